// Capacitance GEMM C = I + alpha^-1 J H^T (line C of Algorithm "MINRES with
// the Laplace-Woodbury preconditioner") on the tcgen05 tensor cores with an
// error-free split of the FP64 operands.
//
// GB300 runs FP64 at 1/64 of the FP32 rate, so the FP64 GEMM is slow, and C
// needs more than single precision: its eigenvalues reach ~1e9, and an
// absolute error of order one in C makes the Woodbury preconditioner
// indefinite (errors of 1e-2 already cost PCG iterations on the ERT
// workloads). The operands are therefore written exactly as sums of BF16
// "digits" and multiplied digit by digit on the tensor cores, with every
// FP32 accumulation kept exact:
//
//  * Chunk scaling: for each row i of J (or H) and each chunk c of 512
//    consecutive K entries an exponent e_ic with max_{k in c} |x_ik| < 2^e_ic.
//    Each entry becomes the integer Y = round(x 2^(48 - e_ic)), |Y| <= 2^48,
//    written in balanced base 128 as seven digits Y = sum_p d_p 128^(6-p),
//    d_1..d_6 in [-64, 63], |d_0| <= 65; each digit is exact in BF16. Scaling per chunk rather
//    than per row keeps the error of the dropped digit pairs proportional to
//    the chunk's own maxima, which matters for sensitivity rows that peak
//    sharply near the electrodes (a 100-fold smaller error in C there).
//  * Digit products d_p d'_q (|.| <= 65 * 64) of the same level l = p + q are
//    summed into one FP32 TMEM accumulator (64 columns per level); pairs with
//    p + q > 6 (weight below 2^-49) are dropped, leaving 28 pairs in 7 levels,
//    issued as 10 MMAs per 16-wide K step (digit p of J against a stack of
//    consecutive digits of H lands on consecutive levels). Over a chunk of
//    512 K entries a level sum is an integer below 512 (2 * 65 * 64 + 5 * 64^2)
//    < 2^24, so the FP32 accumulation is exact. (Base 64, eight digits and
//    1024-entry chunks take 36 pairs for the same 48 bits.)
//  * After every chunk the epilogue warps read the 7 level sums from TMEM,
//    combine them as T_hi = sum_{l<4} S_l 128^(3-l) (exactly, 64-bit integers)
//    and T_lo = sum_{l>=4} S_l 128^(6-l) (FP32, |T_lo| < 2^38), and add
//    2^(e_ic + f_jc - 54) (2^21 T_hi + T_lo) to FP64 accumulators.
//
// Kernel layout: one CTA per (128 x 64 output tile, K range); warp 0 moves
// all seven digit slices of both operands per 32-wide K stage with two bulk
// copies (the digits are stored pre-swizzled in the stage's shared-memory
// image; 64-byte swizzle, double buffered), warp 1 owns TMEM (512 columns, of
// which 7 levels x 64 are used) and issues tcgen05.mma, warps 2..17 drain TMEM. Every
// mbarrier wait is bounded (about one second); on expiry the CTA records
// status bit kStatusTimeout, drains what it started and returns.
#include <cuda_bf16.h>

#include <type_traits>
#include <vector>

#include "df64.cuh"
#include "h1w_internal.cuh"

namespace h1w {
namespace {

constexpr int kSlices = 7;
constexpr int kLevels = 7;                 // digit-pair levels kept: p + q <= 6
static_assert(kLevels == 7, "the epilogue reads levels 0..3 and 4..6");
constexpr int kTileM = 128;                // rows of J per tile (TMEM lanes)
constexpr int kTileN = 64;                 // rows of H per tile (columns per level)
constexpr int kKt = 32;                    // K per stage: 64-byte rows
constexpr int kChunkK = 512;               // K per exact accumulation chunk
constexpr int kItersPerChunk = kChunkK / kKt;
constexpr int kABytes = kSlices * kTileM * kKt * 2;   // 57344
constexpr int kBBytes = kSlices * kTileN * kKt * 2;   // 28672
constexpr int kStageBytes = kABytes + kBBytes;        // 86016 (a multiple of 1024)
constexpr int kStages = 2;
constexpr int kSmemBytes = kStages * kStageBytes + 1024 + 128;
constexpr int kEpiWarps = 16;              // 4 lane quadrants x 4 quarters of the 64 columns
constexpr int kEpiCols = kTileN / 4;       // columns per epilogue thread
constexpr int kGemmThreads = 64 + 32 * kEpiWarps;
constexpr unsigned long long kWaitNs = 1000000000ull;  // one second per wait
// and at most this many polls per wait, should the global timer not advance (a legitimate
// wait, for one copy or one MMA, lasts microseconds)
constexpr uint32_t kWaitPolls = 1u << 24;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t a, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t a) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t a, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(a), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: false when the abort flag is set or wait_ns (normally one second) passes.
__device__ bool mbar_wait(uint32_t a, uint32_t parity, volatile int* abort_flag, uint64_t wait_ns) {
  if (mbar_try(a, parity)) return true;
  const uint64_t t0 = gtimer();
  for (uint32_t n = 1;; ++n) {
    if (mbar_try(a, parity)) return true;
    if ((n & 255) == 0) {
      if (*abort_flag) return false;
      if (gtimer() - t0 > wait_ns || n >= kWaitPolls) return false;
    }
  }
}
// 1D bulk copy global -> shared, completion counted on an mbarrier (16-byte aligned, size % 16 == 0)
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(mbar)
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// K-major operand with 64-byte swizzle: 8-row groups 512 bytes apart.
__device__ __forceinline__ uint64_t desc_sw64(uint32_t saddr) {
  return static_cast<uint64_t>((saddr & 0x3FFFF) >> 4) | (1ull << 16) | (static_cast<uint64_t>(512 >> 4) << 32) |
         (1ull << 46) | (4ull << 61);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
      "[%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

struct OzakiArgs {
  const uint16_t* dA;   // digits of J, stage-tiled (see k_split_digits)
  const uint16_t* dB;   // digits of H, stage-tiled
  const int* eA;        // chunk exponents of J, [global chunk][m]
  const int* eB;        // chunk exponents of H, [global chunk][m]
  long long chunk0;     // global index of the panel's first chunk
  const int2* tiles;    // (128-row block of J, 64-row block of H)
  double* partial;      // [gridDim.y][m][m]
  int* status;
  int m;
  int accumulate;       // add into partial instead of storing
  long long kcta;       // K entries per CTA (multiple of kChunkK)
  long long klen;       // K extent of the digit tensors (multiple of kChunkK)
  long long kvalid;     // K entries of the panel holding data, rounded up to kChunkK (<= klen)
  unsigned long long wait_ns;  // limit of each pipeline wait (one second unless a test shortens it)
  int stall;            // failure-path test: the copy warp issues nothing, so every consumer's wait runs out
};

// 18 warps: four or five per SM sub-partition (16K registers each) cap a thread at 96 registers
__global__ void __launch_bounds__(kGemmThreads, 1) k_ozaki_gemm(OzakiArgs g) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kStages * kStageBytes);
  // bars: 0,1 stage full; 2,3 stage empty; 4 tmem full; 5 tmem empty
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 8);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  int* issued = reinterpret_cast<int*>(tmem_slot + 2);     // stage loads issued
  int* committed = reinterpret_cast<int*>(tmem_slot + 3);  // chunks committed to tmem_full

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int2 tile = g.tiles[blockIdx.x];
  const int row0 = tile.x * kTileM, col0 = tile.y * kTileN;
  const long long kbeg = static_cast<long long>(blockIdx.y) * g.kcta;
  long long kend = kbeg + g.kcta;
  if (kend > g.kvalid) kend = g.kvalid;  // chunks past the data (last panel) are all zero
  const int nchunks = kend > kbeg ? static_cast<int>((kend - kbeg) / kChunkK) : 0;
  const int iters = nchunks * kItersPerChunk;

  if (threadIdx.x == 0) {
    for (int b = 0; b < 4; ++b) mbar_init(smem_u32(&bars[b]), 1);
    mbar_init(smem_u32(&bars[4]), 1);
    mbar_init(smem_u32(&bars[5]), kEpiWarps);
    *abort_flag = 0;
    *issued = 0;
    *committed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(tmem_slot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0 && !g.stall) {
      for (int it = 0; it < iters; ++it) {
        const int s = it & 1;
        const uint32_t ph = (it >> 1) & 1;
        if (!mbar_wait(smem_u32(&bars[2 + s]), ph ^ 1, abort_flag, g.wait_ns)) {
          *abort_flag = 1;
          break;
        }
        const uint32_t full = smem_u32(&bars[s]);
        mbar_expect_tx(full, kStageBytes);
        const long long kb = (kbeg + static_cast<long long>(it) * kKt) / kKt;  // K block in the panel
        const long long nkb = g.klen / kKt;
        const uint32_t dst = smem_u32(smem + s * kStageBytes);
        bulk_load(dst, g.dA + (static_cast<long long>(tile.x) * nkb + kb) * (kABytes / 2), kABytes, full);
        bulk_load(dst + kABytes, g.dB + (static_cast<long long>(tile.y) * nkb + kb) * (kBBytes / 2), kBBytes, full);
        *issued = it + 1;
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // BF16 x BF16 -> FP32, both K-major, M = 128, N = 64 nq. The B slices of a
      // stage are consecutive 64-row blocks, so digit p of J against the
      // stacked digits q0 .. q0 + nq - 1 of H is one MMA whose accumulator
      // columns (p + q0) 64 .. (p + q0 + nq) 64 are exactly the levels p + q.
      uint32_t idesc[5];
#pragma unroll
      for (int nq = 1; nq <= 4; ++nq)
        idesc[nq] = (1u << 4) | (1u << 7) | (1u << 10) | (((nq * kTileN) >> 3) << 17) | ((kTileM >> 4) << 24);
      // (p, q0, nq) covering every pair p + q <= 6 once, N <= 256 per MMA
      constexpr int kMmas = 10;
      constexpr int kP[kMmas] = {0, 0, 1, 1, 2, 2, 3, 4, 5, 6};
      constexpr int kQ0[kMmas] = {0, 4, 0, 4, 0, 4, 0, 0, 0, 0};
      constexpr int kNq[kMmas] = {4, 3, 4, 2, 4, 1, 4, 3, 2, 1};
      int it = 0;
      bool ok = true;
      for (int c = 0; c < nchunks && ok; ++c) {
        if (!mbar_wait(smem_u32(&bars[5]), (c & 1) ^ 1, abort_flag, g.wait_ns)) { ok = false; break; }
        tc_fence_after();
        for (int j = 0; j < kItersPerChunk; ++j, ++it) {
          const int s = it & 1;
          const uint32_t ph = (it >> 1) & 1;
          if (!mbar_wait(smem_u32(&bars[s]), ph, abort_flag, g.wait_ns)) { ok = false; break; }
          tc_fence_after();
          const uint32_t a0 = smem_u32(smem + s * kStageBytes);
          const uint64_t adesc0 = desc_sw64(a0);
          const uint64_t bdesc0 = desc_sw64(a0 + kABytes);
#pragma unroll
          for (int ks = 0; ks < kKt / 16; ++ks) {
#pragma unroll
            for (int u = 0; u < kMmas; ++u) {
              // descriptor start addresses are in 16-byte units
              const uint64_t ad = adesc0 + static_cast<uint64_t>((kP[u] * kTileM * kKt * 2 + ks * 32) >> 4);
              const uint64_t bd = bdesc0 + static_cast<uint64_t>((kQ0[u] * kTileN * kKt * 2 + ks * 32) >> 4);
              // the first MMAs of a chunk (p = 0, both halves) overwrite all 7 levels
              const uint32_t acc = (j == 0 && ks == 0 && kP[u] == 0) ? 0u : 1u;
              mma_bf16(tmem + static_cast<uint32_t>((kP[u] + kQ0[u]) * kTileN), ad, bd, idesc[kNq[u]], acc);
            }
          }
          mma_commit(smem_u32(&bars[2 + s]));
        }
        if (!ok) break;
        mma_commit(smem_u32(&bars[4]));
        *committed = c + 1;
      }
      if (!ok) *abort_flag = 1;
    }
  } else {
    // epilogue: warps 2 .. 2 + kEpiWarps - 1; lane quadrant = warp % 4 (the TMEM lanes a warp
    // may read), column quarter = (warp - 2) / 4. All seven level sums of a chunk are read
    // before TMEM is handed back, and the FP64 work of the chunk comes after, so the next
    // chunk's MMAs wait only for the TMEM loads: the FP64 pipe (1/64 of the FP32 rate) would
    // otherwise stall the tensor cores for several microseconds per chunk.
    const int quad = warp & 3, quarter = (warp - 2) >> 2;
    double acc[kEpiCols];
#pragma unroll
    for (int j = 0; j < kEpiCols; ++j) acc[j] = 0.0;
    const int row = row0 + 32 * quad + lane;
    const int colb = col0 + quarter * kEpiCols;
    const uint32_t tbase = tmem + (static_cast<uint32_t>(32 * quad) << 16) + quarter * kEpiCols;
    for (int c = 0; c < nchunks; ++c) {
      // per-chunk scale factors 2^(e_row + f_col - 54) for this thread's columns
      const long long gch = g.chunk0 + kbeg / kChunkK + c;
      const int er = (row < g.m) ? g.eA[gch * g.m + row] : -100000;
      // lane 0 waits; the warp follows its result so that the .sync.aligned
      // TMEM loads below stay warp-uniform
      int ok = 1;
      if (lane == 0) ok = mbar_wait(smem_u32(&bars[4]), c & 1, abort_flag, g.wait_ns) ? 1 : 0;
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) { if (lane == 0) *abort_flag = 1; break; }
      __syncwarp();
      tc_fence_after();
      // levels 0..3 exactly in 64-bit integers: |T_hi| < 2^24 * 128^3 * 1.01 < 2^46
      long long Thi[kEpiCols];
#pragma unroll
      for (int j = 0; j < kEpiCols; ++j) Thi[j] = 0;
      // two TMEM loads in flight per wait (each wait is a round trip while the tensor cores idle)
#pragma unroll 1
      for (int lev = 0; lev < 4; lev += 2) {
        uint32_t v0[kEpiCols], v1[kEpiCols];
        tmem_ld16(tbase + lev * kTileN, v0);
        tmem_ld16(tbase + (lev + 1) * kTileN, v1);
        tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < kEpiCols; ++j)
          Thi[j] = (Thi[j] * 128 + static_cast<long long>(__float2int_rn(__uint_as_float(v0[j])))) * 128 +
                   static_cast<long long>(__float2int_rn(__uint_as_float(v1[j])));
      }
      // levels 4..6 in FP32: |T_lo| < 2^38, so its rounding (below 2^15 units of the last
      // level) stays under the rounding of the digit split itself
      float Tlo[kEpiCols];
      {
        uint32_t v4[kEpiCols], v5[kEpiCols], v6[kEpiCols];
        tmem_ld16(tbase + 4 * kTileN, v4);
        tmem_ld16(tbase + 5 * kTileN, v5);
        tmem_ld16(tbase + 6 * kTileN, v6);
        tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < kEpiCols; ++j)
          Tlo[j] = fmaf(fmaf(__uint_as_float(v4[j]), 128.f, __uint_as_float(v5[j])), 128.f, __uint_as_float(v6[j]));
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&bars[5]));  // TMEM may be overwritten now
#pragma unroll
      for (int j = 0; j < kEpiCols; ++j) {
        const int col = colb + j;
        const int ec = (col < g.m) ? g.eB[gch * g.m + col] : -100000;
        const int k2 = er + ec - 54;
        // 2^k2 from its bit pattern (0 below the normal range; such chunks are negligible)
        const double scale = (k2 >= -1022 && k2 <= 1023)
                                 ? __longlong_as_double(static_cast<long long>(k2 + 1023) << 52)
                                 : 0.0;
        // 2^21 T_hi + T_lo (the upper group carries the weight 128^3 = 2^21)
        const double val = fma(static_cast<double>(Thi[j]), 2097152.0, static_cast<double>(Tlo[j]));
        acc[j] = fma(val, scale, acc[j]);
      }
    }
    if (!*abort_flag && row < g.m) {
      double* dst = g.partial + static_cast<long long>(blockIdx.y) * g.m * g.m + static_cast<long long>(row) * g.m;
#pragma unroll
      for (int j = 0; j < kEpiCols; ++j) {
        const int col = colb + j;
        if (col < g.m) dst[col] = g.accumulate ? dst[col] + acc[j] : acc[j];
      }
    }
  }

  // teardown: on a timeout wait (bounded) for copies and MMAs still in flight
  __syncthreads();
  if (threadIdx.x == 0 && *abort_flag) {
    atomicOr(g.status, kStatusTimeout);
    const int n = *issued;
    for (int it = (n > 2 ? n - 2 : 0); it < n; ++it) {
      const uint64_t t0 = gtimer();
      for (uint32_t k = 0; !mbar_try(smem_u32(&bars[it & 1]), (it >> 1) & 1) && gtimer() - t0 < kWaitNs &&
                           k < kWaitPolls;
           ++k) {
      }
    }
    const int cc = *committed;
    if (cc > 0) {
      const uint64_t t0 = gtimer();
      for (uint32_t k = 0; !mbar_try(smem_u32(&bars[4]), (cc - 1) & 1) && gtimer() - t0 < kWaitNs && k < kWaitPolls;
           ++k) {
      }
    }
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
  }
}

// ---- operand split ---------------------------------------------------------------

__device__ __forceinline__ long long digits_source(double x, int echunk) {
  // Y = round(|x| 2^(48 - e)) with the sign of x (integer arithmetic on the bits)
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
  const int ex = static_cast<int>((b >> 52) & 0x7FF);
  const long long M = static_cast<long long>((b & 0xFFFFFFFFFFFFFull) | (ex ? (1ull << 52) : 0ull));
  const int sh = 1027 + echunk - (ex ? ex : 1);
  long long Y = 0;
  if (M != 0 && sh >= 1 && sh <= 54) Y = (M + (1ll << (sh - 1))) >> sh;
  return (b >> 63) ? -Y : Y;
}

// The same for one FP32 part of a double-float: |v| < 2^e, so the shift is at least -24
// and |Y| <= 2^48 (integer arithmetic on the bits).
__device__ __forceinline__ long long digits_source_f32(float v, int echunk) {
  const unsigned b = __float_as_uint(v);
  const int ex = static_cast<int>((b >> 23) & 0xFF);
  const long long M = static_cast<long long>((b & 0x7FFFFFu) | (ex ? 0x800000u : 0u));
  const int sh = 102 + echunk - (ex ? ex : 1);
  long long Y = 0;
  if (M != 0 && sh <= 24) Y = sh >= 1 ? (M + (1ll << (sh - 1))) >> sh : M << (-sh);
  return (b >> 31) ? -Y : Y;
}

// Balanced base-128 digits Y = sum_p d_p 128^(6 - p), d_1..d_6 in [-64, 63], |Y| <= 2^48
// (so |d_0| <= 65). The low three digits are fixed by Y modulo 2^21: their value is the
// representative of Y mod 2^21 in [-64 S, 63 S], S = 1 + 128 + 128^2 (a window of exactly
// 2^21 values), so Y splits once into that low part and an exact high part, and each is
// taken apart in 32-bit arithmetic; the digits are those of the digit-by-digit recurrence.
__device__ __forceinline__ void balanced_digits(long long Y, int (&d)[kSlices]) {
  constexpr int kS64 = 64 * (1 + 128 + 16384);
  const int lo = static_cast<int>((Y + kS64) & 0x1FFFFF) - kS64;
  int hi = static_cast<int>((Y - lo) >> 21);
  int y = lo;
#pragma unroll
  for (int p = 6; p >= 4; --p) {
    const int r = ((y + 64) & 127) - 64;
    d[p] = r;
    y = (y - r) >> 7;
  }
#pragma unroll
  for (int p = 3; p >= 1; --p) {
    const int r = ((hi + 64) & 127) - 64;
    d[p] = r;
    hi = (hi - r) >> 7;
  }
  d[0] = hi;
}

// Two small integers (|d| < 2^22) as a packed pair of BF16 values, exactly: adding d to
// the bit pattern of 1.5 * 2^23 and subtracting 1.5 * 2^23 gives float(d); a value of at
// most 8 significant bits leaves the low 16 bits of the float zero, so its upper half is
// the BF16 encoding.
__device__ __forceinline__ uint32_t pack_bf16x2(int d0, int d1) {
  const float f0 = __fsub_rn(__int_as_float(0x4B400000 + d0), 12582912.0f);
  const float f1 = __fsub_rn(__int_as_float(0x4B400000 + d1), 12582912.0f);
  return __byte_perm(__float_as_uint(f0), __float_as_uint(f1), 0x7632);
}

// Seven balanced base-128 digits of each of 8 consecutive K entries, written as one 16-byte
// chunk per digit slice into the stage-tiled, pre-swizzled layout the GEMM copies from:
// [row block][K block of kKt][slice][row in block][kKt], 16-byte chunk c of a row stored at
// c ^ ((row >> 1) & 3) (64-byte swizzle).
__device__ __forceinline__ void store_digits(long long (&Y)[8], int row, long long kc, long long klen, int R,
                                             uint16_t* __restrict__ S) {
  uint32_t packed[kSlices][4];
#pragma unroll
  for (int t = 0; t < 8; t += 2) {
    int da[kSlices], db[kSlices];
    balanced_digits(Y[t], da);
    balanced_digits(Y[t + 1], db);
#pragma unroll
    for (int p = 0; p < kSlices; ++p) packed[p][t >> 1] = pack_bf16x2(da[p], db[p]);
  }
  const int rb = row / R, ri = row % R;
  const long long kb = kc / kKt;
  const int chunk = static_cast<int>((kc % kKt) >> 3);
  const int pchunk = chunk ^ ((ri >> 1) & 3);
  const long long nkb = klen / kKt;
  uint16_t* base = S + ((static_cast<long long>(rb) * nkb + kb) * kSlices) * (R * kKt) + ri * kKt + pchunk * 8;
#pragma unroll
  for (int p = 0; p < kSlices; ++p)
    *reinterpret_cast<uint4*>(base + static_cast<long long>(p) * R * kKt) =
        make_uint4(packed[p][0], packed[p][1], packed[p][2], packed[p][3]);
}

// Split of one K panel [k0, k0 + kw) of X (m rows of N) into digits. A block of
// 64 kSplitRows threads covers kSplitRows consecutive rows and one chunk of 512 K
// entries. A warp takes 8 / kSplitRows K stages of 32 entries; in a stage, lane =
// 4 (row in the group) + 16-byte chunk, so each warp reads row segments of 256 bytes and
// writes kSplitRows consecutive rows (64 kSplitRows bytes) of a stage image per digit
// slice. Per row it finds the chunk exponent e with max |x| < 2^e (-100000 for an
// all-zero chunk), stores it at e[(chunk0 + blockIdx.y) m + row] and writes the digits of
// x 2^(48 - e). Grid: (rows rounded up to R / kSplitRows, klen / 512), rows fastest, so
// that blocks running together fill neighbouring rows of the same stage images. XS is double
// (FP64) or df (double-float, value hi + lo: the exponent comes from the high parts, since
// |hi + lo| <= |hi| (1 + 2^-24) stays within the digit range, and each part is scaled on
// its own, so the value is represented to within 2^(e - 48)).
constexpr int kSplitRows = 1;
constexpr int kSplitThreads = kChunkK / 8 * kSplitRows;  // 8 entries per thread

//
// row0 offsets the rows (a launch may cover a row range of the panel); XD (may be null, FP64
// sources only) receives the double-float conversion of every entry read, the same values as
// k_d2df, so that a pass that needs both reads X once.
template <typename XS>
__global__ void __launch_bounds__(kSplitThreads) k_split_digits(const XS* __restrict__ X, int m, long long N,
                                                                long long k0, long long kw, long long klen, int R,
                                                                long long chunk0, int* __restrict__ e,
                                                                uint16_t* __restrict__ S, int row0 = 0,
                                                                df* __restrict__ XD = nullptr,
                                                                long long pstride = 0) {
  // pstride > 0: one launch over every K panel; blockIdx.y counts the chunks of all panels,
  // and each block finds its panel (offset k0, width kw, digits at S + panel * pstride)
  int by = static_cast<int>(blockIdx.y);
  if (pstride > 0) {
    const int cpp = static_cast<int>(klen / kChunkK);
    const int p = by / cpp;
    by -= p * cpp;
    k0 = static_cast<long long>(p) * klen;
    kw = (N - k0) < klen ? (N - k0) : klen;
    chunk0 = k0 / kChunkK;
    S += static_cast<long long>(p) * pstride;
  }
  constexpr int kGroup = 4 * kSplitRows;   // lanes per stage
  constexpr int kStagesPerWarp = 32 / kGroup;
  constexpr int kWarps = kSplitThreads / 32;
  __shared__ int smax[kWarps][kSplitRows];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int sub = lane / kGroup, rg = (lane >> 2) % kSplitRows, ch = lane & 3;
  const int row = row0 + blockIdx.x * kSplitRows + rg;
  const long long kc =
      static_cast<long long>(by) * kChunkK + (warp * kStagesPerWarp + sub) * kKt + ch * 8;
  constexpr bool kDf = std::is_same<XS, df>::value;
  XS x[8];
  int best = 0;
  // the thread's 8 entries are 64 contiguous bytes: four 16-byte loads when they all lie in
  // the panel and the row start is 16-byte aligned (N even), else entry by entry
  const bool whole = row < m && kc + 8 <= kw && (N & 1) == 0 &&
                     (reinterpret_cast<uintptr_t>(X) & 15) == 0;
  if (whole) {
    const float4* src = reinterpret_cast<const float4*>(X + row * N + k0 + kc);
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const float4 f = src[v];
      if constexpr (kDf) {
        x[2 * v] = df_make(f.x, f.y);
        x[2 * v + 1] = df_make(f.z, f.w);
      } else {
        x[2 * v] = __hiloint2double(__float_as_int(f.y), __float_as_int(f.x));
        x[2 * v + 1] = __hiloint2double(__float_as_int(f.w), __float_as_int(f.z));
      }
    }
  } else {
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const long long k = kc + t;
      if constexpr (kDf) x[t] = (k < kw && row < m) ? X[row * N + k0 + k] : df_make(0.f, 0.f);
      else x[t] = (k < kw && row < m) ? X[row * N + k0 + k] : 0.0;
    }
  }
  if constexpr (!kDf) {
    if (XD && row < m) {  // the double-float copy: 64 contiguous bytes, or entry by entry
      df* dst = XD + row * N + k0 + kc;
      if (whole && (reinterpret_cast<uintptr_t>(XD) & 15) == 0) {
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const df a = df_from_double_fast(x[2 * v]), b = df_from_double_fast(x[2 * v + 1]);
          reinterpret_cast<float4*>(dst)[v] = make_float4(a.hi, a.lo, b.hi, b.lo);
        }
      } else {
#pragma unroll
        for (int t = 0; t < 8; ++t)
          if (kc + t < kw) dst[t] = df_from_double_fast(x[t]);
      }
    }
  }
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    int ex;
    if constexpr (kDf) ex = static_cast<int>((__float_as_uint(x[t].hi) >> 23) & 0xFF);
    else ex = static_cast<int>((static_cast<unsigned long long>(__double_as_longlong(x[t])) >> 52) & 0x7FF);
    best = ex > best ? ex : best;
  }
  // max over the row's lanes of this warp (its chunks and stages), then over the warps
  best = max(best, __shfl_xor_sync(0xffffffffu, best, 1));
  best = max(best, __shfl_xor_sync(0xffffffffu, best, 2));
#pragma unroll
  for (int o = kGroup; o < 32; o <<= 1) best = max(best, __shfl_xor_sync(0xffffffffu, best, o));
  if (ch == 0 && sub == 0) smax[warp][rg] = best;
  __syncthreads();
  best = 0;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) best = max(best, smax[w][rg]);
  int ech;
  if constexpr (kDf) ech = best ? best - 126 : -100000;
  else ech = best ? best - 1022 : -100000;
  if (warp == 0 && sub == 0 && ch == 0 && row < m && static_cast<long long>(by) * kChunkK < kw)
    e[(chunk0 + by) * m + row] = ech;
  long long Y[8];
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    if constexpr (kDf) Y[t] = digits_source_f32(x[t].hi, ech) + digits_source_f32(x[t].lo, ech);
    else Y[t] = digits_source(x[t], ech);
  }
  store_digits(Y, row, kc, klen, R, S);
}

}  // namespace

long long ozaki_panel_width(long long N) {
  long long kp = (N + kChunkK - 1) / kChunkK * kChunkK;
  const long long cap = 262144;
  return kp < cap ? kp : cap;
}

int ozaki_num_tiles(int m) {
  const int rb = (m + kTileM - 1) / kTileM, cb = (m + kTileN - 1) / kTileN;
  int t = 0;
  for (int I = 0; I < rb; ++I)
    for (int J = 2 * I; J < cb; ++J) ++t;
  return t;
}

void ozaki_tiles(int m, std::vector<int>& out) {
  const int rb = (m + kTileM - 1) / kTileM, cb = (m + kTileN - 1) / kTileN;
  out.clear();
  for (int I = 0; I < rb; ++I)
    for (int J = 2 * I; J < cb; ++J) {
      out.push_back(I);
      out.push_back(J);
    }
}

// K splits per panel: the tiles x splits CTAs (one per SM) should fill whole waves of
// the GPU's sms SMs with equal work. Cost = chunks of the busiest CTA x waves, with a
// small charge per split for the partial outputs and their reduction.
int ozaki_splits(int m, long long kp, int sms) {
  const int tiles = ozaki_num_tiles(m);
  const long long nch = kp / kChunkK;
  if (sms < 1) sms = 1;
  if (sms > kMaxSms) sms = kMaxSms;
  int best = 1;
  double best_cost = 1e300;
  const long long lim = 2LL * ((sms + tiles - 1) / tiles);  // ozaki_max_splits
  const long long smax = nch < lim ? nch : lim;
  for (long long sp = 1; sp <= smax; ++sp) {
    const long long per = (nch + sp - 1) / sp;
    const long long waves = (tiles * sp + sms - 1) / sms;
    const double cost = static_cast<double>(per * waves) * (1.0 + 0.01 * static_cast<double>(sp));
    if (cost < best_cost) {
      best_cost = cost;
      best = static_cast<int>(sp);
    }
  }
  return best;
}

int ozaki_max_splits(int m) {
  const int tiles = ozaki_num_tiles(m);
  return 2 * ((kMaxSms + tiles - 1) / tiles);
}

bool ozaki_supported() {
  int dev = 0, major = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  return major == 10;
}

// C partials (FP64, [splits][m][m], upper tiles) of J H^T via the digit split. Each operand
// comes as FP64 (J, H) or, when its double-float copy (Jdf, Hdf) is given, as that.
// Returns false when the kernel attribute cannot be set or the GEMM launch is refused.
bool launch_ozaki_capacitance(const double* J, const double* H, const df* Jdf, const df* Hdf, int m, long long N,
                              const OzakiWork& w, int splits, cudaStream_t s, void (*hook)(void*, int, int),
                              void* hook_arg) {
  const long long kp = w.klen;
  const long long nch = (N + kChunkK - 1) / kChunkK;
  int* eA = w.expo;
  int* eB = w.expo + nch * m;
  if (cudaFuncSetAttribute(k_ozaki_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes) != cudaSuccess)
    return false;

  const int tiles = ozaki_num_tiles(m);
  long long kcta = (kp + splits - 1) / splits;
  kcta = (kcta + kChunkK - 1) / kChunkK * kChunkK;
  int panel = 0;
  for (long long k0 = 0; k0 < N; k0 += kp, ++panel) {
    const long long kw = (N - k0) < kp ? (N - k0) : kp;
    const long long chunk0 = k0 / kChunkK;
    const int rowsA = (m + kTileM - 1) / kTileM * kTileM, rowsB = (m + kTileN - 1) / kTileN * kTileN;
    const unsigned gx = static_cast<unsigned>(kp / kChunkK);
    uint16_t* dA = static_cast<uint16_t*>(w.digitsA);
    uint16_t* dB = static_cast<uint16_t*>(w.digitsB);
    const dim3 ga(rowsA / kSplitRows, gx), gb(rowsB / kSplitRows, gx);
    if (w.j_full) {  // split during line H: this panel's digits in the full-K buffer
      dA += (size_t)panel * kSlices * rowsA * kp;
    } else {
      if (hook) hook(hook_arg, kOzakiSplitJ, 1);
      if (Jdf) k_split_digits<df><<<ga, kSplitThreads, 0, s>>>(Jdf, m, N, k0, kw, kp, kTileM, chunk0, eA, dA);
      else k_split_digits<double><<<ga, kSplitThreads, 0, s>>>(J, m, N, k0, kw, kp, kTileM, chunk0, eA, dA);
      if (hook) hook(hook_arg, kOzakiSplitJ, 0);
    }
    if (hook) hook(hook_arg, kOzakiSplitH, 1);
    if (Hdf) k_split_digits<df><<<gb, kSplitThreads, 0, s>>>(Hdf, m, N, k0, kw, kp, kTileN, chunk0, eB, dB);
    else k_split_digits<double><<<gb, kSplitThreads, 0, s>>>(H, m, N, k0, kw, kp, kTileN, chunk0, eB, dB);
    if (hook) hook(hook_arg, kOzakiSplitH, 0);
    OzakiArgs a;
    a.dA = dA;
    a.dB = dB;
    a.eA = eA;
    a.eB = eB;
    a.chunk0 = chunk0;
    a.tiles = reinterpret_cast<const int2*>(w.tiles);
    a.partial = w.partial;
    a.status = w.status;
    a.m = m;
    a.accumulate = panel > 0 ? 1 : 0;
    a.kcta = kcta;
    a.klen = kp;
    a.kvalid = (kw + kChunkK - 1) / kChunkK * kChunkK;
    a.wait_ns = w.wait_ns ? w.wait_ns : kWaitNs;
    a.stall = w.stall;
    if (hook) hook(hook_arg, kOzakiGemm, 1);
    k_ozaki_gemm<<<dim3(tiles, splits), kGemmThreads, kSmemBytes, s>>>(a);
    if (cudaPeekAtLastError() != cudaSuccess) return false;  // a launch the GPU refused (resources)
    if (hook) hook(hook_arg, kOzakiGemm, 0);
    note_launches(w.j_full ? 2 : 3);
  }
  return true;
}

long long ozaki_chunks(long long N) { return (N + kChunkK - 1) / kChunkK; }

size_t ozaki_j_digits_full_bytes(int m, long long N) {
  const long long kp = ozaki_panel_width(N);
  const long long panels = (N + kp - 1) / kp;
  const long long rowsA = (m + kTileM - 1) / kTileM * kTileM;
  return sizeof(uint16_t) * (size_t)kSlices * rowsA * kp * panels;
}

void launch_split_j_rows(const double* J, int m, long long N, int r0, int r1, const OzakiWork& w, df* Jdf,
                         cudaStream_t s) {
  const long long kp = w.klen;
  const int rowsA = (m + kTileM - 1) / kTileM * kTileM;
  const int rend = r1 >= m ? rowsA : r1;
  if (rend <= r0) return;
  const long long panel_elems = (long long)kSlices * rowsA * kp;
  const long long panels = (N + kp - 1) / kp;
  const dim3 g((unsigned)((rend - r0) / kSplitRows), (unsigned)(panels * (kp / kChunkK)));
  k_split_digits<double><<<g, kSplitThreads, 0, s>>>(J, m, N, 0, kp, kp, kTileM, 0, w.expo,
                                                    static_cast<uint16_t*>(w.digitsA), r0, Jdf, panel_elems);
  note_launches(1);
}
int ozaki_digit_slices() { return kSlices; }

}  // namespace h1w
