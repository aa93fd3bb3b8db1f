// Fused legs of the double-float V-cycle on FV levels whose three axes are all
// coarsened 2:1, with the degree-2 Chebyshev-Jacobi smoother.
//
// Down leg (one kernel): x = S(b), two smoothing steps from x = 0, then the
// restricted residual bc = P^T (b - A x). Up leg (one kernel): x' = x + P xc,
// two smoothing steps from x', result y.
//
// The double-float V-cycle is bound by instruction issue, not by HBM (about
// 40 FP32 instructions per double-float addition or product), so the legs are
// written to need as few double-float operations as possible:
//  * With A = D - N_T (D the diagonal, N_T(u) = sum over axes of T_a times the
//    two face neighbours of u along a), the two Chebyshev steps collapse into
//      down: g = D^-1 b,  x = beta g + gam_c N_T(g),
//      up:   r0 = b + N_T(x') - d_c x',  d0 = del_c r0,
//            y = x' + eta_c r0 + kap_c N_T(d0),
//    with the per-class constants of FusedCoef (exact algebra of the two steps
//    r1 = r0 - A d0, d1 = c1 d0 + c2 D^-1 r1, x += d0 + d1 with d0 = D^-1 r0 / theta).
//    On isotropic levels N_T is T times the plain neighbour sum, and gam_c T and kap_c T
//    are formed once on the host, which saves a product per cell in those two steps.
//  * Values outside the domain are stored as exact zeros in the on-chip
//    buffers, so the stencils sum all six neighbours without boundary tests;
//    the neighbour counts only select the class of the constants.
//  * The prolongation is separable: each coarse plane is interpolated along x,
//    then y, once, and every fine plane combines two such planes along z.
//
// A block owns an xy tile of kFX x kFY fine cells and a range of z planes and
// marches through the planes, keeping the planes each step needs in rings in
// shared memory; every step works on the tile grown by the halo the later
// steps read (3, 2, 1 cells), so neighbouring blocks repeat a little work
// instead of exchanging it. Only b, x and the coarse vectors go through HBM.
#include <algorithm>
#include <atomic>
#include <type_traits>

#include "df64.cuh"
#include "h1w_internal.cuh"
#include "mg_df64_util.cuh"

namespace h1w {
namespace {

using namespace dfmg;

// Tile shape and block size (compile-time). Defaults: 32 x 16 tiles, 256 threads, and
// launch bounds that hold both legs to 85 registers so that three blocks (24 warps) stay
// resident per SM; at two blocks per SM both legs run 10-14 % slower. Larger tiles
// (32 x 32 or 64 x 16 with 512 threads) repeat less halo work but leave the up leg one
// block per SM, which costs more than the halo saves at 128^3.
#ifndef H1W_FUSED_FX
#define H1W_FUSED_FX 32
#endif
#ifndef H1W_FUSED_FY
#define H1W_FUSED_FY 16
#endif
#ifndef H1W_FUSED_THREADS
#define H1W_FUSED_THREADS 256
#endif
#ifndef H1W_FUSED_PRE_MINB
#define H1W_FUSED_PRE_MINB 3
#endif
#ifndef H1W_FUSED_POST_MINB
#define H1W_FUSED_POST_MINB 3
#endif
#ifndef H1W_FUSED_BLOCKS_PER_SM
#define H1W_FUSED_BLOCKS_PER_SM 3
#endif
constexpr int kFX = H1W_FUSED_FX, kFY = H1W_FUSED_FY;           // fine cells of a tile
constexpr int kTX = kFX / 2, kTY = kFY / 2;                     // coarse cells of a tile
constexpr int kW3 = kFX + 6, kH3 = kFY + 6, kA3 = kW3 * kH3;    // tile + 3
constexpr int kW2 = kFX + 4, kH2 = kFY + 4, kA2 = kW2 * kH2;    // tile + 2
constexpr int kW1 = kFX + 2, kH1 = kFY + 2, kA1 = kW1 * kH1;    // tile + 1
constexpr int kHC = kTY + 4;                                    // coarse rows of tile + 2
constexpr int kAX = kHC * kW2;                                  // coarse rows x fine columns
constexpr int kThr = H1W_FUSED_THREADS;
constexpr int kP3 = (kA3 + kThr - 1) / kThr;
constexpr int kP2 = (kA2 + kThr - 1) / kThr;
constexpr int kP1 = (kA1 + kThr - 1) / kThr;
constexpr int kTab = 27;

constexpr int kRX = kH1 * kTX;                                  // fine rows of tile + 1 x coarse columns
constexpr size_t kPreSmem = sizeof(df) * (3 * kA3 + 3 * kA1 + 3 * kA2 + kA1 + 3 * kTab + 1 + kRX + 2 * kTX);  // see k_pre_fused
constexpr size_t kPostSmem = sizeof(df) * (4 * kA2 + 3 * kA2 + kAX + 4 * kA1 + 2 * kA1 + 4 * kTab);  // see k_post_fused

__device__ __forceinline__ bool in_xy(const Level& L, int i, int j) {
  return i >= 0 && i < L.nx && j >= 0 && j < L.ny;
}

// (offset in the plane << 5) | (flag << 4) | xy part of the neighbour class, or -1 outside
// the domain (the launchers require nx ny < 2^26)
__device__ __forceinline__ int xy_desc(const Level& L, int gx, int gy, bool flag = false) {
  if (!in_xy(L, gx, gy)) return -1;
  const int c = ((gx > 0) + (gx < L.nx - 1)) + 3 * ((gy > 0) + (gy < L.ny - 1));
  return ((gy * L.nx + gx) << 5) | (flag ? 16 : 0) | c;
}
__device__ __forceinline__ int desc_off(int d) { return d >> 5; }
__device__ __forceinline__ int desc_cls(int d) { return d & 15; }
__device__ __forceinline__ bool desc_flag(int d) { return (d & 16) != 0; }

__device__ __forceinline__ df scale_w(df v, float w) {
  // weights 1/4 and 1 scale exactly; 3/4 needs a product
  if (w == 0.25f) return df_make(v.hi * 0.25f, v.lo * 0.25f);
  if (w == 1.f) return v;
  return df_mul_f(v, w);
}

// Sum of the six face neighbours at idx (isotropic levels, where N_T = T times it).
__device__ __forceinline__ df nsum6(const df* __restrict__ u0, const df* __restrict__ u1, const df* __restrict__ u2,
                                   int idx, int W) {
  dsum s;
  s.add(u1[idx - 1]);
  s.add(u1[idx + 1]);
  s.add(u1[idx - W]);
  s.add(u1[idx + W]);
  s.add(u0[idx]);
  s.add(u2[idx]);
  return s.get();
}

// N_T(u) at idx of a plane buffer with rows of W cells (u0, u2: planes below and above);
// out-of-domain entries hold zeros.
template <bool ISO>
__device__ __forceinline__ df nsum(const df* __restrict__ u0, const df* __restrict__ u1, const df* __restrict__ u2,
                                   int idx, int W, df T0, df T1, df T2) {
  if (ISO) return df_mul(T0, nsum6(u0, u1, u2, idx, W));
  dsum sx, sy, sz;
  sx.add(u1[idx - 1]);
  sx.add(u1[idx + 1]);
  sy.add(u1[idx - W]);
  sy.add(u1[idx + W]);
  sz.add(u0[idx]);
  sz.add(u2[idx]);
  dsum s;
  s.add(df_mul(T0, sx.get()));
  s.add(df_mul(T1, sy.get()));
  s.add(df_mul(T2, sz.get()));
  return s.get();
}

// Down leg. Grid: (xy tiles, z segments of segK coarse planes, right-hand sides).
template <bool ISO, typename TB>
__global__ void __launch_bounds__(kThr, H1W_FUSED_PRE_MINB) k_pre_fused(Level L, Level Lc, FusedCoef F, const TB* __restrict__ b,
                                                    df* __restrict__ x, df* __restrict__ bc, int segK) {
  extern __shared__ df sm[];
  df* Gp = sm;               // g = D^-1 b over tile + 3, 3 planes
  df* Bp = Gp + 3 * kA3;     // b over tile + 1, 3 planes
  df* Xp = Bp + 3 * kA1;     // smoothed x over tile + 2, 3 planes
  df* Rs = Xp + 3 * kA2;     // residual of one plane over tile + 1
  df* td = Rs + kA1;         // d, dinv, gam by class
  df* tdinv = td + kTab;
  df* tgam = tdinv + kTab;
  df* RX = tgam + kTab + 1;  // residual restricted along x: [fine row of tile + 1][coarse column]
  float4* wxt = reinterpret_cast<float4*>(RX + kRX);  // P^T weights of each coarse column of the tile
  const int tid = threadIdx.x;
  for (int i = tid; i < kTab; i += kThr) {
    td[i] = F.d[i];
    tdinv[i] = F.dinv[i];
    tgam[i] = ISO ? F.gamT[i] : F.gam[i];  // isotropic: T folded in, step 2 sums the neighbours only
  }
  const df T0 = F.T[0], T1 = F.T[1], T2 = F.T[2], beta = F.beta;
  const int ntx = (Lc.nx + kTX - 1) / kTX;
  const int C0x = (int)(blockIdx.x % (unsigned)ntx) * kTX, C0y = (int)(blockIdx.x / (unsigned)ntx) * kTY;
  const int F0x = 2 * C0x, F0y = 2 * C0y;
  const int K0 = (int)blockIdx.y * segK, K1 = min(K0 + segK, Lc.nz);
  const int Z0 = 2 * K0, Z1 = 2 * K1;
  const int64_t pl = (int64_t)L.nx * L.ny, plc = (int64_t)Lc.nx * Lc.ny;
  const TB* bb = b + (int64_t)blockIdx.z * L.N;
  df* xx = x + (int64_t)blockIdx.z * L.N;
  df* cc = bc + (int64_t)blockIdx.z * Lc.N;
  const int u_beg = Z0 - 3, u_end = Z1 + 2;
  // ring slots of planes u, u - 1, u - 2 (rotated once per plane instead of a modulo per access)
  int sl0 = 0, sl1 = 2, sl2 = 1;

  // element descriptors, the same on every plane
  int d3[kP3], r3[kP3], d2[kP2], d1[kP1];
#pragma unroll
  for (int q = 0; q < kP3; ++q) {
    const int e = tid + q * kThr;
    const int lx = e % kW3, ly = e / kW3;
    d3[q] = e < kA3 ? xy_desc(L, F0x - 3 + lx, F0y - 3 + ly) : -1;
    r3[q] = (e < kA3 && lx >= 2 && lx < kW3 - 2 && ly >= 2 && ly < kH3 - 2) ? (ly - 2) * kW1 + lx - 2 : -1;
  }
  int i3[kP2], i2[kP1];  // shared-memory index of the element in the buffer a step reads
#pragma unroll
  for (int q = 0; q < kP2; ++q) {
    const int e = tid + q * kThr;
    const int lx = e % kW2, ly = e / kW2;
    const bool interior = lx >= 2 && lx < 2 + kFX && ly >= 2 && ly < 2 + kFY;
    d2[q] = e < kA2 ? xy_desc(L, F0x - 2 + lx, F0y - 2 + ly, interior) : -1;
    i3[q] = (ly + 1) * kW3 + lx + 1;
  }
#pragma unroll
  for (int q = 0; q < kP1; ++q) {
    const int e = tid + q * kThr;
    const int lx = e % kW1, ly = e / kW1;
    d1[q] = e < kA1 ? xy_desc(L, F0x - 1 + lx, F0y - 1 + ly) : -1;
    i2[q] = (ly + 1) * kW2 + lx + 1;
  }

  df pf[kP3];
  auto fetch = [&](int u) {
    const bool uin = (u >= 0 && u < L.nz);
#pragma unroll
    for (int q = 0; q < kP3; ++q) pf[q] = (uin && d3[q] >= 0) ? load_df(bb, u * pl + desc_off(d3[q])) : dzero();
  };
  fetch(u_beg);

  // restriction, separably: the x pass restricts every fine row of tile + 1 once per coarse
  // column (weights from wxt); then thread c < kTX kTY takes coarse cell c along y and z
  static_assert(kTX * kTY <= kThr, "one thread per coarse cell");
  static_assert(((3 * kA3 + 3 * kA1 + 3 * kA2 + kA1 + 3 * kTab + 1 + kRX) % 2) == 0, "wxt 16-byte aligned");
  if (tid < kTX) {
    float w[4];
    fv_rw(min(C0x + tid, Lc.nx - 1), Lc.nx, 1, w);
    wxt[tid] = make_float4(w[0], w[1], w[2], w[3]);
  }
  const int Ic = tid % kTX, Jc = tid / kTX;
  const int gI = C0x + Ic, gJ = C0y + Jc;
  const bool own = tid < kTX * kTY && gI < Lc.nx && gJ < Lc.ny;
  float wy[4];
  fv_rw(min(gJ, Lc.ny - 1), Lc.ny, 1, wy);
  dsum acc_a, acc_b;  // coarse planes K and K + 1 while fine plane 2K + 1 or 2K + 2 is added
  __syncthreads();

  for (int u = u_beg; u <= u_end; ++u) {
    const int t = u - u_beg;
    // step 1, plane u: g = D^-1 b over tile + 3; b kept over tile + 1
    {
      df* Go = Gp + sl0 * kA3;
      df* Bo = Bp + sl0 * kA1;
      const bool uin = (u >= 0 && u < L.nz);
      const int cz = 9 * ((u > 0) + (u < L.nz - 1));
#pragma unroll
      for (int q = 0; q < kP3; ++q) {
        const int e = tid + q * kThr;
        if (e < kA3) {
          Go[e] = (uin && d3[q] >= 0) ? df_mul(pf[q], tdinv[desc_cls(d3[q]) + cz]) : dzero();
          if (r3[q] >= 0) Bo[r3[q]] = pf[q];
        }
      }
      if (u < u_end) fetch(u + 1);
    }
    __syncthreads();
    // step 2, plane v = u - 1: x = beta g + gam_c N_T(g) over tile + 2
    if (t >= 2) {
      const int v = u - 1;
      const df* G0 = Gp + sl2 * kA3;
      const df* G1 = Gp + sl1 * kA3;
      const df* G2 = Gp + sl0 * kA3;
      df* Xo = Xp + sl1 * kA2;
      const bool vin = (v >= 0 && v < L.nz);
      const bool vout = (v >= Z0 && v < Z1);
      const int cz = 9 * ((v > 0) + (v < L.nz - 1));
#pragma unroll
      for (int q = 0; q < kP2; ++q) {
        const int e = tid + q * kThr;
        if (e < kA2) {
          df xv = dzero();
          if (vin && d2[q] >= 0) {
            const df n = ISO ? nsum6(G0, G1, G2, i3[q], kW3) : nsum<false>(G0, G1, G2, i3[q], kW3, T0, T1, T2);
            dsum s;
            s.add(df_mul(beta, G1[i3[q]]));
            s.add(df_mul(tgam[desc_cls(d2[q]) + cz], n));
            xv = s.get();
            if (vout && desc_flag(d2[q])) xx[v * pl + desc_off(d2[q])] = xv;
          }
          Xo[e] = xv;
        }
      }
      __syncthreads();
    }
    // step 3, plane w = u - 2: residual b + N_T(x) - d_c x over tile + 1, then P^T
    if (t >= 4) {
      const int w = u - 2;
      const df* X0 = Xp + sl0 * kA2;  // plane w - 1 = u - 3 shares the slot of u
      const df* X1 = Xp + sl2 * kA2;
      const df* X2 = Xp + sl1 * kA2;
      const df* B1 = Bp + sl2 * kA1;
      const bool win = (w >= 0 && w < L.nz);
      const int cz = 9 * ((w > 0) + (w < L.nz - 1));
#pragma unroll
      for (int q = 0; q < kP1; ++q) {
        const int e = tid + q * kThr;
        if (e < kA1) {
          df rv = dzero();
          if (win && d1[q] >= 0) {
            const df n = nsum<ISO>(X0, X1, X2, i2[q], kW2, T0, T1, T2);
            dsum s;
            s.add(B1[e]);
            s.add(n);
            s.add(df_neg(df_mul(td[desc_cls(d1[q]) + cz], X1[i2[q]])));
            rv = s.get();
          }
          Rs[e] = rv;
        }
      }
      __syncthreads();
      // P^T within the plane: coarse column I takes fine columns 2I - 1 .. 2I + 2 (tile + 1
      // columns 2I .. 2I + 3), coarse row J fine rows 2J - 1 .. 2J + 2 (tile + 1 rows 2J .. 2J + 3)
      for (int e = tid; e < kRX; e += kThr) {
        const int ly = e / kTX, I = e - ly * kTX;
        const df* row = Rs + ly * kW1 + 2 * I;
        const float4 w = wxt[I];
        dsum sx;
        sx.add(df_mul_f(row[0], w.x));
        sx.add(df_mul_f(row[1], w.y));
        sx.add(df_mul_f(row[2], w.z));
        sx.add(df_mul_f(row[3], w.w));
        RX[e] = sx.get();
      }
      __syncthreads();
      df S = dzero();
      if (own) {
        dsum sy;
#pragma unroll
        for (int b = 0; b < 4; ++b) sy.add(df_mul_f(RX[(2 * Jc + b) * kTX + Ic], wy[b]));
        S = sy.get();
      }
      if (own) {
        float wz[4];
        if (w & 1) {  // w = 2K + 1: tap 2 of coarse plane K, tap 0 of K + 1 (which starts here)
          const int K = (w - 1) >> 1;
          if (K >= 0 && K < Lc.nz) {
            fv_rw(K, Lc.nz, 1, wz);
            if (wz[2] != 0.f) acc_a.add(scale_w(S, wz[2]));
          }
          acc_b = dsum();
          if (K + 1 < Lc.nz) {
            fv_rw(K + 1, Lc.nz, 1, wz);
            if (wz[0] != 0.f) acc_b.add(scale_w(S, wz[0]));
          }
        } else {      // w = 2K: tap 1 of K, tap 3 of K - 1, which is then complete
          const int K = w >> 1;
          if (K < Lc.nz) {
            fv_rw(K, Lc.nz, 1, wz);
            if (wz[1] != 0.f) acc_b.add(scale_w(S, wz[1]));
          }
          if (K - 1 >= 0) {
            fv_rw(K - 1, Lc.nz, 1, wz);
            if (wz[3] != 0.f) acc_a.add(scale_w(S, wz[3]));
          }
          if (K - 1 >= K0 && K - 1 < K1) cc[(K - 1) * plc + (int64_t)gJ * Lc.nx + gI] = acc_a.get();
          acc_a = acc_b;
        }
      }
    }
    const int s_old = sl2;  // the slot of u - 2 takes plane u + 1
    sl2 = sl1;
    sl1 = sl0;
    sl0 = s_old;
  }
}

// Up leg. Grid: (xy tiles, z segments of segZ fine planes (even), right-hand sides).
// y and y64 (either may be null) must not overlap x, xc or b. The march over the planes
// is unrolled by four (the x' and d0 rings hold four planes, r0 two), so those ring slots
// are compile-time constants; the coarse ring (three interpolated coarse planes) is
// indexed at run time.
template <bool ISO, typename TB>
__global__ void __launch_bounds__(kThr, H1W_FUSED_POST_MINB) k_post_fused(Level L, Level Lc, FusedCoef F, const df* __restrict__ x,
                                                     const df* __restrict__ xc, const TB* __restrict__ b,
                                                     df* __restrict__ y, double* __restrict__ y64, int segZ) {
  extern __shared__ df sm[];
  // layout (in df): x' over tile + 2, 4 planes; coarse planes interpolated along x and y over
  // tile + 2, 3 planes; one coarse plane interpolated along x (kHC coarse rows x kW2 fine
  // columns); d0 over tile + 1, 4 planes; r0 over tile + 1, 2 planes; d, del, eta, kap by class
  constexpr int oX = 0, oP = oX + 4 * kA2, oPx = oP + 3 * kA2, oD = oPx + kAX, oR = oD + 4 * kA1;
  constexpr int oTd = oR + 2 * kA1;
  df* Pp = sm + oP;
  df* Px = sm + oPx;
  df* td = sm + oTd;
  df* tdel = td + kTab;
  df* teta = tdel + kTab;
  df* tkap = teta + kTab;
  const int tid = threadIdx.x;
  for (int i = tid; i < kTab; i += kThr) {
    td[i] = F.d[i];
    tdel[i] = F.del[i];
    teta[i] = F.eta[i];
    tkap[i] = ISO ? F.kapT[i] : F.kap[i];  // isotropic: T folded in, step 3 sums the neighbours only
  }
  const df T0 = F.T[0], T1 = F.T[1], T2 = F.T[2];
  const int ntx = (Lc.nx + kTX - 1) / kTX;
  const int C0x = (int)(blockIdx.x % (unsigned)ntx) * kTX, C0y = (int)(blockIdx.x / (unsigned)ntx) * kTY;
  const int F0x = 2 * C0x, F0y = 2 * C0y;
  const int Z0 = (int)blockIdx.y * segZ, Z1 = min(Z0 + segZ, L.nz);
  const int64_t pl = (int64_t)L.nx * L.ny, plc = (int64_t)Lc.nx * Lc.ny;
  const int64_t off = (int64_t)blockIdx.z * L.N;
  const df* xx = x + off;
  const TB* bb = b + off;
  const df* cx = xc + (int64_t)blockIdx.z * Lc.N;
  const int u_beg = Z0 - 2, u_end = Z1 + 1;  // u_beg is even (segZ is even)
  const int Kb = (u_beg >> 1) - 1;  // first coarse plane the block reads
#define CSLOT(K) (((K) - Kb) % 3)

  constexpr int kPI = kFX * kFY / kThr;  // tile cells per thread in step 3
  static_assert(kPI * kThr == kFX * kFY, "whole tile rounds");
  int d2[kP2], d1[kP1], i2[kP1], dI[kPI], iI1[kPI], iI2[kPI];
#pragma unroll
  for (int q = 0; q < kP2; ++q) {
    const int e = tid + q * kThr;
    d2[q] = e < kA2 ? xy_desc(L, F0x - 2 + e % kW2, F0y - 2 + e / kW2) : -1;
  }
#pragma unroll
  for (int q = 0; q < kP1; ++q) {
    const int e = tid + q * kThr;
    const int lx = e % kW1, ly = e / kW1;
    d1[q] = e < kA1 ? xy_desc(L, F0x - 1 + lx, F0y - 1 + ly) : -1;
    i2[q] = (ly + 1) * kW2 + lx + 1;
  }
#pragma unroll
  for (int q = 0; q < kPI; ++q) {
    const int e = tid + q * kThr;
    const int lx = e % kFX, ly = e / kFX;
    dI[q] = xy_desc(L, F0x + lx, F0y + ly);
    iI1[q] = (ly + 1) * kW1 + lx + 1;
    iI2[q] = (ly + 2) * kW2 + lx + 2;
  }

  // coarse plane K interpolated to the fine xy cells of tile + 2, x first, then y (the
  // operand order of the one-kernel prolongation). The 1D weights are 3/4 on the parent
  // coarse cell and 1/4 on the next one towards the fine cell; clamping that neighbour
  // to the grid gives the boundary rule (all weight on the parent) without a branch.
  // Entries for fine cells outside the domain are computed from clamped indices too and
  // never used: step 1 zeroes them. The source offsets are the same on every plane.
  constexpr int kRXp = (kAX + kThr - 1) / kThr;
  int ix0[kRXp], ix1[kRXp], iy0[kP2], iy1[kP2];
#pragma unroll
  for (int r = 0; r < kRXp; ++r) {
    const int e = tid + r * kThr;
    const int jl = e / kW2, fl = e - jl * kW2;
    const int gJ = min(max(C0y - 2 + jl, 0), Lc.ny - 1), gx = F0x - 2 + fl;
    const int I0 = gx >> 1, I1 = (gx & 1) ? I0 + 1 : I0 - 1;
    ix0[r] = gJ * Lc.nx + min(max(I0, 0), Lc.nx - 1);
    ix1[r] = gJ * Lc.nx + min(max(I1, 0), Lc.nx - 1);
  }
#pragma unroll
  for (int q = 0; q < kP2; ++q) {
    const int e = tid + q * kThr;
    const int ey = e / kW2, lx = e - ey * kW2;
    const int gy = F0y - 2 + ey;
    const int J0 = gy >> 1, J1 = (gy & 1) ? J0 + 1 : J0 - 1;
    iy0[q] = (min(max(J0, 0), Lc.ny - 1) - (C0y - 2)) * kW2 + lx;
    iy1[q] = (min(max(J1, 0), Lc.ny - 1) - (C0y - 2)) * kW2 + lx;
  }
  // the coarse values of the next plane to interpolate are loaded a plane ahead into
  // registers (ca, cb), so that their L2 latency hides behind a plane of smoothing
  df ca[kRXp], cb[kRXp];
  bool ck = false;  // the loaded plane is inside the coarse grid
  auto interp_x_load = [&](int K) {
    ck = (K >= 0 && K < Lc.nz);
    const df* plane_c = cx + (ck ? K : 0) * plc;
#pragma unroll
    for (int r = 0; r < kRXp; ++r) {
      const int e = tid + r * kThr;
      const bool in = ck && ((r + 1) * kThr <= kAX || e < kAX);
      ca[r] = in ? plane_c[ix0[r]] : dzero();
      cb[r] = in ? plane_c[ix1[r]] : dzero();
    }
  };
  auto interp_x_store = [&]() {
#pragma unroll
    for (int r = 0; r < kRXp; ++r) {
      const int e = tid + r * kThr;
      if ((r + 1) * kThr <= kAX || e < kAX) {
        df v = dzero();
        if (ck) {
          dsum s;
          s.add(df_mul_f(ca[r], 0.75f));
          s.add(df_make(cb[r].hi * 0.25f, cb[r].lo * 0.25f));
          v = s.get();
        }
        Px[e] = v;
      }
    }
  };
  auto interp_x = [&](int K) {
    interp_x_load(K);
    interp_x_store();
  };
  auto interp_y = [&](int K) {
    df* dst = Pp + CSLOT(K) * kA2;
#pragma unroll
    for (int q = 0; q < kP2; ++q) {
      const int e = tid + q * kThr;
      if ((q + 1) * kThr <= kA2 || e < kA2) {
        const df a = Px[iy0[q]], b1 = Px[iy1[q]];
        dsum s;
        s.add(df_mul_f(a, 0.75f));
        s.add(df_make(b1.hi * 0.25f, b1.lo * 0.25f));
        dst[e] = s.get();
      }
    }
  };
  for (int K = Kb; K < Kb + 3; ++K) {
    interp_x(K);
    __syncthreads();
    interp_y(K);
    __syncthreads();
  }

  // x of the plane step 1 reads next and b of the plane step 2 reads next, loaded one
  // iteration ahead into registers
  df px[kP2], pb[kP1];
  auto fetch_x = [&](int u) {
    const bool in = (u >= 0 && u < L.nz);
#pragma unroll
    for (int q = 0; q < kP2; ++q) px[q] = (in && d2[q] >= 0) ? xx[u * pl + desc_off(d2[q])] : dzero();
  };
  auto fetch_b = [&](int v) {
    const bool in = (v >= 0 && v < L.nz);
#pragma unroll
    for (int q = 0; q < kP1; ++q) pb[q] = (in && d1[q] >= 0) ? load_df(bb, v * pl + desc_off(d1[q])) : dzero();
  };
  fetch_x(u_beg);
  fetch_b(u_beg + 1);  // the first plane step 2 works on

  // one plane of the march: u = u_beg + t with t = 4 j + k; the x' and d0 slot of plane
  // u - i is (k - i) mod 4, the r0 slot (k - i) mod 2
  auto plane = [&](auto kc, int t) {
    constexpr int k = decltype(kc)::value;
    constexpr int x0 = k, x1 = (k + 3) & 3, x2 = (k + 2) & 3, x3 = (k + 1) & 3;  // u, u-1, u-2, u-3
    const int u = u_beg + t;
    // step 1, plane u: x' = x + P xc over tile + 2
    {
      const bool uin = (u >= 0 && u < L.nz);
      int fz[2] = {Kb, Kb};
      float wz[2] = {0.f, 0.f};
      const int nz_ = uin ? fv_prolong_1d(u, Lc.nz, 1, fz, wz) : 0;
      const df* P0 = Pp + CSLOT(fz[0]) * kA2;
      const df* P1 = Pp + CSLOT(fz[nz_ > 1 ? 1 : 0]) * kA2;
#pragma unroll
      for (int q = 0; q < kP2; ++q) {
        const int e = tid + q * kThr;
        if ((q + 1) * kThr <= kA2 || e < kA2) {
          df v = dzero();
          if (uin && d2[q] >= 0) {
            dsum s;
            s.add(px[q]);
            s.add(scale_w(P0[e], wz[0]));
            if (nz_ > 1) s.add(scale_w(P1[e], wz[1]));
            v = s.get();
          }
          sm[oX + x0 * kA2 + e] = v;
        }
      }
      if (u < u_end) fetch_x(u + 1);
      // at u = 2K - 1 the planes K - 1 and K are in use; interpolate K + 1 for u = 2K + 1
      // (its coarse values were loaded at plane u - 1)
      if ((k & 1) && u < u_end) {
        interp_x_store();
        __syncthreads();
        interp_y(((u + 1) >> 1) + 1);
      }
      if (!(k & 1) && u + 1 < u_end) interp_x_load(((u + 2) >> 1) + 1);
    }
    __syncthreads();
    // step 2, plane v = u - 1: r0 = b + N_T(x') - d_c x', d0 = del_c r0 over tile + 1
    if (t >= 2) {
      const int v = u - 1;
      const df* X0 = sm + oX + x2 * kA2;
      const df* X1 = sm + oX + x1 * kA2;
      const df* X2 = sm + oX + x0 * kA2;
      const bool vin = (v >= 0 && v < L.nz);
      const int cz = 9 * ((v > 0) + (v < L.nz - 1));
#pragma unroll
      for (int q = 0; q < kP1; ++q) {
        const int e = tid + q * kThr;
        if ((q + 1) * kThr <= kA1 || e < kA1) {
          df rv = dzero(), dv = dzero();
          if (vin && d1[q] >= 0) {
            const int c = desc_cls(d1[q]) + cz;
            const df n = nsum<ISO>(X0, X1, X2, i2[q], kW2, T0, T1, T2);
            dsum s;
            s.add(pb[q]);
            s.add(n);
            s.add(df_neg(df_mul(td[c], X1[i2[q]])));
            rv = s.get();
            dv = df_mul(tdel[c], rv);
          }
          sm[oR + ((k + 1) & 1) * kA1 + e] = rv;
          sm[oD + x1 * kA1 + e] = dv;
        }
      }
      if (v < Z1) fetch_b(v + 1);
      __syncthreads();
    }
    // step 3, plane w = u - 2 (in [Z0, Z1)): y = x' + eta_c r0 + kap_c N_T(d0) on the tile
    if (t >= 4) {
      const int w = u - 2;
      const df* D0 = sm + oD + x3 * kA1;
      const df* D1 = sm + oD + x2 * kA1;
      const df* D2 = sm + oD + x1 * kA1;
      const df* R1 = sm + oR + (k & 1) * kA1;
      const df* X1 = sm + oX + x2 * kA2;
      const int cz = 9 * ((w > 0) + (w < L.nz - 1));
#pragma unroll
      for (int q = 0; q < kPI; ++q) {
        if (dI[q] >= 0) {
          const int c = desc_cls(dI[q]) + cz;
          const df n = ISO ? nsum6(D0, D1, D2, iI1[q], kW1) : nsum<false>(D0, D1, D2, iI1[q], kW1, T0, T1, T2);
          dsum s;
          s.add(X1[iI2[q]]);
          s.add(df_mul(teta[c], R1[iI1[q]]));
          s.add(df_mul(tkap[c], n));
          const df xv = s.get();
          const int64_t o = off + w * pl + desc_off(dI[q]);
          if (y) y[o] = xv;
          if (y64) y64[o] = df_to_double(xv);
        }
      }
    }
  };
  const int T = u_end - u_beg;
  for (int t = 0; t <= T; t += 4) {
    plane(std::integral_constant<int, 0>{}, t);
    if (t + 1 > T) break;
    plane(std::integral_constant<int, 1>{}, t + 1);
    if (t + 2 > T) break;
    plane(std::integral_constant<int, 2>{}, t + 2);
    if (t + 3 > T) break;
    plane(std::integral_constant<int, 3>{}, t + 3);
  }
#undef CSLOT
}

// z segments: enough blocks for about four waves of resident blocks, with at least
// minp planes per segment (small levels are latency-bound: there, more and shorter
// segments help even though each repeats its halo planes)
int fused_segments(int tiles, int nrhs, int planes, int minp) {
  const int64_t base = (int64_t)tiles * nrhs;
  const int64_t want = 152 * H1W_FUSED_BLOCKS_PER_SM * 4;
  int nseg = (int)std::max<int64_t>(1, (want + base - 1) / base);
  nseg = std::min(nseg, std::max(1, planes / minp));
  return nseg;
}

// dynamic shared memory above 48 KB is opted into once per device and kernel
template <typename K>
bool allow_smem(K kernel, size_t bytes, std::atomic<unsigned long long>& done) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return false;
  const unsigned long long bit = 1ull << dev;
  if (done.load() & bit) return true;
  if (cudaFuncSetAttribute(reinterpret_cast<const void*>(kernel), cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)bytes) != cudaSuccess)
    return false;
  done.fetch_or(bit);
  return true;
}

}  // namespace


namespace {

template <typename TB>
bool pre_fused(const Level& L, const Level& Lc, const FusedCoef& F, int nrhs, const TB* b, df* x, df* bc,
               cudaStream_t s, std::atomic<unsigned long long>* attr) {
  if (!fused_level_ok(L)) return false;
  const bool iso = L.iso != 0;
  if (!(iso ? allow_smem(k_pre_fused<true, TB>, kPreSmem, attr[0])
            : allow_smem(k_pre_fused<false, TB>, kPreSmem, attr[1])))
    return false;
  const int ntx = (Lc.nx + kTX - 1) / kTX, nty = (Lc.ny + kTY - 1) / kTY;
  const int nseg = fused_segments(ntx * nty, nrhs, Lc.nz, Lc.nz >= 64 ? 4 : 1);
  const int segK = (Lc.nz + nseg - 1) / nseg;
  const int nsegs = (Lc.nz + segK - 1) / segK;
  const dim3 grid((unsigned)(ntx * nty), (unsigned)nsegs, (unsigned)nrhs);
  if (iso) k_pre_fused<true, TB><<<grid, kThr, kPreSmem, s>>>(L, Lc, F, b, x, bc, segK);
  else k_pre_fused<false, TB><<<grid, kThr, kPreSmem, s>>>(L, Lc, F, b, x, bc, segK);
  note_launches(1);
  return true;
}

template <typename TB>
bool post_fused(const Level& L, const Level& Lc, const FusedCoef& F, int nrhs, const df* x, const df* xc,
                const TB* b, df* y, double* y64, cudaStream_t s, std::atomic<unsigned long long>* attr) {
  if (!fused_level_ok(L)) return false;
  const bool iso = L.iso != 0;
  if (!(iso ? allow_smem(k_post_fused<true, TB>, kPostSmem, attr[0])
            : allow_smem(k_post_fused<false, TB>, kPostSmem, attr[1])))
    return false;
  const int ntx = (Lc.nx + kTX - 1) / kTX, nty = (Lc.ny + kTY - 1) / kTY;
  const int nseg = fused_segments(ntx * nty, nrhs, L.nz, L.nz >= 128 ? 8 : 2);
  int segZ = (L.nz + nseg - 1) / nseg;
  segZ += segZ & 1;
  const int nsegs = (L.nz + segZ - 1) / segZ;
  const dim3 grid((unsigned)(ntx * nty), (unsigned)nsegs, (unsigned)nrhs);
  if (iso) k_post_fused<true, TB><<<grid, kThr, kPostSmem, s>>>(L, Lc, F, x, xc, b, y, y64, segZ);
  else k_post_fused<false, TB><<<grid, kThr, kPostSmem, s>>>(L, Lc, F, x, xc, b, y, y64, segZ);
  note_launches(1);
  return true;
}

std::atomic<unsigned long long> g_attr_pre[2][2], g_attr_post[2][2];  // [input FP64][iso]

}  // namespace

bool fused_level_ok(const Level& L) {
  return L.cx && L.cy && L.cz && (int64_t)L.nx * L.ny < (int64_t(1) << 26);
}

bool launch_pre_fused_df(const Level& L, const Level& Lc, const FusedCoef& F, int nrhs, const df* b, df* x,
                         df* bc, cudaStream_t s) {
  return pre_fused(L, Lc, F, nrhs, b, x, bc, s, g_attr_pre[0]);
}
bool launch_pre_fused_df(const Level& L, const Level& Lc, const FusedCoef& F, int nrhs, const double* b, df* x,
                         df* bc, cudaStream_t s) {
  return pre_fused(L, Lc, F, nrhs, b, x, bc, s, g_attr_pre[1]);
}
bool launch_post_fused_df(const Level& L, const Level& Lc, const FusedCoef& F, int nrhs, const df* x,
                          const df* xc, const df* b, df* y, double* y64, cudaStream_t s) {
  return post_fused(L, Lc, F, nrhs, x, xc, b, y, y64, s, g_attr_post[0]);
}
bool launch_post_fused_df(const Level& L, const Level& Lc, const FusedCoef& F, int nrhs, const df* x,
                          const df* xc, const double* b, df* y, double* y64, cudaStream_t s) {
  return post_fused(L, Lc, F, nrhs, x, xc, b, y, y64, s, g_attr_post[1]);
}

}  // namespace h1w
