// Dense and Krylov kernels: the skinny passes over J and H (m x N row-major),
// the capacitance GEMM C = I + alpha^-1 J H^T (line C of Algorithm "MINRES
// with the Laplace-Woodbury preconditioner"), the FP64 Cholesky factorization
// (line chol) and triangular solves, the dense coarsest-level solve and the
// PCG vector/scalar updates. Every reduction is deterministic: per-block
// partial sums followed by a fixed-order second stage.
#include <cmath>

#include "h1w_internal.cuh"

namespace h1w {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Deterministic block sum for blockDim.x == kThreads; result valid in thread 0.
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double sh[kThreads / 32];
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double t = 0.0;
  if (wid == 0) {
    t = (lane < kThreads / 32) ? sh[lane] : 0.0;
    t = warp_sum(t);
  }
  return t;
}

// ---- skinny passes ------------------------------------------------------------

constexpr int kRowsChunk = 4096;            // elements of N per block
constexpr int kRowsPerBlock = 8;            // rows of A per block
constexpr int kPerThread = kRowsChunk / kThreads;

// partial[c * m + i] = sum_{k in chunk c} A[i * N + k] * v[k]
__global__ void __launch_bounds__(kThreads) k_rows_dot(const double* __restrict__ A, int m,
                                                       int64_t N, const double* __restrict__ v,
                                                       double* __restrict__ partial) {
  const int64_t k0 = (int64_t)blockIdx.x * kRowsChunk;
  const int r0 = blockIdx.y * kRowsPerBlock;
  double vv[kPerThread];
#pragma unroll
  for (int e = 0; e < kPerThread; ++e) {
    const int64_t k = k0 + threadIdx.x + (int64_t)e * kThreads;
    vv[e] = (k < N) ? v[k] : 0.0;
  }
  __shared__ double sh[kRowsPerBlock][kThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int rr = 0; rr < kRowsPerBlock; ++rr) {
    const int row = r0 + rr;
    double acc = 0.0;
    if (row < m) {
      const double* a = A + (int64_t)row * N;
#pragma unroll
      for (int e = 0; e < kPerThread; ++e) {
        const int64_t k = k0 + threadIdx.x + (int64_t)e * kThreads;
        if (k < N) acc += a[k] * vv[e];
      }
    }
    acc = warp_sum(acc);
    if (lane == 0) sh[rr][wid] = acc;
  }
  __syncthreads();
  if (threadIdx.x < kRowsPerBlock) {
    const int row = r0 + threadIdx.x;
    if (row < m) {
      double t = 0.0;
#pragma unroll
      for (int w = 0; w < kThreads / 32; ++w) t += sh[threadIdx.x][w];
      partial[(int64_t)blockIdx.x * m + row] = t;
    }
  }
}

__global__ void k_reduce_partials(const double* __restrict__ partial, int nchunks, int m,
                                  double scale, double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  double t = 0.0;
  for (int c = 0; c < nchunks; ++c) t += partial[(int64_t)c * m + i];
  out[i] = scale * t;
}

// z_k = (z0_k - (1/alpha) sum_i H[i][k] v_i) / alpha ; partial[block] = sum_k r_k z_k
__global__ void __launch_bounds__(kThreads) k_woodbury_update(
    const double* __restrict__ H, int m, int64_t N, const double* __restrict__ v,
    const double* __restrict__ z0, double alpha, double* __restrict__ z,
    const double* __restrict__ r, double* __restrict__ partial) {
  extern __shared__ double sv[];
  for (int i = threadIdx.x; i < m; i += blockDim.x) sv[i] = v[i];
  __syncthreads();
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double prod = 0.0;
  if (k < N) {
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    const double* col = H + k;
    int i = 0;
    for (; i + 4 <= m; i += 4) {
      a0 += col[(int64_t)(i + 0) * N] * sv[i + 0];
      a1 += col[(int64_t)(i + 1) * N] * sv[i + 1];
      a2 += col[(int64_t)(i + 2) * N] * sv[i + 2];
      a3 += col[(int64_t)(i + 3) * N] * sv[i + 3];
    }
    for (; i < m; ++i) a0 += col[(int64_t)i * N] * sv[i];
    const double hv = (a0 + a1) + (a2 + a3);
    const double zk = (z0[k] - hv / alpha) / alpha;
    z[k] = zk;
    if (r) prod = r[k] * zk;
  }
  if (partial) {
    const double s = block_sum(prod);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
  }
}

// ---- the same two Woodbury passes over H stored as double-floats -----------------
// (the preconditioner's passes; FP32-pipe arithmetic, so they stream at HBM rate)

__device__ __forceinline__ df warp_sum_df(df v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    df t;
    t.hi = __shfl_down_sync(0xffffffffu, v.hi, o);
    t.lo = __shfl_down_sync(0xffffffffu, v.lo, o);
    v = df_add(v, t);
  }
  return v;
}

// partial[c * m + i] = sum_{k in segment c} A[i * N + k] * v[k], A and v
// double-floats. A warp covers a segment of kSegDf entries of one row or of a few
// consecutive rows: lanes stride along the rows (coalesced), each lane accumulates its
// exact products in cascaded sums, and the warp reduces once at the end. Grid: (row
// groups, segments), row groups fastest, so that blocks running together read the same
// segment of neighbouring rows (and of v); the other order was 4 % slower.
constexpr int kSegDf = 8192;


// one cascaded-sum step: (s, e) += p
__device__ __forceinline__ void csum_add(float& s, float& e, df p) {
  const df t = two_sum(s, p.hi);
  s = t.hi;
  e = __fadd_rn(e, __fadd_rn(t.lo, p.lo));
}

// VEC (N even, so that every row starts on a 16-byte boundary): a warp takes kDotRows
// consecutive rows; each lane loads two consecutive entries of v with one 16-byte load and
// uses them for all its rows (v is read once per kDotRows rows), and keeps one cascaded sum
// per row and entry of the pair. Otherwise one row per warp with 8-byte loads.
constexpr int kDotRows = 4;
template <bool VEC>
__global__ void __launch_bounds__(kThreads) k_rows_dot_df(const df* __restrict__ A, int m, int64_t N,
                                                          const df* __restrict__ v, double* __restrict__ partial) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t k0 = (int64_t)blockIdx.y * kSegDf;
  const int64_t kend = (k0 + kSegDf < N) ? k0 + kSegDf : N;
  if (VEC) {
    const int row0 = (blockIdx.x * (kThreads / 32) + wid) * kDotRows;
    if (row0 >= m) return;
    const float4* v4 = reinterpret_cast<const float4*>(v);
    const float4* a4[kDotRows];
#pragma unroll
    for (int r = 0; r < kDotRows; ++r)
      a4[r] = reinterpret_cast<const float4*>(A + (int64_t)min(row0 + r, m - 1) * N);
    float s[kDotRows][2], e[kDotRows][2];
#pragma unroll
    for (int r = 0; r < kDotRows; ++r) s[r][0] = s[r][1] = e[r][0] = e[r][1] = 0.f;
#pragma unroll 2
    for (int64_t j = k0 / 2 + lane; j < kend / 2; j += 32) {
      const float4 y = v4[j];
      const df y0 = df_make(y.x, y.y), y1 = df_make(y.z, y.w);
#pragma unroll
      for (int r = 0; r < kDotRows; ++r) {
        const float4 x = a4[r][j];
        csum_add(s[r][0], e[r][0], df_mul(df_make(x.x, x.y), y0));
        csum_add(s[r][1], e[r][1], df_mul(df_make(x.z, x.w), y1));
      }
    }
#pragma unroll
    for (int r = 0; r < kDotRows; ++r) {
      float s0 = s[r][0], e0 = e[r][0];
      csum_add(s0, e0, fast_two_sum(s[r][1], e[r][1]));
      const df acc = warp_sum_df(fast_two_sum(s0, e0));
      if (lane == 0 && row0 + r < m) partial[(int64_t)blockIdx.y * m + row0 + r] = df_to_double(acc);
    }
  } else {
    const int row = blockIdx.x * (kThreads / 32) + wid;
    if (row >= m) return;
    const df* a = A + (int64_t)row * N;
    float s = 0.f, e = 0.f;
#pragma unroll 8
    for (int64_t k = k0 + lane; k < kend; k += 32) csum_add(s, e, df_mul(a[k], v[k]));
    const df acc = warp_sum_df(fast_two_sum(s, e));
    if (lane == 0) partial[(int64_t)blockIdx.y * m + row] = df_to_double(acc);
  }
}

// z_k = (z0_k - (1/alpha) sum_i H[i][k] v_i) / alpha with H double-floats; partial[block] = sum r_k z_k.
// VEC (N even): each thread takes the two columns 2t, 2t + 1 with one 16-byte load per row
// and two independent cascaded sums.
template <bool VEC>
__global__ void __launch_bounds__(kThreads) k_woodbury_update_df(
    const df* __restrict__ H, int m, int64_t N, const double* __restrict__ v, const double* __restrict__ z0,
    double inv_alpha, double* __restrict__ z, const double* __restrict__ r, double* __restrict__ partial) {
  extern __shared__ df svd[];
  for (int i = threadIdx.x; i < m; i += blockDim.x) svd[i] = df_from_double(v[i]);
  __syncthreads();
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double prod = 0.0;
  if (VEC) {
    const int64_t k = 2 * t;
    if (k < N) {
      float s0 = 0.f, e0 = 0.f, s1 = 0.f, e1 = 0.f;
      const float4* col = reinterpret_cast<const float4*>(H + k);
      const int64_t stride = N / 2;
      for (int i = 0; i < m; ++i) {
        const float4 x = col[(int64_t)i * stride];
        const df w = svd[i];
        csum_add(s0, e0, df_mul(df_make(x.x, x.y), w));
        csum_add(s1, e1, df_mul(df_make(x.z, x.w), w));
      }
      const double h0 = df_to_double(fast_two_sum(s0, e0)), h1 = df_to_double(fast_two_sum(s1, e1));
      const double z0k = (z0[k] - h0 * inv_alpha) * inv_alpha, z1k = (z0[k + 1] - h1 * inv_alpha) * inv_alpha;
      z[k] = z0k;
      z[k + 1] = z1k;
      if (r) prod = r[k] * z0k + r[k + 1] * z1k;
    }
  } else {
    const int64_t k = t;
    if (k < N) {
      float s = 0.f, e = 0.f;
      const df* col = H + k;
      for (int i = 0; i < m; ++i) csum_add(s, e, df_mul(col[(int64_t)i * N], svd[i]));
      const double hv = df_to_double(fast_two_sum(s, e));
      const double zk = (z0[k] - hv * inv_alpha) * inv_alpha;
      z[k] = zk;
      if (r) prod = r[k] * zk;
    }
  }
  if (partial) {
    const double bs = block_sum(prod);
    if (threadIdx.x == 0) partial[blockIdx.x] = bs;
  }
}

// ---- Cholesky (lower, in place, row-major n x n), 32-wide panels --------------

constexpr int kNB = 32;
constexpr int kCholThreads = 256;  // the diagonal block's warp keeps a 32-double row in registers
constexpr int kCholRows = kCholThreads / 32;  // panel rows per block of k_chol_panel

// Cholesky of the nb x nb lower triangle in Ld, in place, by warp 0 of the block (lane r
// holds row r in registers; column c's entries reach the other lanes by shuffles, and each
// pivot costs one square root and one reciprocal), then a barrier for the whole block. Ld
// also receives the reciprocals of the diagonal in column kNB.
__device__ void factor_diag_block(double (*Ld)[kNB + 1], int nb, int* status) {
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    double row[kNB];
    double rdiag = 1.0;  // this lane's reciprocal pivot
#pragma unroll
    for (int j = 0; j < kNB; ++j) row[j] = (lane < nb && j <= lane) ? Ld[lane][j] : 0.0;
#pragma unroll
    for (int c = 0; c < kNB; ++c) {
      if (c < nb) {
        double piv = __shfl_sync(0xffffffffu, row[c], c);
        if (!(piv > 0.0)) {
          if (status && lane == 0) atomicOr(status, kStatusNotSpd);
          piv = 1.0;
        }
        const double inv = rsqrt(piv), d = piv * inv;
        if (lane == c) {
          row[c] = d;
          rdiag = inv;
        } else if (lane > c) {
          row[c] *= inv;
        }
        const double lrc = row[c];
#pragma unroll
        for (int j = c + 1; j < kNB; ++j) {
          const double ljc = __shfl_sync(0xffffffffu, lrc, j);
          if (j < nb && lane >= j) row[j] -= lrc * ljc;
        }
      }
    }
    if (lane < nb) {
#pragma unroll
      for (int j = 0; j < kNB; ++j)
        if (j <= lane) Ld[lane][j] = row[j];
      Ld[lane][kNB] = rdiag;
    }
  }
  __syncthreads();
}

// The diagonal block A11 of the panel at kb, factored in shared memory.
__device__ __forceinline__ int load_factor_diag(const double* A, int n, int kb, double (*Ld)[kNB + 1],
                                                int* status) {
  const int nb = min(kNB, n - kb);
  for (int e = threadIdx.x; e < kNB * kNB; e += blockDim.x) {
    const int r = e / kNB, c = e % kNB;
    if (r < nb && c <= r) Ld[r][c] = A[(int64_t)(kb + r) * n + kb + c];
  }
  __syncthreads();
  factor_diag_block(Ld, nb, status);
  return nb;
}

// L21: one block per kCholRows rows below the panel, one warp per row. Each block factors
// A11 again from A (the factorization is a latency chain of one warp, so repeating it in
// every block costs no time) and solves its rows against it. A11 must still be
// unfactored in A while any of these blocks may start (the blocks of a launch need not
// run together), so block 0 parks L11 where no block of this launch reads (its strict
// lower part transposed into the upper triangle of A11, its diagonal in column kb + 32 of
// rows kb .. kb + 31, all above the diagonal of A and zeroed at the end), and the extra
// block of k_chol_update moves it into place. (The last panel has no rows below it and
// is factored by k_chol_diag.)
__global__ void __launch_bounds__(kCholThreads) k_chol_panel(double* A, int n, int kb, int* status) {
  __shared__ double Ld[kNB][kNB + 1];
  const int nb = load_factor_diag(A, n, kb, Ld, blockIdx.x == 0 ? status : nullptr);
  const int tid = threadIdx.x;
  if (blockIdx.x == 0) {
    for (int e = tid; e < kNB * kNB; e += kCholThreads) {
      const int r = e / kNB, c = e % kNB;
      if (r < nb && c < r) A[(int64_t)(kb + c) * n + kb + r] = Ld[r][c];
      if (r < nb && c == r) A[(int64_t)(kb + r) * n + kb + kNB] = Ld[r][r];
    }
  }
  // rows of this block: solve x L11^T = a for each row (one row per warp)
  const int lane = tid & 31;
  {
    const int row = kb + kNB + blockIdx.x * kCholRows + (tid >> 5);
    if (row >= n) return;
    double a = (lane < nb) ? A[(int64_t)row * n + kb + lane] : 0.0;
    for (int c = 0; c < nb; ++c) {
      double xc = 0.0;
      if (lane == c) xc = a * Ld[c][kNB];  // the reciprocal of the pivot
      xc = __shfl_sync(0xffffffffu, xc, c);
      if (lane == c) a = xc;
      else if (lane > c && lane < nb) a -= xc * Ld[lane][c];
    }
    if (lane < nb) A[(int64_t)row * n + kb + lane] = a;
  }
}

// L11 = chol(A11), written back in place; a non-positive pivot sets kStatusNotSpd.
__device__ __forceinline__ void write_diag_factor(double* A, int n, int kb, double (*Ld)[kNB + 1], int* status) {
  const int nb = load_factor_diag(A, n, kb, Ld, status);
  for (int e = threadIdx.x; e < kNB * kNB; e += blockDim.x) {
    const int r = e / kNB, c = e % kNB;
    if (r < nb && c <= r) A[(int64_t)(kb + r) * n + kb + c] = Ld[r][c];
  }
}

__global__ void __launch_bounds__(kCholThreads) k_chol_diag(double* A, int n, int kb, int* status) {
  __shared__ double Ld[kNB][kNB + 1];
  write_diag_factor(A, n, kb, Ld, status);
}

// trailing update A22 -= L21 L21^T over lower tiles (ti >= tj) of 32 x 32; the block after
// the last tile moves L11 from where k_chol_panel parked it into A11 (none of these
// locations is in A22)
__global__ void __launch_bounds__(256) k_chol_update(double* A, int n, int kb) {
  __shared__ double Li[kNB][kNB + 1];
  __shared__ double Lj[kNB][kNB + 1];
  const int t = blockIdx.x;
  if (t == gridDim.x - 1) {
    const int nb = min(kNB, n - kb);
    for (int e = threadIdx.x; e < kNB * kNB; e += blockDim.x) {
      const int r = e / kNB, c = e % kNB;
      if (r < nb && c < r) A[(int64_t)(kb + r) * n + kb + c] = A[(int64_t)(kb + c) * n + kb + r];
      if (r < nb && c == r) A[(int64_t)(kb + r) * n + kb + r] = A[(int64_t)(kb + r) * n + kb + kNB];
    }
    return;
  }
  int ti = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
  while ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
  while (ti * (ti + 1) / 2 > t) --ti;
  const int tj = t - ti * (ti + 1) / 2;
  const int base = kb + kNB;
  const int ri = base + ti * kNB, rj = base + tj * kNB;
  const int nbk = min(kNB, n - kb);
  for (int e = threadIdx.x; e < kNB * kNB; e += blockDim.x) {
    const int r = e / kNB, c = e % kNB;
    Li[r][c] = (ri + r < n && c < nbk) ? A[(int64_t)(ri + r) * n + kb + c] : 0.0;
    Lj[r][c] = (rj + r < n && c < nbk) ? A[(int64_t)(rj + r) * n + kb + c] : 0.0;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < kNB * kNB; e += blockDim.x) {
    const int r = e / kNB, c = e % kNB;
    if (ri + r >= n || rj + c >= n) continue;
    double s = 0.0;
#pragma unroll 8
    for (int l = 0; l < kNB; ++l) s += Li[r][l] * Lj[c][l];
    A[(int64_t)(ri + r) * n + rj + c] -= s;
  }
}

__global__ void k_zero_upper(double* A, int n) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)n * n) return;
  const int r = (int)(e / n), c = (int)(e % n);
  if (c > r) A[e] = 0.0;
}

// ---- triangular solves, one block per right-hand side --------------------------

// x <- L^-1 x (forward substitution), 32-wide blocks; x in shared memory. The
// 32 x 32 diagonal block is staged in shared memory before its sequential
// solve so that the dependent steps do not wait on global loads.
__global__ void __launch_bounds__(512) k_trsv_lower(const double* __restrict__ L, int n,
                                                    double* __restrict__ xg) {
  extern __shared__ double x[];
  __shared__ double D[kNB][kNB + 1];
  double* xr = xg + (int64_t)blockIdx.x * n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] = xr[i];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int kb = 0; kb < n; kb += kNB) {
    const int nb = min(kNB, n - kb);
    for (int e = threadIdx.x; e < kNB * kNB; e += blockDim.x) {
      const int r = e / kNB, c = e % kNB;
      D[r][c] = (r < nb && c <= r) ? L[(int64_t)(kb + r) * n + kb + c] : 0.0;
    }
    __syncthreads();
    if (wid == 0) {
      double a = (lane < nb) ? x[kb + lane] : 0.0;
      const double inv = (lane < nb) ? 1.0 / D[lane][lane] : 0.0;
      for (int c = 0; c < nb; ++c) {
        double yc = (lane == c) ? a * inv : 0.0;
        yc = __shfl_sync(0xffffffffu, yc, c);
        if (lane == c) a = yc;
        else if (lane > c && lane < nb) a -= yc * D[lane][c];
      }
      if (lane < nb) x[kb + lane] = a;
    }
    __syncthreads();
    for (int i = kb + nb + threadIdx.x; i < n; i += blockDim.x) {
      const double* li = L + (int64_t)i * n + kb;
      double s = 0.0;
#pragma unroll 8
      for (int c = 0; c < nb; ++c) s += li[c] * x[kb + c];
      x[i] -= s;
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) xr[i] = x[i];
}

// x <- L^-T x (backward substitution with the transpose of the lower factor)
__global__ void __launch_bounds__(512) k_trsv_upper_t(const double* __restrict__ L, int n,
                                                      double* __restrict__ xg) {
  extern __shared__ double x[];
  __shared__ double D[kNB][kNB + 1];
  double* xr = xg + (int64_t)blockIdx.x * n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] = xr[i];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nblk = (n + kNB - 1) / kNB;
  for (int bi = nblk - 1; bi >= 0; --bi) {
    const int kb = bi * kNB;
    const int nb = min(kNB, n - kb);
    for (int e = threadIdx.x; e < kNB * kNB; e += blockDim.x) {
      const int r = e / kNB, c = e % kNB;
      D[r][c] = (r < nb && c <= r) ? L[(int64_t)(kb + r) * n + kb + c] : 0.0;
    }
    __syncthreads();
    if (wid == 0) {
      double a = (lane < nb) ? x[kb + lane] : 0.0;
      const double inv = (lane < nb) ? 1.0 / D[lane][lane] : 0.0;
      for (int c = nb - 1; c >= 0; --c) {
        double vc = (lane == c) ? a * inv : 0.0;
        vc = __shfl_sync(0xffffffffu, vc, c);
        if (lane == c) a = vc;
        else if (lane < c) a -= vc * D[c][lane];
      }
      if (lane < nb) x[kb + lane] = a;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kb; i += blockDim.x) {
      double s = 0.0;
#pragma unroll 8
      for (int c = 0; c < nb; ++c) s += L[(int64_t)(kb + c) * n + i] * x[kb + c];
      x[i] -= s;
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) xr[i] = x[i];
}

// ---- both triangular solves of C^-1 s in one cooperative launch ----------------
//
// x <- L^-T L^-1 x for one right-hand side. CTA p owns the 32-row block p. Forward:
// y_p = D_p^-1 (x_p - sum_{J<p} L_pJ y_J), where each update L_pJ y_J is applied as soon
// as block J has published y_J (flag_f[J] == epoch); backward likewise with z_p =
// D_p^-T (y_p - sum_{J>p} L_Jp^T z_J) and flag_b. Only the diagonal solves lie on the
// critical path; the updates of different blocks run on different SMs (a single-block
// solve is bound by the FP64 pipe of one SM). All CTAs must be resident: the launch is
// cooperative. Every wait gives up after wait_ns (one second unless a test shortens it), sets
// kStatusTimeout and returns.
// The flags hold the epoch of the last solve, so they never need resetting.

__device__ __forceinline__ uint64_t trsv_timer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait until flag == epoch (bounded). Thread 0 polls and decides for the whole block, so
// that every thread of the block returns the same answer; false on timeout (or when
// another block already gave up).
__device__ bool trsv_wait(const int* flag, int epoch, int* status, int* s_ok, uint64_t wait_ns) {
  if (threadIdx.x == 0) {
    const uint64_t t0 = trsv_timer();
    unsigned n = 0;
    int ok = 1;
    while (atomicAdd(const_cast<int*>(flag), 0) != epoch) {
      // wait_ns, or 2^22 polls should the global timer not advance (a legitimate wait, for
      // the blocks before this one, lasts well under a millisecond)
      if ((++n & 63) == 0 && (trsv_timer() - t0 > wait_ns || n >= (1u << 22) ||
                              (atomicAdd(status, 0) & kStatusTimeout))) {
        atomicOr(status, kStatusTimeout);
        ok = 0;
        break;
      }
    }
    __threadfence();
    *s_ok = ok;
  }
  __syncthreads();
  return *s_ok != 0;
}

__global__ void __launch_bounds__(256) k_chol_solve_coop(const double* __restrict__ L, int n, double* x,
                                                        int* flag_f, int* flag_b, int epoch_arg,
                                                        const int* epoch_ptr, int* status,
                                                        unsigned long long wait_ns, int stall) {
  // the epoch comes from the host, or (graph replays) from a device counter that a preceding
  // kernel has advanced
  const int epoch = epoch_ptr ? *epoch_ptr : epoch_arg;
  __shared__ double D[kNB][kNB + 1];
  __shared__ double acc[kNB];
  __shared__ int s_ok;
  const int p = blockIdx.x, nblk = gridDim.x;
  const int kb = p * kNB, nb = min(kNB, n - kb);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int e = threadIdx.x; e < kNB * kNB; e += blockDim.x) {
    const int r = e / kNB, c = e % kNB;
    D[r][c] = (r < nb && c <= r) ? L[(int64_t)(kb + r) * n + kb + c] : 0.0;
  }
  if (threadIdx.x < kNB) acc[threadIdx.x] = (threadIdx.x < nb) ? x[kb + threadIdx.x] : 0.0;
  __syncthreads();
  // forward: thread (row r = 4 wid + lane / 8, t = lane % 8) takes columns t, t + 8, t + 16, t + 24
  {
    const int r = 4 * wid + (lane >> 3), t = lane & 7;
    for (int J = 0; J < p; ++J) {
      if (!trsv_wait(flag_f + J, epoch, status, &s_ok, wait_ns)) return;
      const int jb = J * kNB;
      double sacc = 0.0;
      if (r < nb) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int c = t + 8 * k;
          sacc += L[(int64_t)(kb + r) * n + jb + c] * __ldcg(x + jb + c);
        }
      }
      sacc += __shfl_xor_sync(0xffffffffu, sacc, 1);
      sacc += __shfl_xor_sync(0xffffffffu, sacc, 2);
      sacc += __shfl_xor_sync(0xffffffffu, sacc, 4);
      if (t == 0 && r < nb) acc[r] -= sacc;
      __syncthreads();
    }
  }
  if (wid == 0) {
    double a = (lane < nb) ? acc[lane] : 0.0;
    const double inv = (lane < nb) ? 1.0 / D[lane][lane] : 0.0;
    for (int c = 0; c < nb; ++c) {
      double yc = (lane == c) ? a * inv : 0.0;
      yc = __shfl_sync(0xffffffffu, yc, c);
      if (lane == c) a = yc;
      else if (lane > c && lane < nb) a -= yc * D[lane][c];
    }
    if (lane < nb) {
      acc[lane] = a;
      x[kb + lane] = a;
    }
    __threadfence();  // the published values before the flag, from every writing lane
  }
  __syncthreads();
  if (threadIdx.x == 0 && !(stall && p == 0)) {
    __threadfence();
    atomicExch(flag_f + p, epoch);
  }
  // backward: thread (row r = 4 wid + lane % 4, t = lane / 4); rows of L^T are columns of L
  {
    const int r = 4 * wid + (lane & 3), t = lane >> 2;
    for (int J = nblk - 1; J > p; --J) {
      if (!trsv_wait(flag_b + J, epoch, status, &s_ok, wait_ns)) return;
      const int jb = J * kNB, jn = min(kNB, n - jb);
      double sacc = 0.0;
      if (r < nb) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int c = t + 8 * k;
          if (c < jn) sacc += L[(int64_t)(jb + c) * n + kb + r] * __ldcg(x + jb + c);
        }
      }
      sacc += __shfl_xor_sync(0xffffffffu, sacc, 4);
      sacc += __shfl_xor_sync(0xffffffffu, sacc, 8);
      sacc += __shfl_xor_sync(0xffffffffu, sacc, 16);
      if (t == 0 && r < nb) acc[r] -= sacc;
      __syncthreads();
    }
  }
  if (wid == 0) {
    double a = (lane < nb) ? acc[lane] : 0.0;
    const double inv = (lane < nb) ? 1.0 / D[lane][lane] : 0.0;
    for (int c = nb - 1; c >= 0; --c) {
      double vc = (lane == c) ? a * inv : 0.0;
      vc = __shfl_sync(0xffffffffu, vc, c);
      if (lane == c) a = vc;
      else if (lane < c) a -= vc * D[c][lane];
    }
    if (lane < nb) x[kb + lane] = a;
    __threadfence();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicExch(flag_b + p, epoch);
  }
}

// x[r] = X b[r]: one warp per (row, rhs)
__global__ void k_coarse_apply(const double* __restrict__ X, int n, const double* __restrict__ b,
                               double* __restrict__ x) {
  const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  const double* br = b + (int64_t)blockIdx.y * n;
  const double* xr = X + (int64_t)row * n;
  double s = 0.0;
  for (int j = lane; j < n; j += 32) s += xr[j] * br[j];
  s = warp_sum(s);
  if (lane == 0) x[(int64_t)blockIdx.y * n + row] = s;
}

__global__ void k_set_identity(double* X, int n) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)n * n) return;
  X[e] = ((e / n) == (e % n)) ? 1.0 : 0.0;
}

// X holds the columns of the inverse as rows (row r = A^-1 e_r); make it exactly symmetric.
__global__ void k_symmetrize(double* X, int n) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)n * n) return;
  const int r = (int)(e / n), c = (int)(e % n);
  if (c <= r) return;
  const double v = 0.5 * (X[(int64_t)r * n + c] + X[(int64_t)c * n + r]);
  X[(int64_t)r * n + c] = v;
  X[(int64_t)c * n + r] = v;
}

// ---- capacitance GEMM: partial[s][i][j] = sum_{k in split s} J[i][k] H[j][k], upper tiles --

constexpr int kTM = 64, kTK = 16;

__global__ void __launch_bounds__(256) k_cap_gemm(const double* __restrict__ J,
                                                  const double* __restrict__ H, int m, int64_t N,
                                                  int64_t kchunk, double* __restrict__ partial) {
  __shared__ double As[kTK][kTM + 1];
  __shared__ double Bs[kTK][kTM + 1];
  const int t = blockIdx.x;
  int ti = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
  while ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
  while (ti * (ti + 1) / 2 > t) --ti;
  const int tj0 = t - ti * (ti + 1) / 2;  // tj0 <= ti: tile (row tj0, col ti) is upper
  const int i0 = tj0 * kTM, j0 = ti * kTM;
  const int64_t kbeg = (int64_t)blockIdx.y * kchunk;
  const int64_t kend = min(N, kbeg + kchunk);
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  double acc[4][4] = {};
  for (int64_t k = kbeg; k < kend; k += kTK) {
    for (int e = threadIdx.x; e < kTM * kTK; e += blockDim.x) {
      const int r = e / kTK, c = e % kTK;
      const int64_t kk = k + c;
      As[c][r] = (i0 + r < m && kk < kend) ? J[(int64_t)(i0 + r) * N + kk] : 0.0;
      Bs[c][r] = (j0 + r < m && kk < kend) ? H[(int64_t)(j0 + r) * N + kk] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < kTK; ++c) {
      double a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) { a[u] = As[c][ty * 4 + u]; b[u] = Bs[c][tx * 4 + u]; }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] += a[u] * b[v];
    }
    __syncthreads();
  }
  double* P = partial + (int64_t)blockIdx.y * m * m;
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int i = i0 + ty * 4 + u, j = j0 + tx * 4 + v;
      if (i < m && j < m) P[(int64_t)i * m + j] = acc[u][v];
    }
}

// C[i][j] = delta_ij + (1/alpha) sum_s partial[s][min(i,j)][max(i,j)]
__global__ void k_cap_finalize(const double* __restrict__ partial, int splits, int m, double alpha,
                               double* __restrict__ C) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)m * m) return;
  const int i = (int)(e / m), j = (int)(e % m);
  const int a = min(i, j), b = max(i, j);
  double s = 0.0;
  for (int q = 0; q < splits; ++q) s += partial[(int64_t)q * m * m + (int64_t)a * m + b];
  C[e] = (i == j ? 1.0 : 0.0) + s / alpha;
}

// ---- PCG vectors and scalars -----------------------------------------------------
// scalar slots: 0 rz, 1 pq, 2 a, 3 rz_new, 4 beta, 5 rr, 6 bb

__global__ void k_sum_to_scalar(const double* __restrict__ partial, int n, double* dst) {
  double t = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) t += partial[i];
  t = block_sum(t);
  if (threadIdx.x == 0) *dst = t;
}

__global__ void k_pcg_alpha(double* scal) { scal[2] = scal[0] / scal[1]; }

// Device-driven PCG (the loop of h1w_pcg as a graph with a conditional while node). Slots
// beyond the host-driven ones: 7 first, 8 iterations, 9 tol^2 = rtol^2 b.b, 10 maxit,
// 11 true r.r, 12 init (start from x = 0), 13 rtol. The loop body is one PCG iteration
// rotated so that it ends with the convergence test:
//   z = P r; rz_new = r.z; beta (0 the first time); p = z + beta p; w = J p = J z + beta w;
//   q = A p; a = rz / p.q; x += a p; r -= a q; rr = r.r; continue while rr > tol^2 and it < maxit.
__global__ void k_pcg_set_scalars(double* scal, double rtol, int maxit, int init) {
  scal[13] = rtol;
  scal[10] = (double)maxit;
  scal[12] = init ? 1.0 : 0.0;
}

__global__ void __launch_bounds__(kThreads) k_pcg_init(double* __restrict__ x, double* __restrict__ r,
                                                      const double* __restrict__ b, const double* __restrict__ scal,
                                                      int64_t N) {
  if (scal[12] == 0.0) return;  // a restart keeps x and the true residual in r
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < N) {
    x[k] = 0.0;
    r[k] = b[k];
  }
}

__device__ __forceinline__ unsigned pcg_continue(const double* scal) {
  const double rr = scal[5];
  return (isfinite(rr) && rr > scal[9] && scal[8] < scal[10]) ? 1u : 0u;
}

// after b.b (slot 6) and r.r (slot 5) are formed: the tolerance, the counters, the condition
__global__ void k_pcg_start(double* scal, cudaGraphConditionalHandle h) {
  scal[9] = scal[13] * scal[13] * scal[6];
  if (scal[12] != 0.0) scal[8] = 0.0;
  scal[7] = 1.0;
  cudaGraphSetConditional(h, pcg_continue(scal));
}

__global__ void k_pcg_beta_dev(double* scal) {
  if (scal[7] != 0.0) {
    scal[4] = 0.0;
  } else {
    scal[4] = scal[3] / scal[0];
  }
  scal[0] = scal[3];
}

__global__ void k_p_update_dev(double* __restrict__ p, const double* __restrict__ z, double* __restrict__ w,
                               const double* __restrict__ jz, const double* __restrict__ scal, int64_t N, int m) {
  const bool first = scal[7] != 0.0;
  const double beta = scal[4];
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < N) p[k] = first ? z[k] : z[k] + beta * p[k];
  if (k < m) w[k] = first ? jz[k] : jz[k] + beta * w[k];
}

__global__ void k_pcg_alpha_dev(double* scal) {
  scal[2] = scal[0] / scal[1];
  scal[7] = 0.0;
}

__global__ void k_pcg_check(double* scal, cudaGraphConditionalHandle h) {
  scal[8] += 1.0;
  cudaGraphSetConditional(h, pcg_continue(scal));
}

// r = b - q with partial sums of r.r per block
__global__ void __launch_bounds__(kThreads) k_true_residual(double* __restrict__ r, const double* __restrict__ b,
                                                           const double* __restrict__ q, int64_t N,
                                                           double* __restrict__ partial) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double t = 0.0;
  if (k < N) {
    const double v = b[k] - q[k];
    r[k] = v;
    t = v * v;
  }
  t = block_sum(t);
  if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

__global__ void k_bump(int* counter) { *counter += 1; }

__global__ void k_pcg_beta(double* scal) {
  scal[4] = scal[3] / scal[0];
  scal[0] = scal[3];
}

__global__ void __launch_bounds__(kThreads) k_xr_update(double* __restrict__ x, double* __restrict__ r,
                                                        const double* __restrict__ p,
                                                        const double* __restrict__ q,
                                                        const double* __restrict__ scal, int64_t N,
                                                        double* __restrict__ partial) {
  const double a = scal[2];
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double rr = 0.0;
  if (k < N) {
    x[k] += a * p[k];
    const double rv = r[k] - a * q[k];
    r[k] = rv;
    rr = rv * rv;
  }
  const double s = block_sum(rr);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void k_p_update(double* __restrict__ p, const double* __restrict__ z,
                           double* __restrict__ w, const double* __restrict__ jz,
                           const double* __restrict__ scal, int64_t N, int m, int first) {
  const double beta = first ? 0.0 : scal[4];
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < N) p[k] = first ? z[k] : z[k] + beta * p[k];
  if (k < m) w[k] = first ? jz[k] : jz[k] + beta * w[k];
}

__global__ void k_axpby(double* __restrict__ y, double a, const double* __restrict__ x, double b,
                        int64_t N) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < N) y[k] = a * x[k] + b * y[k];
}

__global__ void __launch_bounds__(kThreads) k_dot_partial(const double* __restrict__ a,
                                                          const double* __restrict__ b, int64_t N,
                                                          double* __restrict__ partial) {
  double s = 0.0;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N;
       k += (int64_t)gridDim.x * blockDim.x)
    s += a[k] * b[k];
  s = block_sum(s);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void k_fill(double* y, double v, int64_t N) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < N) y[k] = v;
}

__global__ void k_copy(double* __restrict__ y, const double* __restrict__ x, int64_t N) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < N) y[k] = x[k];
}

inline unsigned nblk(int64_t n, int t = kThreads) { return (unsigned)((n + t - 1) / t); }

}  // namespace

int rows_dot_chunks(int64_t N) { return (int)((N + kRowsChunk - 1) / kRowsChunk); }

void launch_rows_dot(const double* A, int m, int64_t N, const double* v, double* partial,
                     cudaStream_t s) {
  if (m <= 0) return;
  dim3 g(rows_dot_chunks(N), (m + kRowsPerBlock - 1) / kRowsPerBlock);
  k_rows_dot<<<g, kThreads, 0, s>>>(A, m, N, v, partial);
  note_launches(1);
}

void launch_reduce_partials(const double* partial, int nchunks, int m, double scale, double* out,
                            cudaStream_t s) {
  if (m <= 0) return;
  k_reduce_partials<<<nblk(m, 128), 128, 0, s>>>(partial, nchunks, m, scale, out);
  note_launches(1);
}

int rows_dot_df_chunks(int64_t N) { return (int)((N + kSegDf - 1) / kSegDf); }

void launch_rows_dot_df(const df* A, int m, int64_t N, const df* v, double* partial, cudaStream_t s) {
  if (m <= 0) return;
  const int rows_per_block = (kThreads / 32) * ((N % 2 == 0) ? kDotRows : 1);
  dim3 g((m + rows_per_block - 1) / rows_per_block, rows_dot_df_chunks(N));
  if (N % 2 == 0) k_rows_dot_df<true><<<g, kThreads, 0, s>>>(A, m, N, v, partial);
  else k_rows_dot_df<false><<<g, kThreads, 0, s>>>(A, m, N, v, partial);
  note_launches(1);
}

int launch_woodbury_update_df(const df* H, int m, int64_t N, const double* v, const double* z0, double alpha,
                              double* z, const double* r, double* partial, cudaStream_t s) {
  const size_t smem = sizeof(df) * (size_t)(m > 0 ? m : 1);
  const bool vec = N % 2 == 0;
  const unsigned nb = vec ? nblk(N / 2) : nblk(N);
  if (vec) k_woodbury_update_df<true><<<nb, kThreads, smem, s>>>(H, m, N, v, z0, 1.0 / alpha, z, r, partial);
  else k_woodbury_update_df<false><<<nb, kThreads, smem, s>>>(H, m, N, v, z0, 1.0 / alpha, z, r, partial);
  note_launches(1);
  return (int)nb;
}

int colsum_blocks(int64_t N) { return (int)nblk(N); }

void launch_woodbury_update(const double* H, int m, int64_t N, const double* v, const double* z0,
                            double alpha, double* z, const double* r, double* partial,
                            cudaStream_t s) {
  const size_t smem = sizeof(double) * (size_t)(m > 0 ? m : 1);
  k_woodbury_update<<<nblk(N), kThreads, smem, s>>>(H, m, N, v, z0, alpha, z, r, partial);
  note_launches(1);
}

// A = alpha A + J^T J for the dense direct solve: J (m x n, row-major) in 32-row slices
// staged in shared memory, one 32 x 32 tile of A per block, each thread four entries of it.
__global__ void __launch_bounds__(256) k_dense_gn(double* __restrict__ A, int n, double alpha,
                                                  const double* __restrict__ J, int m) {
  __shared__ double Jp[32][33];
  __shared__ double Jq[32][33];
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  const int p0 = blockIdx.y * 32, q0 = blockIdx.x * 32;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int i0 = 0; i0 < m; i0 += 32) {
    for (int r = ty; r < 32; r += 8) {
      const int i = i0 + r;
      Jp[r][tx] = (i < m && p0 + tx < n) ? J[(int64_t)i * n + p0 + tx] : 0.0;
      Jq[r][tx] = (i < m && q0 + tx < n) ? J[(int64_t)i * n + q0 + tx] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int r = 0; r < 32; ++r) {
      const double a = Jq[r][tx];
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[u] = fma(Jp[r][ty + 8 * u], a, acc[u]);
    }
    __syncthreads();
  }
  const int q = q0 + tx;
  if (q >= n) return;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int p = p0 + ty + 8 * u;
    if (p < n) A[(int64_t)p * n + q] = alpha * A[(int64_t)p * n + q] + acc[u];
  }
}

void launch_dense_gn(double* A, int n, double alpha, const double* J, int m, cudaStream_t s) {
  const dim3 grid((n + 31) / 32, (n + 31) / 32);
  k_dense_gn<<<grid, dim3(32, 8), 0, s>>>(A, n, alpha, J, m);
  note_launches(1);
}

void launch_chol(double* A, int n, int* status, cudaStream_t s) {
  for (int kb = 0; kb < n; kb += kNB) {
    const int below = (n - kb - 1) / kNB;  // 32-row blocks after the diagonal block
    if (below > 0) {
      const int rows = n - kb - kNB;
      k_chol_panel<<<(rows + kCholRows - 1) / kCholRows, kCholThreads, 0, s>>>(A, n, kb, status);
      const int tiles = below * (below + 1) / 2;
      k_chol_update<<<tiles + 1, 256, 0, s>>>(A, n, kb);
      note_launches(2);
    } else {
      k_chol_diag<<<1, kCholThreads, 0, s>>>(A, n, kb, status);
      note_launches(1);
    }
  }
  k_zero_upper<<<nblk((int64_t)n * n), kThreads, 0, s>>>(A, n);
  note_launches(1);
}

void launch_trsv_lower(const double* L, int n, double* x, int nrhs, cudaStream_t s) {
  k_trsv_lower<<<nrhs, 512, sizeof(double) * n, s>>>(L, n, x);
  note_launches(1);
}

void launch_trsv_upper_t(const double* L, int n, double* x, int nrhs, cudaStream_t s) {
  k_trsv_upper_t<<<nrhs, 512, sizeof(double) * n, s>>>(L, n, x);
  note_launches(1);
}

bool launch_chol_solve_coop(const double* L, int n, double* x, int* flags, int epoch, const int* epoch_ptr,
                            int* status, unsigned long long wait_ns, int stall, cudaStream_t s) {
  const int nblk = (n + kNB - 1) / kNB;
  int dev = 0, coop = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (!coop || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_chol_solve_coop, 256, 0) != cudaSuccess ||
      nblk > per_sm * sms)
    return false;
  int* flag_f = flags;
  int* flag_b = flags + nblk;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nblk);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (cudaLaunchKernelEx(&cfg, k_chol_solve_coop, L, n, x, flag_f, flag_b, epoch, epoch_ptr, status, wait_ns, stall) !=
      cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  note_launches(1);
  return true;
}

void launch_coarse_apply(const double* X, int n, int nrhs, const double* b, double* x,
                         cudaStream_t s) {
  dim3 g(nblk(n, 8), nrhs);
  k_coarse_apply<<<g, 256, 0, s>>>(X, n, b, x);
  note_launches(1);
}

void launch_set_identity(double* X, int n, cudaStream_t s) {
  k_set_identity<<<nblk((int64_t)n * n), kThreads, 0, s>>>(X, n);
  note_launches(1);
}

void launch_symmetrize_identity_solve(double* X, int n, cudaStream_t s) {
  k_symmetrize<<<nblk((int64_t)n * n), kThreads, 0, s>>>(X, n);
  note_launches(1);
}

int cap_gemm_splits(int m, int64_t N) {
  const int tiles = (m + kTM - 1) / kTM;
  const int utiles = tiles * (tiles + 1) / 2;
  int splits = (4 * 152 + utiles - 1) / utiles;
  const int64_t max_splits = (N + 255) / 256;  // at least 256 columns per split
  if (splits > max_splits) splits = (int)max_splits;
  return splits < 1 ? 1 : splits;
}

void launch_cap_gemm(const double* J, const double* H, int m, int64_t N, double* partial,
                     int splits, cudaStream_t s) {
  const int tiles = (m + kTM - 1) / kTM;
  const int utiles = tiles * (tiles + 1) / 2;
  int64_t kchunk = (N + splits - 1) / splits;
  kchunk = (kchunk + kTK - 1) / kTK * kTK;
  dim3 g(utiles, splits);
  k_cap_gemm<<<g, 256, 0, s>>>(J, H, m, N, kchunk, partial);
  note_launches(1);
}

void launch_cap_finalize(const double* partial, int splits, int m, double alpha, double* C,
                         cudaStream_t s) {
  k_cap_finalize<<<nblk((int64_t)m * m), kThreads, 0, s>>>(partial, splits, m, alpha, C);
  note_launches(1);
}

void launch_sum_to_scalar(const double* partial, int n, double* dst, cudaStream_t s) {
  k_sum_to_scalar<<<1, kThreads, 0, s>>>(partial, n, dst);
  note_launches(1);
}

void launch_pcg_alpha(double* scal, cudaStream_t s) { k_pcg_alpha<<<1, 1, 0, s>>>(scal); }

// ---- the PCG iteration driven from the device (graph replays, no host round trip) ----

void launch_pcg_set_scalars(double* scal, double rtol, int maxit, int init, cudaStream_t s) {
  k_pcg_set_scalars<<<1, 1, 0, s>>>(scal, rtol, maxit, init);
  note_launches(1);
}
void launch_pcg_init(double* x, double* r, const double* b, const double* scal, int64_t N, cudaStream_t s) {
  k_pcg_init<<<nblk(N), kThreads, 0, s>>>(x, r, b, scal, N);
  note_launches(1);
}
void launch_pcg_start(double* scal, cudaGraphConditionalHandle h, cudaStream_t s) {
  k_pcg_start<<<1, 1, 0, s>>>(scal, h);
  note_launches(1);
}
void launch_pcg_beta_dev(double* scal, cudaStream_t s) {
  k_pcg_beta_dev<<<1, 1, 0, s>>>(scal);
  note_launches(1);
}
void launch_p_update_dev(double* p, const double* z, double* w, const double* jz, const double* scal, int64_t N,
                         int m, cudaStream_t s) {
  const int64_t n = N > m ? N : m;
  k_p_update_dev<<<nblk(n), kThreads, 0, s>>>(p, z, w, jz, scal, N, m);
  note_launches(1);
}
void launch_pcg_alpha_dev(double* scal, cudaStream_t s) {
  k_pcg_alpha_dev<<<1, 1, 0, s>>>(scal);
  note_launches(1);
}
void launch_pcg_check(double* scal, cudaGraphConditionalHandle h, cudaStream_t s) {
  k_pcg_check<<<1, 1, 0, s>>>(scal, h);
  note_launches(1);
}
void launch_true_residual(double* r, const double* b, const double* q, int64_t N, double* partial, cudaStream_t s) {
  k_true_residual<<<nblk(N), kThreads, 0, s>>>(r, b, q, N, partial);
  note_launches(1);
}
void launch_bump(int* counter, cudaStream_t s) {
  k_bump<<<1, 1, 0, s>>>(counter);
  note_launches(1);
}
void launch_pcg_beta(double* scal, cudaStream_t s) { k_pcg_beta<<<1, 1, 0, s>>>(scal); }

void launch_xr_update(double* x, double* r, const double* p, const double* q, const double* scal,
                      int64_t N, double* partial, cudaStream_t s) {
  k_xr_update<<<nblk(N), kThreads, 0, s>>>(x, r, p, q, scal, N, partial);
  note_launches(1);
}

void launch_p_update(double* p, const double* z, double* w, const double* jz, const double* scal,
                     int64_t N, int m, bool first, cudaStream_t s) {
  const int64_t n = N > m ? N : m;
  k_p_update<<<nblk(n), kThreads, 0, s>>>(p, z, w, jz, scal, N, m, first ? 1 : 0);
  note_launches(1);
}

void launch_axpby(double* y, double a, const double* x, double b, int64_t N, cudaStream_t s) {
  k_axpby<<<nblk(N), kThreads, 0, s>>>(y, a, x, b, N);
  note_launches(1);
}

int dot_blocks(int64_t N) {
  const int64_t b = nblk(N);
  return (int)(b < 1024 ? b : 1024);
}

void launch_dot_partial(const double* a, const double* b, int64_t N, double* partial,
                        cudaStream_t s) {
  k_dot_partial<<<dot_blocks(N), kThreads, 0, s>>>(a, b, N, partial);
  note_launches(1);
}

void launch_fill(double* y, double v, int64_t N, cudaStream_t s) {
  k_fill<<<nblk(N), kThreads, 0, s>>>(y, v, N);
  note_launches(1);
}

// A device-to-device copy as a kernel: a cudaMemcpyAsync between device buffers goes to a copy
// engine, where it queues behind host-to-device copies of J issued earlier on another stream.
void launch_copy(double* y, const double* x, int64_t N, cudaStream_t s) {
  if (N <= 0) return;
  k_copy<<<nblk(N), kThreads, 0, s>>>(y, x, N);
  note_launches(1);
}

}  // namespace h1w
