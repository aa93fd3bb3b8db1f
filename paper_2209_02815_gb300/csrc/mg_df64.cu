// The V-cycle on FV grids in double-float arithmetic (FP32 pairs, ~48 bits).
//
// The V-cycle is a preconditioner: it must be a fixed, symmetric-to-rounding
// operator that builds H = L-hat^-1 J^T and is applied again inside PCG, but
// it need not be FP64. On GB300 the FP64 version is bound by the FP64 pipe
// (1/64 of the FP32 rate). Here every level vector is stored as a
// double-float (8 bytes, like FP64) and every operation runs on the FP32
// pipes with error-free transformations (df64.cuh), so the kernels become
// bound by memory traffic instead. The operator is the same one the FP64
// kernels (mg_kernels.cu) and the oracle apply: 7-point FV operator, degree-k
// Chebyshev-Jacobi smoothing, cell-centred trilinear transfer with R = P^T,
// dense coarsest solve (kept in FP64).
#include <cstdint>

#include "df64.cuh"
#include "h1w_internal.cuh"
#include "mg_df64_util.cuh"

namespace h1w {
namespace {

using namespace dfmg;

constexpr int kThreads = 256;

// One thread per cell of one right-hand side: grid (ceil(nx / blockDim.x), ny, nz * nrhs).
struct Cell {
  int i, j, k, rhs;
  int64_t p;
};
__device__ __forceinline__ bool cell_of(const Level& L, Cell& c) {
  c.i = blockIdx.x * blockDim.x + threadIdx.x;
  if (c.i >= L.nx) return false;
  c.j = blockIdx.y;
  c.k = (int)(blockIdx.z % (unsigned)L.nz);
  c.rhs = (int)(blockIdx.z / (unsigned)L.nz);
  c.p = ((int64_t)c.k * L.ny + c.j) * L.nx + c.i;
  return true;
}

// (A u)_p for the FV operator, class c = fv_cls(i, j, k)
__device__ __forceinline__ df fv_apply_df(const Level& L, const df* __restrict__ u, int i, int j, int k,
                                          int64_t p, int c) {
  const int64_t sy = L.nx, sz = (int64_t)L.nx * L.ny;
  if (L.iso) {
    dsum s;
    if (i > 0) s.add(u[p - 1]);
    if (i < L.nx - 1) s.add(u[p + 1]);
    if (j > 0) s.add(u[p - sy]);
    if (j < L.ny - 1) s.add(u[p + sy]);
    if (k > 0) s.add(u[p - sz]);
    if (k < L.nz - 1) s.add(u[p + sz]);
    return df_sub(df_mul(L.fvd_diag[c], u[p]), df_mul(L.fvd_T[0], s.get()));
  }
  dsum sx, syy, szz;
  if (i > 0) sx.add(u[p - 1]);
  if (i < L.nx - 1) sx.add(u[p + 1]);
  if (j > 0) syy.add(u[p - sy]);
  if (j < L.ny - 1) syy.add(u[p + sy]);
  if (k > 0) szz.add(u[p - sz]);
  if (k < L.nz - 1) szz.add(u[p + sz]);
  df a = df_mul(L.fvd_diag[c], u[p]);
  a = df_sub(a, df_mul(L.fvd_T[0], sx.get()));
  a = df_sub(a, df_mul(L.fvd_T[1], syy.get()));
  return df_sub(a, df_mul(L.fvd_T[2], szz.get()));
}

__global__ void k_cheb_first_df(Level L, const df* __restrict__ b, df* __restrict__ x, df* __restrict__ r,
                                df* __restrict__ d, int zero_x, df inv_theta) {
  Cell q;
  if (!cell_of(L, q)) return;
  const int64_t off = (int64_t)q.rhs * L.N, p = q.p;
  const int c = fv_cls(L, q.i, q.j, q.k);
  df rv = b[off + p];
  if (!zero_x) rv = df_sub(rv, fv_apply_df(L, x + off, q.i, q.j, q.k, p, c));
  const df dv = df_mul(df_mul(rv, L.fvd_dinv[c]), inv_theta);
  r[off + p] = rv;
  d[off + p] = dv;
  if (zero_x) x[off + p] = dv;  // otherwise x is read by neighbours; the next step adds d
}

__global__ void k_cheb_step_df(Level L, df* __restrict__ r, const df* __restrict__ d_old, df* __restrict__ d_new,
                               df* __restrict__ x, df c1, df c2, int add_old) {
  Cell q;
  if (!cell_of(L, q)) return;
  const int64_t off = (int64_t)q.rhs * L.N, p = q.p;
  const int c = fv_cls(L, q.i, q.j, q.k);
  const df dold = d_old[off + p];
  const df rv = df_sub(r[off + p], fv_apply_df(L, d_old + off, q.i, q.j, q.k, p, c));
  const df dv = df_add(df_mul(c1, dold), df_mul(c2, df_mul(rv, L.fvd_dinv[c])));
  r[off + p] = rv;
  d_new[off + p] = dv;
  x[off + p] = df_add(x[off + p], add_old ? df_add(dold, dv) : dv);
}

__global__ void k_add_df(int64_t n, const df* __restrict__ d, df* __restrict__ x) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p < n) x[p] = df_add(x[p], d[p]);
}

__global__ void k_residual_df(Level L, const df* __restrict__ b, const df* __restrict__ x, df* __restrict__ r) {
  Cell q;
  if (!cell_of(L, q)) return;
  const int64_t off = (int64_t)q.rhs * L.N, p = q.p;
  r[off + p] = df_sub(b[off + p], fv_apply_df(L, x + off, q.i, q.j, q.k, p, fv_cls(L, q.i, q.j, q.k)));
}

__global__ void k_restrict_df(Level Lf, Level Lc, const df* __restrict__ rf, df* __restrict__ bc) {
  Cell q;
  if (!cell_of(Lc, q)) return;
  const df* r = rf + (int64_t)q.rhs * Lf.N;
  float wx[4], wy[4], wz[4];
  fv_rw(q.i, Lc.nx, Lf.cx, wx);
  fv_rw(q.j, Lc.ny, Lf.cy, wy);
  fv_rw(q.k, Lc.nz, Lf.cz, wz);
  // fine index of tap t along an axis: coarsened -> 2I - 1 + t, else I (only t = 1 has weight)
  const int bx = Lf.cx ? 2 * q.i - 1 : q.i - 1, by = Lf.cy ? 2 * q.j - 1 : q.j - 1, bz = Lf.cz ? 2 * q.k - 1 : q.k - 1;
  dsum acc;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    if (wz[c] == 0.f) continue;
    dsum sz;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      if (wy[b] == 0.f) continue;
      const df* row = r + ((int64_t)(bz + c) * Lf.ny + (by + b)) * Lf.nx;
      dsum sx;
#pragma unroll
      for (int a = 0; a < 4; ++a)
        if (wx[a] != 0.f) sx.add(df_mul_f(row[bx + a], wx[a]));
      sz.add(df_mul_f(sx.get(), wy[b]));
    }
    acc.add(df_mul_f(sz.get(), wz[c]));
  }
  bc[(int64_t)q.rhs * Lc.N + q.p] = acc.get();
}

__global__ void k_prolong_add_df(Level Lf, Level Lc, const df* __restrict__ xc, df* __restrict__ xf) {
  Cell q;
  if (!cell_of(Lf, q)) return;
  const df* c = xc + (int64_t)q.rhs * Lc.N;
  int fx[2], fy[2], fz[2];
  float wx[2], wy[2], wz[2];
  const int nx_ = fv_prolong_1d(q.i, Lc.nx, Lf.cx, fx, wx);
  const int ny_ = fv_prolong_1d(q.j, Lc.ny, Lf.cy, fy, wy);
  const int nz_ = fv_prolong_1d(q.k, Lc.nz, Lf.cz, fz, wz);
  dsum acc;
#pragma unroll
  for (int cc = 0; cc < 2; ++cc) {
    if (cc >= nz_) break;
    dsum sz;
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      if (b >= ny_) break;
      const df* row = c + ((int64_t)fz[cc] * Lc.ny + fy[b]) * Lc.nx;
      dsum sx;
#pragma unroll
      for (int a = 0; a < 2; ++a)
        if (a < nx_) sx.add(df_mul_f(row[fx[a]], wx[a]));
      sz.add(df_mul_f(sx.get(), wy[b]));
    }
    acc.add(df_mul_f(sz.get(), wz[cc]));
  }
  const int64_t o = (int64_t)q.rhs * Lf.N + q.p;
  xf[o] = df_add(xf[o], acc.get());
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// x[r] = X b[r] with the FP64 dense inverse of the coarsest operator (n <= kCoarseLimit).
// A block takes kCoarseRows rows (kCoarseRowsPerWarp per warp) of one right-hand side and
// converts that right-hand side to FP64 once, in shared memory, so that the FP64 pipe does
// one FMA per product (a conversion per product took three more FP64 operations). Each row
// keeps lane-strided partial sums over j and one warp reduction, in the same order as one
// warp per row would.
constexpr int kCoarseRowsPerWarp = 4;
constexpr int kCoarseRows = 8 * kCoarseRowsPerWarp;  // 256 threads

__global__ void __launch_bounds__(256) k_coarse_apply_df(const double* __restrict__ X, int n,
                                                         const df* __restrict__ b, df* __restrict__ x) {
  __shared__ double bs[kCoarseLimit];
  const df* br = b + (int64_t)blockIdx.y * n;
  for (int j = threadIdx.x; j < n; j += blockDim.x) bs[j] = df_to_double(br[j]);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int row0 = blockIdx.x * kCoarseRows + (threadIdx.x >> 5) * kCoarseRowsPerWarp;
  if (row0 >= n) return;
  const double* xr[kCoarseRowsPerWarp];
#pragma unroll
  for (int r = 0; r < kCoarseRowsPerWarp; ++r) xr[r] = X + (int64_t)min(row0 + r, n - 1) * n;
  double s[kCoarseRowsPerWarp];
#pragma unroll
  for (int r = 0; r < kCoarseRowsPerWarp; ++r) s[r] = 0.0;
  for (int j = lane; j < n; j += 32) {
    const double bj = bs[j];
#pragma unroll
    for (int r = 0; r < kCoarseRowsPerWarp; ++r) s[r] = fma(xr[r][j], bj, s[r]);
  }
#pragma unroll
  for (int r = 0; r < kCoarseRowsPerWarp; ++r) {
    const double t = warp_sum(s[r]);
    if (lane == 0 && row0 + r < n) x[(int64_t)blockIdx.y * n + row0 + r] = df_from_double(t);
  }
}

// two entries per thread with 16-byte loads and stores (both arrays 16-byte aligned: the
// callers pass workspace slices and row batches of even length); an odd tail is done singly
__global__ void k_d2df(int64_t n, const double* __restrict__ src, df* __restrict__ dst) {
  const int64_t p = 2 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x);
  if (p + 1 < n) {
    const double2 v = *reinterpret_cast<const double2*>(src + p);
    const df a = df_from_double_fast(v.x), b = df_from_double_fast(v.y);
    *reinterpret_cast<float4*>(dst + p) = make_float4(a.hi, a.lo, b.hi, b.lo);
  } else if (p < n) {
    dst[p] = df_from_double_fast(src[p]);
  }
}

__global__ void k_d2df_1(int64_t n, const double* __restrict__ src, df* __restrict__ dst) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p < n) dst[p] = df_from_double_fast(src[p]);
}

__global__ void k_df2d(int64_t n, const df* __restrict__ src, double* __restrict__ dst, df* __restrict__ dst2) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const df v = src[p];
  if (dst) dst[p] = df_to_double(v);
  if (dst2) dst2[p] = v;
}

// grid (ceil(nx / bx), ny, nz * nrhs) and block bx = min(128, nx rounded up to a warp)
inline void geom(const Level& L, int nrhs, dim3& g, dim3& b) {
  const int bx = L.nx >= 128 ? 128 : ((L.nx + 31) / 32) * 32;
  b = dim3(bx);
  g = dim3((unsigned)((L.nx + bx - 1) / bx), (unsigned)L.ny, (unsigned)(L.nz * nrhs));
}
inline unsigned nblk(int64_t n) { return (unsigned)((n + kThreads - 1) / kThreads); }

}  // namespace

void launch_cheb_first_df(const Level& L, int nrhs, const df* b, df* x, df* r, df* d, bool zero_x, df inv_theta,
                          cudaStream_t s) {
  dim3 g, b_;
  geom(L, nrhs, g, b_);
  k_cheb_first_df<<<g, b_, 0, s>>>(L, b, x, r, d, zero_x ? 1 : 0, inv_theta);
  note_launches(1);
}

void launch_cheb_step_df(const Level& L, int nrhs, df* r, const df* d_old, df* d_new, df* x, df c1, df c2,
                         bool add_old, cudaStream_t s) {
  dim3 g, b_;
  geom(L, nrhs, g, b_);
  k_cheb_step_df<<<g, b_, 0, s>>>(L, r, d_old, d_new, x, c1, c2, add_old ? 1 : 0);
  note_launches(1);
}

void launch_add_df(int64_t n, const df* d, df* x, cudaStream_t s) {
  k_add_df<<<nblk(n), kThreads, 0, s>>>(n, d, x);
  note_launches(1);
}

void launch_residual_df(const Level& L, int nrhs, const df* b, const df* x, df* r, cudaStream_t s) {
  dim3 g, b_;
  geom(L, nrhs, g, b_);
  k_residual_df<<<g, b_, 0, s>>>(L, b, x, r);
  note_launches(1);
}

void launch_restrict_df(const Level& Lf, const Level& Lc, int nrhs, const df* rf, df* bc, cudaStream_t s) {
  dim3 g, b_;
  geom(Lc, nrhs, g, b_);
  k_restrict_df<<<g, b_, 0, s>>>(Lf, Lc, rf, bc);
  note_launches(1);
}

void launch_prolong_add_df(const Level& Lf, const Level& Lc, int nrhs, const df* xc, df* xf, cudaStream_t s) {
  dim3 g, b_;
  geom(Lf, nrhs, g, b_);
  k_prolong_add_df<<<g, b_, 0, s>>>(Lf, Lc, xc, xf);
  note_launches(1);
}

void launch_coarse_apply_df(const double* X, int n, int nrhs, const df* b, df* x, cudaStream_t s) {
  k_coarse_apply_df<<<dim3((unsigned)((n + kCoarseRows - 1) / kCoarseRows), nrhs), 256, 0, s>>>(X, n, b, x);
  note_launches(1);
}

void launch_d2df(int64_t n, const double* src, df* dst, cudaStream_t s) {
  // the paired loads need 16-byte alignment; otherwise fall back to the single-entry form
  if ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15) {
    k_d2df_1<<<nblk(n), kThreads, 0, s>>>(n, src, dst);
    note_launches(1);
    return;
  }
  k_d2df<<<nblk((n + 1) / 2), kThreads, 0, s>>>(n, src, dst);
  note_launches(1);
}

void launch_df2d(int64_t n, const df* src, double* dst, df* dst2, cudaStream_t s) {
  k_df2d<<<nblk(n), kThreads, 0, s>>>(n, src, dst, dst2);
  note_launches(1);
}

}  // namespace h1w
