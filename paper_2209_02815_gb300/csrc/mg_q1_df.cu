// The V-cycle on 2D Q1 vertex grids in double-float arithmetic (FP32 pairs, about 48
// bits), the counterpart of the FV kernels in mg_df64.cu.
//
// The Q1 operator of a level is A = Kx (x) My + Mx (x) Ky + Dx (x) Dy with tridiagonal
// 1D factors (Galerkin products on coarse levels keep this form). Its 9-point stencil
// c(a, b) at vertex (i, j) is a sum of three products of 1D entries; evaluating it per
// application would cost about 30 double-float products, so the setup stores the nine
// coefficients and the inverse diagonal of every vertex of every level once, as
// double-floats formed from FP64 (k_q1_stencil_df), and an application is nine
// products and a cascaded sum. Transfers are the vertex ones of the FP64 cycle (linear
// interpolation between even vertices plus the last vertex, R = P^T); their weights 1
// and 1/2 scale double-floats exactly.
#include "df64.cuh"
#include "h1w_internal.cuh"
#include "mg_df64_util.cuh"

namespace h1w {
namespace {

using namespace dfmg;

constexpr int kThreads = 256;

// entry a (-1, 0, 1) of row i of the 1D factor t (0: K, 1: M, 2: D) in q = [6][n]
__device__ __forceinline__ double tri1(const double* q, int n, int t, int i, int a) {
  const double* d = q + (2 * t) * n;
  const double* o = q + (2 * t + 1) * n;
  if (a == 0) return d[i];
  if (a > 0) return (i < n - 1) ? o[i] : 0.0;
  return (i > 0) ? o[i - 1] : 0.0;
}

// stencil [10][N]: entries 3 (b + 1) + (a + 1) for the neighbour (i + a, j + b), 9 = 1 / c(0, 0)
__global__ void k_q1_stencil_df(Level L, df* __restrict__ st) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= L.N) return;
  const int i = (int)(p % L.nx), j = (int)(p / L.nx);
  double c00 = 1.0;
  for (int b = -1; b <= 1; ++b)
    for (int a = -1; a <= 1; ++a) {
      double c = 0.0;
      if (i + a >= 0 && i + a < L.nx && j + b >= 0 && j + b < L.ny)
        c = tri1(L.qx, L.nx, 0, i, a) * tri1(L.qy, L.ny, 1, j, b) + tri1(L.qx, L.nx, 1, i, a) * tri1(L.qy, L.ny, 0, j, b) +
            tri1(L.qx, L.nx, 2, i, a) * tri1(L.qy, L.ny, 2, j, b);
      if (a == 0 && b == 0) c00 = c;
      st[(int64_t)(3 * (b + 1) + (a + 1)) * L.N + p] = df_from_double(c);
    }
  st[9 * L.N + p] = df_from_double(1.0 / c00);
}

// Launch geometry of the vertex kernels: 64 x 4 vertices per block (no index division),
// grid z over the right-hand sides, kRpt of them per thread (the stencil coefficients of a
// vertex are loaded once and applied to each).
constexpr int kBX = 64, kBY = 4;
constexpr int kRpt = 2;

// (A u)_p for kRpt right-hand sides u[k] (offsets off[k] from u); coefficients of neighbours
// outside the grid are zero and skipped; nk right-hand sides are present (1 or kRpt)
// vertex (i, j) lies in the box whose stencil is the constant L.q1c
__device__ __forceinline__ bool q1_uniform(const Level& L, int i, int j) {
  return i >= L.q1_ilo && i <= L.q1_ihi && j >= L.q1_jlo && j <= L.q1_jhi;
}

__device__ __forceinline__ void q1_apply_df(const Level& L, const df* __restrict__ u, const int64_t* off, int nk,
                                            int i, int j, int64_t p, df* out) {
  const df* st = L.q1st;
  dsum s[kRpt];
  if (q1_uniform(L, i, j)) {  // every neighbour exists; the coefficients are the box's (same values)
#pragma unroll
    for (int b = -1; b <= 1; ++b)
#pragma unroll
      for (int a = -1; a <= 1; ++a) {
        const df c = L.q1c[3 * (b + 1) + (a + 1)];
        const int64_t q = p + (int64_t)b * L.nx + a;
#pragma unroll
        for (int k = 0; k < kRpt; ++k)
          if (k < nk) s[k].add(df_mul(c, u[off[k] + q]));
      }
  } else {
#pragma unroll
    for (int b = -1; b <= 1; ++b) {
      if (j + b < 0 || j + b >= L.ny) continue;
#pragma unroll
      for (int a = -1; a <= 1; ++a) {
        if (i + a < 0 || i + a >= L.nx) continue;
        const df c = st[(int64_t)(3 * (b + 1) + (a + 1)) * L.N + p];
        const int64_t q = p + (int64_t)b * L.nx + a;
#pragma unroll
        for (int k = 0; k < kRpt; ++k)
          if (k < nk) s[k].add(df_mul(c, u[off[k] + q]));
      }
    }
  }
#pragma unroll
  for (int k = 0; k < kRpt; ++k) out[k] = s[k].get();
}

__device__ __forceinline__ df q1_dinv(const Level& L, int i, int j, int64_t p) {
  return q1_uniform(L, i, j) ? L.q1c[9] : L.q1st[9 * L.N + p];
}

struct Vtx {
  int i, j, nk;
  int64_t p, off[kRpt];
};
// vertex of this thread on level L and its right-hand sides (blockIdx.z * kRpt + k < nrhs)
__device__ __forceinline__ bool vtx_of(const Level& L, int nrhs, Vtx& v) {
  v.i = (int)(blockIdx.x * kBX + threadIdx.x);
  v.j = (int)(blockIdx.y * kBY + threadIdx.y);
  if (v.i >= L.nx || v.j >= L.ny) return false;
  v.p = (int64_t)v.j * L.nx + v.i;
  const int r0 = (int)blockIdx.z * kRpt;
  v.nk = min(kRpt, nrhs - r0);
#pragma unroll
  for (int k = 0; k < kRpt; ++k) v.off[k] = (int64_t)(r0 + (k < v.nk ? k : 0)) * L.N;
  return true;
}

__global__ void __launch_bounds__(kBX * kBY) k_q1_cheb_first_df(Level L, int nrhs, const df* __restrict__ b,
                                                              df* __restrict__ x, df* __restrict__ r,
                                                              df* __restrict__ d, int zero_x, df inv_theta) {
  Vtx v;
  if (!vtx_of(L, nrhs, v)) return;
  df ax[kRpt];
  if (!zero_x) q1_apply_df(L, x, v.off, v.nk, v.i, v.j, v.p, ax);
  const df dinv = q1_dinv(L, v.i, v.j, v.p);
#pragma unroll
  for (int k = 0; k < kRpt; ++k) {
    if (k >= v.nk) break;
    const int64_t o = v.off[k] + v.p;
    df rv = b[o];
    if (!zero_x) rv = df_sub(rv, ax[k]);
    const df dv = df_mul(df_mul(rv, dinv), inv_theta);
    r[o] = rv;
    d[o] = dv;
    if (zero_x) x[o] = dv;  // otherwise x is read by neighbours; the next step adds d
  }
}

__global__ void __launch_bounds__(kBX * kBY) k_q1_cheb_step_df(Level L, int nrhs, df* __restrict__ r,
                                                             const df* __restrict__ d_old, df* __restrict__ d_new,
                                                             df* __restrict__ x, df c1, df c2, int add_old) {
  Vtx v;
  if (!vtx_of(L, nrhs, v)) return;
  df ad[kRpt];
  q1_apply_df(L, d_old, v.off, v.nk, v.i, v.j, v.p, ad);
  const df dinv = q1_dinv(L, v.i, v.j, v.p);
#pragma unroll
  for (int k = 0; k < kRpt; ++k) {
    if (k >= v.nk) break;
    const int64_t o = v.off[k] + v.p;
    const df dold = d_old[o];
    const df rv = df_sub(r[o], ad[k]);
    const df dv = df_add(df_mul(c1, dold), df_mul(c2, df_mul(rv, dinv)));
    r[o] = rv;
    d_new[o] = dv;
    x[o] = df_add(x[o], add_old ? df_add(dold, dv) : dv);
  }
}

// Degree-2 Chebyshev smoothing in one pass: with A = D - N (N the off-diagonal couplings
// negated), the two steps from x0 give x0 + D^-1 [beta r0 + c2t N(D^-1 r0)], r0 = b - A x0
// (r0 = b from a zero guess), by the identity A (D^-1 r0 / theta) = r0 / theta - N D^-1 r0.
// The sum runs over c_nb dinv_nb r0_nb; vertices whose whole neighbourhood lies in the
// uniform box take c_nb dinv_nb from the level's constants (q1w).
__global__ void __launch_bounds__(kBX * kBY) k_q1_smooth_df(Level L, int nrhs, const df* __restrict__ r0,
                                                          df* __restrict__ x, int zero_x, df beta, df c2t) {
  Vtx v;
  if (!vtx_of(L, nrhs, v)) return;
  dsum s[kRpt];
  const bool inner = v.i > L.q1_ilo && v.i < L.q1_ihi && v.j > L.q1_jlo && v.j < L.q1_jhi;
  if (inner) {
#pragma unroll
    for (int b = -1; b <= 1; ++b)
#pragma unroll
      for (int a = -1; a <= 1; ++a) {
        if (a == 0 && b == 0) continue;
        const df w = L.q1w[3 * (b + 1) + (a + 1)];
        const int64_t q = v.p + (int64_t)b * L.nx + a;
#pragma unroll
        for (int k = 0; k < kRpt; ++k)
          if (k < v.nk) s[k].add(df_mul(w, r0[v.off[k] + q]));
      }
  } else {
    const df* st = L.q1st;
#pragma unroll
    for (int b = -1; b <= 1; ++b) {
      if (v.j + b < 0 || v.j + b >= L.ny) continue;
#pragma unroll
      for (int a = -1; a <= 1; ++a) {
        if ((a == 0 && b == 0) || v.i + a < 0 || v.i + a >= L.nx) continue;
        const int64_t q = v.p + (int64_t)b * L.nx + a;
        const df w = df_mul(st[(int64_t)(3 * (b + 1) + (a + 1)) * L.N + v.p], q1_dinv(L, v.i + a, v.j + b, q));
#pragma unroll
        for (int k = 0; k < kRpt; ++k)
          if (k < v.nk) s[k].add(df_mul(w, r0[v.off[k] + q]));
      }
    }
  }
  const df dinv = q1_dinv(L, v.i, v.j, v.p);
#pragma unroll
  for (int k = 0; k < kRpt; ++k) {
    if (k >= v.nk) break;
    const int64_t o = v.off[k] + v.p;
    // N(D^-1 r0) = -(the sum above)
    const df val = df_mul(dinv, df_sub(df_mul(beta, r0[o]), df_mul(c2t, s[k].get())));
    x[o] = zero_x ? val : df_add(x[o], val);
  }
}

__global__ void __launch_bounds__(kBX * kBY) k_q1_residual_df(Level L, int nrhs, const df* __restrict__ b,
                                                            const df* __restrict__ x, df* __restrict__ r) {
  Vtx v;
  if (!vtx_of(L, nrhs, v)) return;
  df ax[kRpt];
  q1_apply_df(L, x, v.off, v.nk, v.i, v.j, v.p, ax);
#pragma unroll
  for (int k = 0; k < kRpt; ++k) {
    if (k >= v.nk) break;
    r[v.off[k] + v.p] = df_sub(b[v.off[k] + v.p], ax[k]);
  }
}

// 1D Q1 transfers: a fine vertex is a coarse vertex iff it is even or the last one
__device__ __forceinline__ bool q1c(int f, int nf) { return ((f & 1) == 0) || f == nf - 1; }

__device__ __forceinline__ int q1_rst(int I, int nf, int coarsened, int* f, float* w) {
  if (!coarsened) { f[0] = I; w[0] = 1.f; return 1; }
  const int f0 = min(2 * I, nf - 1);
  int c = 0;
  f[c] = f0; w[c++] = 1.f;
  if (f0 - 1 >= 0 && !q1c(f0 - 1, nf)) { f[c] = f0 - 1; w[c++] = 0.5f; }
  if (f0 + 1 <= nf - 1 && !q1c(f0 + 1, nf)) { f[c] = f0 + 1; w[c++] = 0.5f; }
  return c;
}

__device__ __forceinline__ int q1_prl(int i, int nf, int nc, int coarsened, int* f, float* w) {
  if (!coarsened) { f[0] = i; w[0] = 1.f; return 1; }
  if ((i & 1) == 0) { f[0] = i >> 1; w[0] = 1.f; return 1; }
  if (i == nf - 1) { f[0] = nc - 1; w[0] = 1.f; return 1; }
  f[0] = (i - 1) >> 1; w[0] = 0.5f;
  f[1] = (i + 1) >> 1; w[1] = 0.5f;
  return 2;
}

__device__ __forceinline__ df halve(df v, float w) {  // w is 1 or 1/2: exact
  return w == 1.f ? v : df_make(v.hi * 0.5f, v.lo * 0.5f);
}

__global__ void __launch_bounds__(kBX * kBY) k_q1_restrict_df(Level Lf, Level Lc, const df* __restrict__ rf,
                                                            df* __restrict__ bc) {
  const int I = (int)(blockIdx.x * kBX + threadIdx.x), J = (int)(blockIdx.y * kBY + threadIdx.y);
  if (I >= Lc.nx || J >= Lc.ny) return;
  const int64_t p = (int64_t)J * Lc.nx + I;
  const df* r = rf + (int64_t)blockIdx.z * Lf.N;
  int fx[3], fy[3];
  float wx[3], wy[3];
  const int nx_ = q1_rst(I, Lf.nx, Lf.cx, fx, wx);
  const int ny_ = q1_rst(J, Lf.ny, Lf.cy, fy, wy);
  dsum acc;
  for (int b = 0; b < ny_; ++b) {
    const df* row = r + (int64_t)fy[b] * Lf.nx;
    dsum sx;
    for (int a = 0; a < nx_; ++a) sx.add(halve(row[fx[a]], wx[a]));
    acc.add(halve(sx.get(), wy[b]));
  }
  bc[(int64_t)blockIdx.z * Lc.N + p] = acc.get();
}

__global__ void __launch_bounds__(kBX * kBY) k_q1_prolong_add_df(Level Lf, Level Lc, const df* __restrict__ xc,
                                                               df* __restrict__ xf) {
  const int i = (int)(blockIdx.x * kBX + threadIdx.x), j = (int)(blockIdx.y * kBY + threadIdx.y);
  if (i >= Lf.nx || j >= Lf.ny) return;
  const int64_t p = (int64_t)j * Lf.nx + i;
  const df* c = xc + (int64_t)blockIdx.z * Lc.N;
  int fx[2], fy[2];
  float wx[2], wy[2];
  const int nx_ = q1_prl(i, Lf.nx, Lc.nx, Lf.cx, fx, wx);
  const int ny_ = q1_prl(j, Lf.ny, Lc.ny, Lf.cy, fy, wy);
  dsum acc;
  for (int b = 0; b < ny_; ++b) {
    const df* row = c + (int64_t)fy[b] * Lc.nx;
    dsum sx;
    for (int a = 0; a < nx_; ++a) sx.add(halve(row[fx[a]], wx[a]));
    acc.add(halve(sx.get(), wy[b]));
  }
  const int64_t o = (int64_t)blockIdx.z * Lf.N + p;
  xf[o] = df_add(xf[o], acc.get());
}

inline dim3 grid_of(int64_t n, int nrhs) { return dim3((unsigned)((n + kThreads - 1) / kThreads), (unsigned)nrhs); }
// the vertex kernels: 64 x 4 vertices per block, z = groups of `per` right-hand sides
inline dim3 grid2(const Level& L, int nrhs, int per) {
  return dim3((unsigned)((L.nx + kBX - 1) / kBX), (unsigned)((L.ny + kBY - 1) / kBY), (unsigned)((nrhs + per - 1) / per));
}
const dim3 kBlock2(kBX, kBY);

}  // namespace

void launch_q1_stencil_df(const Level& L, df* st, cudaStream_t s) {
  k_q1_stencil_df<<<grid_of(L.N, 1), kThreads, 0, s>>>(L, st);
  note_launches(1);
}
void launch_q1_cheb_first_df(const Level& L, int nrhs, const df* b, df* x, df* r, df* d, bool zero_x, df inv_theta,
                             cudaStream_t s) {
  k_q1_cheb_first_df<<<grid2(L, nrhs, kRpt), kBlock2, 0, s>>>(L, nrhs, b, x, r, d, zero_x ? 1 : 0, inv_theta);
  note_launches(1);
}
void launch_q1_cheb_step_df(const Level& L, int nrhs, df* r, const df* d_old, df* d_new, df* x, df c1, df c2,
                            bool add_old, cudaStream_t s) {
  k_q1_cheb_step_df<<<grid2(L, nrhs, kRpt), kBlock2, 0, s>>>(L, nrhs, r, d_old, d_new, x, c1, c2, add_old ? 1 : 0);
  note_launches(1);
}
void launch_q1_smooth_df(const Level& L, int nrhs, const df* r0, df* x, bool zero_x, df beta, df c2t,
                         cudaStream_t s) {
  k_q1_smooth_df<<<grid2(L, nrhs, kRpt), kBlock2, 0, s>>>(L, nrhs, r0, x, zero_x ? 1 : 0, beta, c2t);
  note_launches(1);
}
void launch_q1_residual_df(const Level& L, int nrhs, const df* b, const df* x, df* r, cudaStream_t s) {
  k_q1_residual_df<<<grid2(L, nrhs, kRpt), kBlock2, 0, s>>>(L, nrhs, b, x, r);
  note_launches(1);
}
void launch_q1_restrict_df(const Level& Lf, const Level& Lc, int nrhs, const df* rf, df* bc, cudaStream_t s) {
  k_q1_restrict_df<<<grid2(Lc, nrhs, 1), kBlock2, 0, s>>>(Lf, Lc, rf, bc);
  note_launches(1);
}
void launch_q1_prolong_add_df(const Level& Lf, const Level& Lc, int nrhs, const df* xc, df* xf, cudaStream_t s) {
  k_q1_prolong_add_df<<<grid2(Lf, nrhs, 1), kBlock2, 0, s>>>(Lf, Lc, xc, xf);
  note_launches(1);
}

}  // namespace h1w
