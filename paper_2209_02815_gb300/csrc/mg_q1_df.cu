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

// (A u)_p; coefficients of neighbours outside the grid are zero and skipped
__device__ __forceinline__ df q1_apply_df(const Level& L, const df* __restrict__ u, int i, int j, int64_t p) {
  const df* st = L.q1st;
  dsum s;
#pragma unroll
  for (int b = -1; b <= 1; ++b) {
    if (j + b < 0 || j + b >= L.ny) continue;
#pragma unroll
    for (int a = -1; a <= 1; ++a) {
      if (i + a < 0 || i + a >= L.nx) continue;
      s.add(df_mul(st[(int64_t)(3 * (b + 1) + (a + 1)) * L.N + p], u[p + (int64_t)b * L.nx + a]));
    }
  }
  return s.get();
}

struct Vtx {
  int i, j;
  int64_t p, off;
};
__device__ __forceinline__ bool vtx_of(const Level& L, Vtx& v) {
  v.p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v.p >= L.N) return false;
  v.i = (int)(v.p % L.nx);
  v.j = (int)(v.p / L.nx);
  v.off = (int64_t)blockIdx.y * L.N;
  return true;
}

__global__ void k_q1_cheb_first_df(Level L, const df* __restrict__ b, df* __restrict__ x, df* __restrict__ r,
                                   df* __restrict__ d, int zero_x, df inv_theta) {
  Vtx v;
  if (!vtx_of(L, v)) return;
  df rv = b[v.off + v.p];
  if (!zero_x) rv = df_sub(rv, q1_apply_df(L, x + v.off, v.i, v.j, v.p));
  const df dv = df_mul(df_mul(rv, L.q1st[9 * L.N + v.p]), inv_theta);
  r[v.off + v.p] = rv;
  d[v.off + v.p] = dv;
  if (zero_x) x[v.off + v.p] = dv;  // otherwise x is read by neighbours; the next step adds d
}

__global__ void k_q1_cheb_step_df(Level L, df* __restrict__ r, const df* __restrict__ d_old,
                                  df* __restrict__ d_new, df* __restrict__ x, df c1, df c2, int add_old) {
  Vtx v;
  if (!vtx_of(L, v)) return;
  const int64_t o = v.off + v.p;
  const df dold = d_old[o];
  const df rv = df_sub(r[o], q1_apply_df(L, d_old + v.off, v.i, v.j, v.p));
  const df dv = df_add(df_mul(c1, dold), df_mul(c2, df_mul(rv, L.q1st[9 * L.N + v.p])));
  r[o] = rv;
  d_new[o] = dv;
  x[o] = df_add(x[o], add_old ? df_add(dold, dv) : dv);
}

__global__ void k_q1_residual_df(Level L, const df* __restrict__ b, const df* __restrict__ x, df* __restrict__ r) {
  Vtx v;
  if (!vtx_of(L, v)) return;
  r[v.off + v.p] = df_sub(b[v.off + v.p], q1_apply_df(L, x + v.off, v.i, v.j, v.p));
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

__global__ void k_q1_restrict_df(Level Lf, Level Lc, const df* __restrict__ rf, df* __restrict__ bc) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= Lc.N) return;
  const int I = (int)(p % Lc.nx), J = (int)(p / Lc.nx);
  const df* r = rf + (int64_t)blockIdx.y * Lf.N;
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
  bc[(int64_t)blockIdx.y * Lc.N + p] = acc.get();
}

__global__ void k_q1_prolong_add_df(Level Lf, Level Lc, const df* __restrict__ xc, df* __restrict__ xf) {
  Vtx v;
  if (!vtx_of(Lf, v)) return;
  const df* c = xc + (int64_t)blockIdx.y * Lc.N;
  int fx[2], fy[2];
  float wx[2], wy[2];
  const int nx_ = q1_prl(v.i, Lf.nx, Lc.nx, Lf.cx, fx, wx);
  const int ny_ = q1_prl(v.j, Lf.ny, Lc.ny, Lf.cy, fy, wy);
  dsum acc;
  for (int b = 0; b < ny_; ++b) {
    const df* row = c + (int64_t)fy[b] * Lc.nx;
    dsum sx;
    for (int a = 0; a < nx_; ++a) sx.add(halve(row[fx[a]], wx[a]));
    acc.add(halve(sx.get(), wy[b]));
  }
  const int64_t o = v.off + v.p;
  xf[o] = df_add(xf[o], acc.get());
}

inline dim3 grid_of(int64_t n, int nrhs) { return dim3((unsigned)((n + kThreads - 1) / kThreads), (unsigned)nrhs); }

}  // namespace

void launch_q1_stencil_df(const Level& L, df* st, cudaStream_t s) {
  k_q1_stencil_df<<<grid_of(L.N, 1), kThreads, 0, s>>>(L, st);
  note_launches(1);
}
void launch_q1_cheb_first_df(const Level& L, int nrhs, const df* b, df* x, df* r, df* d, bool zero_x, df inv_theta,
                             cudaStream_t s) {
  k_q1_cheb_first_df<<<grid_of(L.N, nrhs), kThreads, 0, s>>>(L, b, x, r, d, zero_x ? 1 : 0, inv_theta);
  note_launches(1);
}
void launch_q1_cheb_step_df(const Level& L, int nrhs, df* r, const df* d_old, df* d_new, df* x, df c1, df c2,
                            bool add_old, cudaStream_t s) {
  k_q1_cheb_step_df<<<grid_of(L.N, nrhs), kThreads, 0, s>>>(L, r, d_old, d_new, x, c1, c2, add_old ? 1 : 0);
  note_launches(1);
}
void launch_q1_residual_df(const Level& L, int nrhs, const df* b, const df* x, df* r, cudaStream_t s) {
  k_q1_residual_df<<<grid_of(L.N, nrhs), kThreads, 0, s>>>(L, b, x, r);
  note_launches(1);
}
void launch_q1_restrict_df(const Level& Lf, const Level& Lc, int nrhs, const df* rf, df* bc, cudaStream_t s) {
  k_q1_restrict_df<<<grid_of(Lc.N, nrhs), kThreads, 0, s>>>(Lf, Lc, rf, bc);
  note_launches(1);
}
void launch_q1_prolong_add_df(const Level& Lf, const Level& Lc, int nrhs, const df* xc, df* xf, cudaStream_t s) {
  k_q1_prolong_add_df<<<grid_of(Lf.N, nrhs), kThreads, 0, s>>>(Lf, Lc, xc, xf);
  note_launches(1);
}

}  // namespace h1w
