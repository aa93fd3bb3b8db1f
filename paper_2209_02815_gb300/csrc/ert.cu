// The ERT forward model and its Jacobian on the context's finite-volume grid (Sec. 4.1,
// Eqs. 4.1-4.5): h1w_forward and h1w_adjoint.
//
// Model. sigma = exp(m) per cell; the conductance of the face between neighbours a, b
// along axis k is G_k 2 s_a s_b / (s_a + s_b) (G_k = face area / centre distance, the
// level's Tx, Ty, Tz); a box face marked Dirichlet (the paper's gamma_D) couples its
// boundary cells to a ghost value 0 at distance h_k / 2 (conductance 2 G_k s_a), the
// other box faces are zero-flux. Electrode e injects a unit current into its cell c_e,
// so the pole field is u_e = A^-1 e_{c_e}, and measurement i with electrodes (A, B, M, N)
// (-1: at infinity) is g_i = k_i (v(c_M) - v(c_N)), v = u_A - u_B (Eq. 4.3 with the
// geometric factor of Eq. 4.5). By reciprocity A^-1 (e_M - e_N) = u_M - u_N = w, so the
// derivative of Eq. 4.4 is J_ic = -k_i w^T (dA / dm_c) v: a sum over the faces of cell c
// of d(conductance)/dm_c times the jumps of v and w across the face.
//
// Forward solve. All n_e pole fields at once by PCG in FP64 (flexible beta, since the
// preconditioner is applied in FP32) on A, preconditioned by two FP32 V-cycles on the same
// operator (the second from the first's result; kErtCycles): the context's hierarchy and its trilinear transfers (R = P^T), Chebyshev-
// Jacobi smoothing of degree 2 on [lambda / 10, lambda] with the Gershgorin bound
// lambda = 2 of D^-1 A (one stencil pass per smoothing, k_smooth32), and coarse operators
// rediscretized from the geometric mean of the children's conductivities; the coarsest
// level is solved with a dense inverse from the FP64 Cholesky factor. A thread of the
// cycle's kernels takes one cell for kFpt fields, so it reads the cell's coefficients once.
//
// Jacobian. One block takes 32 consecutive cells: it stages the jumps of every field
// across the six faces of each cell, and the conductance derivatives, in shared memory,
// then every warp forms J_ic for its measurements with the 32 cells on its lanes. The
// same kernel accumulates J^T r without storing J.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "h1w_internal.cuh"
#include "mg_df64_util.cuh"

namespace h1w {
namespace {

constexpr int kThreads = 256;
constexpr int kJacCells = 32;
constexpr int kJacWarps = 8;
constexpr int kDotBlocks = 64;   // partial sums per field in the dot kernels
constexpr double kLambda = 2.0;  // Gershgorin bound of D^-1 A for this operator

struct Bump {
  char* base;
  size_t off = 0;
  template <class T>
  T* take(size_t count) {
    off = (off + 255) & ~size_t(255);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += sizeof(T) * (count ? count : 1);
    return p;
  }
};

struct Coef32 {
  const float *tx, *ty, *tz, *dg, *dinv;  // t*: conductance to the + neighbour (0 at the last cell)
};

struct Layout {
  int* cell;
  int4* abmn;
  double* k;
  float2* nkdf;  // -k_i as double-floats (hi, lo)
  double* sig[kMaxLevels];
  double *tx64, *ty64, *tz64, *dg64;
  float *tx[kMaxLevels], *ty[kMaxLevels], *tz[kMaxLevels], *dg[kMaxLevels], *dinv[kMaxLevels];
  float *x[kMaxLevels], *b[kMaxLevels], *r[kMaxLevels];
  double *Ac, *Xc;
  float* Xf;
  int* status;
  double *r64, *z64, *p64, *q64;
  double* partial;  // [2][n_e][kDotBlocks]
  double* jvp;      // [m][blocks of the Jacobian kernel]: partial sums of J p
  double* scal;     // [kScal][n_e]
};

enum { kRho = 0, kAlpha, kBeta, kRR, kActive, kScal };

size_t layout(Layout& W, char* base, const Level* lev, int nlev, int n_e, int m) {
  Bump B{base};
  const int64_t N = lev[0].N;
  W.cell = B.take<int>(n_e);
  W.abmn = B.take<int4>(m);
  W.k = B.take<double>(m);
  W.nkdf = B.take<float2>(m);
  for (int l = 0; l < nlev; ++l) W.sig[l] = B.take<double>(lev[l].N);
  W.tx64 = B.take<double>(N);
  W.ty64 = B.take<double>(N);
  W.tz64 = B.take<double>(N);
  W.dg64 = B.take<double>(N);
  for (int l = 0; l < nlev; ++l) {
    const int64_t n = lev[l].N;
    W.tx[l] = B.take<float>(n);
    W.ty[l] = B.take<float>(n);
    W.tz[l] = B.take<float>(n);
    W.dg[l] = B.take<float>(n);
    W.dinv[l] = B.take<float>(n);
    W.x[l] = B.take<float>(n * n_e);
    W.b[l] = B.take<float>(n * n_e);
    W.r[l] = B.take<float>(n * n_e);
  }
  const int64_t nc = lev[nlev - 1].N;
  W.Ac = B.take<double>(nc * nc);
  W.Xc = B.take<double>(nc * nc);
  W.Xf = B.take<float>(nc * nc);
  W.status = B.take<int>(1);
  W.r64 = B.take<double>(N * n_e);
  W.z64 = B.take<double>(N * n_e);
  W.p64 = B.take<double>(N * n_e);
  W.q64 = B.take<double>(N * n_e);
  W.partial = B.take<double>(2 * (size_t)n_e * kDotBlocks);
  W.jvp = B.take<double>((size_t)m * (size_t)((N + kJacCells - 1) / kJacCells));
  W.scal = B.take<double>((size_t)kScal * n_e);
  return B.off + 256;
}

// (i, j, k) of cell p in 32-bit unsigned arithmetic (the forward checks N < 2^31): 64-bit
// division is a long software sequence, and the one-field-per-thread kernels pay it per field
__device__ __forceinline__ void cell_ijk(const Level& L, int64_t p, int& i, int& j, int& k) {
  const unsigned u = (unsigned)p, nx = (unsigned)L.nx, ny = (unsigned)L.ny;
  const unsigned q = u / nx;
  i = (int)(u - q * nx);
  k = (int)(q / ny);
  j = (int)(q - (unsigned)k * ny);
}

__device__ __forceinline__ double harmonic_face(double G, double a, double b) { return G * 2.0 * a * b / (a + b); }

inline unsigned nblk(int64_t n) { return (unsigned)((n + kThreads - 1) / kThreads); }

// ---- conductivities and coefficients --------------------------------------------

__global__ void k_exp(int64_t N, const double* __restrict__ m, double* __restrict__ s) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p < N) s[p] = exp(m[p]);
}

// coarse conductivity = geometric mean of the children's
__global__ void k_coarsen_sigma(Level Lf, Level Lc, const double* __restrict__ sf, double* __restrict__ sc) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= Lc.N) return;
  int I, J, K;
  cell_ijk(Lc, p, I, J, K);
  const int nx = Lf.cx ? 2 : 1, ny = Lf.cy ? 2 : 1, nz = Lf.cz ? 2 : 1;
  double acc = 0.0;
  for (int c = 0; c < nz; ++c)
    for (int b = 0; b < ny; ++b)
      for (int a = 0; a < nx; ++a) {
        const int64_t f = ((int64_t)(K * nz + c) * Lf.ny + (J * ny + b)) * Lf.nx + (I * nx + a);
        acc += log(sf[f]);
      }
  sc[p] = exp(acc / (nx * ny * nz));
}

// Conductances to the + neighbours and the diagonal of one level; FP64 copies and the
// dense matrix (coarsest level) when asked. A Dirichlet face adds ghost * G_k * sigma to the
// diagonal: ghost = 2 on the fine level (the model: u = 0 half a cell away). The coarse
// levels only precondition, and there ghost = 4, so that the coarse operator matches P^T A P
// on constants (a coarse boundary cell collects four fine ghost faces of 2 G_k sigma with
// prolongation weight 1, while its own G_k is twice the fine one).
__global__ void k_coef(Level L, const double* __restrict__ sig, unsigned dirichlet, double ghost, float* tx,
                       float* ty, float* tz, float* dg, float* dinv, double* tx64, double* ty64, double* tz64,
                       double* dg64, double* A) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= L.N) return;
  int i, j, k;
  cell_ijk(L, p, i, j, k);
  const double s = sig[p];
  const int64_t sx = 1, sy = L.nx, sz = (int64_t)L.nx * L.ny;
  const double G[3] = {L.Tx, L.Ty, L.Tz};
  const int idx[3] = {i, j, k}, n[3] = {L.nx, L.ny, L.nz};
  const int64_t st[3] = {sx, sy, sz};
  double tplus[3], d = 0.0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    double tm = 0.0, tp = 0.0;
    if (idx[a] > 0) tm = harmonic_face(G[a], s, sig[p - st[a]]);
    else if (dirichlet >> (2 * a) & 1) d += ghost * G[a] * s;
    if (idx[a] < n[a] - 1) tp = harmonic_face(G[a], s, sig[p + st[a]]);
    else if (dirichlet >> (2 * a + 1) & 1) d += ghost * G[a] * s;
    d += tm + tp;
    tplus[a] = tp;
    if (A) {
      if (idx[a] > 0) A[p * L.N + p - st[a]] = -tm;
      if (idx[a] < n[a] - 1) A[p * L.N + p + st[a]] = -tp;
    }
  }
  tx[p] = (float)tplus[0];
  ty[p] = (float)tplus[1];
  tz[p] = (float)tplus[2];
  dg[p] = (float)d;
  dinv[p] = (float)(1.0 / d);
  if (tx64) {
    tx64[p] = tplus[0];
    ty64[p] = tplus[1];
    tz64[p] = tplus[2];
    dg64[p] = d;
  }
  if (A) A[p * L.N + p] = d;
}

// ---- the operator ------------------------------------------------------------------

template <class T>
struct Stencil {
  T c, xm, xp, ym, yp, zm, zp;  // diagonal and the six couplings (0 where there is no face)
  int64_t sy, sz;
  bool hxm, hxp, hym, hyp, hzm, hzp;
};

template <class T>
__device__ __forceinline__ Stencil<T> load_stencil(const Level& L, const T* tx, const T* ty, const T* tz, const T* dg,
                                                   int64_t p) {
  int i, j, k;
  cell_ijk(L, p, i, j, k);
  Stencil<T> S;
  S.sy = L.nx;
  S.sz = (int64_t)L.nx * L.ny;
  S.hxm = i > 0; S.hxp = i < L.nx - 1;
  S.hym = j > 0; S.hyp = j < L.ny - 1;
  S.hzm = k > 0; S.hzp = k < L.nz - 1;
  S.c = dg[p];
  S.xp = tx[p]; S.yp = ty[p]; S.zp = tz[p];
  S.xm = S.hxm ? tx[p - 1] : T(0);
  S.ym = S.hym ? ty[p - S.sy] : T(0);
  S.zm = S.hzm ? tz[p - S.sz] : T(0);
  return S;
}

template <class T>
__device__ __forceinline__ T stencil_apply(const Stencil<T>& S, const T* __restrict__ x, int64_t p) {
  T y = S.c * x[p];
  if (S.hxm) y -= S.xm * x[p - 1];
  if (S.hxp) y -= S.xp * x[p + 1];
  if (S.hym) y -= S.ym * x[p - S.sy];
  if (S.hyp) y -= S.yp * x[p + S.sy];
  if (S.hzm) y -= S.zm * x[p - S.sz];
  if (S.hzp) y -= S.zp * x[p + S.sz];
  return y;
}

// y_e = A x_e (FP64, level 0), one thread per cell over all fields
__global__ void k_apply64(Level L, const double* tx, const double* ty, const double* tz, const double* dg, int nrhs,
                          const double* __restrict__ x, double* __restrict__ y) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= L.N) return;
  const Stencil<double> S = load_stencil<double>(L, tx, ty, tz, dg, p);
  for (int e = 0; e < nrhs; ++e) y[e * L.N + p] = stencil_apply(S, x + e * L.N, p);
}

// ---- FP32 V-cycle -------------------------------------------------------------------

// The FP32 cycle's kernels take kFpt fields per thread: a cell's stencil coefficients and
// its index arithmetic serve all of them. Their 1D grid runs the field groups of a cell
// block next to each other (group = block index modulo the group count), so the coefficients
// come from DRAM once and from L2 for the other groups; with the groups outermost every
// group re-read them from DRAM.
constexpr int kFpt = 8;
// V-cycles per application of the forward's preconditioner: the FP32 cycle costs less than
// an outer FP64 iteration (the operator runs on the FP64 pipe), so two cycles pay: 14 -> 9
// iterations and 54.6 -> 51.9 ms per forward at 128^3 with 32 fields (three: 7, 53.3 ms)
constexpr int kErtCycles = 2;

// The degree-2 Chebyshev-Jacobi smoothing collapses into one stencil pass. With A = D - N
// (N(u)_i = sum over the faces of cell i of t u_nb), d0 = D^-1 r0 / theta, r1 = r0 - A d0 and
// x += d0 + c1 d0 + c2 D^-1 r1, the identity A d0 = r0 / theta - N d0 gives
//   x += D^-1 [beta r0 + (c2 / theta) N(D^-1 r0)],  beta = (1 + c1) / theta + c2 (1 - 1 / theta),
// with r0 = b for the zero initial guess of the pre-smoothing and r0 = b - A x for the
// post-smoothing. One pass reads r0 (with its neighbours) and x and writes x, where the
// two-step form wrote r, d and x twice.
__global__ void k_smooth32(Level L, Coef32 C, int ne, const float* __restrict__ r0, float* __restrict__ x,
                           int zero_x, float beta, float c2t) {
  const unsigned ng = (unsigned)((ne + kFpt - 1) / kFpt), grp = blockIdx.x % ng;  // field groups fastest
  const int64_t p = (int64_t)(blockIdx.x / ng) * blockDim.x + threadIdx.x;
  if (p >= L.N) return;
  const Stencil<float> S = load_stencil<float>(L, C.tx, C.ty, C.tz, C.dg, p);
  const float di = C.dinv[p];
  // face conductance times the neighbour's D^-1 (0 where there is no neighbour)
  const float wxm = S.hxm ? S.xm * C.dinv[p - 1] : 0.f, wxp = S.hxp ? S.xp * C.dinv[p + 1] : 0.f;
  const float wym = S.hym ? S.ym * C.dinv[p - S.sy] : 0.f, wyp = S.hyp ? S.yp * C.dinv[p + S.sy] : 0.f;
  const float wzm = S.hzm ? S.zm * C.dinv[p - S.sz] : 0.f, wzp = S.hzp ? S.zp * C.dinv[p + S.sz] : 0.f;
#pragma unroll
  for (int f = 0; f < kFpt; ++f) {
    const int e = (int)grp * kFpt + f;
    if (e >= ne) break;
    const int64_t o = (int64_t)e * L.N;
    const float* r = r0 + o;
    float n = 0.f;
    if (S.hxm) n += wxm * r[p - 1];
    if (S.hxp) n += wxp * r[p + 1];
    if (S.hym) n += wym * r[p - S.sy];
    if (S.hyp) n += wyp * r[p + S.sy];
    if (S.hzm) n += wzm * r[p - S.sz];
    if (S.hzp) n += wzp * r[p + S.sz];
    const float dx = di * (beta * r[p] + c2t * n);
    x[o + p] = zero_x ? dx : x[o + p] + dx;
  }
}

__global__ void k_resid32(Level L, Coef32 C, int ne, const float* __restrict__ b, const float* __restrict__ x,
                          float* __restrict__ r) {
  const unsigned ng = (unsigned)((ne + kFpt - 1) / kFpt), grp = blockIdx.x % ng;  // field groups fastest
  const int64_t p = (int64_t)(blockIdx.x / ng) * blockDim.x + threadIdx.x;
  if (p >= L.N) return;
  const Stencil<float> S = load_stencil<float>(L, C.tx, C.ty, C.tz, C.dg, p);
#pragma unroll
  for (int f = 0; f < kFpt; ++f) {
    const int e = (int)grp * kFpt + f;
    if (e >= ne) break;
    const int64_t o = (int64_t)e * L.N;
    r[o + p] = b[o + p] - stencil_apply(S, x + o, p);
  }
}

// Cell-centred trilinear transfer weights of one axis (2:1 agglomeration), as in the
// context's cycle: prolongation 3/4 from the parent and 1/4 from the parent's
// neighbour on the child's side (the parent alone at the boundary); R = P^T. Both
// footprints have a fixed size (4 fine cells per coarse cell, 2 coarse cells per fine
// cell) with in-range indices and weight 0 where a point does not exist, so the loops
// unroll and all loads of a thread are independent.
__device__ __forceinline__ void rst_1d(int I, int nc, int coarsened, int f[4], float w[4]) {
  if (!coarsened) {
    f[0] = f[1] = f[2] = f[3] = I;
    w[0] = 1.f; w[1] = w[2] = w[3] = 0.f;
    return;
  }
  const bool lo = I >= 1, hi = I + 1 < nc;
  f[0] = lo ? 2 * I - 1 : 2 * I;
  f[1] = 2 * I;
  f[2] = 2 * I + 1;
  f[3] = hi ? 2 * I + 2 : 2 * I + 1;
  w[0] = lo ? 0.25f : 0.f;
  w[1] = lo ? 0.75f : 1.f;
  w[2] = hi ? 0.75f : 1.f;
  w[3] = hi ? 0.25f : 0.f;
}

__device__ __forceinline__ void prl_1d(int i, int nc, int coarsened, int f[2], float w[2]) {
  if (!coarsened) { f[0] = f[1] = i; w[0] = 1.f; w[1] = 0.f; return; }
  const int I = i >> 1;
  const int J = (i & 1) ? I + 1 : I - 1;
  const bool has = J >= 0 && J < nc;
  f[0] = I; f[1] = has ? J : I;
  w[0] = has ? 0.75f : 1.f; w[1] = has ? 0.25f : 0.f;
}

// grid: (coarse cells / 256, fields)
__global__ void k_restrict32(Level Lf, Level Lc, int ne, const float* __restrict__ rf, float* __restrict__ bc) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= Lc.N) return;
  int I, J, K;
  cell_ijk(Lc, p, I, J, K);
  int fx[4], fy[4], fz[4];
  float wx[4], wy[4], wz[4];
  rst_1d(I, Lc.nx, Lf.cx, fx, wx);
  rst_1d(J, Lc.ny, Lf.cy, fy, wy);
  rst_1d(K, Lc.nz, Lf.cz, fz, wz);
  {  // one field per thread here: the restriction is bound by the latency of its 64 loads
    const int e = (int)blockIdx.y;
    if (e >= ne) return;
    const float* r = rf + (int64_t)e * Lf.N;
    float acc = 0.f;
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const float* row = r + ((int64_t)fz[c] * Lf.ny + fy[b]) * Lf.nx;
        const float s = wx[0] * row[fx[0]] + wx[1] * row[fx[1]] + wx[2] * row[fx[2]] + wx[3] * row[fx[3]];
        acc += wy[b] * wz[c] * s;
      }
    bc[(int64_t)e * Lc.N + p] = acc;
  }
}

// The restriction on a level whose x axis is coarsened: a thread takes the coarse pair
// (2t, 2t + 1) of one row, whose x footprints are fine cells 4t - 1 .. 4t + 2 and
// 4t + 1 .. 4t + 4, and reads each fine row segment once: 4t .. 4t + 3 as two 8-byte loads
// (fine rows have an even length, so 4t is 8-byte aligned), 4t - 1 and 4t + 4 alone where
// they exist. Half the load instructions of one coarse cell per thread. Grid: (pairs / 256,
// fields); every other coarse quantity as in k_restrict32.
__global__ void k_restrict32_pairs(Level Lf, Level Lc, int ne, const float* __restrict__ rf,
                                   float* __restrict__ bc) {
  const int nx2 = (Lc.nx + 1) >> 1;
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t npair = (int64_t)nx2 * Lc.ny * Lc.nz;
  if (q >= npair) return;
  const unsigned u = (unsigned)q;
  const unsigned row = u / (unsigned)nx2;
  const int t = (int)(u - row * (unsigned)nx2);
  const int K = (int)(row / (unsigned)Lc.ny), J = (int)(row - (unsigned)K * Lc.ny);
  const int e = (int)blockIdx.y;
  if (e >= ne) return;
  const int I0 = 2 * t, I1 = I0 + 1;
  const bool has1 = I1 < Lc.nx;
  // x weights of the two coarse cells at fine offsets -1 .. 4 from 4t (0 where not used)
  float a[6], b[6];
  {
    const bool lo0 = I0 >= 1, hi0 = I0 + 1 < Lc.nx;
    a[0] = lo0 ? 0.25f : 0.f; a[1] = lo0 ? 0.75f : 1.f; a[2] = hi0 ? 0.75f : 1.f; a[3] = hi0 ? 0.25f : 0.f;
    a[4] = 0.f; a[5] = 0.f;
    const bool hi1 = I1 + 1 < Lc.nx;
    b[0] = 0.f; b[1] = 0.f;
    b[2] = has1 ? 0.25f : 0.f; b[3] = has1 ? 0.75f : 0.f;
    b[4] = has1 ? (hi1 ? 0.75f : 1.f) : 0.f; b[5] = (has1 && hi1) ? 0.25f : 0.f;
  }
  int fy[4], fz[4];
  float wy[4], wz[4];
  rst_1d(J, Lc.ny, Lf.cy, fy, wy);
  rst_1d(K, Lc.nz, Lf.cz, fz, wz);
  const int x0 = 4 * t;
  const bool left = x0 >= 1, right = x0 + 4 < Lf.nx, mid2 = x0 + 2 < Lf.nx;
  const float* r = rf + (int64_t)e * Lf.N;
  float acc0 = 0.f, acc1 = 0.f;
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int bb = 0; bb < 4; ++bb) {
      const float* rw = r + ((int64_t)fz[c] * Lf.ny + fy[bb]) * Lf.nx + x0;
      const float2 m0 = *reinterpret_cast<const float2*>(rw);
      const float2 m1 = mid2 ? *reinterpret_cast<const float2*>(rw + 2) : make_float2(0.f, 0.f);
      const float vl = left ? rw[-1] : 0.f, vr = right ? rw[4] : 0.f;
      const float w = wy[bb] * wz[c];
      acc0 += w * (a[0] * vl + a[1] * m0.x + a[2] * m0.y + a[3] * m1.x);
      acc1 += w * (b[2] * m0.y + b[3] * m1.x + b[4] * m1.y + b[5] * vr);
    }
  float* out = bc + (int64_t)e * Lc.N + ((int64_t)K * Lc.ny + J) * Lc.nx + I0;
  out[0] = acc0;
  if (has1) out[1] = acc1;
}

// grid: (fine cells / 256, fields)
__global__ void k_prolong_add32(Level Lf, Level Lc, int ne, const float* __restrict__ xc, float* __restrict__ xf) {
  const unsigned ng = (unsigned)((ne + kFpt - 1) / kFpt), grp = blockIdx.x % ng;  // field groups fastest
  const int64_t p = (int64_t)(blockIdx.x / ng) * blockDim.x + threadIdx.x;
  if (p >= Lf.N) return;
  int i, j, k;
  cell_ijk(Lf, p, i, j, k);
  int fx[2], fy[2], fz[2];
  float wx[2], wy[2], wz[2];
  prl_1d(i, Lc.nx, Lf.cx, fx, wx);
  prl_1d(j, Lc.ny, Lf.cy, fy, wy);
  prl_1d(k, Lc.nz, Lf.cz, fz, wz);
#pragma unroll
  for (int f = 0; f < kFpt; ++f) {
    const int e = (int)grp * kFpt + f;
    if (e >= ne) break;
    const float* c = xc + (int64_t)e * Lc.N;
    float acc = 0.f;
#pragma unroll
    for (int cc = 0; cc < 2; ++cc)
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        const float* row = c + ((int64_t)fz[cc] * Lc.ny + fy[b]) * Lc.nx;
        acc += wy[b] * wz[cc] * (wx[0] * row[fx[0]] + wx[1] * row[fx[1]]);
      }
    xf[(int64_t)e * Lf.N + p] += acc;
  }
}

// The prolongation on a level whose x axis is coarsened: a thread takes the fine pair
// (2I, 2I + 1) of one row, the two children of coarse cell I, which read coarse cells I - 1,
// I and I + 1 of each coarse row (three loads for two fine cells instead of four) and are
// read and written as one 8-byte pair. Same arithmetic, in the same order, as
// k_prolong_add32; the field groups of a pair block are adjacent in the 1D grid.
__global__ void k_prolong_add32_pairs(Level Lf, Level Lc, int ne, const float* __restrict__ xc,
                                      float* __restrict__ xf) {
  const unsigned ng = (unsigned)((ne + kFpt - 1) / kFpt), grp = blockIdx.x % ng;
  const int64_t q = (int64_t)(blockIdx.x / ng) * blockDim.x + threadIdx.x;
  const int64_t npair = (int64_t)Lc.nx * Lf.ny * Lf.nz;
  if (q >= npair) return;
  const unsigned u = (unsigned)q;
  const unsigned row = u / (unsigned)Lc.nx;
  const int I = (int)(u - row * (unsigned)Lc.nx);
  const int k = (int)(row / (unsigned)Lf.ny), j = (int)(row - (unsigned)k * Lf.ny);
  int fy[2], fz[2];
  float wy[2], wz[2];
  prl_1d(j, Lc.ny, Lf.cy, fy, wy);
  prl_1d(k, Lc.nz, Lf.cz, fz, wz);
  const bool hl = I >= 1, hr = I + 1 < Lc.nx;
  const float a0 = hl ? 0.75f : 1.f, a1 = hl ? 0.25f : 0.f;  // fine 2I: the parent and its left neighbour
  const float b0 = hr ? 0.75f : 1.f, b1 = hr ? 0.25f : 0.f;  // fine 2I + 1: the parent and its right one
  const int Il = hl ? I - 1 : I, Ir = hr ? I + 1 : I;
  const int64_t pf = ((int64_t)k * Lf.ny + j) * Lf.nx + 2 * I;
#pragma unroll
  for (int f = 0; f < kFpt; ++f) {
    const int e = (int)grp * kFpt + f;
    if (e >= ne) break;
    const float* c = xc + (int64_t)e * Lc.N;
    float s0 = 0.f, s1 = 0.f;
#pragma unroll
    for (int cc = 0; cc < 2; ++cc)
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        const float* rw = c + ((int64_t)fz[cc] * Lc.ny + fy[b]) * Lc.nx;
        const float vm = rw[I];
        s0 += wy[b] * wz[cc] * (a0 * vm + a1 * rw[Il]);
        s1 += wy[b] * wz[cc] * (b0 * vm + b1 * rw[Ir]);
      }
    float2* xp = reinterpret_cast<float2*>(xf + (int64_t)e * Lf.N + pf);
    float2 v = *xp;
    v.x += s0;
    v.y += s1;
    *xp = v;
  }
}

// x_e = X b_e on the coarsest level (X: dense inverse, n x n, FP32)
__global__ void k_dense_apply32(const float* __restrict__ X, int n, const float* __restrict__ b, float* __restrict__ x) {
  extern __shared__ float sb[];
  const int e = blockIdx.y;
  for (int j = threadIdx.x; j < n; j += blockDim.x) sb[j] = b[(int64_t)e * n + j];
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float* row = X + (int64_t)i * n;
  float acc = 0.f;
  for (int j = 0; j < n; ++j) acc += row[j] * sb[j];
  x[(int64_t)e * n + i] = acc;
}

__global__ void k_d2f(int64_t n, const double* __restrict__ a, float* __restrict__ b) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p < n) b[p] = (float)a[p];
}

// ---- PCG vector kernels (FP64, grid: (kDotBlocks, fields)) ---------------------------

__device__ __forceinline__ double block_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[k];
  __syncthreads();
  return s;
}

// x = 0, r = e_{c_e}, b32 = (float) r
__global__ void k_init(int64_t N, const int* __restrict__ cell, double* __restrict__ x, double* __restrict__ r,
                       float* __restrict__ b32) {
  const int e = blockIdx.y;
  const int c = cell[e];
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (int64_t)gridDim.x * blockDim.x) {
    const double v = (p == c) ? 1.0 : 0.0;
    x[e * N + p] = 0.0;
    r[e * N + p] = v;
    b32[e * N + p] = (float)v;
  }
}

// r = e_{c_e} - q (q = A u), b32 = (float) r; u is left as it is
__global__ void k_init_warm(int64_t N, const int* __restrict__ cell, const double* __restrict__ q,
                            double* __restrict__ r, float* __restrict__ b32) {
  const int e = blockIdx.y;
  const int c = cell[e];
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (int64_t)gridDim.x * blockDim.x) {
    const double v = ((p == c) ? 1.0 : 0.0) - q[e * N + p];
    r[e * N + p] = v;
    b32[e * N + p] = (float)v;
  }
}

// partial[0] = a . b, partial[1] = c . d (when c is given), per field
__global__ void k_dots(int64_t N, const double* __restrict__ a, const double* __restrict__ b,
                       const double* __restrict__ c, const double* __restrict__ d, double* __restrict__ partial) {
  __shared__ double red[kThreads / 32];
  const int e = blockIdx.y, ne = gridDim.y;
  double s0 = 0.0, s1 = 0.0;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = e * N + p;
    s0 += a[o] * b[o];
    if (c) s1 += c[o] * d[o];
  }
  s0 = block_sum(s0, red);
  s1 = block_sum(s1, red);
  if (threadIdx.x == 0) {
    partial[(int64_t)e * gridDim.x + blockIdx.x] = s0;
    partial[((int64_t)ne + e) * gridDim.x + blockIdx.x] = s1;
  }
}

// z = (double) z32; partials r . z and z . q
// A float as the equal double, by assembling the IEEE 754 bit fields with integer
// instructions (a conversion instruction runs on the FP64 pipe, which GB300 issues at 1/64
// of the FP32 rate). Zeros keep their sign; subnormal floats (below 2^-126, about 1.2e-38)
// become zero; infinities and NaNs keep their class. In J = -k_i (hi + lo) this drops lo
// only when |lo| < 2^-126, i.e. |hi| below about 2^-102 (2e-31): such an entry keeps
// its hi part, and its absolute error stays below |k_i| 2^-126.
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xFFu;
  if (e == 0u) return __hiloint2double(static_cast<int>(u & 0x80000000u), 0);
  const unsigned e11 = (e == 0xFFu) ? 0x7FFu : e + (1023u - 127u);
  const unsigned hi = (u & 0x80000000u) | (e11 << 20) | ((u & 0x7FFFFFu) >> 3);
  return __hiloint2double(static_cast<int>(hi), static_cast<int>(u << 29));
}

// A double as a float by its bit fields, rounding toward zero: the FP32 cycle's input needs
// no correct rounding, and this keeps the conversion off the FP64 pipe. Magnitudes below the
// float normal range become zero, above it infinity; NaNs stay NaNs.
__device__ __forceinline__ float d2f_trunc(double d) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(d));
  const unsigned hi = static_cast<unsigned>(b >> 32), lo = static_cast<unsigned>(b);
  const unsigned sign = hi & 0x80000000u;
  const int e = static_cast<int>((hi >> 20) & 0x7FFu);
  const unsigned m = ((hi & 0xFFFFFu) << 3) | (lo >> 29);  // the top 23 significand bits
  if (e == 0x7FF) return __uint_as_float(sign | 0x7F800000u | (m ? 0x400000u : 0u));
  const int ef = e - 1023 + 127;
  if (ef <= 0) return __uint_as_float(sign);
  if (ef >= 255) return __uint_as_float(sign | 0x7F800000u);
  return __uint_as_float(sign | (static_cast<unsigned>(ef) << 23) | m);
}

// The preconditioned residual z stays in the cycle's FP32 output; the PCG kernels widen it
// to FP64 where they read it, by f2d_bits (no FP64-pipe conversion, no FP64 copy of z).
__global__ void k_z_dots(int64_t N, const float* __restrict__ z32, const double* __restrict__ r,
                         const double* __restrict__ q, double* __restrict__ partial) {
  __shared__ double red[kThreads / 32];
  const int e = blockIdx.y, ne = gridDim.y;
  double s0 = 0.0, s1 = 0.0;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = e * N + p;
    const double zv = f2d_bits(z32[o]);
    s0 += r[o] * zv;
    if (q) s1 += zv * q[o];
  }
  s0 = block_sum(s0, red);
  s1 = block_sum(s1, red);
  if (threadIdx.x == 0) {
    partial[(int64_t)e * gridDim.x + blockIdx.x] = s0;
    partial[((int64_t)ne + e) * gridDim.x + blockIdx.x] = s1;
  }
}

// x += alpha p; r -= alpha q; b32 = r in FP32 (truncated); partial r . r
__global__ void k_xr(int64_t N, const double* __restrict__ scal, double* __restrict__ x, double* __restrict__ r,
                     const double* __restrict__ p_, const double* __restrict__ q, float* __restrict__ b32,
                     double* __restrict__ partial) {
  __shared__ double red[kThreads / 32];
  const int e = blockIdx.y, ne = gridDim.y;
  const double a = scal[kAlpha * ne + e];
  double s0 = 0.0;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = e * N + p;
    x[o] += a * p_[o];
    const double rv = r[o] - a * q[o];
    r[o] = rv;
    b32[o] = d2f_trunc(rv);
    s0 += rv * rv;
  }
  s0 = block_sum(s0, red);
  if (threadIdx.x == 0) partial[(int64_t)e * gridDim.x + blockIdx.x] = s0;
}

// p = z + beta p (first: p = z)
__global__ void k_pupd(int64_t N, const double* __restrict__ scal, const float* __restrict__ z32,
                       double* __restrict__ p_, int first) {
  const int e = blockIdx.y, ne = gridDim.y;
  const double be = first ? 0.0 : scal[kBeta * ne + e];
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = e * N + p;
    const double zv = f2d_bits(z32[o]);
    p_[o] = first ? zv : zv + be * p_[o];
  }
}

// Per-field scalar updates from the partial sums (one thread per field).
// mode 0: rho = r.z (start); 1: alpha = rho / p.q (0 once converged or at breakdown);
// 2: rr = r.r, active = rr > tol2; 3: beta = z.(r - r_old) / rho = -alpha z.q / rho (the
// flexible form, since r - r_old = -alpha q), rho = r.z.
__global__ void k_scalars(int mode, int ne, int nb, const double* __restrict__ partial, double* __restrict__ scal,
                          double tol2) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  double s0 = 0.0, s1 = 0.0;
  for (int b = 0; b < nb; ++b) {
    s0 += partial[(int64_t)e * nb + b];
    s1 += partial[((int64_t)ne + e) * nb + b];
  }
  double* S = scal;
  if (mode == 0) {
    S[kRho * ne + e] = s0;
    S[kActive * ne + e] = 1.0;
  } else if (mode == 1) {
    const double rho = S[kRho * ne + e];
    S[kAlpha * ne + e] = (S[kActive * ne + e] != 0.0 && s0 > 0.0 && rho > 0.0) ? rho / s0 : 0.0;
  } else if (mode == 2) {
    S[kRR * ne + e] = s0;
    if (!(s0 > tol2)) S[kActive * ne + e] = 0.0;
  } else {
    const double rho = S[kRho * ne + e];
    const double a = S[kAlpha * ne + e];
    S[kBeta * ne + e] = (rho > 0.0 && S[kActive * ne + e] != 0.0) ? -a * s1 / rho : 0.0;
    S[kRho * ne + e] = s0;
  }
}

// ---- measurements and the Jacobian ---------------------------------------------------

__device__ __forceinline__ double field_at(const double* U, int64_t N, const int* cell, int e, int f) {
  return (e >= 0 && f >= 0) ? U[(int64_t)e * N + cell[f]] : 0.0;
}

__global__ void k_measure(const double* __restrict__ U, int64_t N, const int* __restrict__ cell,
                          const int4* __restrict__ abmn, const double* __restrict__ k, int m, double* __restrict__ g) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const int4 q = abmn[i];
  const double vm = field_at(U, N, cell, q.x, q.z) - field_at(U, N, cell, q.y, q.z);
  const double vn = field_at(U, N, cell, q.x, q.w) - field_at(U, N, cell, q.y, q.w);
  g[i] = k[i] * (vm - vn);
}

// Shared layout: D[e][face][cell] jumps u_e(c) - u_e(neighbour) (u_e(c) across a Dirichlet
// face, 0 across a zero-flux one), then W[face][cell] = d(conductance)/dm_c, both formed in
// FP64 and stored as double-floats, then the warps' partial sums of J^T r. The products
// and sums of a row run in double-float arithmetic (about 48 bits) on the FP32 pipes, which
// GB300 issues at 64 times its FP64 rate; only the scaling by -k_i is FP64.

// MODE kRows writes the rows of J, kJTr writes J^T r (r = rv), kJvp writes the per-block
// partial sums of J p (p = rv, indexed by cell) to J[i * gridDim.x + block].
enum { kRows = 0, kJTr = 1, kJvp = 2 };

template <int MODE>
__global__ void __launch_bounds__(kJacWarps * 32) k_jacobian(Level L, const double* __restrict__ U, int ne,
                                                             const double* __restrict__ sig, unsigned dirichlet,
                                                             const int4* __restrict__ abmn, const float2* __restrict__ nkf,
                                                             int m, const double* __restrict__ rv, double* __restrict__ J,
                                                             double* __restrict__ JTr) {
  extern __shared__ double sm[];
  df* D = reinterpret_cast<df*>(sm);
  df* Wf = D + (size_t)ne * 6 * kJacCells;
  double* red = reinterpret_cast<double*>(Wf + 6 * kJacCells);
  const int64_t N = L.N;
  const int64_t p0 = (int64_t)blockIdx.x * kJacCells;
  const int64_t st[3] = {1, L.nx, (int64_t)L.nx * L.ny};
  const int nn[3] = {L.nx, L.ny, L.nz};
  const double G[3] = {L.Tx, L.Ty, L.Tz};
  for (int t = threadIdx.x; t < 6 * kJacCells; t += blockDim.x) {
    const int f = t / kJacCells, c = t % kJacCells;
    const int64_t p = p0 + c;
    double w = 0.0;
    if (p < N) {
      int ijk[3];
      cell_ijk(L, p, ijk[0], ijk[1], ijk[2]);
      const int a = f >> 1, side = f & 1;
      const bool inside = side ? ijk[a] < nn[a] - 1 : ijk[a] > 0;
      const double s = sig[p];
      if (inside) {
        const double o = sig[side ? p + st[a] : p - st[a]];
        const double den = s + o;
        w = G[a] * 2.0 * s * o * o / (den * den);
      } else if (dirichlet >> f & 1) {
        w = 2.0 * G[a] * s;
      }
    }
    Wf[t] = df_from_double_fast(w);
  }
  for (int t = threadIdx.x; t < ne * kJacCells; t += blockDim.x) {
    const int e = t / kJacCells, c = t % kJacCells;
    const int64_t p = p0 + c;
    df* De = D + (size_t)e * 6 * kJacCells;
    if (p < N) {
      int ijk[3];
      cell_ijk(L, p, ijk[0], ijk[1], ijk[2]);
      const double* u = U + (int64_t)e * N;
      const double up = u[p];
#pragma unroll
      for (int f = 0; f < 6; ++f) {
        const int a = f >> 1, side = f & 1;
        const bool inside = side ? ijk[a] < nn[a] - 1 : ijk[a] > 0;
        // W is 0 on zero-flux faces
        De[f * kJacCells + c] = df_from_double_fast(inside ? up - u[side ? p + st[a] : p - st[a]] : up);
      }
    } else {
#pragma unroll
      for (int f = 0; f < 6; ++f) De[f * kJacCells + c] = df_make(0.f, 0.f);
    }
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, c = threadIdx.x & 31;
  const int64_t p = p0 + c;
  df w6[6];
#pragma unroll
  for (int f = 0; f < 6; ++f) w6[f] = Wf[f * kJacCells + c];
  // A warp takes a contiguous range of measurements. Survey rows are ordered by source
  // (A, B), so consecutive rows of a warp share it: t_f = W_f (D_A - D_B) is formed once per
  // source and warp, and each row costs one difference, one product and one sum term per
  // face. (Dealt out round-robin, each warp met a new source every other row.)
  double acc_r = 0.0;
  const double pc = (MODE == kJvp && p < N) ? rv[p] : 0.0;
  int la = -2, lb = -2;
  df t6[6];
  const int per = (m + kJacWarps - 1) / kJacWarps;
  const int i_end = min(m, (warp + 1) * per);
  for (int i = warp * per; i < i_end; ++i) {
    const int4 q = abmn[i];
    if (q.x != la || q.y != lb) {  // warp-uniform
      la = q.x;
      lb = q.y;
      const df* DA = la >= 0 ? D + (size_t)la * 6 * kJacCells + c : nullptr;
      const df* DB = lb >= 0 ? D + (size_t)lb * 6 * kJacCells + c : nullptr;
#pragma unroll
      for (int f = 0; f < 6; ++f) {
        const df dv = DA ? (DB ? df_sub(DA[f * kJacCells], DB[f * kJacCells]) : DA[f * kJacCells])
                         : (DB ? df_neg(DB[f * kJacCells]) : df_make(0.f, 0.f));
        t6[f] = df_mul(w6[f], dv);
      }
    }
    const df* DM = q.z >= 0 ? D + (size_t)q.z * 6 * kJacCells + c : nullptr;
    const df* DN = q.w >= 0 ? D + (size_t)q.w * 6 * kJacCells + c : nullptr;
    dfmg::dsum acc;
    if (DM && DN) {
#pragma unroll
      for (int f = 0; f < 6; ++f) acc.add(df_mul(t6[f], df_sub(DM[f * kJacCells], DN[f * kJacCells])));
    } else if (DM || DN) {
      const df* D1 = DM ? DM : DN;
#pragma unroll
      for (int f = 0; f < 6; ++f) acc.add(df_mul(t6[f], D1[f * kJacCells]));
    }
    df sum = acc.get();
    if (!DM && DN) sum = df_neg(sum);
    const float2 nk = nkf[i];
    const df vd = df_mul(sum, df_make(nk.x, nk.y));  // -k_i * sum
    const double val = f2d_bits(vd.hi) + f2d_bits(vd.lo);
    if (MODE == kRows) {
      if (p < N) J[(int64_t)i * N + p] = val;
    } else if (MODE == kJTr) {
      acc_r = fma(rv[i], val, acc_r);
    } else {  // the warp's 32 cells of row i
      double v = val * pc;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (c == 0) J[(int64_t)i * gridDim.x + blockIdx.x] = v;
    }
  }
  if (MODE == kJTr) {
    red[warp * kJacCells + c] = acc_r;
    __syncthreads();
    if (warp == 0 && p < N) {
      double s = 0.0;
      for (int w = 0; w < kJacWarps; ++w) s += red[w * kJacCells + c];
      JTr[p] = s;
    }
  }
}

// Jp_i = sum over blocks of the partial sums of row i (one block per row, fixed order)
__global__ void k_row_sums(const double* __restrict__ partial, int nb, double* __restrict__ out) {
  __shared__ double red[kThreads / 32];
  const double* row = partial + (int64_t)blockIdx.x * nb;
  double s = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) s += row[b];
  s = block_sum(s, red);
  if (threadIdx.x == 0) out[blockIdx.x] = s;
}

size_t jac_smem(int ne) { return sizeof(double) * ((size_t)ne * 6 * kJacCells + 6 * kJacCells + kJacWarps * kJacCells); }

// ---- host driver ---------------------------------------------------------------------

struct Cheb {
  float beta, c2t;  // the collapsed degree-2 step (k_smooth32): beta and c2 / theta
};

// ratio 0: the FV cell grids' interval [lambda / 10, lambda] (14 forward iterations at 128^3
// for ratios 8 to 16, 15 at 20 and 18 at 30)
Cheb cheb_coefs(double ratio) {
  const double lo = kLambda / (ratio > 0.0 ? ratio : 10.0), hi = kLambda;
  const double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo), sg = theta / delta;
  const double rho0 = 1.0 / sg;
  const double rho1 = 1.0 / (2.0 * sg - rho0);
  const double it = 1.0 / theta, c1 = rho1 * rho0, c2 = 2.0 * rho1 / delta;
  return Cheb{(float)((1.0 + c1) * it + c2 * (1.0 - it)), (float)(c2 * it)};
}

Coef32 coef_of(const Layout& W, int l) { return Coef32{W.tx[l], W.ty[l], W.tz[l], W.dg[l], W.dinv[l]}; }

// x = kErtCycles V-cycles on b (level-0 buffers W.b[0] -> W.x[0]; a further cycle starts from the
// previous x); W.r[l] holds the residuals
void vcycle32(const Layout& W, const Level* lev, int nl, int ne, const Cheb& K, cudaStream_t s) {
  const unsigned ng = (unsigned)((ne + kFpt - 1) / kFpt);
  for (int cyc = 0; cyc < kErtCycles; ++cyc) {
    for (int l = 0; l < nl - 1; ++l) {
      const Coef32 C = coef_of(W, l);
      const unsigned nb = nblk(lev[l].N);
      if (l == 0 && cyc > 0) {  // a further cycle starts from the current x: smooth the residual
        k_resid32<<<nb * ng, kThreads, 0, s>>>(lev[l], C, ne, W.b[l], W.x[l], W.r[l]);
        k_smooth32<<<nb * ng, kThreads, 0, s>>>(lev[l], C, ne, W.r[l], W.x[l], 0, K.beta, K.c2t);
        note_launches(2);
      } else {
        k_smooth32<<<nb * ng, kThreads, 0, s>>>(lev[l], C, ne, W.b[l], W.x[l], 1, K.beta, K.c2t);
        note_launches(1);
      }
      k_resid32<<<nb * ng, kThreads, 0, s>>>(lev[l], C, ne, W.b[l], W.x[l], W.r[l]);
      if (lev[l].cx && (reinterpret_cast<uintptr_t>(W.r[l]) & 7) == 0) {  // 8-byte loads need an aligned workspace
        const int64_t npair = (int64_t)((lev[l + 1].nx + 1) / 2) * lev[l + 1].ny * lev[l + 1].nz;
        k_restrict32_pairs<<<dim3(nblk(npair), ne), kThreads, 0, s>>>(lev[l], lev[l + 1], ne, W.r[l], W.b[l + 1]);
      } else {
        k_restrict32<<<dim3(nblk(lev[l + 1].N), ne), kThreads, 0, s>>>(lev[l], lev[l + 1], ne, W.r[l], W.b[l + 1]);
      }
      note_launches(2);
    }
    const int nc = (int)lev[nl - 1].N;
    k_dense_apply32<<<dim3((nc + kThreads - 1) / kThreads, ne), kThreads, sizeof(float) * nc, s>>>(W.Xf, nc, W.b[nl - 1],
                                                                                                    W.x[nl - 1]);
    note_launches(1);
    for (int l = nl - 2; l >= 0; --l) {
      const Coef32 C = coef_of(W, l);
      const unsigned nb = nblk(lev[l].N);
      if (lev[l].cx && (reinterpret_cast<uintptr_t>(W.x[l]) & 7) == 0) {  // 8-byte pairs need an aligned workspace
        const int64_t npair = (int64_t)lev[l + 1].nx * lev[l].ny * lev[l].nz;
        k_prolong_add32_pairs<<<nblk(npair) * ng, kThreads, 0, s>>>(lev[l], lev[l + 1], ne, W.x[l + 1], W.x[l]);
      } else {
        k_prolong_add32<<<nb * ng, kThreads, 0, s>>>(lev[l], lev[l + 1], ne, W.x[l + 1], W.x[l]);
      }
      k_resid32<<<nb * ng, kThreads, 0, s>>>(lev[l], C, ne, W.b[l], W.x[l], W.r[l]);
      k_smooth32<<<nb * ng, kThreads, 0, s>>>(lev[l], C, ne, W.r[l], W.x[l], 0, K.beta, K.c2t);
      note_launches(3);
    }
  }
}

h1w_status validate_survey(const Level* lev, const h1w_survey* sv, std::string& err) {
  if (lev[0].N >= (int64_t(1) << 31)) {
    err = "ert: grids of 2^31 cells or more are not supported";
    return H1W_EUNSUPPORTED;
  }
  if (!sv || sv->n_e < 1 || sv->n_e > H1W_ERT_MAX_ELECTRODES || sv->m < 0 || !sv->cell ||
      (sv->m > 0 && (!sv->abmn || !sv->k))) {
    err = "survey: need 1..H1W_ERT_MAX_ELECTRODES electrodes, m >= 0 and non-NULL arrays";
    return H1W_EINVAL;
  }
  if (sv->dirichlet == 0 || sv->dirichlet >= 64u) {
    err = "survey: dirichlet must mark at least one of the six box faces (bits 0..5)";
    return H1W_EINVAL;
  }
  for (int e = 0; e < sv->n_e; ++e)
    if (sv->cell[e] < 0 || sv->cell[e] >= lev[0].N) {
      err = "survey: electrode cell out of range";
      return H1W_EINVAL;
    }
  for (int64_t q = 0; q < 4 * (int64_t)sv->m; ++q)
    if (sv->abmn[q] < -1 || sv->abmn[q] >= sv->n_e) {
      err = "survey: electrode index out of range in abmn";
      return H1W_EINVAL;
    }
  return H1W_OK;
}

h1w_status check_cuda(cudaStream_t s, std::string& err, const char* where) {
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    err = std::string(where) + ": " + cudaGetErrorString(e);
    return H1W_ECUDA;
  }
  return H1W_OK;
}

h1w_status upload_survey(const Layout& W, const h1w_survey* sv, cudaStream_t s) {
  cudaMemcpyAsync(W.cell, sv->cell, sizeof(int) * sv->n_e, cudaMemcpyHostToDevice, s);
  if (sv->m > 0) {
    cudaMemcpyAsync(W.abmn, sv->abmn, sizeof(int4) * sv->m, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(W.k, sv->k, sizeof(double) * sv->m, cudaMemcpyHostToDevice, s);
    std::vector<float2> nk(sv->m);
    for (int i = 0; i < sv->m; ++i) {
      const double v = -sv->k[i];
      nk[i].x = static_cast<float>(v);
      nk[i].y = static_cast<float>(v - static_cast<double>(nk[i].x));
    }
    // pageable source: the copy has read it when the call returns
    cudaMemcpyAsync(W.nkdf, nk.data(), sizeof(float2) * sv->m, cudaMemcpyHostToDevice, s);
  }
  return H1W_OK;
}

// Conductivities and operator coefficients of every level; the coarsest level's dense inverse.
h1w_status build_operator(const Layout& W, const Level* lev, int nl, const double* logsigma, unsigned dirichlet,
                          cudaStream_t s, std::string& err) {
  k_exp<<<nblk(lev[0].N), kThreads, 0, s>>>(lev[0].N, logsigma, W.sig[0]);
  note_launches(1);
  for (int l = 1; l < nl; ++l) {
    k_coarsen_sigma<<<nblk(lev[l].N), kThreads, 0, s>>>(lev[l - 1], lev[l], W.sig[l - 1], W.sig[l]);
    note_launches(1);
  }
  const int nc = (int)lev[nl - 1].N;
  cudaMemsetAsync(W.Ac, 0, sizeof(double) * nc * nc, s);
  for (int l = 0; l < nl; ++l) {
    const bool top = l == 0, bottom = l == nl - 1;
    k_coef<<<nblk(lev[l].N), kThreads, 0, s>>>(lev[l], W.sig[l], dirichlet, top ? 2.0 : 4.0, W.tx[l], W.ty[l],
                                               W.tz[l], W.dg[l],
                                               W.dinv[l], top ? W.tx64 : nullptr, top ? W.ty64 : nullptr,
                                               top ? W.tz64 : nullptr, top ? W.dg64 : nullptr, bottom ? W.Ac : nullptr);
    note_launches(1);
  }
  cudaMemsetAsync(W.status, 0, sizeof(int), s);
  launch_chol(W.Ac, nc, W.status, s);
  launch_set_identity(W.Xc, nc, s);
  launch_trsv_lower(W.Ac, nc, W.Xc, nc, s);
  launch_trsv_upper_t(W.Ac, nc, W.Xc, nc, s);
  launch_symmetrize_identity_solve(W.Xc, nc, s);
  k_d2f<<<nblk((int64_t)nc * nc), kThreads, 0, s>>>((int64_t)nc * nc, W.Xc, W.Xf);
  note_launches(1);
  int status = 0;
  cudaMemcpyAsync(&status, W.status, sizeof(int), cudaMemcpyDeviceToHost, s);
  h1w_status st = check_cuda(s, err, "ert operator");
  if (st != H1W_OK) return st;
  if (status & kStatusNotSpd) {
    err = "ert: coarsest-level matrix is not positive definite";
    return H1W_ENOTSPD;
  }
  return H1W_OK;
}

}  // namespace

size_t ert_workspace_bytes(const Level* lev, int nlev, int n_e, int m) {
  if (n_e < 1 || n_e > H1W_ERT_MAX_ELECTRODES || m < 0) return 0;
  Layout W;
  return layout(W, nullptr, lev, nlev, n_e, m);
}

h1w_status ert_forward(const Level* lev, int nl, cudaStream_t s, const h1w_survey* sv, const double* logsigma,
                       double* U, double* g, void* ws, size_t ws_bytes, double rtol, int maxit, bool warm,
                       double cheb_ratio, h1w_info* info, std::string& err) {
  h1w_status st = validate_survey(lev, sv, err);
  if (st != H1W_OK) return st;
  if (!logsigma || !U || (sv->m > 0 && !g) || !ws || !(rtol > 0.0) || maxit < 1) {
    err = "h1w_forward: NULL logsigma/U/g/workspace, rtol <= 0 or maxit < 1";
    return H1W_EINVAL;
  }
  const int ne = sv->n_e;
  Layout W;
  if (layout(W, nullptr, lev, nl, ne, sv->m) > ws_bytes) {
    err = "h1w_forward: workspace smaller than h1w_ert_workspace_size";
    return H1W_EINVAL;
  }
  layout(W, static_cast<char*>(ws), lev, nl, ne, sv->m);
  upload_survey(W, sv, s);
  st = build_operator(W, lev, nl, logsigma, sv->dirichlet, s, err);
  if (st != H1W_OK) return st;

  const Level& L0 = lev[0];
  const int64_t N = L0.N;
  const dim3 vg(kDotBlocks, ne);
  const unsigned sb = (unsigned)((ne + 127) / 128);
  const double tol2 = rtol * rtol;  // ||f_e|| = 1
  const Cheb K = cheb_coefs(cheb_ratio);
  std::vector<double> rr(ne);
  if (warm) {  // r = e_c - A u from the fields in U
    k_apply64<<<nblk(N), kThreads, 0, s>>>(L0, W.tx64, W.ty64, W.tz64, W.dg64, ne, U, W.q64);
    k_init_warm<<<vg, kThreads, 0, s>>>(N, W.cell, W.q64, W.r64, W.b[0]);
    note_launches(2);
  } else {
    k_init<<<vg, kThreads, 0, s>>>(N, W.cell, U, W.r64, W.b[0]);
    note_launches(1);
  }
  vcycle32(W, lev, nl, ne, K, s);
  k_z_dots<<<vg, kThreads, 0, s>>>(N, W.x[0], W.r64, nullptr, W.partial);
  k_scalars<<<sb, 128, 0, s>>>(0, ne, kDotBlocks, W.partial, W.scal, tol2);
  k_pupd<<<vg, kThreads, 0, s>>>(N, W.scal, W.x[0], W.p64, 1);
  note_launches(3);
  int it = 0;
  bool done = false;
  double worst = 1.0;
  while (!done && it < maxit) {
    ++it;
    k_apply64<<<nblk(N), kThreads, 0, s>>>(L0, W.tx64, W.ty64, W.tz64, W.dg64, ne, W.p64, W.q64);
    k_dots<<<vg, kThreads, 0, s>>>(N, W.p64, W.q64, nullptr, nullptr, W.partial);
    k_scalars<<<sb, 128, 0, s>>>(1, ne, kDotBlocks, W.partial, W.scal, tol2);
    k_xr<<<vg, kThreads, 0, s>>>(N, W.scal, U, W.r64, W.p64, W.q64, W.b[0], W.partial);
    k_scalars<<<sb, 128, 0, s>>>(2, ne, kDotBlocks, W.partial, W.scal, tol2);
    note_launches(5);
    cudaMemcpyAsync(rr.data(), W.scal + kRR * ne, sizeof(double) * ne, cudaMemcpyDeviceToHost, s);
    st = check_cuda(s, err, "h1w_forward");
    if (st != H1W_OK) return st;
    worst = 0.0;
    for (int e = 0; e < ne; ++e) worst = std::max(worst, rr[e]);
    if (!(worst == worst)) {
      err = "h1w_forward: NaN residual";
      return H1W_ENOTCONV;
    }
    if (worst <= tol2) {
      done = true;
      break;
    }
    vcycle32(W, lev, nl, ne, K, s);
    k_z_dots<<<vg, kThreads, 0, s>>>(N, W.x[0], W.r64, W.q64, W.partial);
    k_scalars<<<sb, 128, 0, s>>>(3, ne, kDotBlocks, W.partial, W.scal, tol2);
    k_pupd<<<vg, kThreads, 0, s>>>(N, W.scal, W.x[0], W.p64, 0);
    note_launches(3);
  }
  if (sv->m > 0) {
    k_measure<<<(sv->m + 127) / 128, 128, 0, s>>>(U, N, W.cell, W.abmn, W.k, sv->m, g);
    note_launches(1);
  }
  if (info) {
    // true residual ||e_{c_e} - A u_e|| in FP64, worst field
    k_apply64<<<nblk(N), kThreads, 0, s>>>(L0, W.tx64, W.ty64, W.tz64, W.dg64, ne, U, W.q64);
    k_init<<<vg, kThreads, 0, s>>>(N, W.cell, W.z64, W.r64, W.b[0]);
    note_launches(2);
    launch_copy(W.p64, W.q64, (int64_t)N * ne, s);
    launch_axpby(W.p64, 1.0, W.r64, -1.0, N * ne, s);  // p = r - q
    k_dots<<<vg, kThreads, 0, s>>>(N, W.p64, W.p64, nullptr, nullptr, W.partial);
    k_scalars<<<sb, 128, 0, s>>>(2, ne, kDotBlocks, W.partial, W.scal, 0.0);
    note_launches(2);
    cudaMemcpyAsync(rr.data(), W.scal + kRR * ne, sizeof(double) * ne, cudaMemcpyDeviceToHost, s);
    st = check_cuda(s, err, "h1w_forward");
    if (st != H1W_OK) return st;
    double tw = 0.0;
    for (int e = 0; e < ne; ++e) tw = std::max(tw, rr[e]);
    info->iters = it;
    info->restarts = 0;
    info->rel_res_true = std::sqrt(tw);
    info->rel_res_rec = std::sqrt(worst);
  } else {
    st = check_cuda(s, err, "h1w_forward");
    if (st != H1W_OK) return st;
  }
  if (!done) {
    err = "h1w_forward: PCG did not reach rtol within maxit";
    return H1W_ENOTCONV;
  }
  return H1W_OK;
}

h1w_status ert_adjoint(const Level* lev, int nl, cudaStream_t s, const h1w_survey* sv, const double* logsigma,
                       const double* U, const double* r, double* JTr, double* J, void* ws, size_t ws_bytes,
                       std::string& err) {
  h1w_status st = validate_survey(lev, sv, err);
  if (st != H1W_OK) return st;
  if (!logsigma || !U || !ws || (JTr && !r) || (!JTr && !J)) {
    err = "h1w_adjoint: NULL logsigma/U/workspace, JTr without r, or neither JTr nor J";
    return H1W_EINVAL;
  }
  const int ne = sv->n_e;
  Layout W;
  if (layout(W, nullptr, lev, nl, ne, sv->m) > ws_bytes) {
    err = "h1w_adjoint: workspace smaller than h1w_ert_workspace_size";
    return H1W_EINVAL;
  }
  layout(W, static_cast<char*>(ws), lev, nl, ne, sv->m);
  upload_survey(W, sv, s);
  const Level& L0 = lev[0];
  k_exp<<<nblk(L0.N), kThreads, 0, s>>>(L0.N, logsigma, W.sig[0]);
  note_launches(1);
  const size_t smem = jac_smem(ne);
  const unsigned grid = (unsigned)((L0.N + kJacCells - 1) / kJacCells);
  if (J) {
    cudaFuncSetAttribute(k_jacobian<kRows>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_jacobian<kRows><<<grid, kJacWarps * 32, smem, s>>>(L0, U, ne, W.sig[0], sv->dirichlet, W.abmn, W.nkdf, sv->m,
                                                         nullptr, J, nullptr);
    note_launches(1);
  }
  if (JTr) {
    cudaFuncSetAttribute(k_jacobian<kJTr>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_jacobian<kJTr><<<grid, kJacWarps * 32, smem, s>>>(L0, U, ne, W.sig[0], sv->dirichlet, W.abmn, W.nkdf, sv->m, r,
                                                        nullptr, JTr);
    note_launches(1);
  }
  return check_cuda(s, err, "h1w_adjoint");
}

h1w_status ert_jvp(const Level* lev, int nl, cudaStream_t s, const h1w_survey* sv, const double* logsigma,
                   const double* U, const double* pvec, double* Jp, void* ws, size_t ws_bytes, std::string& err) {
  h1w_status st = validate_survey(lev, sv, err);
  if (st != H1W_OK) return st;
  if (!logsigma || !U || !pvec || (sv->m > 0 && !Jp) || !ws) {
    err = "h1w_ert_jvp: NULL logsigma/U/p/Jp/workspace";
    return H1W_EINVAL;
  }
  const int ne = sv->n_e;
  Layout W;
  if (layout(W, nullptr, lev, nl, ne, sv->m) > ws_bytes) {
    err = "h1w_ert_jvp: workspace smaller than h1w_ert_workspace_size";
    return H1W_EINVAL;
  }
  if (sv->m == 0) return H1W_OK;
  layout(W, static_cast<char*>(ws), lev, nl, ne, sv->m);
  upload_survey(W, sv, s);
  const Level& L0 = lev[0];
  k_exp<<<nblk(L0.N), kThreads, 0, s>>>(L0.N, logsigma, W.sig[0]);
  const size_t smem = jac_smem(ne);
  const unsigned grid = (unsigned)((L0.N + kJacCells - 1) / kJacCells);
  cudaFuncSetAttribute(k_jacobian<kJvp>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_jacobian<kJvp><<<grid, kJacWarps * 32, smem, s>>>(L0, U, ne, W.sig[0], sv->dirichlet, W.abmn, W.nkdf, sv->m, pvec,
                                                      W.jvp, nullptr);
  k_row_sums<<<sv->m, kThreads, 0, s>>>(W.jvp, (int)grid, Jp);
  note_launches(3);
  return check_cuda(s, err, "h1w_ert_jvp");
}

}  // namespace h1w
