// Matrix-free multigrid kernels for L-hat^-1 ~ (K + M)^-1 on structured grids:
// stencil residuals, Chebyshev-Jacobi smoothing steps, restriction R = P^T,
// prolongation P, the Gershgorin bound of D^-1 A and the coarsest dense matrix.
//
// The paper applies an algebraic multigrid cycle as the Laplace
// preconditioner S-hat^-1 (Sec. 3.2) as a black box; on the structured grids
// of this library that cycle is geometric and matrix-free:
//  * FV (3D cell-centred): 7-point operator with face transmissibilities
//    T_d and cell volume V (the lowest-order Raviart-Thomas Schur complement
//    with diagonal Q, Sec. 2.3 / 3.2); every level is the same operator
//    rediscretized; transfer by cell-centred trilinear interpolation.
//  * Q1 (2D vertex): A = Kx (x) My + Mx (x) Ky + Dx (x) Dy with tridiagonal 1D
//    factors; coarse levels are Galerkin products, which keep this form.
// All kernels are batched over right-hand sides: blockIdx.y selects one of
// nrhs vectors stored back to back (stride N of the level).
#include "h1w_internal.cuh"

namespace h1w {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ double tri(const double* q, int n, int t, int i, int a) {
  const double* d = q + (2 * t) * n;
  const double* o = q + (2 * t + 1) * n;
  if (a == 0) return d[i];
  if (a > 0) return (i < n - 1) ? o[i] : 0.0;
  return (i > 0) ? o[i - 1] : 0.0;
}

struct FV {
  static constexpr int kDisc = H1W_FV_CELL;
  __device__ static int cls(const Level& L, int i, int j, int k) {
    return ((i > 0) + (i < L.nx - 1)) + 3 * ((j > 0) + (j < L.ny - 1)) + 9 * ((k > 0) + (k < L.nz - 1));
  }
  __device__ static double diag(const Level& L, int i, int j, int k) { return L.fv_diag[cls(L, i, j, k)]; }
  __device__ static double dinv(const Level& L, int i, int j, int k) { return L.fv_dinv[cls(L, i, j, k)]; }
  // returns (A u)_p; dg and di receive the diagonal A_pp and its inverse
  __device__ static double apply(const Level& L, const double* u, int i, int j, int k, int64_t p,
                                 double& dg, double& di) {
    const int64_t sy = L.nx, sz = (int64_t)L.nx * L.ny;
    const int c = cls(L, i, j, k);
    dg = L.fv_diag[c];
    di = L.fv_dinv[c];
    if (L.iso) {
      double s = 0.0;
      if (i > 0) s += u[p - 1];
      if (i < L.nx - 1) s += u[p + 1];
      if (j > 0) s += u[p - sy];
      if (j < L.ny - 1) s += u[p + sy];
      if (k > 0) s += u[p - sz];
      if (k < L.nz - 1) s += u[p + sz];
      return dg * u[p] - L.Tx * s;
    }
    double sx_ = 0.0, sy_ = 0.0, sz_ = 0.0;
    if (i > 0) sx_ += u[p - 1];
    if (i < L.nx - 1) sx_ += u[p + 1];
    if (j > 0) sy_ += u[p - sy];
    if (j < L.ny - 1) sy_ += u[p + sy];
    if (k > 0) sz_ += u[p - sz];
    if (k < L.nz - 1) sz_ += u[p + sz];
    return dg * u[p] - L.Tx * sx_ - L.Ty * sy_ - L.Tz * sz_;
  }
  __device__ static double apply(const Level& L, const double* u, int i, int j, int k, int64_t p,
                                 double& dg) {
    double di;
    return apply(L, u, i, j, k, p, dg, di);
  }
  __device__ static double gersh(const Level& L, int i, int j, int k) {
    const double d = diag(L, i, j, k);
    return (2.0 * d - L.V) / d;
  }
};

struct Q1 {
  static constexpr int kDisc = H1W_Q1_VERTEX;
  __device__ static double diag(const Level& L, int i, int j, int) {
    return tri(L.qx, L.nx, 0, i, 0) * tri(L.qy, L.ny, 1, j, 0) +
           tri(L.qx, L.nx, 1, i, 0) * tri(L.qy, L.ny, 0, j, 0) +
           tri(L.qx, L.nx, 2, i, 0) * tri(L.qy, L.ny, 2, j, 0);
  }
  __device__ static double dinv(const Level& L, int i, int j, int k) { return 1.0 / diag(L, i, j, k); }
  __device__ static double apply(const Level& L, const double* u, int i, int j, int k, int64_t p,
                                 double& dg, double& di) {
    const double a = apply(L, u, i, j, k, p, dg);
    di = 1.0 / dg;
    return a;
  }
  __device__ static double apply(const Level& L, const double* u, int i, int j, int, int64_t p,
                                 double& dg) {
    const int nx = L.nx, ny = L.ny;
    double kxm = tri(L.qx, nx, 0, i, -1), kx0 = tri(L.qx, nx, 0, i, 0), kxp = tri(L.qx, nx, 0, i, 1);
    double mxm = tri(L.qx, nx, 1, i, -1), mx0 = tri(L.qx, nx, 1, i, 0), mxp = tri(L.qx, nx, 1, i, 1);
    double dxm = tri(L.qx, nx, 2, i, -1), dx0 = tri(L.qx, nx, 2, i, 0), dxp = tri(L.qx, nx, 2, i, 1);
    double acc = 0.0;
#pragma unroll
    for (int b = -1; b <= 1; ++b) {
      const int jj = j + b;
      if (jj < 0 || jj >= ny) continue;
      const double* row = u + (p - i) + (int64_t)b * nx;
      const double um = (i > 0) ? row[i - 1] : 0.0;
      const double u0 = row[i];
      const double up = (i < nx - 1) ? row[i + 1] : 0.0;
      const double fk = kxm * um + kx0 * u0 + kxp * up;
      const double fm = mxm * um + mx0 * u0 + mxp * up;
      const double fd = dxm * um + dx0 * u0 + dxp * up;
      acc += tri(L.qy, ny, 1, j, b) * fk + tri(L.qy, ny, 0, j, b) * fm + tri(L.qy, ny, 2, j, b) * fd;
    }
    dg = kx0 * tri(L.qy, ny, 1, j, 0) + mx0 * tri(L.qy, ny, 0, j, 0) + dx0 * tri(L.qy, ny, 2, j, 0);
    return acc;
  }
  __device__ static double coef(const Level& L, int i, int j, int a, int b) {
    return tri(L.qx, L.nx, 0, i, a) * tri(L.qy, L.ny, 1, j, b) +
           tri(L.qx, L.nx, 1, i, a) * tri(L.qy, L.ny, 0, j, b) +
           tri(L.qx, L.nx, 2, i, a) * tri(L.qy, L.ny, 2, j, b);
  }
  __device__ static double gersh(const Level& L, int i, int j, int) {
    double s = 0.0;
    for (int b = -1; b <= 1; ++b)
      for (int a = -1; a <= 1; ++a) {
        if (i + a < 0 || i + a >= L.nx || j + b < 0 || j + b >= L.ny) continue;
        s += fabs(coef(L, i, j, a, b));
      }
    return s / coef(L, i, j, 0, 0);
  }
};

__device__ __forceinline__ void decompose(const Level& L, int64_t p, int& i, int& j, int& k) {
  i = (int)(p % L.nx);
  const int64_t t = p / L.nx;
  j = (int)(t % L.ny);
  k = (int)(t / L.ny);
}

template <class D>
__global__ void k_cheb_first(Level L, const double* __restrict__ b, double* __restrict__ x,
                             double* __restrict__ r, double* __restrict__ d, int zero_x,
                             double inv_theta) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= L.N) return;
  const int64_t off = (int64_t)blockIdx.y * L.N;
  int i, j, k;
  decompose(L, p, i, j, k);
  double dg, di, rv;
  if (zero_x) {
    di = D::dinv(L, i, j, k);
    rv = b[off + p];
  } else {
    const double ax = D::apply(L, x + off, i, j, k, p, dg, di);
    rv = b[off + p] - ax;
  }
  const double dv = rv * di * inv_theta;
  r[off + p] = rv;
  d[off + p] = dv;
  // x is read through the stencil by neighbouring threads, so it is only
  // written here when it was not read (zero_x); otherwise the next pointwise
  // step adds d (add_old in k_cheb_step).
  if (zero_x) x[off + p] = dv;
}

template <class D>
__global__ void k_cheb_step(Level L, double* __restrict__ r, const double* __restrict__ d_old,
                            double* __restrict__ d_new, double* __restrict__ x, double c1,
                            double c2, int add_old) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= L.N) return;
  const int64_t off = (int64_t)blockIdx.y * L.N;
  int i, j, k;
  decompose(L, p, i, j, k);
  double dg, di;
  const double ad = D::apply(L, d_old + off, i, j, k, p, dg, di);
  const double rv = r[off + p] - ad;
  const double dv = c1 * d_old[off + p] + c2 * (rv * di);
  r[off + p] = rv;
  d_new[off + p] = dv;
  x[off + p] += add_old ? d_old[off + p] + dv : dv;
}

__global__ void k_add(int64_t n, const double* __restrict__ d, double* __restrict__ x) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p < n) x[p] += d[p];
}

template <class D>
__global__ void k_residual(Level L, const double* __restrict__ b, const double* __restrict__ x,
                           double* __restrict__ r) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= L.N) return;
  const int64_t off = (int64_t)blockIdx.y * L.N;
  int i, j, k;
  decompose(L, p, i, j, k);
  double dg;
  r[off + p] = b[off + p] - D::apply(L, x + off, i, j, k, p, dg);
}

// ---- transfer weights --------------------------------------------------------

// FV, coarse cell I on an axis: fine cells and weights of row I of P^T.
__device__ __forceinline__ int fv_restrict_1d(int I, int nc, int coarsened, int* f, double* w) {
  if (!coarsened) { f[0] = I; w[0] = 1.0; return 1; }
  int c = 0;
  if (I >= 1) { f[c] = 2 * I - 1; w[c++] = 0.25; }
  f[c] = 2 * I;     w[c++] = (I >= 1) ? 0.75 : 1.0;
  f[c] = 2 * I + 1; w[c++] = (I + 1 < nc) ? 0.75 : 1.0;
  if (I + 1 < nc) { f[c] = 2 * I + 2; w[c++] = 0.25; }
  return c;
}

// FV, fine cell i: coarse cells and weights of row i of P.
__device__ __forceinline__ int fv_prolong_1d(int i, int nc, int coarsened, int* f, double* w) {
  if (!coarsened) { f[0] = i; w[0] = 1.0; return 1; }
  const int I = i >> 1;
  const int J = (i & 1) ? I + 1 : I - 1;
  if (J >= 0 && J < nc) { f[0] = I; w[0] = 0.75; f[1] = J; w[1] = 0.25; return 2; }
  f[0] = I; w[0] = 1.0;
  return 1;
}

// Q1: a fine vertex f is a coarse vertex iff f is even or f is the last vertex.
__device__ __forceinline__ bool q1_is_coarse(int f, int nf) { return ((f & 1) == 0) || f == nf - 1; }

__device__ __forceinline__ int q1_restrict_1d(int I, int nf, int coarsened, int* f, double* w) {
  if (!coarsened) { f[0] = I; w[0] = 1.0; return 1; }
  const int f0 = min(2 * I, nf - 1);
  int c = 0;
  f[c] = f0; w[c++] = 1.0;
  if (f0 - 1 >= 0 && !q1_is_coarse(f0 - 1, nf)) { f[c] = f0 - 1; w[c++] = 0.5; }
  if (f0 + 1 <= nf - 1 && !q1_is_coarse(f0 + 1, nf)) { f[c] = f0 + 1; w[c++] = 0.5; }
  return c;
}

__device__ __forceinline__ int q1_prolong_1d(int i, int nf, int nc, int coarsened, int* f,
                                             double* w) {
  if (!coarsened) { f[0] = i; w[0] = 1.0; return 1; }
  if ((i & 1) == 0) { f[0] = i >> 1; w[0] = 1.0; return 1; }
  if (i == nf - 1) { f[0] = nc - 1; w[0] = 1.0; return 1; }
  f[0] = (i - 1) >> 1; w[0] = 0.5;
  f[1] = (i + 1) >> 1; w[1] = 0.5;
  return 2;
}

template <int DISC>
__global__ void k_restrict(Level Lf, Level Lc, const double* __restrict__ rf,
                           double* __restrict__ bc) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= Lc.N) return;
  const double* r = rf + (int64_t)blockIdx.y * Lf.N;
  int I, J, K;
  decompose(Lc, p, I, J, K);
  int fx[4], fy[4], fz[4];
  double wx[4], wy[4], wz[4];
  int nx_, ny_, nz_;
  if (DISC == H1W_FV_CELL) {
    nx_ = fv_restrict_1d(I, Lc.nx, Lf.cx, fx, wx);
    ny_ = fv_restrict_1d(J, Lc.ny, Lf.cy, fy, wy);
    nz_ = fv_restrict_1d(K, Lc.nz, Lf.cz, fz, wz);
  } else {
    nx_ = q1_restrict_1d(I, Lf.nx, Lf.cx, fx, wx);
    ny_ = q1_restrict_1d(J, Lf.ny, Lf.cy, fy, wy);
    nz_ = 1; fz[0] = 0; wz[0] = 1.0;
  }
  double acc = 0.0;
  for (int c = 0; c < nz_; ++c)
    for (int b = 0; b < ny_; ++b) {
      const double wyz = wy[b] * wz[c];
      const double* row = r + ((int64_t)fz[c] * Lf.ny + fy[b]) * Lf.nx;
      double s = 0.0;
      for (int a = 0; a < nx_; ++a) s += wx[a] * row[fx[a]];
      acc += wyz * s;
    }
  bc[(int64_t)blockIdx.y * Lc.N + p] = acc;
}

template <int DISC>
__global__ void k_prolong_add(Level Lf, Level Lc, const double* __restrict__ xc,
                              double* __restrict__ xf) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= Lf.N) return;
  const double* c = xc + (int64_t)blockIdx.y * Lc.N;
  int i, j, k;
  decompose(Lf, p, i, j, k);
  int fx[2], fy[2], fz[2];
  double wx[2], wy[2], wz[2];
  int nx_, ny_, nz_;
  if (DISC == H1W_FV_CELL) {
    nx_ = fv_prolong_1d(i, Lc.nx, Lf.cx, fx, wx);
    ny_ = fv_prolong_1d(j, Lc.ny, Lf.cy, fy, wy);
    nz_ = fv_prolong_1d(k, Lc.nz, Lf.cz, fz, wz);
  } else {
    nx_ = q1_prolong_1d(i, Lf.nx, Lc.nx, Lf.cx, fx, wx);
    ny_ = q1_prolong_1d(j, Lf.ny, Lc.ny, Lf.cy, fy, wy);
    nz_ = 1; fz[0] = 0; wz[0] = 1.0;
  }
  double acc = 0.0;
  for (int cc = 0; cc < nz_; ++cc)
    for (int b = 0; b < ny_; ++b) {
      const double* row = c + ((int64_t)fz[cc] * Lc.ny + fy[b]) * Lc.nx;
      double s = 0.0;
      for (int a = 0; a < nx_; ++a) s += wx[a] * row[fx[a]];
      acc += wy[b] * wz[cc] * s;
    }
  xf[(int64_t)blockIdx.y * Lf.N + p] += acc;
}

template <class D>
__global__ void k_gershgorin(Level L, unsigned long long* out_bits) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= L.N) return;
  int i, j, k;
  decompose(L, p, i, j, k);
  const double g = D::gersh(L, i, j, k);
  // positive doubles order like their bit patterns
  atomicMax(out_bits, (unsigned long long)__double_as_longlong(g));
}

template <class D>
__global__ void k_assemble_dense(Level L, double* A) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= L.N) return;
  int i, j, k;
  decompose(L, p, i, j, k);
  double* row = A + p * L.N;
  if (D::kDisc == H1W_FV_CELL) {
    const int64_t sy = L.nx, sz = (int64_t)L.nx * L.ny;
    row[p] = FV::diag(L, i, j, k);
    if (i > 0) row[p - 1] = -L.Tx;
    if (i < L.nx - 1) row[p + 1] = -L.Tx;
    if (j > 0) row[p - sy] = -L.Ty;
    if (j < L.ny - 1) row[p + sy] = -L.Ty;
    if (k > 0) row[p - sz] = -L.Tz;
    if (k < L.nz - 1) row[p + sz] = -L.Tz;
  } else {
    for (int b = -1; b <= 1; ++b)
      for (int a = -1; a <= 1; ++a) {
        if (i + a < 0 || i + a >= L.nx || j + b < 0 || j + b >= L.ny) continue;
        row[p + (int64_t)b * L.nx + a] = Q1::coef(L, i, j, a, b);
      }
  }
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Deterministic block sum (blockDim.x == kThreads); result valid in thread 0.
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double sh[kThreads / 32];
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double t = 0.0;
  if (wid == 0) {
    t = (lane < kThreads / 32) ? sh[lane] : 0.0;
    t = warp_sum(t);
  }
  return t;
}

template <class D>
__global__ void __launch_bounds__(kThreads) k_apply_op(Level L, double ca, const double* __restrict__ p,
                                                       double cj, const double* __restrict__ J,
                                                       const double* __restrict__ w, int m,
                                                       double* __restrict__ out,
                                                       double* __restrict__ partial) {
  extern __shared__ double sw[];
  for (int i = threadIdx.x; i < m; i += blockDim.x) sw[i] = w[i];
  __syncthreads();
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double prod = 0.0;
  if (q < L.N) {
    int i, j, k;
    decompose(L, q, i, j, k);
    double dg;
    double v = ca * D::apply(L, p, i, j, k, q, dg);
    if (m > 0) {
      double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
      const double* col = J + q;
      int r = 0;
      for (; r + 4 <= m; r += 4) {
        a0 += col[(int64_t)(r + 0) * L.N] * sw[r + 0];
        a1 += col[(int64_t)(r + 1) * L.N] * sw[r + 1];
        a2 += col[(int64_t)(r + 2) * L.N] * sw[r + 2];
        a3 += col[(int64_t)(r + 3) * L.N] * sw[r + 3];
      }
      for (; r < m; ++r) a0 += col[(int64_t)r * L.N] * sw[r];
      v += cj * ((a0 + a1) + (a2 + a3));
    }
    out[q] = v;
    prod = p[q] * v;
  }
  if (partial) {
    const double s = block_sum(prod);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
  }
}

// out = ca * (A p) + cj * sum_i Jd[i][k] w[i], with J as double-floats (the
// stencil part in FP64); partial[block] = sum_k p_k out_k when partial != null.

// VEC (N even): each thread takes the two cells 2t, 2t + 1, reading the two entries of each
// row of Jd with one 16-byte load, with one cascaded sum per cell.
template <class D, bool VEC>
__global__ void __launch_bounds__(kThreads) k_apply_op_df(Level L, double ca, const double* __restrict__ p,
                                                          double cj, const df* __restrict__ Jd,
                                                          const double* __restrict__ w, int m,
                                                          double* __restrict__ out,
                                                          double* __restrict__ partial) {
  extern __shared__ df swd[];
  for (int i = threadIdx.x; i < m; i += blockDim.x) swd[i] = df_from_double(w[i]);
  __syncthreads();
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  constexpr int kC = VEC ? 2 : 1;
  const int64_t q0 = kC * t0;
  double prod = 0.0;
  if (q0 < L.N) {
    float s[kC], e[kC];
#pragma unroll
    for (int c = 0; c < kC; ++c) s[c] = e[c] = 0.f;
    if (m > 0) {
      if (VEC) {
        const float4* col = reinterpret_cast<const float4*>(Jd + q0);
        const int64_t stride = L.N / 2;
        for (int r = 0; r < m; ++r) {
          const float4 x = col[(int64_t)r * stride];
          const df wr = swd[r];
          const df t0_ = df_mul(df_make(x.x, x.y), wr), t1_ = df_mul(df_make(x.z, x.w), wr);
          df u = two_sum(s[0], t0_.hi);
          s[0] = u.hi;
          e[0] = __fadd_rn(e[0], __fadd_rn(u.lo, t0_.lo));
          u = two_sum(s[kC - 1], t1_.hi);
          s[kC - 1] = u.hi;
          e[kC - 1] = __fadd_rn(e[kC - 1], __fadd_rn(u.lo, t1_.lo));
        }
      } else {
        const df* col = Jd + q0;
        for (int r = 0; r < m; ++r) {
          const df t = df_mul(col[(int64_t)r * L.N], swd[r]);
          const df u = two_sum(s[0], t.hi);
          s[0] = u.hi;
          e[0] = __fadd_rn(e[0], __fadd_rn(u.lo, t.lo));
        }
      }
    }
#pragma unroll
    for (int c = 0; c < kC; ++c) {
      const int64_t q = q0 + c;
      int i, j, k;
      decompose(L, q, i, j, k);
      double dg;
      double v = ca * D::apply(L, p, i, j, k, q, dg);
      if (m > 0) v += cj * df_to_double(fast_two_sum(s[c], e[c]));
      out[q] = v;
      prod += p[q] * v;
    }
  }
  if (partial) {
    const double t = block_sum(prod);
    if (threadIdx.x == 0) partial[blockIdx.x] = t;
  }
}

inline dim3 grid_for(int64_t N, int nrhs) {
  return dim3((unsigned)((N + kThreads - 1) / kThreads), (unsigned)nrhs);
}

}  // namespace

#define H1W_DISPATCH(disc, KERNEL, ...)                   \
  do {                                                    \
    if ((disc) == H1W_FV_CELL) KERNEL<FV>__VA_ARGS__;     \
    else KERNEL<Q1>__VA_ARGS__;                           \
  } while (0)

void launch_cheb_first(int disc, const Level& L, int nrhs, const double* b, double* x, double* r,
                       double* d, bool zero_x, double inv_theta, cudaStream_t s) {
  H1W_DISPATCH(disc, k_cheb_first, <<<grid_for(L.N, nrhs), kThreads, 0, s>>>(L, b, x, r, d, zero_x ? 1 : 0, inv_theta));
  note_launches(1);
}

void launch_cheb_step(int disc, const Level& L, int nrhs, double* r, const double* d_old,
                      double* d_new, double* x, double c1, double c2, bool add_old, cudaStream_t s) {
  H1W_DISPATCH(disc, k_cheb_step, <<<grid_for(L.N, nrhs), kThreads, 0, s>>>(L, r, d_old, d_new, x, c1, c2, add_old ? 1 : 0));
  note_launches(1);
}

void launch_add(int64_t n, const double* d, double* x, cudaStream_t s) {
  k_add<<<(unsigned)((n + kThreads - 1) / kThreads), kThreads, 0, s>>>(n, d, x);
  note_launches(1);
}

void launch_residual(int disc, const Level& L, int nrhs, const double* b, const double* x,
                     double* r, cudaStream_t s) {
  H1W_DISPATCH(disc, k_residual, <<<grid_for(L.N, nrhs), kThreads, 0, s>>>(L, b, x, r));
  note_launches(1);
}

void launch_restrict(int disc, const Level& Lf, const Level& Lc, int nrhs, const double* rf,
                     double* bc, cudaStream_t s) {
  if (disc == H1W_FV_CELL)
    k_restrict<H1W_FV_CELL><<<grid_for(Lc.N, nrhs), kThreads, 0, s>>>(Lf, Lc, rf, bc);
  else
    k_restrict<H1W_Q1_VERTEX><<<grid_for(Lc.N, nrhs), kThreads, 0, s>>>(Lf, Lc, rf, bc);
  note_launches(1);
}

void launch_prolong_add(int disc, const Level& Lf, const Level& Lc, int nrhs, const double* xc,
                        double* xf, cudaStream_t s) {
  if (disc == H1W_FV_CELL)
    k_prolong_add<H1W_FV_CELL><<<grid_for(Lf.N, nrhs), kThreads, 0, s>>>(Lf, Lc, xc, xf);
  else
    k_prolong_add<H1W_Q1_VERTEX><<<grid_for(Lf.N, nrhs), kThreads, 0, s>>>(Lf, Lc, xc, xf);
  note_launches(1);
}

void launch_gershgorin(int disc, const Level& L, unsigned long long* out_bits, cudaStream_t s) {
  H1W_DISPATCH(disc, k_gershgorin, <<<grid_for(L.N, 1), kThreads, 0, s>>>(L, out_bits));
  note_launches(1);
}

void launch_assemble_dense(int disc, const Level& L, double* A, cudaStream_t s) {
  H1W_DISPATCH(disc, k_assemble_dense, <<<grid_for(L.N, 1), kThreads, 0, s>>>(L, A));
  note_launches(1);
}

int apply_op_blocks(const Level& L) { return (int)((L.N + kThreads - 1) / kThreads); }

void launch_apply_op_df(int disc, const Level& L, double ca, const double* p, double cj, const df* Jd,
                        const double* w, int m, double* out, double* partial, int* nblocks_out, cudaStream_t s) {
  const bool vec = L.N % 2 == 0;
  const int nb = vec ? (int)((L.N / 2 + kThreads - 1) / kThreads) : apply_op_blocks(L);
  if (nblocks_out) *nblocks_out = nb;
  const size_t smem = sizeof(df) * (size_t)(m > 0 ? m : 1);
  if (disc == H1W_FV_CELL) {
    if (vec) k_apply_op_df<FV, true><<<nb, kThreads, smem, s>>>(L, ca, p, cj, Jd, w, m, out, partial);
    else k_apply_op_df<FV, false><<<nb, kThreads, smem, s>>>(L, ca, p, cj, Jd, w, m, out, partial);
  } else {
    if (vec) k_apply_op_df<Q1, true><<<nb, kThreads, smem, s>>>(L, ca, p, cj, Jd, w, m, out, partial);
    else k_apply_op_df<Q1, false><<<nb, kThreads, smem, s>>>(L, ca, p, cj, Jd, w, m, out, partial);
  }
  note_launches(1);
}

void launch_apply_op(int disc, const Level& L, double ca, const double* p, double cj,
                     const double* J, const double* w, int m, double* out, double* partial,
                     int* nblocks_out, cudaStream_t s) {
  const int nb = apply_op_blocks(L);
  if (nblocks_out) *nblocks_out = nb;
  const size_t smem = sizeof(double) * (size_t)(m > 0 ? m : 1);
  H1W_DISPATCH(disc, k_apply_op, <<<nb, kThreads, smem, s>>>(L, ca, p, cj, J, w, m, out, partial));
  note_launches(1);
}

}  // namespace h1w
