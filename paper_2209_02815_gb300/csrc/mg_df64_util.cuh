// Device helpers shared by the double-float multigrid kernels (mg_df64.cu,
// mg_fused.cu): the FV neighbour class, cascaded double-float summation and the
// 1D weights of the cell-centred transfer operators.
#pragma once

#include "df64.cuh"
#include "h1w_internal.cuh"

namespace h1w {
namespace dfmg {

__device__ __forceinline__ int fv_cls(const Level& L, int i, int j, int k) {
  return ((i > 0) + (i < L.nx - 1)) + 3 * ((j > 0) + (j < L.ny - 1)) + 9 * ((k > 0) + (k < L.nz - 1));
}

__device__ __forceinline__ df dzero() { return df_make(0.f, 0.f); }

// Cascaded summation of double-floats: the high parts are added with TwoSum,
// their rounding errors and the low parts are collected in one float, and the
// result is renormalized once. For the handful of terms summed here the
// error stays near 2^-46 of the largest term. The first term is taken as it is
// (s = hi, e = lo): adding it to an empty sum by TwoSum gives the same two floats
// (up to the sign of a zero) for 8 instructions that IEEE rules keep the compiler
// from removing. Where the adds are unrolled, `first` is known at compile time.
struct dsum {
  float s = 0.f, e = 0.f;
  bool first = true;
  __device__ __forceinline__ void add(df v) {
    if (first) {
      s = v.hi;
      e = v.lo;
      first = false;
      return;
    }
    const df t = two_sum(s, v.hi);
    s = t.hi;
    e = __fadd_rn(e, __fadd_rn(t.lo, v.lo));
  }
  __device__ __forceinline__ df get() const { return fast_two_sum(s, e); }
};

// FV 1D transfer weights (rows of P^T and of P), as in mg_kernels.cu: P takes 3/4 of the
// parent coarse cell and 1/4 of the next one towards the fine cell, and only the parent at
// the ends of an axis (constant extrapolation)
__device__ __forceinline__ int fv_restrict_1d(int I, int nc, int coarsened, int* f, float* w) {
  if (!coarsened) { f[0] = I; w[0] = 1.f; return 1; }
  int c = 0;
  if (I >= 1) { f[c] = 2 * I - 1; w[c++] = 0.25f; }
  f[c] = 2 * I;     w[c++] = (I >= 1) ? 0.75f : 1.f;
  f[c] = 2 * I + 1; w[c++] = (I + 1 < nc) ? 0.75f : 1.f;
  if (I + 1 < nc) { f[c] = 2 * I + 2; w[c++] = 0.25f; }
  return c;
}

__device__ __forceinline__ int fv_prolong_1d(int i, int nc, int coarsened, int* f, float* w) {
  if (!coarsened) { f[0] = i; w[0] = 1.f; return 1; }
  const int I = i >> 1;
  const int J = (i & 1) ? I + 1 : I - 1;
  if (J >= 0 && J < nc) { f[0] = I; w[0] = 0.75f; f[1] = J; w[1] = 0.25f; return 2; }
  f[0] = I; w[0] = 1.f;
  return 1;
}

// weights of row I of the 1D P^T at fine offsets 2I-1, 2I, 2I+1, 2I+2 (0 where absent)
__device__ __forceinline__ void fv_rw(int I, int nc, int coarsened, float* w) {
  if (!coarsened) { w[0] = 0.f; w[1] = 1.f; w[2] = 0.f; w[3] = 0.f; return; }
  w[0] = (I >= 1) ? 0.25f : 0.f;
  w[1] = (I >= 1) ? 0.75f : 1.f;
  w[2] = (I + 1 < nc) ? 0.75f : 1.f;
  w[3] = (I + 1 < nc) ? 0.25f : 0.f;
}

}  // namespace dfmg
}  // namespace h1w
