/*
 * FP64 CPU oracle: operator apply and unpreconditioned conjugate gradients.
 * TEST INFRASTRUCTURE ONLY: used by the test suite, smoke() and the CPU
 * baseline legs of bench.py; the product library never links it.
 *
 * Operator (the Gauss-Newton system of Eq. 2.9 scaled by beta, with the mass
 * term; alpha is the paper's beta):
 *     q = alpha * (K + M) p + J^T (J p)
 * with K + M an assembled CSR matrix and J a dense m x N row-major matrix.
 * J^T J is never formed (Sec. 3.2, complexity discussion).
 *
 * CG: plain conjugate gradients from x0 = 0, stopping when the recursively
 * updated residual satisfies ||r||_2 <= rtol ||b||_2 (the Euclidean rule used
 * for the paper's experiments, Sec. 4).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int h1wo_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* q = alpha * A p + J^T (J p); w (length m) is scratch owned by the caller. */
void h1wo_apply(int64_t N, const int64_t* indptr, const int64_t* indices, const double* data,
                double alpha, int64_t m, const double* J, const double* p, double* q, double* w) {
  for (int64_t i = 0; i < m; ++i) {
    const double* row = J + i * N;
    double s = 0.0;
#pragma omp parallel for reduction(+ : s) schedule(static)
    for (int64_t k = 0; k < N; ++k) s += row[k] * p[k];
    w[i] = s;
  }
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < N; ++k) {
    double acc = 0.0;
    for (int64_t e = indptr[k]; e < indptr[k + 1]; ++e) acc += data[e] * p[indices[e]];
    double jt = 0.0;
    for (int64_t i = 0; i < m; ++i) jt += J[i * N + k] * w[i];
    q[k] = alpha * acc + jt;
  }
}

static double dot(int64_t N, const double* a, const double* b) {
  double s = 0.0;
#pragma omp parallel for reduction(+ : s) schedule(static)
  for (int64_t k = 0; k < N; ++k) s += a[k] * b[k];
  return s;
}

/* Unpreconditioned CG. Returns iterations; *relres = final recursive ||r||/||b||.
 * x (output) and r, p, q (scratch, length N), w (scratch, length m) are caller-owned. */
int64_t h1wo_cg(int64_t N, const int64_t* indptr, const int64_t* indices, const double* data,
                double alpha, int64_t m, const double* J, const double* b, double rtol,
                int64_t maxit, double* x, double* r, double* p, double* q, double* w,
                double* relres) {
  memset(x, 0, sizeof(double) * N);
  memcpy(r, b, sizeof(double) * N);
  memcpy(p, b, sizeof(double) * N);
  double bnorm = sqrt(dot(N, b, b));
  double rr = bnorm * bnorm;
  int64_t it = 0;
  if (bnorm == 0.0) { *relres = 0.0; return 0; }
  while (it < maxit && sqrt(rr) > rtol * bnorm) {
    h1wo_apply(N, indptr, indices, data, alpha, m, J, p, q, w);
    double a = rr / dot(N, p, q);
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < N; ++k) { x[k] += a * p[k]; r[k] -= a * q[k]; }
    double rr_new = dot(N, r, r);
    double beta = rr_new / rr;
    rr = rr_new;
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < N; ++k) p[k] = r[k] + beta * p[k];
    ++it;
  }
  *relres = sqrt(rr) / bnorm;
  return it;
}
