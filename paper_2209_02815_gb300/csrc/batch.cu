// h1w_solve_batch: many independent H1-regularized Gauss-Newton systems at once.
//
// Each system has its own context (its grid, measurements, workspace and stream) and is
// solved by the same two calls as a single system, h1w_capacitance and h1w_pcg. Those
// calls wait on their own stream (PCG reads its residual norm every iteration), so a
// single host thread would leave the GPU idle between the launches of one system. Here a
// pool of host threads takes the systems off a shared counter, one system per thread at a
// time, and the systems' kernels overlap on their separate streams: the small grids of a
// batch fill the GPU together where one alone cannot.
#include <algorithm>
#include <atomic>
#include <thread>
#include <vector>

#include "h1w_internal.cuh"

extern "C" h1w_status h1w_solve_batch(h1w_ctx* const* ctxs, int32_t count, const int32_t* m,
                                      const double* const* J, const double* const* b, double* const* x,
                                      double rtol, int32_t maxit, int32_t threads, h1w_info* info,
                                      h1w_status* status) {
  if (count < 0 || (count > 0 && (!ctxs || !m || !J || !b || !x)))
    return h1w::set_global_error(H1W_EINVAL, "h1w_solve_batch: NULL arrays or negative count");
  for (int32_t i = 0; i < count; ++i)
    if (!ctxs[i]) return h1w::set_global_error(H1W_EINVAL, "h1w_solve_batch: NULL context");
  if (count == 0) return H1W_OK;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return h1w::set_global_error(H1W_ECUDA, "h1w_solve_batch: no device");
  const int nthreads = std::max(1, std::min<int>(threads > 0 ? threads : 8, count));
  std::atomic<int> next{0};
  std::vector<h1w_status> st(count, H1W_OK);
  auto worker = [&]() {
    cudaSetDevice(dev);  // host threads start on device 0
    for (int i = next.fetch_add(1); i < count; i = next.fetch_add(1)) {
      h1w_status s = h1w_capacitance(ctxs[i], m[i], J[i]);
      if (s == H1W_OK) s = h1w_pcg(ctxs[i], b[i], x[i], rtol, maxit, info ? info + i : nullptr);
      st[i] = s;
    }
  };
  std::vector<std::thread> pool;
  pool.reserve(nthreads - 1);
  for (int t = 1; t < nthreads; ++t) pool.emplace_back(worker);
  worker();
  for (auto& t : pool) t.join();
  h1w_status first = H1W_OK;
  for (int32_t i = 0; i < count; ++i) {
    if (status) status[i] = st[i];
    if (first == H1W_OK && st[i] != H1W_OK) first = st[i];
  }
  if (first != H1W_OK) h1w::set_global_error(first, "h1w_solve_batch: a system failed (see its context's last error)");
  return first;
}
