// h1w_apply_op_static: the system operator q = alpha (K + M) p + J^T (J p)
// for callers that cannot allocate device memory.
//
// The regular entry points take their scratch from a workspace the caller
// allocates. Some callers cannot do that: code whose device memory is owned
// by another allocator (a framework's caching pool or a fixed-size arena
// planned ahead of time) and that must not call cudaMalloc itself, because
// cudaMalloc synchronizes the whole device and takes memory outside that
// budget. For them this entry point keeps its scratch (the per-chunk partial
// sums of J p, the m-vector J p and, for Q1 grids, the 1D element
// coefficients) in one file-scope __device__ array of fixed size, which every
// GPU that loads the library holds until the process exits. It calls no
// cudaMalloc, cudaFree or allocating library routine.
//
// Host code only ever sees a host-side stand-in under the array's name, so
// the device address is looked up once per device with
// cudaGetSymbolAddress, with that device current, and passed to the kernels.
#include <mutex>
#include <string>

#include "h1w_internal.cuh"

namespace h1w {
namespace {

constexpr int64_t kStaticScratchDoubles = int64_t(1) << 20;  // 8 MiB per device
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_static_scratch[kStaticScratchDoubles];

std::mutex g_scratch_mu;
double* g_scratch_dev[kMaxDevices] = {};

// Fine-level Q1 1D factors [Kd, Ko, Md, Mo, Dd, Do] of linear elements with
// natural boundary conditions (the same values the context's setup uploads).
__global__ void k_q1_fine_coeffs(int n, double h, double* q) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const bool end = (i == 0 || i == n - 1);
  q[0 * n + i] = (end ? 1.0 : 2.0) / h;
  q[2 * n + i] = (end ? 1.0 : 2.0) * h / 3.0;
  q[4 * n + i] = (end ? 0.5 : 1.0) * h;
  q[1 * n + i] = (i < n - 1) ? -1.0 / h : 0.0;
  q[3 * n + i] = (i < n - 1) ? h / 6.0 : 0.0;
  q[5 * n + i] = 0.0;
}

int64_t round256(int64_t doubles) { return (doubles + 31) / 32 * 32; }

}  // namespace
}  // namespace h1w

using namespace h1w;

extern "C" h1w_status h1w_apply_op_static(const h1w_grid* g, int32_t m, const double* J,
                                          const double* p, double* q, void* stream) {
  if (!g) return set_global_error(H1W_EINVAL, "grid is NULL");
  if (!((g->dim == 2 && g->disc == H1W_Q1_VERTEX) || (g->dim == 3 && g->disc == H1W_FV_CELL)))
    return set_global_error(H1W_EUNSUPPORTED, "supported: dim 2 with H1W_Q1_VERTEX, dim 3 with H1W_FV_CELL");
  int64_t N = 1;
  for (int a = 0; a < g->dim; ++a) {
    if (g->n[a] < 2 || !(g->h[a] > 0.0)) return set_global_error(H1W_EINVAL, "bad grid size or spacing");
    N *= g->n[a];
  }
  if (!(g->alpha > 0.0)) return set_global_error(H1W_EINVAL, "alpha must be positive");
  if (m < 0 || m > kMaxM) return set_global_error(H1W_EINVAL, "m out of range [0, 4096]");
  if (!p || !q || p == q || (m > 0 && !J))
    return set_global_error(H1W_EINVAL, "p, q (distinct) and J (when m > 0) must be non-NULL");

  // layout of the static scratch for this call
  const int64_t chunks = rows_dot_chunks(N);
  const int64_t off_w = round256(chunks * (m > 0 ? m : 0));
  const int64_t off_q = off_w + round256(m > 0 ? m : 1);
  const int64_t nq = (g->disc == H1W_Q1_VERTEX) ? 6 * (int64_t)(g->n[0] + g->n[1]) : 0;
  const int64_t need = off_q + nq;
  if (need > kStaticScratchDoubles)
    return set_global_error(
        H1W_EINVAL, "h1w_apply_op_static: grid and m need " + std::to_string(need) +
                        " doubles of static scratch, more than its fixed size of " +
                        std::to_string(kStaticScratchDoubles) +
                        " (use h1w_setup with a workspace instead)");

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_global_error(H1W_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return set_global_error(H1W_EUNSUPPORTED, "device index beyond 63");
  double* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_dev[dev]) {
      void* ptr = nullptr;
      e = cudaGetSymbolAddress(&ptr, g_static_scratch);
      if (e != cudaSuccess)
        return set_global_error(H1W_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_scratch_dev[dev] = static_cast<double*>(ptr);
    }
    base = g_scratch_dev[dev];
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  double* partial = base;
  double* w = base + off_w;
  Level L{};
  L.nx = g->n[0];
  L.ny = g->n[1];
  L.nz = g->dim == 3 ? g->n[2] : 1;
  L.N = N;
  if (g->disc == H1W_FV_CELL) {
    const double hx = g->h[0], hy = g->h[1], hz = g->h[2];
    L.Tx = hy * hz / hx; L.Ty = hx * hz / hy; L.Tz = hx * hy / hz; L.V = hx * hy * hz;
    L.iso = (L.Tx == L.Ty && L.Ty == L.Tz) ? 1 : 0;
    for (int cz = 0; cz < 3; ++cz)
      for (int cy = 0; cy < 3; ++cy)
        for (int cx = 0; cx < 3; ++cx)
          L.fv_diag[cx + 3 * cy + 9 * cz] = L.V + L.Tx * cx + L.Ty * cy + L.Tz * cz;
  } else {
    double* qx = base + off_q;
    double* qy = qx + 6 * (int64_t)L.nx;
    k_q1_fine_coeffs<<<(L.nx + 127) / 128, 128, 0, s>>>(L.nx, g->h[0], qx);
    k_q1_fine_coeffs<<<(L.ny + 127) / 128, 128, 0, s>>>(L.ny, g->h[1], qy);
    note_launches(2);
    L.qx = qx;
    L.qy = qy;
  }
  // Every partial sum and every entry of w is written before it is read, so
  // no part of the scratch needs clearing between calls.
  if (m > 0) {
    launch_rows_dot(J, m, N, p, partial, s);
    launch_reduce_partials(partial, (int)chunks, m, 1.0, w, s);
  }
  launch_apply_op(g->disc, L, g->alpha, p, 1.0, J, w, m, q, nullptr, nullptr, s);
  e = cudaGetLastError();
  if (e != cudaSuccess) return set_global_error(H1W_ECUDA, std::string("h1w_apply_op_static: ") + cudaGetErrorString(e));
  return H1W_OK;
}
