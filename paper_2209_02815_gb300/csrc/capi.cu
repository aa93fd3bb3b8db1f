// Host runtime and C ABI of h1w: workspace planning, multigrid hierarchy
// construction, the batched V-cycle driver, the capacitance setup (lines H,
// C, chol of Algorithm "MINRES with the Laplace-Woodbury preconditioner"),
// the Woodbury preconditioner apply (Sec. 3.2) and the PCG driver with the
// Euclidean stopping rule of Sec. 4. All device memory comes from the
// caller's workspace; nothing here allocates device memory.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <new>
#include <string>
#include <vector>

#include "h1w_internal.cuh"

using namespace h1w;

std::atomic<long long> h1w::g_kernel_launches{0};

namespace {

thread_local std::string g_setup_error;

struct Bump {
  char* base;   // nullptr while sizing
  size_t off = 0;
  template <class T>
  T* take(size_t count) {
    off = (off + 255) & ~size_t(255);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += sizeof(T) * (count ? count : 1);
    return p;
  }
};

struct LevelBufs {
  double *x, *b, *r, *da, *db;
};

// One set of row-batch copies of J from page-locked host memory into a device buffer
// (h1w_capacitance_from_host, h1w_prefetch_J). The events are recorded on the copy stream
// around each batch's copy; the capacitance that consumes the set waits on end[b] before
// batch b's V-cycles.
struct HostCopy {
  const double* host = nullptr;
  const double* dev = nullptr;
  int m = 0;
  bool active = false;
  bool prefetched = false;   // issued by h1w_prefetch_J, ahead of the capacitance that consumes it
  std::vector<int> edge;
  std::vector<cudaEvent_t> beg, end;
};

}  // namespace

struct h1w_ctx {
  h1w_grid grid;
  h1w_options opt;
  int disc;
  int m_max;
  cudaStream_t stream;
  int nlev;
  Level lev[kMaxLevels];
  ChebCoef cheb[kMaxLevels];
  FusedCoef fco[kMaxLevels];
  LevelBufs buf[kMaxLevels];
  std::vector<double> qhost[kMaxLevels][2];  // Q1 1D coefficients (host copy)
  double* qdev;          // Q1 coefficients, all levels
  df* q1st;              // Q1 double-float stencil tables, all levels
  double* coarse_X;      // dense inverse of the coarsest operator
  double* coarse_L;      // scratch for its factorization
  int* dstatus;          // device status word
  unsigned long long* dbits;
  // capacitance state
  int m;                 // current number of measurements (-1: none yet)
  const double* J;       // borrowed
  double* H;             // m_max x N (FP64 paths only)
  df* Hdf;               // m_max x N, H as double-floats (double-float V-cycle only)
  df* Jdf;               // m_max x N, J as double-floats for the cycle and the Krylov passes
  df* vdf;               // N, a vector converted to double-floats
  double* C;             // m_max x m_max
  double* Lc;            // m_max x m_max
  double* gemm_partial;
  int64_t gemm_partial_len;
  OzakiWork oz;                  // tensor-core capacitance buffers (cap_gemm = 0)
  std::vector<int> oz_tiles_host;
  int oz_tiles_m = -1;           // m of the tile list on the device
  // Krylov vectors
  double *r, *z, *z0, *p, *q;
  double *svec, *jz, *w, *wtmp;
  double* partial;       // reductions over N (per-block)
  int64_t partial_len;
  double* scal;          // scalar slots
  // phase timing: 0 H start, 1 H end / C start, 2 C end, 3 chol end, 4 pcg start, 5 pcg end
  cudaEvent_t ev[6];
  bool have_ev;
  // per-kernel timing: event pairs around selected launches, summed per category
  static constexpr int kTimed = 1024;
  cudaEvent_t kev[kTimed][2];
  int kcat[kTimed];
  int nk;
  bool timing_on;
  bool time_vc = false;  // record the finest-level fused V-cycle kernels (line H only)
  int num_sms = 152;     // SMs of the context's device
  int* trsv_flags = nullptr;  // per-block flags of the cooperative C^-1 solve
  int trsv_epoch = 0;
  unsigned long long wait_ns = 1000000000ull;  // limit of every bounded device wait
  int stall = H1W_STALL_NONE;                  // failure-path test injection (h1w_inject_stall)
  // device-driven PCG: the loop as a CUDA graph with a conditional while node
  bool capturing = false;       // launches are being captured: no per-kernel timing, no host reads
  int* gflags = nullptr;        // flags of the cooperative C^-1 solve inside graphs
  int* gepoch = nullptr;        // device epoch counter for them
  double* gb = nullptr;         // right-hand side and solution of the single-system graph
  double* gx = nullptr;
  cudaStream_t body_stream = nullptr;  // captures the loop body
  cudaStream_t cap_stream = nullptr;   // captures the graphs (the context's stream may be the legacy one)
  // cached single-system graphs: two, so that a caller alternating between two device copies
  // of J (double-buffered host copies) finds both; the true residual bakes J's address in
  struct PcgGraph {
    cudaGraphExec_t exec = nullptr;
    int m = -1;
    const double* J = nullptr;
    int stall = 0;
    unsigned long long wait = 0;
    long long l_pre = 0, l_body = 0, l_post = 0;
    unsigned long long used = 0;  // last use, for replacing the older one
  } pcg_g[2];
  int pcg_cur = 0;              // the entry pcg_graph_ready chose
  unsigned long long pcg_clock = 0;
  long long pcg_l_pre = 0, pcg_l_body = 0, pcg_l_post = 0;  // kernels per part of the last captured graph
  unsigned long long uid = 0;   // process-unique id (batch graph cache keys)
  cudaStream_t copy_stream = nullptr;   // host-to-device copies of h1w_capacitance_from_host
  HostCopy hcopy[2];                     // pending or running copies of J (at most two)
  cudaEvent_t order_ev = nullptr;        // orders a copy after the work queued on the stream
  std::vector<cudaEvent_t> cyc_beg, cyc_end;  // per row batch: its V-cycles start and end
  // profile of the last h1w_capacitance_from_host, ms from the start of its line H
  std::vector<int> prof_rows;
  std::vector<float> prof_copy_beg, prof_copy_end, prof_cyc_beg, prof_cyc_end;
  cudaStream_t cycle_stream = nullptr;  // the preconditioner's V-cycle, beside its H^T r pass
  cudaEvent_t cycle_ev[2] = {};
  float cat_ms[16];
  int cat_n[16];
  long long launches_cap, launches_pcg;
  std::string err;
};

namespace {

}  // namespace

h1w_status h1w::set_global_error(h1w_status st, const std::string& msg) {
  g_setup_error = msg;
  return st;
}

namespace {

enum { kCatGemm = 0, kCatJdot = 1, kCatOp = 2, kCatHdot = 3, kCatHupd = 4, kCatDown = 5, kCatUp = 6,
       kCatSplitJ = 7, kCatSplitH = 8, kCatD2df = 9, kCatCount = 10 };

void timed_begin(h1w_ctx* c) {
  if (c->timing_on && !c->capturing && c->have_ev && c->nk < h1w_ctx::kTimed)
    cudaEventRecord(c->kev[c->nk][0], c->stream);
}
void timed_end(h1w_ctx* c, int cat) {
  if (c->timing_on && !c->capturing && c->have_ev && c->nk < h1w_ctx::kTimed) {
    cudaEventRecord(c->kev[c->nk][1], c->stream);
    c->kcat[c->nk++] = cat;
  }
}
// after the stream has been synchronized: add the recorded pairs into the
// category sums, first clearing the categories in reset_mask
void timed_collect(h1w_ctx* c, unsigned reset_mask) {
  for (int k = 0; k < kCatCount; ++k)
    if (reset_mask & (1u << k)) { c->cat_ms[k] = 0.f; c->cat_n[k] = 0; }
  for (int t = 0; t < c->nk; ++t) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c->kev[t][0], c->kev[t][1]) == cudaSuccess) {
      c->cat_ms[c->kcat[t]] += ms;
      c->cat_n[c->kcat[t]] += 1;
    }
  }
  c->nk = 0;
  cudaGetLastError();
}

h1w_status fail(h1w_ctx* c, h1w_status st, const std::string& msg) {
  if (c) c->err = msg;
  else g_setup_error = msg;
  return st;
}

h1w_status cuda_check(h1w_ctx* c, const char* where) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    return fail(c, H1W_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
  return H1W_OK;
}

void q1_fine_1d(int n, double h, std::vector<double>& q) {
  // [Kd, Ko, Md, Mo, Dd, Do] for linear elements with natural boundary conditions
  q.assign(6 * (size_t)n, 0.0);
  for (int i = 0; i < n; ++i) {
    const bool end = (i == 0 || i == n - 1);
    q[0 * n + i] = (end ? 1.0 : 2.0) / h;
    q[2 * n + i] = (end ? 1.0 : 2.0) * h / 3.0;
    q[4 * n + i] = (end ? 0.5 : 1.0) * h;
    if (i < n - 1) {
      q[1 * n + i] = -1.0 / h;
      q[3 * n + i] = h / 6.0;
      q[5 * n + i] = 0.0;
    }
  }
}

// 1D Q1 prolongation entries of fine vertex f: (coarse index, weight)
int q1_p_entries(int f, int nf, int nc, int* I, double* w) {
  if ((f & 1) == 0) { I[0] = f >> 1; w[0] = 1.0; return 1; }
  if (f == nf - 1) { I[0] = nc - 1; w[0] = 1.0; return 1; }
  I[0] = (f - 1) >> 1; w[0] = 0.5;
  I[1] = (f + 1) >> 1; w[1] = 0.5;
  return 2;
}

// Galerkin product P^T T P of the three tridiagonal pairs in q (size nf -> nc)
void q1_coarse_1d(const std::vector<double>& q, int nf, int nc, std::vector<double>& out) {
  out.assign(6 * (size_t)nc, 0.0);
  for (int t = 0; t < 3; ++t) {
    const double* d = q.data() + (2 * t) * nf;
    const double* o = q.data() + (2 * t + 1) * nf;
    double* cd = out.data() + (2 * t) * nc;
    double* co = out.data() + (2 * t + 1) * nc;
    for (int f = 0; f < nf; ++f) {
      int If[2]; double wf[2];
      const int nfe = q1_p_entries(f, nf, nc, If, wf);
      for (int g = std::max(0, f - 1); g <= std::min(nf - 1, f + 1); ++g) {
        const double tfg = (g == f) ? d[f] : (g > f ? o[f] : o[g]);
        if (tfg == 0.0) continue;
        int Ig[2]; double wg[2];
        const int nge = q1_p_entries(g, nf, nc, Ig, wg);
        for (int a = 0; a < nfe; ++a)
          for (int b = 0; b < nge; ++b) {
            const int I = If[a], Jc = Ig[b];
            const double v = wf[a] * tfg * wg[b];
            if (I == Jc) cd[I] += v;
            else if (Jc == I + 1) co[I] += 0.5 * v;   // (I, I+1) and (I+1, I) both land here
            else if (I == Jc + 1) co[Jc] += 0.5 * v;
          }
      }
    }
  }
}

// The longest index range around the middle of a 1D Q1 factor set q = [Kd, Ko, Md, Mo, Dd, Do]
// (n entries each) on which every vertex's entries (diagonal, and the couplings to both
// neighbours) equal the middle vertex's bit for bit; the end vertices are never included
// (they lack a neighbour). Empty (lo > hi) when n < 3.
void q1_uniform_range(const std::vector<double>& q, int n, int& lo, int& hi) {
  lo = 1;
  hi = 0;
  if (n < 3) return;
  auto same = [&](int i, int r) {
    for (int t = 0; t < 3; ++t) {
      const double* d = q.data() + (2 * t) * n;
      const double* o = q.data() + (2 * t + 1) * n;
      if (std::memcmp(&d[i], &d[r], sizeof(double)) || std::memcmp(&o[i], &o[r], sizeof(double)) ||
          std::memcmp(&o[i - 1], &o[r - 1], sizeof(double)))
        return false;
    }
    return true;
  };
  const int r = n / 2;
  lo = hi = r;
  while (lo - 1 >= 1 && same(lo - 1, r)) --lo;
  while (hi + 1 <= n - 2 && same(hi + 1, r)) ++hi;
}

struct Plan {
  int nlev = 0;
  int n[kMaxLevels][3];
  double h[kMaxLevels][3];
  int c[kMaxLevels][3];
  bool ok = false;
  std::string why;
};

Plan plan_levels(const h1w_grid& g) {
  Plan P;
  int n[3] = {g.n[0], g.n[1], g.dim == 3 ? g.n[2] : 1};
  double h[3] = {g.h[0], g.h[1], g.dim == 3 ? g.h[2] : 1.0};
  for (int l = 0; l < kMaxLevels; ++l) {
    for (int a = 0; a < 3; ++a) { P.n[l][a] = n[a]; P.h[l][a] = h[a]; P.c[l][a] = 0; }
    P.nlev = l + 1;
    const int64_t N = (int64_t)n[0] * n[1] * n[2];
    if (N <= kCoarseTarget) break;
    bool any = false;
    int nn[3] = {n[0], n[1], n[2]};
    for (int a = 0; a < g.dim; ++a) {
      bool co;
      if (g.disc == H1W_Q1_VERTEX) co = n[a] >= 3;
      else co = (n[a] % 2 == 0) && n[a] >= 4;
      if (co) {
        P.c[l][a] = 1;
        any = true;
        nn[a] = (g.disc == H1W_Q1_VERTEX) ? ((n[a] - 1) / 2 + 1 + ((n[a] - 1) % 2)) : n[a] / 2;
        h[a] *= 2.0;
      }
    }
    if (!any) break;
    if (l == kMaxLevels - 1) { P.why = "too many multigrid levels"; return P; }
    for (int a = 0; a < 3; ++a) n[a] = nn[a];
  }
  const int l = P.nlev - 1;
  const int64_t Nc = (int64_t)P.n[l][0] * P.n[l][1] * P.n[l][2];
  if (Nc > kCoarseLimit) {
    P.why = "grid cannot be coarsened to <= 1024 unknowns (coarsest has " + std::to_string(Nc) + ")";
    return P;
  }
  P.ok = true;
  return P;
}

// Interval ratio of the Chebyshev smoother: the caller's, else the discretization's (the
// ratios that gave the fewest PCG iterations over isotropic and anisotropic grids of each kind).
double cheb_ratio_of(int disc, const h1w_options& o) {
  if (o.cheb_ratio > 0.0) return o.cheb_ratio;
  return disc == H1W_Q1_VERTEX ? 6.0 : 10.0;
}

h1w_status validate(const h1w_grid* g, int32_t m_max, const h1w_options* o, std::string& why) {
  if (!g) { why = "grid is NULL"; return H1W_EINVAL; }
  if (!((g->dim == 2 && g->disc == H1W_Q1_VERTEX) || (g->dim == 3 && g->disc == H1W_FV_CELL))) {
    why = "supported: dim 2 with H1W_Q1_VERTEX, dim 3 with H1W_FV_CELL";
    return H1W_EUNSUPPORTED;
  }
  for (int a = 0; a < g->dim; ++a) {
    if (g->n[a] < 2 || g->n[a] > (1 << 20)) { why = "n out of range"; return H1W_EINVAL; }
    if (!(g->h[a] > 0.0) || !std::isfinite(g->h[a])) { why = "h must be positive"; return H1W_EINVAL; }
  }
  if (g->dim == 2 && g->n[2] != 1) { why = "n[2] must be 1 in 2D"; return H1W_EINVAL; }
  if (!(g->alpha > 0.0) || !std::isfinite(g->alpha)) { why = "alpha must be positive"; return H1W_EINVAL; }
  if (m_max < 0 || m_max > kMaxM) { why = "m_max out of range [0, 4096]"; return H1W_EINVAL; }
  if (o) {
    if (o->cheb_degree < 1 || o->cheb_degree > 7) { why = "cheb_degree out of range [1, 7]"; return H1W_EINVAL; }
    if (o->rhs_block < 1 || o->rhs_block > 256) { why = "rhs_block out of range [1, 256]"; return H1W_EINVAL; }
    if (o->max_restarts < 0 || o->max_restarts > 100) { why = "max_restarts out of range"; return H1W_EINVAL; }
    if (o->cap_gemm != 0 && o->cap_gemm != 1) { why = "cap_gemm must be 0 or 1"; return H1W_EINVAL; }
    if (o->mg_arith != 0 && o->mg_arith != 1) { why = "mg_arith must be 0 or 1"; return H1W_EINVAL; }
    if (o->mg_unfused != 0 && o->mg_unfused != 1) { why = "mg_unfused must be 0 or 1"; return H1W_EINVAL; }
    if (o->precond != 0 && o->precond != 1) { why = "precond must be 0 or 1"; return H1W_EINVAL; }
    if (o->pcg_mode != 0 && o->pcg_mode != 1) { why = "pcg_mode must be 0 or 1"; return H1W_EINVAL; }
    if (o->j_digits != 0 && o->j_digits != 1) { why = "j_digits must be 0 or 1"; return H1W_EINVAL; }
    if (!(o->cheb_ratio == 0.0 || (o->cheb_ratio >= 1.5 && o->cheb_ratio <= 1000.0))) {
      why = "cheb_ratio neither 0 nor in [1.5, 1000]";
      return H1W_EINVAL;
    }
  }
  return H1W_OK;
}

int64_t gemm_partial_len(int m_max, int64_t N, bool ozaki) {
  int64_t best = 1;
  for (int m = 1; m <= m_max; ++m) {
    best = std::max(best, (int64_t)cap_gemm_splits(m, N) * m * m);
    if (ozaki)  // any SM count: the setup uses the device's own
      best = std::max(best, (int64_t)ozaki_max_splits(m) * m * m);
  }
  return best;
}

// right-hand sides per batched V-cycle: the option, but no more than the capacitance
// phase ever batches (m_max rows), so small-m contexts do not size buffers for 128
int block_rhs(const h1w_options& o, int m_max) { return std::max(1, std::min(o.rhs_block, m_max)); }

// Lays out every buffer; with ctx->... pointers filled when base != nullptr.
size_t layout(h1w_ctx* c, const Plan& P, const h1w_grid& g, int m_max, const h1w_options& o,
              char* base) {
  Bump B{base};
  const int nb = block_rhs(o, m_max);
  const int64_t N0 = (int64_t)P.n[0][0] * P.n[0][1] * P.n[0][2];
  int64_t qlen = 0;
  for (int l = 0; l < P.nlev; ++l) qlen += 6 * (int64_t)(P.n[l][0] + P.n[l][1]);
  double* qdev = B.take<double>(g.disc == H1W_Q1_VERTEX ? qlen : 1);
  int64_t stlen = 1;
  if (g.disc == H1W_Q1_VERTEX && o.mg_arith == 0) {
    stlen = 0;
    for (int l = 0; l < P.nlev; ++l) stlen += 10 * (int64_t)P.n[l][0] * P.n[l][1] * P.n[l][2];
  }
  df* q1st = B.take<df>(stlen);
  LevelBufs bufs[kMaxLevels];
  // the fused legs on the finest level read b from the caller and write x only: its r, b
  // and Chebyshev vectors are then not needed
  const bool fused0 = (g.disc == H1W_FV_CELL) && o.mg_arith == 0 && o.mg_unfused == 0 && o.cheb_degree == 2 &&
                      P.nlev > 1 && P.c[0][0] && P.c[0][1] && P.c[0][2] &&
                      (int64_t)P.n[0][0] * P.n[0][1] < (int64_t(1) << 26);
  for (int l = 0; l < P.nlev; ++l) {
    const int64_t Nl = (int64_t)P.n[l][0] * P.n[l][1] * P.n[l][2];
    const int64_t nw = (l == 0 && fused0) ? 1 : nb * Nl;
    bufs[l].x = B.take<double>(nb * Nl);  // level 0: used by the double-float cycle
    bufs[l].b = B.take<double>(nw);
    bufs[l].r = B.take<double>(nw);
    bufs[l].da = B.take<double>(nw);
    bufs[l].db = B.take<double>(nw);
  }
  const int l = P.nlev - 1;
  const int64_t Nc = (int64_t)P.n[l][0] * P.n[l][1] * P.n[l][2];
  double* cX = B.take<double>(Nc * Nc);
  double* cL = B.take<double>(Nc * Nc);
  int* dstatus = B.take<int>(4);
  int* tflags = B.take<int>(2 * ((m_max + 31) / 32 + 1));
  int* gflags = B.take<int>(2 * ((m_max + 31) / 32 + 1) + 1);  // graph flags, then the epoch counter
  unsigned long long* dbits = B.take<unsigned long long>(4);
  const bool use_df = o.mg_arith == 0;
  // FP64 H: not needed when the cycle is double-float and C runs on the tensor cores
  double* H = B.take<double>((use_df && o.cap_gemm == 0) ? 1 : (int64_t)m_max * N0);
  df* Hdf = use_df ? B.take<df>((int64_t)m_max * N0) : nullptr;
  df* Jdf = use_df ? B.take<df>((int64_t)m_max * N0) : nullptr;
  df* vdf = use_df ? B.take<df>(N0) : nullptr;
  double* C = B.take<double>((int64_t)m_max * m_max);
  double* Lc = B.take<double>((int64_t)m_max * m_max);
  const bool oz = (o.cap_gemm == 0) && m_max > 0;
  const int64_t gpl = gemm_partial_len(m_max, N0, oz);
  double* gp = B.take<double>(gpl);
  const long long kp = ozaki_panel_width(N0);
  OzakiWork ow{};
  if (oz) {
    // the digits of J for every K panel when they fit the cap: line H then splits J as it
    // converts it to double-floats, and line C reads J no more (one pass over J saved)
    const size_t jfull = ozaki_j_digits_full_bytes(m_max, N0);
    ow.j_full = o.j_digits == 1 && use_df && o.precond == 0 && jfull <= (size_t)kJDigitsFullMax;
    ow.digitsA = ow.j_full ? static_cast<void*>(B.take<uint8_t>(jfull))
                           : static_cast<void*>(B.take<uint16_t>((size_t)ozaki_digit_slices() * ((m_max + 127) / 128 * 128) * kp));
    ow.digitsB = B.take<uint16_t>((size_t)ozaki_digit_slices() * ((m_max + 63) / 64 * 64) * kp);
    ow.expo = B.take<int>(2 * (size_t)m_max * ozaki_chunks(N0));
    ow.tiles = B.take<int>(2 * (size_t)ozaki_num_tiles(m_max));
    ow.klen = kp;
  }
  double* r = B.take<double>(N0);
  double* z = B.take<double>(N0);
  double* z0 = B.take<double>(N0);
  double* p = B.take<double>(N0);
  double* q = B.take<double>(N0);
  double* svec = B.take<double>(m_max);
  double* jz = B.take<double>(m_max);
  double* w = B.take<double>(m_max);
  double* wtmp = B.take<double>(m_max);
  const int64_t plen = std::max<int64_t>({(int64_t)rows_dot_chunks(N0) * std::max(m_max, 1),
                                          (int64_t)colsum_blocks(N0), (int64_t)dot_blocks(N0)});
  double* partial = B.take<double>(plen);
  double* scal = B.take<double>(16);
  double* gb = B.take<double>(N0);
  double* gx = B.take<double>(N0);
  if (c) {
    c->qdev = qdev;
    c->q1st = q1st;
    for (int k = 0; k < P.nlev; ++k) c->buf[k] = bufs[k];
    c->coarse_X = cX; c->coarse_L = cL; c->dstatus = dstatus; c->dbits = dbits; c->trsv_flags = tflags;
    c->H = H; c->C = C; c->Lc = Lc; c->gemm_partial = gp; c->gemm_partial_len = gpl;
    c->Hdf = Hdf; c->vdf = vdf; c->Jdf = Jdf;
    c->oz = ow;
    c->oz.partial = gp;
    c->oz.status = dstatus;
    c->r = r; c->z = z; c->z0 = z0; c->p = p; c->q = q;
    c->svec = svec; c->jz = jz; c->w = w; c->wtmp = wtmp;
    c->partial = partial; c->partial_len = plen; c->scal = scal;
    c->gflags = gflags; c->gepoch = gflags + 2 * ((m_max + 31) / 32 + 1); c->gb = gb; c->gx = gx;
  }
  return B.off + 256;
}

// ---- multigrid driver -------------------------------------------------------------

void smooth(h1w_ctx* c, int l, int nrhs, const double* b, double* x, bool zero_x) {
  const Level& L = c->lev[l];
  const ChebCoef& K = c->cheb[l];
  double* da = c->buf[l].da;
  double* db = c->buf[l].db;
  launch_cheb_first(c->disc, L, nrhs, b, x, c->buf[l].r, da, zero_x, K.inv_theta, c->stream);
  // with a nonzero start the first correction d_0 is added by the next step
  bool pending = !zero_x;
  for (int j = 1; j < c->opt.cheb_degree; ++j) {
    launch_cheb_step(c->disc, L, nrhs, c->buf[l].r, da, db, x, K.c1[j], K.c2[j], pending, c->stream);
    pending = false;
    std::swap(da, db);
  }
  if (pending) launch_add((int64_t)nrhs * L.N, da, x, c->stream);
}

// x = L-hat^-1 b for nrhs <= rhs_block vectors (b, x: level-0 sized, contiguous)
void vcycle_block(h1w_ctx* c, int nrhs, const double* b0, double* x0) {
  const int nl = c->nlev;
  if (nl == 1) {
    launch_coarse_apply(c->coarse_X, (int)c->lev[0].N, nrhs, b0, x0, c->stream);
    return;
  }
  const double* bp[kMaxLevels];
  double* xp[kMaxLevels];
  bp[0] = b0; xp[0] = x0;
  for (int l = 1; l < nl; ++l) { bp[l] = c->buf[l].b; xp[l] = c->buf[l].x; }
  for (int l = 0; l < nl - 1; ++l) {
    smooth(c, l, nrhs, bp[l], xp[l], true);
    launch_residual(c->disc, c->lev[l], nrhs, bp[l], xp[l], c->buf[l].r, c->stream);
    launch_restrict(c->disc, c->lev[l], c->lev[l + 1], nrhs, c->buf[l].r, c->buf[l + 1].b, c->stream);
  }
  launch_coarse_apply(c->coarse_X, (int)c->lev[nl - 1].N, nrhs, bp[nl - 1], xp[nl - 1], c->stream);
  for (int l = nl - 2; l >= 0; --l) {
    launch_prolong_add(c->disc, c->lev[l], c->lev[l + 1], nrhs, xp[l + 1], xp[l], c->stream);
    smooth(c, l, nrhs, bp[l], xp[l], false);
  }
}

// ---- the same cycle in double-float arithmetic (FV grids) -------------------------

inline df* dfp(double* p) { return reinterpret_cast<df*>(p); }

void smooth_df(h1w_ctx* c, int l, int nrhs, const df* b, df* x, bool zero_x) {
  const Level& L = c->lev[l];
  const ChebCoef& K = c->cheb[l];
  df* r = dfp(c->buf[l].r);
  df* da = dfp(c->buf[l].da);
  df* db = dfp(c->buf[l].db);
  const bool q1 = c->disc == H1W_Q1_VERTEX;
  if (q1 && c->opt.cheb_degree == 2) {  // the two steps in one pass (after the residual, from a nonzero x)
    if (!zero_x) launch_q1_residual_df(L, nrhs, b, x, r, c->stream);
    launch_q1_smooth_df(L, nrhs, zero_x ? b : r, x, zero_x, K.beta_df, K.c2t_df, c->stream);
    return;
  }
  if (q1) launch_q1_cheb_first_df(L, nrhs, b, x, r, da, zero_x, K.inv_theta_df, c->stream);
  else launch_cheb_first_df(L, nrhs, b, x, r, da, zero_x, K.inv_theta_df, c->stream);
  bool pending = !zero_x;
  for (int j = 1; j < c->opt.cheb_degree; ++j) {
    if (q1) launch_q1_cheb_step_df(L, nrhs, r, da, db, x, K.c1_df[j], K.c2_df[j], pending, c->stream);
    else launch_cheb_step_df(L, nrhs, r, da, db, x, K.c1_df[j], K.c2_df[j], pending, c->stream);
    pending = false;
    std::swap(da, db);
  }
  if (pending) launch_add_df((int64_t)nrhs * L.N, da, x, c->stream);
}

// level l smooths with the fused down/up kernels (FV, all axes coarsened, degree-2 smoother)
bool fused_level(const h1w_ctx* c, int l) {
  return c->disc == H1W_FV_CELL && c->opt.mg_unfused == 0 && c->opt.cheb_degree == 2 && l < c->nlev - 1 &&
         fused_level_ok(c->lev[l]);
}

// x = L-hat^-1 b for nrhs <= rhs_block right-hand sides given as double-floats (b0, level-0
// sized, contiguous); the result goes to x64 (FP64) and/or xdf (double-floats).
// Returns false if a fused kernel could not be configured.
bool vcycle_block_df(h1w_ctx* c, int nrhs, const df* b0, const double* b0_64, double* x64, df* xdf) {
  const int nl = c->nlev;
  cudaStream_t s = c->stream;
  const df* bl[kMaxLevels];
  const df* xf[kMaxLevels];
  // FP64 right-hand sides: the fused finest-level kernels split them on the fly; every other
  // consumer gets a double-float copy
  if (b0_64 && !(nl > 1 && fused_level(c, 0))) {
    launch_d2df((int64_t)nrhs * c->lev[0].N, b0_64, dfp(c->buf[0].b), s);
    b0 = dfp(c->buf[0].b);
    b0_64 = nullptr;
  }
  bl[0] = b0;
  for (int l = 1; l < nl; ++l) bl[l] = dfp(c->buf[l].b);
  for (int l = 0; l < nl - 1; ++l) {
    df* x = dfp(c->buf[l].x);
    if (fused_level(c, l)) {
      if (l == 0 && c->time_vc) timed_begin(c);
      const bool ok = (l == 0 && b0_64)
                          ? launch_pre_fused_df(c->lev[0], c->lev[1], c->fco[0], nrhs, b0_64, x, dfp(c->buf[1].b), s)
                          : launch_pre_fused_df(c->lev[l], c->lev[l + 1], c->fco[l], nrhs, bl[l], x,
                                                dfp(c->buf[l + 1].b), s);
      if (!ok) return false;
      if (l == 0 && c->time_vc) timed_end(c, kCatDown);
    } else {
      smooth_df(c, l, nrhs, bl[l], x, true);
      if (c->disc == H1W_Q1_VERTEX) {
        launch_q1_residual_df(c->lev[l], nrhs, bl[l], x, dfp(c->buf[l].r), s);
        launch_q1_restrict_df(c->lev[l], c->lev[l + 1], nrhs, dfp(c->buf[l].r), dfp(c->buf[l + 1].b), s);
      } else {
        launch_residual_df(c->lev[l], nrhs, bl[l], x, dfp(c->buf[l].r), s);
        launch_restrict_df(c->lev[l], c->lev[l + 1], nrhs, dfp(c->buf[l].r), dfp(c->buf[l + 1].b), s);
      }
    }
  }
  launch_coarse_apply_df(c->coarse_X, (int)c->lev[nl - 1].N, nrhs, bl[nl - 1], dfp(c->buf[nl - 1].x), s);
  xf[nl - 1] = dfp(c->buf[nl - 1].x);
  bool written = false;
  for (int l = nl - 2; l >= 0; --l) {
    if (fused_level(c, l)) {
      df* y = (l == 0) ? xdf : dfp(c->buf[l].r);   // r is free on the up leg
      double* y64 = (l == 0) ? x64 : nullptr;
      if (l == 0 && c->time_vc) timed_begin(c);
      const bool ok = (l == 0 && b0_64)
                          ? launch_post_fused_df(c->lev[0], c->lev[1], c->fco[0], nrhs, dfp(c->buf[0].x), xf[1],
                                                 b0_64, y, y64, s)
                          : launch_post_fused_df(c->lev[l], c->lev[l + 1], c->fco[l], nrhs, dfp(c->buf[l].x),
                                                 xf[l + 1], bl[l], y, y64, s);
      if (!ok) return false;
      if (l == 0 && c->time_vc) timed_end(c, kCatUp);
      xf[l] = y;
      written = (l == 0);
    } else {
      df* x = dfp(c->buf[l].x);
      if (c->disc == H1W_Q1_VERTEX) launch_q1_prolong_add_df(c->lev[l], c->lev[l + 1], nrhs, xf[l + 1], x, s);
      else launch_prolong_add_df(c->lev[l], c->lev[l + 1], nrhs, xf[l + 1], x, s);
      smooth_df(c, l, nrhs, bl[l], x, false);
      xf[l] = x;
    }
  }
  if (!written) launch_df2d((int64_t)nrhs * c->lev[0].N, xf[0], x64, xdf, s);
  return true;
}

bool uses_df(const h1w_ctx* c) { return c->opt.mg_arith == 0; }

// x = L-hat^-1 b for nrhs vectors. b comes in FP64 (b64) or, on the double-float cycle,
// as double-floats (bdf, preferred when given). The result goes to x64 and/or, on the
// double-float cycle, xdf. Returns false if a fused kernel could not be configured.
bool vcycle_many(h1w_ctx* c, int nrhs, const double* b64, const df* bdf, double* x64, df* xdf) {
  const int64_t N = c->lev[0].N;
  const int nb = block_rhs(c->opt, c->m_max);
  for (int r0 = 0; r0 < nrhs; r0 += nb) {
    const int nr = std::min(nb, nrhs - r0);
    const int64_t o = (int64_t)r0 * N;
    if (uses_df(c)) {
      if (!vcycle_block_df(c, nr, bdf ? bdf + o : nullptr, bdf ? nullptr : b64 + o, x64 ? x64 + o : nullptr,
                           xdf ? xdf + o : nullptr))
        return false;
    } else {
      vcycle_block(c, nr, b64 + o, x64 + o);
    }
  }
  return true;
}

// w = J v (m-vector), through per-chunk partials
void j_times(h1w_ctx* c, const double* A, const double* v, double* out, double scale = 1.0) {
  const int64_t N = c->lev[0].N;
  if (c->m <= 0) return;
  timed_begin(c);
  launch_rows_dot(A, c->m, N, v, c->partial, c->stream);
  timed_end(c, kCatJdot);
  launch_reduce_partials(c->partial, rows_dot_chunks(N), c->m, scale, out, c->stream);
}

// w = J v through the double-float copy of J (Krylov passes)
void j_times_df(h1w_ctx* c, const double* v, double* out) {
  const int64_t N = c->lev[0].N;
  if (c->m <= 0) return;
  launch_d2df(N, v, c->vdf, c->stream);
  timed_begin(c);
  launch_rows_dot_df(c->Jdf, c->m, N, c->vdf, c->partial, c->stream);
  timed_end(c, kCatJdot);
  launch_reduce_partials(c->partial, rows_dot_df_chunks(N), c->m, 1.0, out, c->stream);
}

// z = P^-1 r; when rz_slot >= 0 also scal[rz_slot] = r . z. False if the cycle could not run.
bool apply_prec_impl(h1w_ctx* c, const double* r, double* z, int rz_slot) {
  const int64_t N = c->lev[0].N;
  const int m = c->opt.precond == 1 ? 0 : c->m;  // Laplace only: z = alpha^-1 L-hat^-1 r
  const bool dfp_ = uses_df(c) && m > 0;
  // z0 = L-hat^-1 r and s = H^T r (with y = C^-1 s) do not depend on each other: on the
  // double-float path the cycle, bound by latency, runs on a second stream while the pass,
  // bound by HBM, runs on the context's; the update z = (z0 - H y / alpha) / alpha joins them
  const bool side = dfp_ && c->cycle_stream;
  if (uses_df(c)) {                                 // r as double-floats: input of the cycle and of H^T r
    launch_d2df(N, r, c->vdf, c->stream);
    if (side) {
      cudaEventRecord(c->cycle_ev[0], c->stream);
      cudaStreamWaitEvent(c->cycle_stream, c->cycle_ev[0], 0);
      const cudaStream_t main = c->stream;
      c->stream = c->cycle_stream;  // every launch of the cycle goes to the context's stream
      const bool ok = vcycle_many(c, 1, nullptr, c->vdf, c->z0, nullptr);
      c->stream = main;
      cudaEventRecord(c->cycle_ev[1], c->cycle_stream);
      if (!ok) {
        cudaStreamWaitEvent(c->stream, c->cycle_ev[1], 0);
        return false;
      }
    } else if (!vcycle_many(c, 1, nullptr, c->vdf, c->z0, nullptr)) {
      return false;
    }
  } else {
    vcycle_many(c, 1, r, nullptr, c->z0, nullptr);
  }
  if (m > 0) {
    if (dfp_) {                                     // s = H^T r (double-float pass)
      timed_begin(c);
      launch_rows_dot_df(c->Hdf, m, N, c->vdf, c->partial, c->stream);
      timed_end(c, kCatHdot);
      launch_reduce_partials(c->partial, rows_dot_df_chunks(N), m, 1.0, c->svec, c->stream);
    } else {
      timed_begin(c);
      launch_rows_dot(c->H, m, N, r, c->partial, c->stream);  // s = H^T r
      timed_end(c, kCatHdot);
      launch_reduce_partials(c->partial, rows_dot_chunks(N), m, 1.0, c->svec, c->stream);
    }
    // y = C^-1 s by the two triangular solves: backward stable, so the Woodbury formula sees
    // C + dC with |dC| ~ eps |C|. A product with an explicitly formed C^-1 is not (each
    // column carries its own rounding), which for |C| ~ 1e10 breaks the preconditioner.
    bool coop = false;
    if (c->capturing) {  // replayed graphs: the epoch lives on the device and advances per solve
      launch_bump(c->gepoch, c->stream);
      coop = launch_chol_solve_coop(c->Lc, m, c->svec, c->gflags, 0, c->gepoch, c->dstatus, c->wait_ns,
                                    c->stall == H1W_STALL_PREC_SOLVE ? 1 : 0, c->stream);
    } else {
      if (c->trsv_epoch == 0x7FFFFFFF) {  // flags hold epochs 1 .. 2^31 - 1
        cudaMemsetAsync(c->trsv_flags, 0, sizeof(int) * 2 * ((c->m_max + 31) / 32 + 1), c->stream);
        c->trsv_epoch = 0;
      }
      coop = launch_chol_solve_coop(c->Lc, m, c->svec, c->trsv_flags, ++c->trsv_epoch, nullptr, c->dstatus,
                                    c->wait_ns, c->stall == H1W_STALL_PREC_SOLVE ? 1 : 0, c->stream);
    }
    if (!coop) {
      launch_trsv_lower(c->Lc, m, c->svec, 1, c->stream);
      launch_trsv_upper_t(c->Lc, m, c->svec, 1, c->stream);
    }
  }
  if (side) cudaStreamWaitEvent(c->stream, c->cycle_ev[1], 0);  // z0 is ready
  timed_begin(c);
  int nparts = colsum_blocks(N);
  if (dfp_)
    nparts = launch_woodbury_update_df(c->Hdf, m, N, c->svec, c->z0, c->grid.alpha, z, rz_slot >= 0 ? r : nullptr,
                                       rz_slot >= 0 ? c->partial : nullptr, c->stream);
  else
    launch_woodbury_update(c->H, m, N, c->svec, c->z0, c->grid.alpha, z, rz_slot >= 0 ? r : nullptr,
                           rz_slot >= 0 ? c->partial : nullptr, c->stream);
  timed_end(c, kCatHupd);
  if (rz_slot >= 0) launch_sum_to_scalar(c->partial, nparts, c->scal + rz_slot, c->stream);
  return true;
}

// q = alpha (K+M) p + J^T w with w = J p given; scal[pq_slot] = p . q when pq_slot >= 0
void apply_op_w(h1w_ctx* c, const double* p, const double* w, double* q, int pq_slot, bool krylov = false) {
  int nb = 0;
  timed_begin(c);
  if (krylov && uses_df(c) && c->m > 0)
    launch_apply_op_df(c->disc, c->lev[0], c->grid.alpha, p, 1.0, c->Jdf, w, c->m, q,
                       pq_slot >= 0 ? c->partial : nullptr, &nb, c->stream);
  else
    launch_apply_op(c->disc, c->lev[0], c->grid.alpha, p, 1.0, c->J, w, c->m > 0 ? c->m : 0, q,
                    pq_slot >= 0 ? c->partial : nullptr, &nb, c->stream);
  timed_end(c, kCatOp);
  if (pq_slot >= 0) launch_sum_to_scalar(c->partial, nb, c->scal + pq_slot, c->stream);
}

double read_scalar(h1w_ctx* c, int slot) {
  double v = 0.0;
  cudaMemcpyAsync(&v, c->scal + slot, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  cudaStreamSynchronize(c->stream);
  return v;
}

// Enqueues on c->stream, which must be capturing into a graph, the whole PCG solve of
// A x = b driven from the device: x = 0 and r = b (unless slot init is 0: a restart from
// the true residual already in r), b.b and r.r, the loop as a conditional while node whose
// body is one PCG iteration ending with the convergence test, and the FP64 true residual
// r = b - A x with r.r in slot 11. Returns false when a graph call fails (text in c->err).
bool capture_pcg(h1w_ctx* c, const double* b, double* x, bool clear_status) {
  const int64_t N = c->lev[0].N;
  const int m = c->m;
  const cudaStream_t s = c->stream;
  const long long l0 = g_kernel_launches.load();
  // bounded waits of the C^-1 solves report in the status word (kept when the capacitance of
  // the same graph has written to it)
  if (clear_status) cudaMemsetAsync(c->dstatus, 0, sizeof(int), s);
  launch_pcg_init(x, c->r, b, c->scal, N, s);
  launch_dot_partial(b, b, N, c->partial, s);
  launch_sum_to_scalar(c->partial, dot_blocks(N), c->scal + kSlotBB, s);
  launch_dot_partial(c->r, c->r, N, c->partial, s);
  launch_sum_to_scalar(c->partial, dot_blocks(N), c->scal + kSlotRR, s);
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  if (cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, nullptr, nullptr, nullptr) != cudaSuccess ||
      cs != cudaStreamCaptureStatusActive) {
    c->err = "pcg graph: the stream is not capturing";
    return false;
  }
  cudaGraphConditionalHandle h;
  if (cudaGraphConditionalHandleCreate(&h, g, 0, 0) != cudaSuccess) {
    c->err = "pcg graph: cudaGraphConditionalHandleCreate failed";
    return false;
  }
  launch_pcg_start(c->scal, h, s);
  if (cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, nullptr, &nd) != cudaSuccess) {
    c->err = "pcg graph: cudaStreamGetCaptureInfo failed";
    return false;
  }
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  if (cudaGraphAddNode(&node, g, deps, nullptr, nd, &cp) != cudaSuccess ||
      cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies) != cudaSuccess) {
    c->err = "pcg graph: adding the conditional while node failed";
    return false;
  }
  const long long l1 = g_kernel_launches.load();
  // the body: one PCG iteration, captured on the body stream into the node's graph
  if (!c->body_stream && cudaStreamCreateWithFlags(&c->body_stream, cudaStreamNonBlocking) != cudaSuccess) {
    c->err = "pcg graph: cannot create the body stream";
    return false;
  }
  if (cudaStreamBeginCaptureToGraph(c->body_stream, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                    cudaStreamCaptureModeRelaxed) != cudaSuccess) {
    c->err = "pcg graph: cudaStreamBeginCaptureToGraph failed";
    return false;
  }
  c->stream = c->body_stream;
  bool ok = apply_prec_impl(c, c->r, c->z, kSlotRZN);
  if (ok) {
    if (uses_df(c)) j_times_df(c, c->z, c->jz);
    else j_times(c, c->J, c->z, c->jz);
    launch_pcg_beta_dev(c->scal, c->stream);
    launch_p_update_dev(c->p, c->z, c->w, c->jz, c->scal, N, m > 0 ? m : 0, c->stream);
    apply_op_w(c, c->p, c->w, c->q, kSlotPQ, true);
    launch_pcg_alpha_dev(c->scal, c->stream);
    launch_xr_update(x, c->r, c->p, c->q, c->scal, N, c->partial, c->stream);
    launch_sum_to_scalar(c->partial, colsum_blocks(N), c->scal + kSlotRR, c->stream);
    launch_pcg_check(c->scal, h, c->stream);
  }
  c->stream = s;
  cudaGraph_t body = nullptr;
  const cudaError_t eb = cudaStreamEndCapture(c->body_stream, &body);
  if (!ok || eb != cudaSuccess) {
    c->err = !ok ? "pcg graph: multigrid kernel attribute failed"
                 : std::string("pcg graph: capture of the loop body failed: ") + cudaGetErrorString(eb);
    cudaGetLastError();
    return false;
  }
  const long long l2 = g_kernel_launches.load();
  // after the loop: the FP64 true residual with the caller's J
  j_times(c, c->J, x, c->wtmp);
  apply_op_w(c, x, c->wtmp, c->q, -1);
  launch_true_residual(c->r, b, c->q, N, c->partial, s);
  launch_sum_to_scalar(c->partial, colsum_blocks(N), c->scal + kSlotRRTrue, s);
  const long long l3 = g_kernel_launches.load();
  c->pcg_l_pre = l1 - l0;
  c->pcg_l_body = l2 - l1;
  c->pcg_l_post = l3 - l2;
  return true;
}

// Builds (or reuses) the single-system graph of c: b from c->gb, x into c->gx.
h1w_status pcg_graph_ready(h1w_ctx* c) {
  for (int i = 0; i < 2; ++i) {
    h1w_ctx::PcgGraph& e = c->pcg_g[i];
    if (e.exec && e.m == c->m && e.J == c->J && e.stall == c->stall && e.wait == c->wait_ns) {
      e.used = ++c->pcg_clock;
      c->pcg_cur = i;
      return H1W_OK;
    }
  }
  // replace an empty entry, else the one used longest ago
  const int slot = !c->pcg_g[0].exec ? 0 : !c->pcg_g[1].exec ? 1 : (c->pcg_g[0].used <= c->pcg_g[1].used ? 0 : 1);
  h1w_ctx::PcgGraph& G = c->pcg_g[slot];
  if (G.exec) {
    cudaGraphExecDestroy(G.exec);
    G.exec = nullptr;
  }
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return cuda_check(c, "pcg graph");
  if (!c->cap_stream && cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
    return fail(c, H1W_ECUDA, "pcg graph: cannot create the capture stream");
  const cudaStream_t orig = c->stream;
  c->stream = c->cap_stream;
  c->capturing = true;
  if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
    c->capturing = false;
    c->stream = orig;
    return fail(c, H1W_ECUDA, "pcg graph: cudaStreamBeginCapture failed");
  }
  const bool ok = capture_pcg(c, c->gb, c->gx, true);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(c->stream, &g);
  c->capturing = false;
  c->stream = orig;
  if (!ok || e != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return fail(c, H1W_ECUDA, ok ? std::string("pcg graph: capture failed: ") + cudaGetErrorString(e) : c->err);
  }
  const cudaError_t ei = cudaGraphInstantiate(&G.exec, g, 0);
  cudaGraphDestroy(g);
  if (ei != cudaSuccess) {
    G.exec = nullptr;
    cudaGetLastError();
    return fail(c, H1W_ECUDA, std::string("pcg graph: instantiation failed: ") + cudaGetErrorString(ei));
  }
  G.m = c->m;
  G.J = c->J;
  G.stall = c->stall;
  G.wait = c->wait_ns;
  G.l_pre = c->pcg_l_pre;
  G.l_body = c->pcg_l_body;
  G.l_post = c->pcg_l_post;
  G.used = ++c->pcg_clock;
  c->pcg_cur = slot;
  return H1W_OK;
}

// The preconditioner's second stream (double-float path with measurements): highest priority,
// so that the cycle's small kernels are not queued behind the blocks of the pass beside them.
bool ensure_cycle_stream(h1w_ctx* c) {
  if (!(uses_df(c) && c->m > 0) || c->cycle_stream) return true;
  int lo = 0, hi = 0;
  cudaDeviceGetStreamPriorityRange(&lo, &hi);
  bool made = cudaStreamCreateWithPriority(&c->cycle_stream, cudaStreamNonBlocking, hi) == cudaSuccess;
  for (int e = 0; e < 2 && made; ++e)
    made = cudaEventCreateWithFlags(&c->cycle_ev[e], cudaEventDisableTiming) == cudaSuccess;
  return made;
}

// h1w_pcg with the loop driven from the device: one graph launch per (re)start, one host
// read of the scalars after each.
h1w_status pcg_graph_solve(h1w_ctx* c, const double* b, double* x, double rtol, int maxit, h1w_info* info) {
  const int64_t N = c->lev[0].N;
  const cudaStream_t s = c->stream;
  h1w_status st = pcg_graph_ready(c);
  if (st != H1W_OK) return st;
  const h1w_ctx::PcgGraph& G = c->pcg_g[c->pcg_cur];
  const long long l0 = g_kernel_launches.load();
  if (c->have_ev) cudaEventRecord(c->ev[4], s);
  h1w::launch_copy(c->gb, b, (int64_t)N, s);
  h1w_info inf{0, 0, 0.0, 0.0};
  double sc[16] = {};
  long long launched = 0;
  for (int restart = 0; restart <= c->opt.max_restarts; ++restart) {
    launch_pcg_set_scalars(c->scal, rtol, maxit, restart == 0 ? 1 : 0, s);
    const int it0 = (int)sc[kSlotIt];
    if (cudaGraphLaunch(G.exec, s) != cudaSuccess) return cuda_check(c, "pcg graph launch");
    cudaMemcpyAsync(sc, c->scal, sizeof(sc), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return cuda_check(c, "pcg graph");
    const int it = (int)sc[kSlotIt];
    launched += G.l_pre + (long long)(it - it0) * G.l_body + G.l_post;
    inf.iters = it;
    const double bb = sc[kSlotBB];
    inf.rel_res_true = bb > 0.0 ? std::sqrt(sc[kSlotRRTrue] / bb) : 0.0;
    inf.rel_res_rec = bb > 0.0 ? std::sqrt(sc[kSlotRR] / bb) : 0.0;
    if (inf.rel_res_true <= rtol || it >= maxit || !std::isfinite(inf.rel_res_true)) break;
    ++inf.restarts;
  }
  h1w::launch_copy(x, c->gx, (int64_t)N, s);
  if (c->have_ev) cudaEventRecord(c->ev[5], s);
  int dst = 0;
  cudaMemcpyAsync(&dst, c->dstatus, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return cuda_check(c, "pcg graph");
  c->launches_pcg = g_kernel_launches.load() - l0 + launched;
  for (int k = kCatJdot; k <= kCatHupd; ++k) { c->cat_ms[k] = 0.f; c->cat_n[k] = 0; }
  if (info) *info = inf;
  st = cuda_check(c, "pcg graph");
  if (st != H1W_OK) return st;
  if (dst & kStatusTimeout) return fail(c, H1W_ETIMEOUT, "pcg: a bounded device wait ran out");
  if (!(inf.rel_res_true <= rtol)) return fail(c, H1W_ENOTCONV, "PCG did not reach rtol within maxit");
  return H1W_OK;
}

}  // namespace

extern "C" {

void h1w_default_options(h1w_options* opt) {
  if (!opt) return;
  opt->cheb_degree = 2;
  opt->rhs_block = 128;
  opt->max_restarts = 3;
  opt->cap_gemm = 0;
  opt->mg_arith = 0;
  opt->mg_unfused = 0;
  opt->precond = 0;
  opt->pcg_mode = 0;
  opt->cheb_ratio = 0.0;
  opt->j_digits = 1;
}

size_t h1w_workspace_size(const h1w_grid* grid, int32_t m_max, const h1w_options* opt) {
  h1w_options o;
  h1w_default_options(&o);
  if (opt) o = *opt;
  std::string why;
  if (validate(grid, m_max, &o, why) != H1W_OK) return 0;
  Plan P = plan_levels(*grid);
  if (!P.ok) return 0;
  return layout(nullptr, P, *grid, m_max, o, nullptr);
}

h1w_status h1w_setup(const h1w_grid* grid, int32_t m_max, const h1w_options* opt, void* workspace,
                     size_t ws_bytes, void* stream, h1w_ctx** out) {
  if (!out) return fail(nullptr, H1W_EINVAL, "out is NULL");
  *out = nullptr;
  h1w_options o;
  h1w_default_options(&o);
  if (opt) o = *opt;
  std::string why;
  h1w_status st = validate(grid, m_max, &o, why);
  if (st != H1W_OK) return fail(nullptr, st, why);
  Plan P = plan_levels(*grid);
  if (!P.ok) return fail(nullptr, H1W_EUNSUPPORTED, P.why);
  const size_t need = layout(nullptr, P, *grid, m_max, o, nullptr);
  if (!workspace) return fail(nullptr, H1W_EINVAL, "workspace is NULL");
  if (reinterpret_cast<uintptr_t>(workspace) % 256) return fail(nullptr, H1W_EINVAL, "workspace must be 256-byte aligned");
  if (ws_bytes < need)
    return fail(nullptr, H1W_ENOMEM, "workspace too small: need " + std::to_string(need) + " bytes");
  h1w_ctx* c = new (std::nothrow) h1w_ctx();
  if (!c) return fail(nullptr, H1W_ENOMEM, "host allocation of the context failed");
  c->grid = *grid;
  c->opt = o;
  c->disc = grid->disc;
  c->m_max = m_max;
  c->stream = reinterpret_cast<cudaStream_t>(stream);
  {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && sms > 0)
      c->num_sms = sms;
  }
  c->nlev = P.nlev;
  c->m = -1;
  c->J = nullptr;
  layout(c, P, *grid, m_max, o, static_cast<char*>(workspace));
  cudaMemsetAsync(c->trsv_flags, 0, sizeof(int) * 2 * ((m_max + 31) / 32 + 1), c->stream);
  cudaMemsetAsync(c->gflags, 0, sizeof(int) * (2 * ((m_max + 31) / 32 + 1) + 1), c->stream);
  {
    static std::atomic<unsigned long long> next_uid{1};
    c->uid = next_uid.fetch_add(1);
  }
  c->have_ev = true;
  for (int e = 0; e < 6; ++e)
    if (cudaEventCreate(&c->ev[e]) != cudaSuccess) c->have_ev = false;
  for (int t = 0; t < h1w_ctx::kTimed && c->have_ev; ++t)
    for (int e = 0; e < 2; ++e)
      if (cudaEventCreate(&c->kev[t][e]) != cudaSuccess) c->have_ev = false;
  c->nk = 0;
  c->timing_on = false;
  for (int k = 0; k < 16; ++k) { c->cat_ms[k] = 0.f; c->cat_n[k] = 0; }
  c->launches_cap = c->launches_pcg = 0;

  // level descriptors
  int64_t qoff = 0, stoff = 0;
  for (int l = 0; l < P.nlev; ++l) {
    Level& L = c->lev[l];
    L = Level{};
    L.nx = P.n[l][0]; L.ny = P.n[l][1]; L.nz = P.n[l][2];
    L.N = (int64_t)L.nx * L.ny * L.nz;
    L.cx = P.c[l][0]; L.cy = P.c[l][1]; L.cz = P.c[l][2];
    if (c->disc == H1W_FV_CELL) {
      const double hx = P.h[l][0], hy = P.h[l][1], hz = P.h[l][2];
      L.Tx = hy * hz / hx; L.Ty = hx * hz / hy; L.Tz = hx * hy / hz; L.V = hx * hy * hz;
      L.iso = (L.Tx == L.Ty && L.Ty == L.Tz) ? 1 : 0;
      for (int cz = 0; cz < 3; ++cz)
        for (int cy = 0; cy < 3; ++cy)
          for (int cx = 0; cx < 3; ++cx) {
            const double dg = L.V + L.Tx * cx + L.Ty * cy + L.Tz * cz;
            L.fv_diag[cx + 3 * cy + 9 * cz] = dg;
            L.fv_dinv[cx + 3 * cy + 9 * cz] = 1.0 / dg;
            L.fvd_diag[cx + 3 * cy + 9 * cz] = df_host(dg);
            L.fvd_dinv[cx + 3 * cy + 9 * cz] = df_host(1.0 / dg);
          }
      L.fvd_T[0] = df_host(L.Tx);
      L.fvd_T[1] = df_host(L.Ty);
      L.fvd_T[2] = df_host(L.Tz);
    } else {
      for (int a = 0; a < 2; ++a) {
        if (l == 0) q1_fine_1d(P.n[0][a], grid->h[a], c->qhost[0][a]);
        else if (P.c[l - 1][a]) q1_coarse_1d(c->qhost[l - 1][a], P.n[l - 1][a], P.n[l][a], c->qhost[l][a]);
        else c->qhost[l][a] = c->qhost[l - 1][a];
      }
      double* qx = c->qdev + qoff;
      qoff += 6 * (int64_t)L.nx;
      double* qy = c->qdev + qoff;
      qoff += 6 * (int64_t)L.ny;
      cudaMemcpyAsync(qx, c->qhost[l][0].data(), sizeof(double) * 6 * L.nx, cudaMemcpyHostToDevice, c->stream);
      cudaMemcpyAsync(qy, c->qhost[l][1].data(), sizeof(double) * 6 * L.ny, cudaMemcpyHostToDevice, c->stream);
      L.qx = qx; L.qy = qy;
      if (o.mg_arith == 0) {
        df* st = c->q1st + stoff;
        stoff += 10 * L.N;
        launch_q1_stencil_df(L, st, c->stream);
        L.q1st = st;
        // the vertices whose 1D factor entries equal those of the middle vertex have the
        // middle vertex's stencil: the kernels take it from the Level instead of the table
        int lo[2], hi[2];
        for (int a = 0; a < 2; ++a) q1_uniform_range(c->qhost[l][a], a == 0 ? L.nx : L.ny, lo[a], hi[a]);
        L.q1_ilo = lo[0]; L.q1_ihi = hi[0]; L.q1_jlo = lo[1]; L.q1_jhi = hi[1];
        for (int k = 0; k < 10; ++k) L.q1c[k] = df_make(0.f, 0.f);
        if (lo[0] <= hi[0] && lo[1] <= hi[1]) {
          const int64_t pm = (int64_t)((lo[1] + hi[1]) / 2) * L.nx + (lo[0] + hi[0]) / 2;
          for (int k = 0; k < 10; ++k)
            cudaMemcpyAsync(&L.q1c[k], st + (int64_t)k * L.N + pm, sizeof(df), cudaMemcpyDeviceToHost, c->stream);
          if (cudaStreamSynchronize(c->stream) != cudaSuccess) { L.q1_ilo = 1; L.q1_ihi = 0; }
        }
        const double dinv_box = (double)L.q1c[9].hi + (double)L.q1c[9].lo;
        for (int k = 0; k < 9; ++k) L.q1w[k] = df_host(((double)L.q1c[k].hi + (double)L.q1c[k].lo) * dinv_box);
      }
    }
  }
  // Gershgorin bounds and Chebyshev coefficients
  for (int l = 0; l < P.nlev; ++l) {
    cudaMemsetAsync(c->dbits, 0, sizeof(unsigned long long), c->stream);
    launch_gershgorin(c->disc, c->lev[l], c->dbits, c->stream);
    unsigned long long bits = 0;
    cudaMemcpyAsync(&bits, c->dbits, sizeof(bits), cudaMemcpyDeviceToHost, c->stream);
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) {
      st = cuda_check(c, "setup");
      g_setup_error = c->err;
      delete c;
      return st == H1W_OK ? H1W_ECUDA : st;
    }
    double lam;
    std::memcpy(&lam, &bits, sizeof(lam));
    c->lev[l].lam = lam;
    const double lo = lam / cheb_ratio_of(c->disc, o), hi = lam;
    const double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo), sigma = theta / delta;
    ChebCoef& K = c->cheb[l];
    K.inv_theta = 1.0 / theta;
    K.inv_theta_df = df_host(K.inv_theta);
    double rho_prev = 1.0 / sigma;
    for (int j = 1; j < o.cheb_degree; ++j) {
      const double rho = 1.0 / (2.0 * sigma - rho_prev);
      K.c1[j] = rho * rho_prev;
      K.c2[j] = 2.0 * rho / delta;
      K.c1_df[j] = df_host(K.c1[j]);
      K.c2_df[j] = df_host(K.c2[j]);
      rho_prev = rho;
    }
    if (o.cheb_degree == 2) {
      K.beta_df = df_host(K.inv_theta * (1.0 + K.c1[1]) + K.c2[1] * (1.0 - K.inv_theta));
      K.c2t_df = df_host(K.c2[1] * K.inv_theta);
    }
    if (c->disc == H1W_FV_CELL && o.cheb_degree == 2) {   // constants of the fused smoothing legs
      const Level& L = c->lev[l];
      FusedCoef& F = c->fco[l];
      const double it = K.inv_theta, c1 = K.c1[1], c2 = K.c2[1];
      const double beta = it * (1.0 + c1) + c2 * (1.0 - it);
      for (int k = 0; k < 27; ++k) {
        const double d = L.fv_diag[k], di = 1.0 / d;
        F.d[k] = df_host(d);
        F.dinv[k] = df_host(di);
        F.gam[k] = df_host(c2 * it * di);
        F.del[k] = df_host(it * di);
        F.eta[k] = df_host(beta * di);
        F.kap[k] = df_host(c2 * di);
        F.gamT[k] = df_host(c2 * it * di * L.Tx);
        F.kapT[k] = df_host(c2 * di * L.Tx);
      }
      F.T[0] = df_host(L.Tx);
      F.T[1] = df_host(L.Ty);
      F.T[2] = df_host(L.Tz);
      F.beta = df_host(beta);
    }
  }
  // coarsest level: dense matrix, Cholesky, explicit symmetric inverse
  {
    const Level& L = c->lev[P.nlev - 1];
    const int n = (int)L.N;
    cudaMemsetAsync(c->coarse_L, 0, sizeof(double) * n * n, c->stream);
    launch_assemble_dense(c->disc, L, c->coarse_L, c->stream);
    cudaMemsetAsync(c->dstatus, 0, sizeof(int), c->stream);
    launch_chol(c->coarse_L, n, c->dstatus, c->stream);
    launch_set_identity(c->coarse_X, n, c->stream);
    launch_trsv_lower(c->coarse_L, n, c->coarse_X, n, c->stream);
    launch_trsv_upper_t(c->coarse_L, n, c->coarse_X, n, c->stream);
    launch_symmetrize_identity_solve(c->coarse_X, n, c->stream);
    int status = 0;
    cudaMemcpyAsync(&status, c->dstatus, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess || cudaGetLastError() != cudaSuccess) {
      g_setup_error = std::string("setup: ") + cudaGetErrorString(e);
      delete c;
      return H1W_ECUDA;
    }
    if (status & kStatusNotSpd) {
      g_setup_error = "coarsest-level matrix is not positive definite";
      delete c;
      return H1W_ENOTSPD;
    }
  }
  *out = c;
  return H1W_OK;
}

// Lines H, C, chol. With J_host given, the rows of J are first copied from it into J
// (device) on the context's copy stream, one rhs_block batch at a time, each batch's
// conversion and V-cycles waiting only for that batch's copy.
static h1w_status capacitance_core(h1w_ctx* c, int32_t m, const double* J, const double* J_host);

// Row batches: rhs_block rows each. With J coming from the host the batches ramp up from
// 16 rows by a factor of about 1.25 (rounded up to multiples of 8): the cycles start after
// a short first copy, and while a batch runs the copy of the next, slightly larger one
// completes (a cycle costs somewhat more per row than the copy of the row over the host
// link), so the cycles rarely wait for data.
static std::vector<int> batch_edges(const h1w_ctx* c, int m, bool from_host) {
  const int nb = block_rhs(c->opt, c->m_max);
  std::vector<int> edge{0};
  for (int r0 = 0, bs = from_host ? std::min(nb, 16) : nb; r0 < m;) {
    r0 = std::min(m, r0 + bs);
    edge.push_back(r0);
    if (from_host) bs = std::min(nb, (bs + bs / 4 + 7) / 8 * 8);
  }
  return edge;
}

static bool make_events(std::vector<cudaEvent_t>& v, size_t n) {
  while (v.size() < n) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return false;
    v.push_back(e);
  }
  return true;
}

// Queues the copies of J_host into J_dev on the copy stream, after the work already queued
// on the context's stream (which may still read J_dev), one row batch at a time.
static h1w_status issue_host_copies(h1w_ctx* c, HostCopy& h, int m, const double* J_host, const double* J_dev) {
  const int64_t N = c->lev[0].N;
  if (!c->copy_stream && cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking) != cudaSuccess)
    return fail(c, H1W_ECUDA, "capacitance_from_host: cannot create the copy stream");
  if (!c->order_ev && cudaEventCreateWithFlags(&c->order_ev, cudaEventDisableTiming) != cudaSuccess)
    return fail(c, H1W_ECUDA, "capacitance_from_host: cannot create an event");
  h.edge = batch_edges(c, m, true);
  const int nbatch = (int)h.edge.size() - 1;
  // fresh events for every copy set: re-recording the events that the context's stream waited
  // on when this set's previous copies were consumed held that stream back until the new
  // copies had finished (measured: the next step's work waited about one copy of J)
  for (cudaEvent_t e : h.beg) cudaEventDestroy(e);
  for (cudaEvent_t e : h.end) cudaEventDestroy(e);
  h.beg.clear();
  h.end.clear();
  if (!make_events(h.beg, nbatch) || !make_events(h.end, nbatch))
    return fail(c, H1W_ECUDA, "capacitance_from_host: cannot create an event");
  cudaEventRecord(c->order_ev, c->stream);
  cudaStreamWaitEvent(c->copy_stream, c->order_ev, 0);
  for (int bi = 0; bi < nbatch; ++bi) {
    const int64_t r0 = h.edge[bi], nr = h.edge[bi + 1] - h.edge[bi];
    cudaEventRecord(h.beg[bi], c->copy_stream);
    cudaMemcpyAsync(const_cast<double*>(J_dev) + r0 * N, J_host + r0 * N, sizeof(double) * nr * N,
                    cudaMemcpyHostToDevice, c->copy_stream);
    cudaEventRecord(h.end[bi], c->copy_stream);
  }
  h.host = J_host;
  h.dev = J_dev;
  h.m = m;
  h.active = true;
  h.prefetched = false;
  return cuda_check(c, "capacitance_from_host: copies");
}

// the pending copy set of (J_host, J_dev, m), or a new one queued now; null on failure
static HostCopy* host_copies_for(h1w_ctx* c, int m, const double* J_host, const double* J_dev, h1w_status& st) {
  st = H1W_OK;
  for (HostCopy& h : c->hcopy)
    if (h.active && h.host == J_host && h.dev == J_dev && h.m == m) return &h;
  for (HostCopy& h : c->hcopy)
    if (!h.active) {
      st = issue_host_copies(c, h, m, J_host, J_dev);
      return st == H1W_OK ? &h : nullptr;
    }
  st = fail(c, H1W_ESTATE, "capacitance_from_host: two other prefetches of J are pending");
  return nullptr;
}

// every return waits for the copies of J_host, so that none outlives the call
static h1w_status capacitance_impl(h1w_ctx* c, int32_t m, const double* J, const double* J_host) {
  const h1w_status st = capacitance_core(c, m, J, J_host);
  if (J_host) {
    for (HostCopy& h : c->hcopy)
      if (h.active && h.host == J_host && h.dev == J && h.m == m) {
        if (!h.end.empty() && h.edge.size() > 1) cudaEventSynchronize(h.end[h.edge.size() - 2]);
        h.active = false;
      }
  }
  return st;
}

// The GEMM's tile list for m rows, uploaded only when m differs from the last upload: a copy
// from host memory on the context's stream would queue on a copy engine behind a pending
// prefetch of J.
static void upload_tiles(h1w_ctx* c, int m) {
  if (c->oz_tiles_m == m) return;
  ozaki_tiles(m, c->oz_tiles_host);
  cudaMemcpyAsync(c->oz.tiles, c->oz_tiles_host.data(), sizeof(int) * c->oz_tiles_host.size(),
                  cudaMemcpyHostToDevice, c->stream);
  c->oz_tiles_m = m;
}

// Host-side preparation of a capacitance that will be captured into a graph: the GEMM's tile
// list for m rows, uploaded (a capture cannot copy from pageable host memory). Synchronizes.
static h1w_status capacitance_prepare(h1w_ctx* c, int32_t m) {
  if (m > 0 && c->opt.cap_gemm == 0 && c->opt.precond == 0) upload_tiles(c, m);
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return cuda_check(c, "capacitance_prepare");
  return cuda_check(c, "capacitance_prepare");
}

static h1w_status capacitance_core(h1w_ctx* c, int32_t m, const double* J, const double* J_host) {
  const int64_t N = c->lev[0].N;
  c->m = m;
  c->J = J;
  const long long l0 = g_kernel_launches.load();
  if (m == 0) { c->launches_cap = 0; return H1W_OK; }
  HostCopy* hc = nullptr;
  if (J_host) {
    h1w_status st = H1W_OK;
    hc = host_copies_for(c, m, J_host, J, st);
    if (!hc) return st;
  }
  // V-cycle batches: the copy batches when this call issued the copies (they grow from 16
  // rows, so the cycles start early and follow the copy), else the standard rhs_block
  // batches, each waiting for the copy batch that holds its last row (a prefetched copy is
  // usually complete, and small batches would only cost cycle efficiency)
  const bool own = hc && !hc->prefetched;
  const std::vector<int> edge = own ? hc->edge : batch_edges(c, m, false);
  const int nbatch = (int)edge.size() - 1;
  std::vector<int> cov_first, cov_last;   // per V-cycle batch: copy batches of its first and last rows
  if (hc) {
    const int ncb = (int)hc->edge.size() - 1;
    for (int bi = 0, j = 0; bi < nbatch; ++bi) {
      while (j < ncb - 1 && hc->edge[j + 1] <= edge[bi]) ++j;
      cov_first.push_back(j);
      int k = j;
      while (k < ncb - 1 && hc->edge[k + 1] < edge[bi + 1]) ++k;
      cov_last.push_back(k);
    }
    if (!make_events(c->cyc_beg, nbatch) || !make_events(c->cyc_end, nbatch))
      return fail(c, H1W_ECUDA, "capacitance_from_host: cannot create an event");
  }
  if (c->have_ev && !c->capturing) cudaEventRecord(c->ev[0], c->stream);
  if (c->opt.precond == 1) {  // Laplace-only preconditioner: J for the operator, no lines H, C, chol
    for (int bi = 0; bi < nbatch; ++bi) {
      const int64_t r0 = edge[bi], nr = edge[bi + 1] - edge[bi], o = r0 * N;
      if (hc) cudaStreamWaitEvent(c->stream, hc->end[cov_last[bi]], 0);
      if (uses_df(c)) launch_d2df(nr * N, J + o, c->Jdf + o, c->stream);
    }
    for (int k = 1; k < 4 && c->have_ev && !c->capturing; ++k) cudaEventRecord(c->ev[k], c->stream);
    c->launches_cap = g_kernel_launches.load() - l0;
    if (c->capturing) return cuda_check(c, "capacitance");
    const cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return fail(c, H1W_ECUDA, std::string("capacitance: ") + cudaGetErrorString(e));
    return cuda_check(c, "capacitance");
  }
  // line H; on the double-float cycle the tensor-core split reads H as double-floats, so the
  // FP64 copy of H is only written for the FP64 paths
  const bool h_df_only = uses_df(c) && c->opt.cap_gemm == 0;
  c->nk = 0;
  c->timing_on = c->time_vc = true;
  bool vc_ok = true;
  for (int bi = 0; bi < nbatch && vc_ok; ++bi) {
    const int64_t r0 = edge[bi], nr = edge[bi + 1] - edge[bi], o = r0 * N;
    if (hc) {
      cudaStreamWaitEvent(c->stream, hc->end[cov_last[bi]], 0);
      cudaEventRecord(c->cyc_beg[bi], c->stream);
    }
    if (uses_df(c)) {  // J for the cycle and the Krylov passes (and, with j_full, J's digits for line C)
      timed_begin(c);
      if (c->oz.j_full && c->opt.cap_gemm == 0)
        launch_split_j_rows(J, m, N, (int)r0, (int)(r0 + nr), c->oz, c->Jdf, c->stream);
      else
        launch_d2df(nr * N, J + o, c->Jdf + o, c->stream);
      timed_end(c, kCatD2df);
    }
    vc_ok = vcycle_many(c, (int)nr, J + o, uses_df(c) ? c->Jdf + o : nullptr, h_df_only ? nullptr : c->H + o,
                        c->Hdf ? c->Hdf + o : nullptr);
    if (hc) cudaEventRecord(c->cyc_end[bi], c->stream);
  }
  c->timing_on = c->time_vc = false;
  if (!vc_ok) return fail(c, H1W_ECUDA, "capacitance: multigrid kernel attribute failed");
  if (c->have_ev && !c->capturing) cudaEventRecord(c->ev[1], c->stream);
  cudaMemsetAsync(c->dstatus, 0, sizeof(int), c->stream);
  int splits = 0;
  if (c->opt.cap_gemm == 0) {                                       // line C, tensor cores
    if (!ozaki_supported()) return fail(c, H1W_EUNSUPPORTED, "tensor-core capacitance GEMM needs sm_100-class GPU");
    if (!c->capturing) upload_tiles(c, m);  // a capture finds the list uploaded by capacitance_prepare
    splits = ozaki_splits(m, c->oz.klen, c->num_sms);
    c->oz.wait_ns = c->wait_ns;
    c->oz.stall = c->stall == H1W_STALL_CAP_GEMM ? 1 : 0;
    c->timing_on = true;
    const bool ok = launch_ozaki_capacitance(
        J, c->H, nullptr, h_df_only ? c->Hdf : nullptr, m, N, c->oz, splits, c->stream,
        [](void* p, int which, int begin) {
          h1w_ctx* cx = static_cast<h1w_ctx*>(p);
          if (begin) timed_begin(cx);
          else timed_end(cx, which == kOzakiGemm ? kCatGemm : which == kOzakiSplitJ ? kCatSplitJ : kCatSplitH);
        },
        c);
    c->timing_on = false;
    if (!ok)
      return fail(c, H1W_ECUDA, std::string("capacitance: tensor-core GEMM not launched: ") +
                                    cudaGetErrorString(cudaGetLastError()));
  } else {                                                          // line C, FP64 CUDA cores
    splits = cap_gemm_splits(m, N);
    c->timing_on = true;
    timed_begin(c);
    launch_cap_gemm(J, c->H, m, N, c->gemm_partial, splits, c->stream);
    timed_end(c, kCatGemm);
    c->timing_on = false;
  }
  if (c->have_ev && !c->capturing) cudaEventRecord(c->ev[2], c->stream);
  launch_cap_finalize(c->gemm_partial, splits, m, c->grid.alpha, c->C, c->stream);
  h1w::launch_copy(c->Lc, c->C, (int64_t)m * m, c->stream);
  launch_chol(c->Lc, m, c->dstatus, c->stream);                    // line chol
  if (c->have_ev && !c->capturing) cudaEventRecord(c->ev[3], c->stream);
  c->launches_cap = g_kernel_launches.load() - l0;
  if (c->capturing) return cuda_check(c, "capacitance");  // the status word is read after the graph ran
  int status = 0;
  cudaMemcpyAsync(&status, c->dstatus, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return fail(c, H1W_ECUDA, std::string("capacitance: ") + cudaGetErrorString(e));
  timed_collect(c, (1u << kCatGemm) | (1u << kCatDown) | (1u << kCatUp) | (1u << kCatSplitJ) | (1u << kCatSplitH) |
                       (1u << kCatD2df));
  if (hc && c->have_ev) {  // when each batch's copy began and ended, and its cycles began and ended
    cudaEventSynchronize(hc->end[hc->edge.size() - 2]);
    auto rel = [&](cudaEvent_t e) {
      float ms = 0.f;
      return cudaEventElapsedTime(&ms, c->ev[0], e) == cudaSuccess ? ms : 0.f;
    };
    c->prof_rows.assign(nbatch, 0);
    c->prof_copy_beg.assign(nbatch, 0.f);
    c->prof_copy_end.assign(nbatch, 0.f);
    c->prof_cyc_beg.assign(nbatch, 0.f);
    c->prof_cyc_end.assign(nbatch, 0.f);
    for (int bi = 0; bi < nbatch; ++bi) {
      c->prof_rows[bi] = edge[bi + 1] - edge[bi];
      c->prof_copy_beg[bi] = rel(hc->beg[cov_first[bi]]);
      c->prof_copy_end[bi] = rel(hc->end[cov_last[bi]]);
      c->prof_cyc_beg[bi] = rel(c->cyc_beg[bi]);
      c->prof_cyc_end[bi] = rel(c->cyc_end[bi]);
    }
    cudaGetLastError();
  }
  h1w_status st = cuda_check(c, "capacitance");
  if (st != H1W_OK) return st;
  if (status & kStatusTimeout) {
    c->m = -1;
    return fail(c, H1W_ETIMEOUT, "capacitance GEMM: a bounded device wait ran out");
  }
  if (status & kStatusNotSpd) {
    c->m = -1;
    return fail(c, H1W_ENOTSPD, "capacitance matrix is not numerically positive definite");
  }
  return H1W_OK;
}

h1w_status h1w_capacitance(h1w_ctx* c, int32_t m, const double* J) {
  if (!c) return H1W_EINVAL;
  if (m < 0 || m > c->m_max) return fail(c, H1W_EINVAL, "m out of range [0, m_max]");
  if (m > 0 && !J) return fail(c, H1W_EINVAL, "J is NULL");
  return capacitance_impl(c, m, J, nullptr);
}

h1w_status h1w_capacitance_from_host(h1w_ctx* c, int32_t m, const double* J_host, double* J_dev) {
  if (!c) return H1W_EINVAL;
  if (m < 0 || m > c->m_max) return fail(c, H1W_EINVAL, "m out of range [0, m_max]");
  if (m > 0 && (!J_host || !J_dev)) return fail(c, H1W_EINVAL, "J_host and J_dev must be non-NULL");
  return capacitance_impl(c, m, J_dev, m > 0 ? J_host : nullptr);
}

// The device's address of page-locked host memory, or null when p is not such memory.
static const double* host_view(const void* p) {
  cudaPointerAttributes a{};
  if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (a.type != cudaMemoryTypeHost || !a.devicePointer) return nullptr;
  return static_cast<const double*>(a.devicePointer);
}

h1w_status h1w_pcg_host(h1w_ctx* c, const double* b_host, double* x_host, double rtol, int32_t maxit,
                        h1w_info* info) {
  if (!c) return H1W_EINVAL;
  if (!b_host || !x_host || b_host == x_host)
    return fail(c, H1W_EINVAL, "pcg_host: b_host and x_host must be distinct non-NULL pointers");
  const double* bd = host_view(b_host);
  double* xd = const_cast<double*>(host_view(x_host));
  if (!bd || !xd) return fail(c, H1W_EINVAL, "pcg_host: b_host and x_host must be page-locked host memory");
  const int64_t N = c->lev[0].N;
  if (c->m < 0) return fail(c, H1W_ESTATE, "call h1w_capacitance first");
  h1w::launch_copy(c->gb, bd, N, c->stream);   // b in, read by a kernel
  const h1w_status st = h1w_pcg(c, c->gb, c->gx, rtol, maxit, info);
  if (st != H1W_OK && st != H1W_ENOTCONV) return st;
  h1w::launch_copy(xd, c->gx, N, c->stream);   // x out (also the last iterate on ENOTCONV)
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return cuda_check(c, "pcg_host");
  const h1w_status sc = cuda_check(c, "pcg_host");
  return sc != H1W_OK ? sc : st;
}

h1w_status h1w_prefetch_J(h1w_ctx* c, int32_t m, const double* J_host, double* J_dev) {
  if (!c) return H1W_EINVAL;
  if (m < 1 || m > c->m_max) return fail(c, H1W_EINVAL, "prefetch_J: m out of range [1, m_max]");
  if (!J_host || !J_dev) return fail(c, H1W_EINVAL, "prefetch_J: J_host and J_dev must be non-NULL");
  for (HostCopy& h : c->hcopy)
    if (h.active && h.dev == J_dev && !(h.host == J_host && h.m == m))
      return fail(c, H1W_ESTATE, "prefetch_J: another copy into J_dev is pending");
  h1w_status st = H1W_OK;
  HostCopy* h = host_copies_for(c, m, J_host, J_dev, st);
  if (h) h->prefetched = true;
  return st;
}

h1w_status h1w_get_copy_profile(const h1w_ctx* c, int32_t cap, int32_t* nbatch, int32_t* rows, float* copy_begin_ms,
                                float* copy_end_ms, float* cycle_begin_ms, float* cycle_end_ms) {
  if (!c || cap < 0) return H1W_EINVAL;
  const int n = (int)c->prof_rows.size();
  if (nbatch) *nbatch = n;
  for (int i = 0; i < std::min(n, (int)cap); ++i) {
    if (rows) rows[i] = c->prof_rows[i];
    if (copy_begin_ms) copy_begin_ms[i] = c->prof_copy_beg[i];
    if (copy_end_ms) copy_end_ms[i] = c->prof_copy_end[i];
    if (cycle_begin_ms) cycle_begin_ms[i] = c->prof_cyc_beg[i];
    if (cycle_end_ms) cycle_end_ms[i] = c->prof_cyc_end[i];
  }
  return H1W_OK;
}

h1w_status h1w_apply_prec(h1w_ctx* c, const double* r, double* z) {
  if (!c) return H1W_EINVAL;
  if (!r || !z || r == z) return fail(c, H1W_EINVAL, "r and z must be distinct non-NULL pointers");
  if (c->m < 0) return fail(c, H1W_ESTATE, "call h1w_capacitance first");
  if (!apply_prec_impl(c, r, z, -1)) return fail(c, H1W_ECUDA, "apply_prec: multigrid kernel attribute failed");
  return cuda_check(c, "apply_prec");
}

h1w_status h1w_apply_op(h1w_ctx* c, const double* p, double* q) {
  if (!c) return H1W_EINVAL;
  if (!p || !q || p == q) return fail(c, H1W_EINVAL, "p and q must be distinct non-NULL pointers");
  if (c->m < 0) return fail(c, H1W_ESTATE, "call h1w_capacitance first");
  j_times(c, c->J, p, c->wtmp);
  apply_op_w(c, p, c->wtmp, q, -1);
  return cuda_check(c, "apply_op");
}

h1w_status h1w_vcycle(h1w_ctx* c, int32_t nrhs, const double* b, double* x) {
  if (!c) return H1W_EINVAL;
  if (nrhs < 0 || (nrhs > 0 && (!b || !x))) return fail(c, H1W_EINVAL, "bad vcycle arguments");
  if (nrhs == 0) return H1W_OK;
  if (!vcycle_many(c, nrhs, b, nullptr, x, nullptr))
    return fail(c, H1W_ECUDA, "vcycle: multigrid kernel attribute failed");
  return cuda_check(c, "vcycle");
}

h1w_status h1w_gn_rhs(h1w_ctx* c, const double* dm, const double* d, double* b) {
  if (!c) return H1W_EINVAL;
  if (!dm || !b || dm == b) return fail(c, H1W_EINVAL, "dm and b must be distinct non-NULL pointers");
  if (c->m < 0) return fail(c, H1W_ESTATE, "call h1w_capacitance first");
  if (c->m > 0 && !d) return fail(c, H1W_EINVAL, "d is NULL");
  launch_apply_op(c->disc, c->lev[0], -c->grid.alpha, dm, -1.0, c->J, d, c->m, b, nullptr, nullptr,
                  c->stream);
  return cuda_check(c, "gn_rhs");
}

h1w_status h1w_pcg(h1w_ctx* c, const double* b, double* x, double rtol, int32_t maxit,
                   h1w_info* info) {
  if (!c) return H1W_EINVAL;
  if (!b || !x || b == x) return fail(c, H1W_EINVAL, "b and x must be distinct non-NULL pointers");
  if (!(rtol > 0.0) || maxit < 0) return fail(c, H1W_EINVAL, "rtol must be > 0 and maxit >= 0");
  if (c->m < 0) return fail(c, H1W_ESTATE, "call h1w_capacitance first");
  const int64_t N = c->lev[0].N;
  const int m = c->m;
  cudaStream_t s = c->stream;
  enum { RZ = 0, PQ = 1, A = 2, RZN = 3, BETA = 4, RR = 5, BB = 6 };
  if (!ensure_cycle_stream(c)) return fail(c, H1W_ECUDA, "pcg: cannot create the cycle stream or its events");
  if (c->opt.pcg_mode == 0) return pcg_graph_solve(c, b, x, rtol, maxit, info);
  const long long l0 = g_kernel_launches.load();
  if (c->have_ev) cudaEventRecord(c->ev[4], s);
  c->nk = 0;
  c->timing_on = true;
  cudaMemsetAsync(c->dstatus, 0, sizeof(int), s);  // bounded waits of the C^-1 solves report here
  launch_dot_partial(b, b, N, c->partial, s);
  launch_sum_to_scalar(c->partial, dot_blocks(N), c->scal + BB, s);
  const double bnorm = std::sqrt(read_scalar(c, BB));
  cudaMemsetAsync(x, 0, sizeof(double) * N, s);
  h1w_info inf{0, 0, 0.0, 0.0};
  if (bnorm == 0.0) {
    if (info) *info = inf;
    if (c->have_ev) cudaEventRecord(c->ev[5], s);
    cudaStreamSynchronize(s);
    c->timing_on = false;
    c->nk = 0;
    c->launches_pcg = g_kernel_launches.load() - l0;
    return cuda_check(c, "pcg");
  }
  h1w::launch_copy(c->r, b, (int64_t)N, s);
  double rr = bnorm * bnorm;
  const double tol = rtol * bnorm;
  int it = 0;
  double rel_true = 1.0;
  bool prec_failed = false;
  for (int restart = 0; restart <= c->opt.max_restarts; ++restart) {
    if (!apply_prec_impl(c, c->r, c->z, RZ)) { prec_failed = true; break; }
    if (uses_df(c)) j_times_df(c, c->z, c->jz);
    else j_times(c, c->J, c->z, c->jz);
    launch_p_update(c->p, c->z, c->w, c->jz, c->scal, N, m > 0 ? m : 0, true, s);
    while (it < maxit && std::sqrt(rr) > tol) {
      apply_op_w(c, c->p, c->w, c->q, PQ, true);
      launch_pcg_alpha(c->scal, s);
      launch_xr_update(x, c->r, c->p, c->q, c->scal, N, c->partial, s);
      launch_sum_to_scalar(c->partial, colsum_blocks(N), c->scal + RR, s);
      rr = read_scalar(c, RR);
      ++it;
      if (!std::isfinite(rr)) break;
      if (std::sqrt(rr) <= tol) break;
      if (!apply_prec_impl(c, c->r, c->z, RZN)) { prec_failed = true; break; }
      if (uses_df(c)) j_times_df(c, c->z, c->jz);
      else j_times(c, c->J, c->z, c->jz);
      launch_pcg_beta(c->scal, s);
      launch_p_update(c->p, c->z, c->w, c->jz, c->scal, N, m > 0 ? m : 0, false, s);
    }
    if (prec_failed) break;
    // true residual r = b - A x
    j_times(c, c->J, x, c->wtmp);
    apply_op_w(c, x, c->wtmp, c->q, -1);
    h1w::launch_copy(c->r, c->q, (int64_t)N, s);
    launch_axpby(c->r, 1.0, b, -1.0, N, s);
    launch_dot_partial(c->r, c->r, N, c->partial, s);
    launch_sum_to_scalar(c->partial, dot_blocks(N), c->scal + RR, s);
    const double rr_rec = rr;
    rr = read_scalar(c, RR);
    rel_true = std::sqrt(rr) / bnorm;
    inf.rel_res_rec = std::sqrt(rr_rec) / bnorm;
    if (rel_true <= rtol || it >= maxit || !std::isfinite(rel_true)) break;
    ++inf.restarts;
  }
  inf.iters = it;
  inf.rel_res_true = rel_true;
  if (info) *info = inf;
  if (c->have_ev) {
    cudaEventRecord(c->ev[5], s);
    cudaEventSynchronize(c->ev[5]);
  }
  c->timing_on = false;
  timed_collect(c, (1u << kCatJdot) | (1u << kCatOp) | (1u << kCatHdot) | (1u << kCatHupd));
  c->launches_pcg = g_kernel_launches.load() - l0;
  h1w_status st = cuda_check(c, "pcg");
  if (st != H1W_OK) return st;
  if (prec_failed) return fail(c, H1W_ECUDA, "pcg: multigrid kernel attribute failed");
  int dst = 0;
  cudaMemcpyAsync(&dst, c->dstatus, sizeof(int), cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  if (dst & kStatusTimeout) return fail(c, H1W_ETIMEOUT, "pcg: a bounded device wait ran out");
  if (!(rel_true <= rtol)) return fail(c, H1W_ENOTCONV, "PCG did not reach rtol within maxit");
  return H1W_OK;
}

// ---- many systems in one graph ------------------------------------------------------

namespace {

struct BatchGraph {
  std::vector<unsigned long long> key;
  cudaGraphExec_t exec = nullptr;
  std::vector<long long> l_pre, l_body, l_post, l_cap;
};
std::mutex g_batch_mu;
BatchGraph g_batch;                    // the last batch graph (replayed while its key matches)
cudaStream_t g_batch_origin = nullptr;  // capture origin and launch stream
int g_batch_dev = -1;

unsigned long long bits_of(double v) {
  unsigned long long u;
  std::memcpy(&u, &v, sizeof(u));
  return u;
}

}  // namespace

h1w_status h1w_solve_batch_graph(h1w_ctx* const* ctxs, int32_t count, const int32_t* m, const double* const* J,
                                 const double* const* b, double* const* x, double rtol, int32_t maxit,
                                 h1w_info* info, h1w_status* status) {
  if (count < 0 || (count > 0 && (!ctxs || !m || !J || !b || !x)))
    return h1w::set_global_error(H1W_EINVAL, "h1w_solve_batch_graph: NULL arrays or negative count");
  if (!(rtol > 0.0) || maxit < 0) return h1w::set_global_error(H1W_EINVAL, "h1w_solve_batch_graph: bad rtol/maxit");
  for (int32_t i = 0; i < count; ++i) {
    h1w_ctx* c = ctxs[i];
    if (!c) return h1w::set_global_error(H1W_EINVAL, "h1w_solve_batch_graph: NULL context");
    if (m[i] < 0 || m[i] > c->m_max || (m[i] > 0 && !J[i]) || !b[i] || !x[i] || b[i] == x[i])
      return h1w::set_global_error(H1W_EINVAL, "h1w_solve_batch_graph: bad m, J, b or x of system " +
                                                   std::to_string(i));
    if (c->opt.precond != 0 && m[i] > 0)
      return h1w::set_global_error(H1W_EUNSUPPORTED, "h1w_solve_batch_graph: needs precond = 0");
    for (int32_t k = 0; k < i; ++k)
      if (ctxs[k] == c) return h1w::set_global_error(H1W_EINVAL, "h1w_solve_batch_graph: contexts must be distinct");
  }
  if (count == 0) return H1W_OK;
  std::lock_guard<std::mutex> lock(g_batch_mu);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return h1w::set_global_error(H1W_ECUDA, "h1w_solve_batch_graph: no device");
  std::vector<unsigned long long> key{(unsigned long long)count, bits_of(rtol), (unsigned long long)maxit,
                                      (unsigned long long)dev};
  for (int32_t i = 0; i < count; ++i) {
    const h1w_ctx* c = ctxs[i];
    key.insert(key.end(), {c->uid, (unsigned long long)m[i], (unsigned long long)(uintptr_t)J[i],
                           (unsigned long long)(uintptr_t)b[i], (unsigned long long)(uintptr_t)x[i],
                           (unsigned long long)c->stall, c->wait_ns});
  }
  for (int32_t i = 0; i < count; ++i) {  // host state of each system, as h1w_capacitance sets it
    h1w_ctx* c = ctxs[i];
    c->m = m[i];
    c->J = J[i];
    if (!ensure_cycle_stream(c)) return fail(c, H1W_ECUDA, "batch graph: cannot create the cycle stream");
    if (!c->cap_stream && cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
      return fail(c, H1W_ECUDA, "batch graph: cannot create the capture stream");
  }
  if (g_batch_dev != dev || !g_batch_origin) {
    if (cudaStreamCreateWithFlags(&g_batch_origin, cudaStreamNonBlocking) != cudaSuccess)
      return h1w::set_global_error(H1W_ECUDA, "h1w_solve_batch_graph: cannot create the origin stream");
    g_batch_dev = dev;
    if (g_batch.exec) cudaGraphExecDestroy(g_batch.exec);
    g_batch = BatchGraph{};
  }
  if (!g_batch.exec || g_batch.key != key) {
    if (g_batch.exec) cudaGraphExecDestroy(g_batch.exec);
    g_batch = BatchGraph{};
    for (int32_t i = 0; i < count; ++i) {
      const h1w_status st = capacitance_prepare(ctxs[i], m[i]);
      if (st != H1W_OK) return st;
    }
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> join(count, nullptr);
    bool ok = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) == cudaSuccess;
    for (int32_t i = 0; i < count && ok; ++i)
      ok = cudaEventCreateWithFlags(&join[i], cudaEventDisableTiming) == cudaSuccess;
    std::string why;
    if (ok && cudaStreamBeginCapture(g_batch_origin, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
      ok = false;
      why = "cudaStreamBeginCapture failed";
    }
    if (ok) {
      cudaEventRecord(fork, g_batch_origin);
      g_batch.l_pre.assign(count, 0);
      g_batch.l_body.assign(count, 0);
      g_batch.l_post.assign(count, 0);
      g_batch.l_cap.assign(count, 0);
      for (int32_t i = 0; i < count && ok; ++i) {
        h1w_ctx* c = ctxs[i];
        const cudaStream_t orig = c->stream;
        c->stream = c->cap_stream;
        c->capturing = true;
        cudaStreamWaitEvent(c->stream, fork, 0);
        const long long l0 = g_kernel_launches.load();
        if (capacitance_core(c, m[i], J[i], nullptr) != H1W_OK) {
          ok = false;
          why = c->err;
        }
        g_batch.l_cap[i] = g_kernel_launches.load() - l0;
        if (ok) {
          launch_pcg_set_scalars(c->scal, rtol, maxit, 1, c->stream);
          ok = capture_pcg(c, b[i], x[i], m[i] == 0);
          if (!ok) why = c->err;
          g_batch.l_pre[i] = c->pcg_l_pre + 1;
          g_batch.l_body[i] = c->pcg_l_body;
          g_batch.l_post[i] = c->pcg_l_post;
        }
        cudaEventRecord(join[i], c->stream);
        cudaStreamWaitEvent(g_batch_origin, join[i], 0);
        c->capturing = false;
        c->stream = orig;
      }
      cudaGraph_t g = nullptr;
      const cudaError_t e = cudaStreamEndCapture(g_batch_origin, &g);
      if (ok && (e != cudaSuccess || !g)) {
        ok = false;
        why = std::string("capture failed: ") + cudaGetErrorString(e);
      }
      if (ok) {
        const cudaError_t ei = cudaGraphInstantiate(&g_batch.exec, g, 0);
        if (ei != cudaSuccess) {
          ok = false;
          g_batch.exec = nullptr;
          why = std::string("instantiation failed: ") + cudaGetErrorString(ei);
        }
      }
      if (g) cudaGraphDestroy(g);
    }
    for (int32_t i = 0; i < count; ++i) ctxs[i]->capturing = false;
    if (fork) cudaEventDestroy(fork);
    for (cudaEvent_t e : join)
      if (e) cudaEventDestroy(e);
    cudaGetLastError();
    if (!ok) {
      g_batch = BatchGraph{};
      return h1w::set_global_error(H1W_ECUDA, "h1w_solve_batch_graph: " + why);
    }
    g_batch.key = key;
  }
  for (int32_t i = 0; i < count; ++i) {  // the graph starts after the work queued on each system's stream
    if (!ctxs[i]->order_ev && cudaEventCreateWithFlags(&ctxs[i]->order_ev, cudaEventDisableTiming) != cudaSuccess)
      return fail(ctxs[i], H1W_ECUDA, "batch graph: cannot create an event");
    cudaEventRecord(ctxs[i]->order_ev, ctxs[i]->stream);
    cudaStreamWaitEvent(g_batch_origin, ctxs[i]->order_ev, 0);
  }
  if (cudaGraphLaunch(g_batch.exec, g_batch_origin) != cudaSuccess || cudaStreamSynchronize(g_batch_origin) != cudaSuccess)
    return h1w::set_global_error(H1W_ECUDA, std::string("h1w_solve_batch_graph: ") +
                                                cudaGetErrorString(cudaGetLastError()));
  h1w_status first = H1W_OK;
  for (int32_t i = 0; i < count; ++i) {
    h1w_ctx* c = ctxs[i];
    double sc[16] = {};
    int dst = 0;
    cudaMemcpy(sc, c->scal, sizeof(sc), cudaMemcpyDeviceToHost);
    cudaMemcpy(&dst, c->dstatus, sizeof(int), cudaMemcpyDeviceToHost);
    h1w_info inf{0, 0, 0.0, 0.0};
    inf.iters = (int)sc[kSlotIt];
    const double bb = sc[kSlotBB];
    inf.rel_res_true = bb > 0.0 ? std::sqrt(sc[kSlotRRTrue] / bb) : 0.0;
    inf.rel_res_rec = bb > 0.0 ? std::sqrt(sc[kSlotRR] / bb) : 0.0;
    c->launches_cap = g_batch.l_cap[i];
    c->launches_pcg = g_batch.l_pre[i] + (long long)inf.iters * g_batch.l_body[i] + g_batch.l_post[i];
    h1w_status st = H1W_OK;
    if (dst & kStatusNotSpd) {
      c->m = -1;
      st = fail(c, H1W_ENOTSPD, "capacitance matrix is not numerically positive definite");
    } else if (dst & kStatusTimeout) {
      st = fail(c, H1W_ETIMEOUT, "batch graph: a bounded device wait ran out");
    } else if (!(inf.rel_res_true <= rtol) && inf.iters < maxit && std::isfinite(inf.rel_res_true)) {
      // the recursive residual met rtol but the true one did not: continue this system with
      // restarts from its true residual, as h1w_pcg does
      st = h1w_pcg(c, b[i], x[i], rtol, maxit, &inf);
    } else if (!(inf.rel_res_true <= rtol)) {
      st = fail(c, H1W_ENOTCONV, "PCG did not reach rtol within maxit");
    }
    if (info) info[i] = inf;
    if (status) status[i] = st;
    if (first == H1W_OK && st != H1W_OK) first = st;
  }
  if (cudaGetLastError() != cudaSuccess)
    return h1w::set_global_error(H1W_ECUDA, "h1w_solve_batch_graph: a CUDA call failed");
  if (first != H1W_OK)
    h1w::set_global_error(first, "h1w_solve_batch_graph: a system failed (see its context's last error)");
  return first;
}

// ---- autotuner: right-hand sides per batched V-cycle --------------------------------

namespace {

constexpr int kTuneCandidates[] = {8, 16, 32, 64, 128, 256};

struct TuneKey {
  int disc, n0, n1, n2, m, cheb, unfused;
  bool operator<(const TuneKey& o) const {
    return std::tie(disc, n0, n1, n2, m, cheb, unfused) < std::tie(o.disc, o.n0, o.n1, o.n2, o.m, o.cheb, o.unfused);
  }
};
std::mutex g_tune_mu;
std::map<TuneKey, std::pair<int, float>> g_tune_cache;

// distinct effective block sizes: a context never batches more than m rows
std::vector<int> tune_candidates(int m) {
  std::vector<int> out;
  for (int rb : kTuneCandidates) {
    const int eff = std::min(rb, std::max(m, 1));
    if (out.empty() || out.back() != eff) out.push_back(eff);
  }
  return out;
}

}  // namespace

size_t h1w_autotune_workspace_size(const h1w_grid* grid, int32_t m, const h1w_options* base) {
  h1w_options o;
  h1w_default_options(&o);
  if (base) o = *base;
  size_t need = 0;
  for (int rb : tune_candidates(m)) {
    o.rhs_block = rb;
    const size_t s = h1w_workspace_size(grid, m, &o);
    if (s == 0) return 0;
    need = std::max(need, s);
  }
  return need;
}

h1w_status h1w_autotune(const h1w_grid* grid, int32_t m, const h1w_options* base, void* workspace, size_t ws_bytes,
                        void* stream, h1w_options* out, float* ms_per_rhs) {
  if (!grid || !out) return h1w::set_global_error(H1W_EINVAL, "h1w_autotune: grid and out must be non-NULL");
  h1w_options o;
  h1w_default_options(&o);
  if (base) o = *base;
  *out = o;
  if (ms_per_rhs) *ms_per_rhs = 0.f;
  if (m <= 0 || o.mg_arith != 0 || o.precond != 0) return H1W_OK;  // nothing to tune on these paths
  const TuneKey key{grid->disc, grid->n[0], grid->n[1], grid->n[2], m, o.cheb_degree, o.mg_unfused};
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      out->rhs_block = it->second.first;
      if (ms_per_rhs) *ms_per_rhs = it->second.second;
      return H1W_OK;
    }
  }
  const size_t need = h1w_autotune_workspace_size(grid, m, &o);
  if (need == 0) return h1w::set_global_error(H1W_EINVAL, "h1w_autotune: invalid grid or options");
  if (!workspace || ws_bytes < need)
    return h1w::set_global_error(H1W_ENOMEM, "h1w_autotune: workspace too small: need " + std::to_string(need));
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return h1w::set_global_error(H1W_ECUDA, "h1w_autotune: cannot create events");
  std::vector<std::pair<int, float>> timed_rb;
  h1w_status st = H1W_OK;
  for (int rb : tune_candidates(m)) {
    h1w_options oc = o;
    oc.rhs_block = rb;
    h1w_ctx* c = nullptr;
    st = h1w_setup(grid, m, &oc, workspace, ws_bytes, stream, &c);
    if (st != H1W_OK) break;
    const int nr = std::min(rb, m);
    // any finite values will do: the cycle's cost does not depend on them
    launch_fill(reinterpret_cast<double*>(c->Jdf), 1e-3, (int64_t)nr * c->lev[0].N, c->stream);
    bool ok = vcycle_many(c, nr, nullptr, c->Jdf, nullptr, c->Hdf);  // warm-up (kernel attributes)
    cudaEventRecord(e0, c->stream);
    for (int r = 0; r < 2 && ok; ++r) ok = vcycle_many(c, nr, nullptr, c->Jdf, nullptr, c->Hdf);
    cudaEventRecord(e1, c->stream);
    float ms = 0.f;
    const bool timed = cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
    h1w_destroy(c);
    if (!ok || !timed) {
      st = h1w::set_global_error(H1W_ECUDA, "h1w_autotune: timing the batched V-cycle failed");
      break;
    }
    timed_rb.push_back({rb, ms / (2.0f * nr)});
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != H1W_OK) return st;
  // the smallest block within 5 % of the fastest: the V-cycle buffers grow with the block
  float fastest = timed_rb[0].second;
  for (const auto& t : timed_rb) fastest = std::min(fastest, t.second);
  int best = timed_rb.back().first;
  float best_ms = timed_rb.back().second;
  for (const auto& t : timed_rb)
    if (t.second <= 1.05f * fastest) {
      best = t.first;
      best_ms = t.second;
      break;
    }
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache[key] = {best, best_ms};
  }
  out->rhs_block = best;
  if (ms_per_rhs) *ms_per_rhs = best_ms;
  return H1W_OK;
}

h1w_status h1w_capacitance_factors(h1w_ctx* c, double* C, double* L) {
  if (!c) return H1W_EINVAL;
  if (c->m < 0) return fail(c, H1W_ESTATE, "call h1w_capacitance first");
  if (c->opt.precond == 1) return fail(c, H1W_ESTATE, "precond = 1 forms no capacitance matrix");
  const size_t bytes = sizeof(double) * c->m * c->m;
  if (C && bytes) h1w::launch_copy(C, c->C, (int64_t)c->m * c->m, c->stream);
  if (L && bytes) h1w::launch_copy(L, c->Lc, (int64_t)c->m * c->m, c->stream);
  return cuda_check(c, "capacitance_factors");
}

h1w_status h1w_get_timings(const h1w_ctx* c, h1w_timings* out) {
  if (!c || !out) return H1W_EINVAL;
  h1w_timings t{};
  if (c->have_ev) {
    auto el = [&](int a, int b) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, c->ev[a], c->ev[b]) != cudaSuccess) ms = 0.f;
      return ms;
    };
    if (c->m > 0) {
      t.t_H_ms = el(0, 1);
      t.t_C_ms = el(1, 2);
      t.t_chol_ms = el(2, 3);
    }
    t.t_pcg_ms = el(4, 5);
  }
  cudaGetLastError();  // elapsed-time queries on unrecorded events are not errors here
  t.launches_capacitance = c->launches_cap;
  t.launches_pcg = c->launches_pcg;
  t.t_gemm_kernel_ms = c->cat_ms[kCatGemm];
  t.t_jdot_ms = c->cat_ms[kCatJdot];
  t.t_op_ms = c->cat_ms[kCatOp];
  t.t_hdot_ms = c->cat_ms[kCatHdot];
  t.t_hupd_ms = c->cat_ms[kCatHupd];
  t.n_gemm_kernel = c->cat_n[kCatGemm];
  t.n_jdot = c->cat_n[kCatJdot];
  t.n_op = c->cat_n[kCatOp];
  t.n_hdot = c->cat_n[kCatHdot];
  t.n_hupd = c->cat_n[kCatHupd];
  t.t_vc_down_ms = c->cat_ms[kCatDown];
  t.t_vc_up_ms = c->cat_ms[kCatUp];
  t.n_vc_down = c->cat_n[kCatDown];
  t.n_vc_up = c->cat_n[kCatUp];
  t.t_split_j_ms = c->cat_ms[kCatSplitJ];
  t.t_split_h_ms = c->cat_ms[kCatSplitH];
  t.t_d2df_ms = c->cat_ms[kCatD2df];
  t.n_split_j = c->cat_n[kCatSplitJ];
  t.n_split_h = c->cat_n[kCatSplitH];
  t.n_d2df = c->cat_n[kCatD2df];
  *out = t;
  return H1W_OK;
}

h1w_status h1w_level_info(const h1w_ctx* c, int32_t level, int32_t* nlevels, int32_t* n) {
  if (!c) return H1W_EINVAL;
  if (nlevels) *nlevels = c->nlev;
  if (n) {
    if (level < 0 || level >= c->nlev) return H1W_EINVAL;
    n[0] = c->lev[level].nx; n[1] = c->lev[level].ny; n[2] = c->lev[level].nz;
  }
  return H1W_OK;
}

const char* h1w_last_error(const h1w_ctx* c) {
  if (!c) return g_setup_error.c_str();
  return c->err.c_str();
}

size_t h1w_direct_workspace_size(const h1w_ctx* c) {
  if (!c || c->lev[0].N > H1W_DIRECT_MAX_N) return 0;
  return sizeof(double) * (size_t)c->lev[0].N * (size_t)c->lev[0].N + 256;
}

h1w_status h1w_solve_direct(h1w_ctx* c, const double* b, double* x, void* workspace, size_t ws_bytes) {
  if (!c) return h1w::set_global_error(H1W_EINVAL, "h1w_solve_direct: NULL context");
  if (!b || !x || !workspace) return fail(c, H1W_EINVAL, "h1w_solve_direct: NULL argument");
  const size_t need = h1w_direct_workspace_size(c);
  if (need == 0) return fail(c, H1W_EUNSUPPORTED, "h1w_solve_direct: grid larger than H1W_DIRECT_MAX_N");
  if (ws_bytes < need - 256) return fail(c, H1W_EINVAL, "h1w_solve_direct: workspace too small");
  if (c->m < 0) return fail(c, H1W_ESTATE, "call h1w_capacitance first");
  const int n = (int)c->lev[0].N;
  double* A = static_cast<double*>(workspace);
  cudaMemsetAsync(A, 0, sizeof(double) * (size_t)n * n, c->stream);
  launch_assemble_dense(c->disc, c->lev[0], A, c->stream);          // K + M
  launch_dense_gn(A, n, c->grid.alpha, c->J, c->m, c->stream);       // alpha (K + M) + J^T J
  cudaMemsetAsync(c->dstatus, 0, sizeof(int), c->stream);
  launch_chol(A, n, c->dstatus, c->stream);
  if (x != b) h1w::launch_copy(x, b, (int64_t)n, c->stream);
  launch_trsv_lower(A, n, x, 1, c->stream);
  launch_trsv_upper_t(A, n, x, 1, c->stream);
  int status = 0;
  cudaMemcpyAsync(&status, c->dstatus, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  const cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return fail(c, H1W_ECUDA, std::string("h1w_solve_direct: ") + cudaGetErrorString(e));
  const h1w_status st = cuda_check(c, "h1w_solve_direct");
  if (st != H1W_OK) return st;
  if (status & kStatusNotSpd) return fail(c, H1W_ENOTSPD, "h1w_solve_direct: matrix is not numerically positive definite");
  return H1W_OK;
}

size_t h1w_ert_workspace_size(const h1w_ctx* c, int32_t n_e, int32_t m) {
  if (!c || c->disc != H1W_FV_CELL) return 0;
  return h1w::ert_workspace_bytes(c->lev, c->nlev, n_e, m);
}

h1w_status h1w_forward(h1w_ctx* c, const h1w_survey* survey, const double* logsigma, double* U, double* g,
                       void* workspace, size_t ws_bytes, double rtol, int32_t maxit, uint32_t flags,
                       h1w_info* info) {
  if (!c) return h1w::set_global_error(H1W_EINVAL, "h1w_forward: NULL context");
  if (c->disc != H1W_FV_CELL) return fail(c, H1W_EUNSUPPORTED, "h1w_forward: needs an H1W_FV_CELL grid");
  std::string err;
  if (flags & ~H1W_FORWARD_WARM_START) return fail(c, H1W_EINVAL, "h1w_forward: unknown flags");
  const h1w_status st = h1w::ert_forward(c->lev, c->nlev, c->stream, survey, logsigma, U, g, workspace, ws_bytes,
                                         rtol, maxit, (flags & H1W_FORWARD_WARM_START) != 0, c->opt.cheb_ratio,
                                         info, err);
  return st == H1W_OK ? st : fail(c, st, err);
}

h1w_status h1w_adjoint(h1w_ctx* c, const h1w_survey* survey, const double* logsigma, const double* U,
                       const double* r, double* JTr, double* J, void* workspace, size_t ws_bytes) {
  if (!c) return h1w::set_global_error(H1W_EINVAL, "h1w_adjoint: NULL context");
  if (c->disc != H1W_FV_CELL) return fail(c, H1W_EUNSUPPORTED, "h1w_adjoint: needs an H1W_FV_CELL grid");
  std::string err;
  const h1w_status st =
      h1w::ert_adjoint(c->lev, c->nlev, c->stream, survey, logsigma, U, r, JTr, J, workspace, ws_bytes, err);
  return st == H1W_OK ? st : fail(c, st, err);
}

h1w_status h1w_ert_jvp(h1w_ctx* c, const h1w_survey* survey, const double* logsigma, const double* U,
                       const double* p, double* Jp, void* workspace, size_t ws_bytes) {
  if (!c) return h1w::set_global_error(H1W_EINVAL, "h1w_ert_jvp: NULL context");
  if (c->disc != H1W_FV_CELL) return fail(c, H1W_EUNSUPPORTED, "h1w_ert_jvp: needs an H1W_FV_CELL grid");
  std::string err;
  const h1w_status st = h1w::ert_jvp(c->lev, c->nlev, c->stream, survey, logsigma, U, p, Jp, workspace, ws_bytes, err);
  return st == H1W_OK ? st : fail(c, st, err);
}

h1w_status h1w_gn_step(h1w_ctx* c, const h1w_survey* survey, const double* g_obs, const double* m_ref,
                       double* mvec, double* U, double* J, double* g, double* scratch, void* ert_ws,
                       size_t ert_ws_bytes, double rtol_fwd, double rtol, int32_t maxit, uint32_t fwd_flags,
                       h1w_gn_info* info) {
  if (!c) return h1w::set_global_error(H1W_EINVAL, "h1w_gn_step: NULL context");
  if (!survey || !g_obs || !m_ref || !mvec || !J || !g || !scratch)
    return fail(c, H1W_EINVAL, "h1w_gn_step: NULL argument");
  if (survey->m < 1 || survey->m > c->m_max) return fail(c, H1W_EINVAL, "h1w_gn_step: need 1 <= survey->m <= m_max");
  const int64_t N = c->lev[0].N;
  const int m = survey->m;
  double* dmr = scratch;        // m - m_ref
  double* b = scratch + N;      // GN right-hand side
  double* dm = scratch + 2 * N;  // the step
  double* d = scratch + 3 * N;  // g_m - g_obs
  h1w_info fi{}, pi{};
  h1w_status st = h1w_forward(c, survey, mvec, U, g, ert_ws, ert_ws_bytes, rtol_fwd, maxit, fwd_flags, &fi);
  if (st != H1W_OK) return st;
  st = h1w_adjoint(c, survey, mvec, U, nullptr, nullptr, J, ert_ws, ert_ws_bytes);
  if (st != H1W_OK) return st;
  h1w::launch_copy(d, g, (int64_t)m, c->stream);
  h1w::launch_axpby(d, -1.0, g_obs, 1.0, m, c->stream);
  h1w::launch_copy(dmr, mvec, (int64_t)N, c->stream);
  h1w::launch_axpby(dmr, -1.0, m_ref, 1.0, N, c->stream);
  std::vector<double> dh(m);
  cudaMemcpyAsync(dh.data(), d, sizeof(double) * m, cudaMemcpyDeviceToHost, c->stream);
  st = h1w_capacitance(c, m, J);
  if (st != H1W_OK) return st;
  st = h1w_gn_rhs(c, dmr, d, b);
  if (st != H1W_OK) return st;
  st = h1w_pcg(c, b, dm, rtol, maxit, &pi);
  if (st != H1W_OK) return st;
  h1w::launch_axpby(mvec, 1.0, dm, 1.0, N, c->stream);
  h1w::launch_dot_partial(dm, dm, N, c->partial, c->stream);
  std::vector<double> part(h1w::dot_blocks(N));
  cudaMemcpyAsync(part.data(), c->partial, sizeof(double) * part.size(), cudaMemcpyDeviceToHost, c->stream);
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return cuda_check(c, "h1w_gn_step");
  st = cuda_check(c, "h1w_gn_step");
  if (st != H1W_OK) return st;
  if (info) {
    double mis = 0.0, sn = 0.0;
    for (double v : dh) mis += v * v;
    for (double v : part) sn += v;
    info->fwd_iters = fi.iters;
    info->gn_iters = pi.iters;
    info->misfit = std::sqrt(mis);
    info->rel_res_true = pi.rel_res_true;
    info->step_norm = std::sqrt(sn);
  }
  return H1W_OK;
}

h1w_status h1w_set_pcg_mode(h1w_ctx* c, int32_t mode) {
  if (!c) return h1w::set_global_error(H1W_EINVAL, "h1w_set_pcg_mode: NULL context");
  if (mode != 0 && mode != 1) return fail(c, H1W_EINVAL, "h1w_set_pcg_mode: mode must be 0 or 1");
  c->opt.pcg_mode = mode;
  return H1W_OK;
}

h1w_status h1w_inject_stall(h1w_ctx* c, int32_t kind, int64_t wait_limit_ns) {
  if (!c) return h1w::set_global_error(H1W_EINVAL, "h1w_inject_stall: NULL context");
  if (kind != H1W_STALL_NONE && kind != H1W_STALL_CAP_GEMM && kind != H1W_STALL_PREC_SOLVE)
    return fail(c, H1W_EINVAL, "h1w_inject_stall: unknown kind");
  if (wait_limit_ns < 0 || wait_limit_ns > 60000000000ll)
    return fail(c, H1W_EINVAL, "h1w_inject_stall: wait_limit_ns out of range [0, 60 s]");
  c->stall = kind;
  c->wait_ns = wait_limit_ns > 0 ? (unsigned long long)wait_limit_ns : 1000000000ull;
  return H1W_OK;
}

h1w_status h1w_cholesky(h1w_ctx* c, int32_t n, double* A) {
  if (!c) return h1w::set_global_error(H1W_EINVAL, "h1w_cholesky: NULL context");
  if (n < 1 || n > H1W_CHOLESKY_MAX_N) return fail(c, H1W_EINVAL, "h1w_cholesky: n out of range");
  if (!A) return fail(c, H1W_EINVAL, "h1w_cholesky: A is NULL");
  cudaMemsetAsync(c->dstatus, 0, sizeof(int), c->stream);
  launch_chol(A, n, c->dstatus, c->stream);
  int status = 0;
  cudaMemcpyAsync(&status, c->dstatus, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  const cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return fail(c, H1W_ECUDA, std::string("h1w_cholesky: ") + cudaGetErrorString(e));
  const h1w_status st = cuda_check(c, "h1w_cholesky");
  if (st != H1W_OK) return st;
  if (status & kStatusNotSpd)
    return fail(c, H1W_ENOTSPD, "h1w_cholesky: a pivot is not positive (the matrix is not numerically SPD)");
  return H1W_OK;
}

void h1w_destroy(h1w_ctx* c) {
  if (!c) return;
  if (c->copy_stream) {
    cudaStreamSynchronize(c->copy_stream);
    cudaStreamDestroy(c->copy_stream);
  }
  for (HostCopy& h : c->hcopy) {
    for (cudaEvent_t e : h.beg) cudaEventDestroy(e);
    for (cudaEvent_t e : h.end) cudaEventDestroy(e);
  }
  for (cudaEvent_t e : c->cyc_beg) cudaEventDestroy(e);
  for (cudaEvent_t e : c->cyc_end) cudaEventDestroy(e);
  if (c->order_ev) cudaEventDestroy(c->order_ev);
  if (c->cycle_stream) {
    cudaStreamSynchronize(c->cycle_stream);
    cudaStreamDestroy(c->cycle_stream);
    for (int e = 0; e < 2; ++e)
      if (c->cycle_ev[e]) cudaEventDestroy(c->cycle_ev[e]);
  }
  for (h1w_ctx::PcgGraph& e : c->pcg_g)
    if (e.exec) cudaGraphExecDestroy(e.exec);
  if (c->body_stream) {
    cudaStreamSynchronize(c->body_stream);
    cudaStreamDestroy(c->body_stream);
  }
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->have_ev) {
    for (int e = 0; e < 6; ++e) cudaEventDestroy(c->ev[e]);
    for (int t = 0; t < h1w_ctx::kTimed; ++t)
      for (int e = 0; e < 2; ++e) cudaEventDestroy(c->kev[t][e]);
  }
  delete c;
}

}  // extern "C"
