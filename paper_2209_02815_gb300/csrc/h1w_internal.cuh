// Internal declarations shared by the h1w CUDA translation units.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <string>
#include <vector>

#include "df64.cuh"
#include "h1w.h"

namespace h1w {

constexpr int kMaxLevels = 16;
constexpr int kCoarseTarget = 512;   // stop coarsening once a level has <= this many unknowns
constexpr int kCoarseLimit = 1024;   // largest coarsest level accepted for the dense solve
constexpr int kMaxM = 4096;          // largest number of measurements accepted

// One multigrid level. Plain data, passed to kernels by value.
//  FV (3D cell-centred): (A u)_c = V u_c + sum_d T_d sum_{nb c' along d} (u_c - u_c').
//  Q1 (2D vertex): A = Kx (x) My + Mx (x) Ky + Dx (x) Dy with symmetric
//  tridiagonal 1D factors stored as six arrays of length n per axis:
//  [Kd, Ko, Md, Mo, Dd, Do] (diagonal, and coupling (i, i+1) at index i).
struct Level {
  int nx, ny, nz;
  int64_t N;
  double Tx, Ty, Tz, V;         // FV coefficients
  const double* qx;              // Q1 x-axis coefficients [6][nx] (device)
  const double* qy;              // Q1 y-axis coefficients [6][ny] (device)
  const df* q1st;                // Q1 double-float cycle: per-vertex stencil [9][N] and 1/diag [N] (device)
  // Q1: the box of vertices [q1_ilo, q1_ihi] x [q1_jlo, q1_jhi] whose stencil and 1/diag equal
  // q1c (the table's entries there, read back at setup); empty when ilo > ihi
  int q1_ilo, q1_ihi, q1_jlo, q1_jhi;
  df q1c[10];
  df q1w[9];                     // q1c[k] q1c[9]: a coupling times the box's inverse diagonal
  double lam;                    // upper bound of spec(D^-1 A) (Gershgorin)
  int cx, cy, cz;                // axis coarsened towards the next level
  int iso;                       // FV with Tx == Ty == Tz
  // FV diagonal and its inverse by neighbour counts (cx + 3 cy + 9 cz, each 0..2)
  double fv_diag[27];
  double fv_dinv[27];
  // the same FV coefficients as double-floats (double-float V-cycle)
  df fvd_diag[27];
  df fvd_dinv[27];
  df fvd_T[3];
};

// Per-class coefficients of the fused degree-2 smoothing legs (mg_fused.cu), class
// c = cx + 3 cy + 9 cz by neighbour counts: d = diagonal of A, dinv = 1 / d,
// gam = c2 / (theta d), del = 1 / (theta d), eta = beta / d, kap = c2 / d with
// beta = (1 + c1) / theta + c2 (1 - 1 / theta) (theta, c1, c2 of the level's smoother);
// T = face coefficients (Tx, Ty, Tz).
struct FusedCoef {
  df d[27], dinv[27], gam[27], del[27], eta[27], kap[27];
  df gamT[27], kapT[27];  // gam T and kap T on isotropic levels (T = T[0] = T[1] = T[2])
  df T[3];
  df beta;
};

struct ChebCoef {
  double inv_theta;   // 1 / theta
  double c1[8];       // rho_j rho_{j-1} for step j (1-based; index 0 unused)
  double c2[8];       // 2 rho_j / delta
  df inv_theta_df, c1_df[8], c2_df[8];  // the same as double-floats
  // degree 2 collapsed into one pass: x += D^-1 [beta r0 + c2t N(D^-1 r0)], A = D - N
  df beta_df, c2t_df;
};

// Kernels launched by this library in this process (every launcher adds its count).
extern std::atomic<long long> g_kernel_launches;
inline void note_launches(int k) { g_kernel_launches.fetch_add(k, std::memory_order_relaxed); }

// Records msg as the thread's last error (h1w_last_error(NULL)) and returns st.
h1w_status set_global_error(h1w_status st, const std::string& msg);

// Device status word bits (written by kernels, read back by the host).
enum : int { kStatusNotSpd = 1, kStatusTimeout = 2 };

// Device buffers of the tensor-core capacitance GEMM (ozaki_gemm.cu).
struct OzakiWork {
  void* digitsA;                 // BF16 digits of a K panel of J, stage-tiled (128-row blocks)
  void* digitsB;                 // BF16 digits of the same panel of H, stage-tiled (64-row blocks)
  int* expo;                     // chunk exponents [N/1024][m] of J, then of H
  int* tiles;                    // [2 * tiles] (row block, column block)
  double* partial;               // [splits][m][m]
  int* status;                   // device status word
  long long klen;                // K panel width (multiple of 2048)
  unsigned long long wait_ns;    // limit of each bounded wait (0: one second)
  int stall;                     // failure-path test: withhold the operand copies (see h1w_inject_stall)
  bool j_full = false;           // digitsA holds every K panel of J, split during line H
                                 // (launch_split_j_rows); line C then splits only H
};
long long ozaki_panel_width(long long N);
long long ozaki_chunks(long long N);
int ozaki_digit_slices();  // BF16 digit slices per operand entry
int ozaki_num_tiles(int m);
constexpr int kMaxSms = 256;  // SM counts above this are treated as this many
// K splits per panel for a GPU with sms SMs; never above ozaki_max_splits(m)
int ozaki_splits(int m, long long kp, int sms);
int ozaki_max_splits(int m);
bool ozaki_supported();
// Each operand as FP64 (J, H) or, when its double-float copy (Jdf, Hdf) is given, as that.
// hook (may be null) is called as hook(hook_arg, which, 1) before and hook(hook_arg, which, 0)
// after each launch, which = kOzakiSplitJ, kOzakiSplitH (digit splits) or kOzakiGemm.
enum { kOzakiGemm = 0, kOzakiSplitJ = 1, kOzakiSplitH = 2 };
// J digits of every K panel kept between lines H and C while they take at most this much
constexpr long long kJDigitsFullMax = 32LL << 30;
size_t ozaki_j_digits_full_bytes(int m, long long N);
// Line H's conversion of J rows [r0, r1) to double-floats (Jdf) fused with their digit split
// for every K panel into the full-K buffer of w (w.j_full): one pass over those rows of J.
// The launch that ends at row m also zeroes the digits of the last row block's padding rows.
void launch_split_j_rows(const double* J, int m, long long N, int r0, int r1, const OzakiWork& w, df* Jdf,
                         cudaStream_t s);
bool launch_ozaki_capacitance(const double* J, const double* H, const df* Jdf, const df* Hdf, int m, long long N,
                              const OzakiWork& w, int splits, cudaStream_t s, void (*hook)(void*, int, int),
                              void* hook_arg);
void ozaki_tiles(int m, std::vector<int>& out);

// ---- kernel launchers (mg_kernels.cu) --------------------------------------
// r = b - A x (r = b when zero_x); d = D^-1 r / theta; x = d only when zero_x
void launch_cheb_first(int disc, const Level& L, int nrhs, const double* b, double* x, double* r,
                       double* d, bool zero_x, double inv_theta, cudaStream_t s);
// r -= A d_old; d_new = c1 d_old + c2 D^-1 r; x += d_new (+ d_old when add_old)
void launch_cheb_step(int disc, const Level& L, int nrhs, double* r, const double* d_old,
                      double* d_new, double* x, double c1, double c2, bool add_old, cudaStream_t s);
void launch_add(int64_t n, const double* d, double* x, cudaStream_t s);
void launch_residual(int disc, const Level& L, int nrhs, const double* b, const double* x,
                     double* r, cudaStream_t s);
void launch_restrict(int disc, const Level& Lf, const Level& Lc, int nrhs, const double* rf,
                     double* bc, cudaStream_t s);
void launch_prolong_add(int disc, const Level& Lf, const Level& Lc, int nrhs, const double* xc,
                        double* xf, cudaStream_t s);
void launch_gershgorin(int disc, const Level& L, unsigned long long* out_bits, cudaStream_t s);
void launch_assemble_dense(int disc, const Level& L, double* A, cudaStream_t s);
// out = ca * (A p) + cj * sum_i J[i][k] w[i]; partial[block] = sum_k p_k out_k when partial != null.
void launch_apply_op(int disc, const Level& L, double ca, const double* p, double cj,
                     const double* J, const double* w, int m, double* out, double* partial,
                     int* nblocks_out, cudaStream_t s);
int apply_op_blocks(const Level& L);
// the same with J stored as double-floats (Jd, m x N)
void launch_apply_op_df(int disc, const Level& L, double ca, const double* p, double cj, const df* Jd,
                        const double* w, int m, double* out, double* partial, int* nblocks_out, cudaStream_t s);
// ---- double-float V-cycle on FV grids (mg_df64.cu) ----------------------------
void launch_cheb_first_df(const Level& L, int nrhs, const df* b, df* x, df* r, df* d, bool zero_x, df inv_theta,
                          cudaStream_t s);
void launch_cheb_step_df(const Level& L, int nrhs, df* r, const df* d_old, df* d_new, df* x, df c1, df c2,
                         bool add_old, cudaStream_t s);
void launch_add_df(int64_t n, const df* d, df* x, cudaStream_t s);
void launch_residual_df(const Level& L, int nrhs, const df* b, const df* x, df* r, cudaStream_t s);
void launch_restrict_df(const Level& Lf, const Level& Lc, int nrhs, const df* rf, df* bc, cudaStream_t s);
void launch_prolong_add_df(const Level& Lf, const Level& Lc, int nrhs, const df* xc, df* xf, cudaStream_t s);
void launch_coarse_apply_df(const double* X, int n, int nrhs, const df* b, df* x, cudaStream_t s);
void launch_d2df(int64_t n, const double* src, df* dst, cudaStream_t s);
// dst = src as FP64; dst2 (may be null) receives a copy of the double-floats
void launch_df2d(int64_t n, const df* src, double* dst, df* dst2, cudaStream_t s);
// The double-float cycle on 2D Q1 levels (one kernel per step): per-vertex stencil tables
// (launch_q1_stencil_df fills L.q1st's storage from L.qx, L.qy), smoothing steps, residual
// and vertex transfers, as the FV ones above.
void launch_q1_stencil_df(const Level& L, df* st, cudaStream_t s);
void launch_q1_cheb_first_df(const Level& L, int nrhs, const df* b, df* x, df* r, df* d, bool zero_x, df inv_theta,
                             cudaStream_t s);
void launch_q1_cheb_step_df(const Level& L, int nrhs, df* r, const df* d_old, df* d_new, df* x, df c1, df c2,
                            bool add_old, cudaStream_t s);
void launch_q1_smooth_df(const Level& L, int nrhs, const df* r0, df* x, bool zero_x, df beta, df c2t,
                         cudaStream_t s);
void launch_q1_residual_df(const Level& L, int nrhs, const df* b, const df* x, df* r, cudaStream_t s);
void launch_q1_restrict_df(const Level& Lf, const Level& Lc, int nrhs, const df* rf, df* bc, cudaStream_t s);
void launch_q1_prolong_add_df(const Level& Lf, const Level& Lc, int nrhs, const df* xc, df* xf, cudaStream_t s);

// Fused smoothing passes on a level with all three axes coarsened 2:1 and the degree-2
// smoother: down leg (x = S(b) from zero, bc = P^T (b - A x)) and up leg (y = S(x + P xc)
// started from the corrected x; y and/or y64 may be null, not both). False if the level
// does not qualify or the kernel attribute for its shared memory could not be set
// (nothing launched).
bool fused_level_ok(const Level& L);  // all axes coarsened and nx ny < 2^26
// b (the level's right-hand sides) as double-floats or as FP64 (split on the fly).
bool launch_pre_fused_df(const Level& L, const Level& Lc, const FusedCoef& F, int nrhs, const df* b, df* x,
                         df* bc, cudaStream_t s);
bool launch_pre_fused_df(const Level& L, const Level& Lc, const FusedCoef& F, int nrhs, const double* b, df* x,
                         df* bc, cudaStream_t s);
bool launch_post_fused_df(const Level& L, const Level& Lc, const FusedCoef& F, int nrhs, const df* x,
                          const df* xc, const df* b, df* y, double* y64, cudaStream_t s);
bool launch_post_fused_df(const Level& L, const Level& Lc, const FusedCoef& F, int nrhs, const df* x,
                          const df* xc, const double* b, df* y, double* y64, cudaStream_t s);

// ---- dense / Krylov kernels (dense_kernels.cu) ------------------------------
// partial[c * m + i] = sum_{k in chunk c} A[i * lda + k] v[k]
int rows_dot_chunks(int64_t N);
void launch_rows_dot(const double* A, int m, int64_t N, const double* v, double* partial,
                     cudaStream_t s);
// out[i] = scale * sum_c partial[c * m + i]
void launch_reduce_partials(const double* partial, int nchunks, int m, double scale, double* out,
                            cudaStream_t s);
// z_k = (z0_k - (1/alpha) sum_i H[i][k] v_i) / alpha; partial[block] = sum r_k z_k
int colsum_blocks(int64_t N);
void launch_woodbury_update(const double* H, int m, int64_t N, const double* v, const double* z0,
                            double alpha, double* z, const double* r, double* partial,
                            cudaStream_t s);
// the same two preconditioner passes with H (and v) stored as double-floats
int rows_dot_df_chunks(int64_t N);
void launch_rows_dot_df(const df* A, int m, int64_t N, const df* v, double* partial, cudaStream_t s);
// returns the number of block partials of r . z written to partial (at most colsum_blocks(N))
int launch_woodbury_update_df(const df* H, int m, int64_t N, const double* v, const double* z0, double alpha,
                              double* z, const double* r, double* partial, cudaStream_t s);
void launch_chol(double* A, int n, int* status, cudaStream_t s);
// A = alpha A + J^T J (A n x n, J m x n, row-major)
void launch_dense_gn(double* A, int n, double alpha, const double* J, int m, cudaStream_t s);
// in-place triangular solves with the lower factor L (n x n): x <- L^-1 x, x <- L^-T x
void launch_trsv_lower(const double* L, int n, double* x, int nrhs, cudaStream_t s);
void launch_trsv_upper_t(const double* L, int n, double* x, int nrhs, cudaStream_t s);
// x <- L^-T L^-1 x for one right-hand side in one cooperative launch of ceil(n / 32) CTAs.
// flags: 2 ceil(n / 32) ints, zero before the first call; epoch > 0 and different from the
// previous call's. Each wait gives up after wait_ns. stall (failure-path test): the first
// block publishes no result, so the waits of the others run out. False if the device
// cannot keep all CTAs resident (nothing launched).
// epoch_ptr (may be null): a device counter holding the epoch instead of `epoch` (graph replays,
// where a preceding launch_bump advances it).
bool launch_chol_solve_coop(const double* L, int n, double* x, int* flags, int epoch, const int* epoch_ptr,
                            int* status, unsigned long long wait_ns, int stall, cudaStream_t s);
void launch_coarse_apply(const double* X, int n, int nrhs, const double* b, double* x,
                         cudaStream_t s);
void launch_symmetrize_identity_solve(double* X, int n, cudaStream_t s);
void launch_set_identity(double* X, int n, cudaStream_t s);
int cap_gemm_splits(int m, int64_t N);
void launch_cap_gemm(const double* J, const double* H, int m, int64_t N, double* partial,
                     int splits, cudaStream_t s);
void launch_cap_finalize(const double* partial, int splits, int m, double alpha, double* C,
                         cudaStream_t s);
// Krylov scalar kernels: scal is a small device array (see ScalarSlot in capi.cu)
void launch_sum_to_scalar(const double* partial, int n, double* dst, cudaStream_t s);
void launch_pcg_alpha(double* scal, cudaStream_t s);
// The PCG loop driven from the device (a graph with a conditional while node): scalar slots
// 7 first, 8 iterations, 9 tol^2, 10 maxit, 11 true r.r, 12 init, 13 rtol (see dense_kernels.cu).
enum : int { kSlotRZ = 0, kSlotPQ = 1, kSlotA = 2, kSlotRZN = 3, kSlotBeta = 4, kSlotRR = 5, kSlotBB = 6,
             kSlotFirst = 7, kSlotIt = 8, kSlotTol2 = 9, kSlotMaxit = 10, kSlotRRTrue = 11, kSlotInit = 12,
             kSlotRtol = 13 };
void launch_pcg_set_scalars(double* scal, double rtol, int maxit, int init, cudaStream_t s);
void launch_pcg_init(double* x, double* r, const double* b, const double* scal, int64_t N, cudaStream_t s);
void launch_pcg_start(double* scal, cudaGraphConditionalHandle h, cudaStream_t s);
void launch_pcg_beta_dev(double* scal, cudaStream_t s);
void launch_p_update_dev(double* p, const double* z, double* w, const double* jz, const double* scal, int64_t N,
                         int m, cudaStream_t s);
void launch_pcg_alpha_dev(double* scal, cudaStream_t s);
void launch_pcg_check(double* scal, cudaGraphConditionalHandle h, cudaStream_t s);
void launch_true_residual(double* r, const double* b, const double* q, int64_t N, double* partial, cudaStream_t s);
void launch_bump(int* counter, cudaStream_t s);
void launch_pcg_beta(double* scal, cudaStream_t s);
void launch_xr_update(double* x, double* r, const double* p, const double* q, const double* scal,
                      int64_t N, double* partial, cudaStream_t s);
void launch_p_update(double* p, const double* z, double* w, const double* jz, const double* scal,
                     int64_t N, int m, bool first, cudaStream_t s);
void launch_axpby(double* y, double a, const double* x, double b, int64_t N, cudaStream_t s);
void launch_dot_partial(const double* a, const double* b, int64_t N, double* partial,
                        cudaStream_t s);
int dot_blocks(int64_t N);
void launch_fill(double* y, double v, int64_t N, cudaStream_t s);
void launch_copy(double* y, const double* x, int64_t N, cudaStream_t s);

// ---- ERT forward model and Jacobian (ert.cu), on a context's FV hierarchy ----------
size_t ert_workspace_bytes(const Level* lev, int nlev, int n_e, int m);
h1w_status ert_forward(const Level* lev, int nlev, cudaStream_t s, const h1w_survey* sv, const double* logsigma,
                       double* U, double* g, void* ws, size_t ws_bytes, double rtol, int maxit, bool warm,
                       double cheb_ratio, h1w_info* info, std::string& err);
h1w_status ert_jvp(const Level* lev, int nlev, cudaStream_t s, const h1w_survey* sv, const double* logsigma,
                   const double* U, const double* p, double* Jp, void* ws, size_t ws_bytes, std::string& err);
h1w_status ert_adjoint(const Level* lev, int nlev, cudaStream_t s, const h1w_survey* sv, const double* logsigma,
                       const double* U, const double* r, double* JTr, double* J, void* ws, size_t ws_bytes,
                       std::string& err);

}  // namespace h1w
