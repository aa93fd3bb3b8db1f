/*
 * h1w: GB300 (sm_103a) solver for the Gauss-Newton linear system of
 * H1-regularized parameter identification,
 *
 *     (alpha (K + M) + J^T J) x = b,
 *
 * preconditioned through the Sherman-Morrison-Woodbury formula around a fast
 * Laplace solver (Blechta & Ernst, arXiv 2209.02815). Notation: alpha is the
 * paper's regularization weight beta; K is the Neumann stiffness operator of
 * the term int |grad m|^2 (operator L of Eq. 2.8); M is a mass operator that
 * makes K + M definite; J (m x N) is the measurement Jacobian of Eq. 2.15.
 *
 * Discretizations: H1W_Q1_VERTEX (2D bilinear elements on an nx x ny vertex
 * grid, row-sum lumped mass) and H1W_FV_CELL (3D cell-centred finite volumes
 * on an nx x ny x nz cell grid: the lowest-order Raviart-Thomas Schur
 * complement with diagonal Q that the paper uses as its Laplace
 * approximation S-hat in Sec. 3.2). Vectors are indexed x fastest:
 * p = (k * ny + j) * nx + i.
 *
 * Conventions for every entry point:
 *  - Array arguments are DEVICE pointers (FP64 unless stated) on the GPU the
 *    context was created on, read and written in stream order on the context's
 *    stream. The caller owns them. J is row-major [m][N] (one row per
 *    measurement, the rows of Eq. 2.15).
 *  - Device memory: the library allocates none. The caller passes one
 *    workspace of at least h1w_workspace_size() bytes (256-byte aligned) to
 *    h1w_setup; the context keeps pointers into it until h1w_destroy.
 *  - Errors are returned as h1w_status codes; no exceptions cross this
 *    boundary, and no device trap or assert is used. h1w_last_error() gives
 *    a text description. Kernels report failures (a non-positive Cholesky
 *    pivot) through a device status word that the host reads back.
 *  - Calls that return solver results (h1w_capacitance, h1w_pcg) synchronize
 *    the stream before returning; the others are asynchronous.
 *  - A context is not thread safe; distinct contexts are independent.
 */
#ifndef H1W_H
#define H1W_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  H1W_OK = 0,
  H1W_EINVAL = 1,        /* invalid argument (null pointer, bad size, bad grid) */
  H1W_ENOMEM = 2,        /* workspace smaller than h1w_workspace_size() */
  H1W_ECUDA = 3,         /* a CUDA runtime call or kernel launch failed */
  H1W_ENOTCONV = 4,      /* PCG did not reach rtol within maxit (x holds the last iterate) */
  H1W_ENOTSPD = 5,       /* Cholesky met a non-positive pivot (capacitance or coarse matrix) */
  H1W_ETIMEOUT = 6,      /* a bounded device-side wait ran out (the kernel returned early) */
  H1W_EUNSUPPORTED = 7,  /* grid that the multigrid hierarchy cannot coarsen to <= 1024 unknowns */
  H1W_ESTATE = 8         /* call out of order (e.g. h1w_pcg before h1w_capacitance) */
} h1w_status;

enum { H1W_Q1_VERTEX = 1, H1W_FV_CELL = 2 };

typedef struct {
  int32_t dim;     /* 2 (with H1W_Q1_VERTEX) or 3 (with H1W_FV_CELL) */
  int32_t disc;    /* H1W_Q1_VERTEX or H1W_FV_CELL */
  int32_t n[3];    /* vertices (Q1) or cells (FV) per axis, x first; n[2] = 1 in 2D */
  double h[3];     /* mesh spacing per axis (> 0) */
  double alpha;    /* regularization weight (> 0), the paper's beta */
} h1w_grid;

typedef struct {
  int32_t cheb_degree;   /* Chebyshev smoother degree per half-cycle (1..7, default 2) */
  int32_t rhs_block;     /* right-hand sides per batched V-cycle while building H (1..256, default 128;
                            a context uses at most m_max of them and sizes its buffers so) */
  int32_t max_restarts;  /* true-residual restarts allowed in h1w_pcg (default 3) */
  int32_t cap_gemm;      /* line C: 0 = tensor cores on an exact BF16 digit split of the FP64
                            operands (48-bit, default), 1 = FP64 CUDA cores */
  int32_t mg_arith;      /* arithmetic of the V-cycle and of the passes over J and H inside PCG:
                            0 = double-float (FP32 pairs, about 48 bits, default), 1 = FP64 */
  int32_t mg_unfused;    /* double-float cycle: 0 = levels with all axes coarsened and the degree-2
                            smoother run each leg (smoothing, residual and transfer) as one kernel
                            (default), 1 = one kernel per step. Both give identical results. */
  int32_t precond;       /* preconditioner of h1w_pcg / h1w_apply_prec: 0 = Laplace-Woodbury
                            alpha^-1 [L^-1 - alpha^-1 H C^-1 H^T] (default); 1 = Laplace only,
                            alpha^-1 L^-1, the paper's variant without the capacitance matrix
                            (Sec. 3.2), for which h1w_capacitance skips lines H, C and chol */
  int32_t pcg_mode;      /* h1w_pcg: 0 = the iteration driven from the device: the loop is a CUDA graph
                            with a conditional while node, the scalars stay on the GPU and the host
                            waits once per (re)start (default; the context keeps the graphs of the two
                            J addresses used last, so alternating between two device copies of J
                            captures each once); 1 = a host loop that reads the residual norm back
                            every iteration and times individual kernels (h1w_get_timings) */
  double cheb_ratio;     /* the Chebyshev smoother targets [lambda / cheb_ratio, lambda] of D^-1 A, lambda the
                            Gershgorin bound; 1.5 .. 1000, or 0 (default) for the discretization's
                            ratio: 10 on FV cell grids, 6 on Q1 vertex grids. It also sets the interval
                            of h1w_forward's FP32 cycle (10 at 0) */
  int32_t j_digits;      /* line C on the tensor cores: 1 (default) = while J is converted to double-floats
                            in line H, also split it into the GEMM's digits for every K panel, kept in
                            the workspace when they take at most 32 GB (14 bytes per entry of J, rows
                            rounded up to 128), so that line C reads J no more; 0 = split J per K panel
                            in line C (the workspace holds one panel's digits) */
} h1w_options;

typedef struct {
  int32_t iters;         /* PCG iterations performed */
  int32_t restarts;      /* restarts from the true residual */
  double rel_res_true;   /* ||b - A x||_2 / ||b||_2, recomputed in FP64 at exit */
  double rel_res_rec;    /* last recursively updated ||r||_2 / ||b||_2 */
} h1w_info;

/* Device-side phase times of the last calls on a context, taken with CUDA
 * events on the context's stream (the paper reports the same breakdown as
 * t_H, t_C, t_chol and the solver time, Table 4.1), and the number of kernels
 * the library launched in them. */
typedef struct {
  float t_H_ms;                 /* line H: batched V-cycles of the last h1w_capacitance */
  float t_C_ms;                 /* line C: operand preparation and the capacitance GEMM */
  float t_chol_ms;              /* forming C from the GEMM partials and its Cholesky factor */
  float t_pcg_ms;               /* the last h1w_pcg, launch to convergence */
  int64_t launches_capacitance; /* kernels launched by the last h1w_capacitance */
  int64_t launches_pcg;         /* kernels launched by the last h1w_pcg */
  /* device time and launch count of individual kernels in those two calls */
  float t_gemm_kernel_ms;       /* capacitance GEMM kernel launches (line C) */
  float t_jdot_ms;              /* passes J z over J inside PCG */
  float t_op_ms;                /* operator kernel (stencil + J^T w) inside PCG */
  float t_hdot_ms;              /* passes H^T r over H inside PCG */
  float t_hupd_ms;              /* passes z = (z0 - H v / alpha) / alpha over H inside PCG */
  int32_t n_gemm_kernel, n_jdot, n_op, n_hdot, n_hupd, reserved;
  float t_vc_down_ms;           /* fused down-leg kernel of the finest level (line H, double-float cycle) */
  float t_vc_up_ms;             /* fused up-leg kernel of the finest level (line H, double-float cycle) */
  int32_t n_vc_down, n_vc_up;
  float t_split_j_ms;           /* digit split of J before each GEMM panel (line C, tensor cores) */
  float t_split_h_ms;           /* digit split of H before each GEMM panel (line C, tensor cores) */
  float t_d2df_ms;              /* FP64 -> double-float conversion of J's row batches (line H) */
  int32_t n_split_j, n_split_h, n_d2df, reserved2;
} h1w_timings;

typedef struct h1w_ctx h1w_ctx;

/* Fills *opt with the defaults listed in h1w_options. */
void h1w_default_options(h1w_options* opt);

/* Bytes of device workspace needed for this grid and at most m_max
 * measurements (opt may be NULL for defaults). Returns 0 for invalid input. */
size_t h1w_workspace_size(const h1w_grid* grid, int32_t m_max, const h1w_options* opt);

/* Builds the multigrid hierarchy for L-hat^-1 (one symmetric V-cycle on K + M;
 * the paper's AMG line of Algorithm "Gauss-Newton with iterative solver",
 * here a matrix-free geometric cycle) inside `workspace` and returns a
 * context bound to `stream` (a cudaStream_t; NULL = legacy default stream).
 * The coarsest-level Cholesky factor is computed on the GPU. */
h1w_status h1w_setup(const h1w_grid* grid, int32_t m_max, const h1w_options* opt, void* workspace,
                     size_t ws_bytes, void* stream, h1w_ctx** out);

/* Lines H, C and chol of Algorithm "MINRES with the Laplace-Woodbury
 * preconditioner": H = L-hat^-1 J^T (m batched V-cycles), C = I + alpha^-1 J H
 * (formed from its upper triangle and mirrored), C = L L^T. With
 * cap_gemm = 0 the product J H^T runs on the tensor cores: each chunk of
 * 1024 consecutive entries of a row of J and of H is scaled by its own power
 * of two, rounded to 48 bits and written exactly as eight BF16 digits; digit
 * products are accumulated exactly in FP32 chunks and combined in FP64
 * (error below 2^-47 of the chunk maxima). J (m x N, row-major, device) is
 * borrowed: it must stay valid and unchanged until the next h1w_capacitance or
 * h1w_destroy. 0 <= m <= m_max; m = 0 gives the Laplace-only preconditioner.
 * Synchronizes; H1W_ENOTSPD if C is not numerically positive definite. */
h1w_status h1w_capacitance(h1w_ctx* ctx, int32_t m, const double* J);

/* The same lines with J supplied in page-locked HOST memory: J_host (m x N,
 * row-major, e.g. from cudaHostAlloc) is copied into the caller's DEVICE
 * buffer J_dev (m x N), which then is the borrowed J of the context, exactly as
 * J of h1w_capacitance. The copy runs on a second stream of the context in row
 * batches of rhs_block, and each batch's V-cycles start as soon as its own
 * rows have arrived, so the copy overlaps line H. No counterpart in the paper
 * (its data never leave the host). J_host must stay valid until the call
 * returns; the results equal those of h1w_capacitance on the same J.
 * Synchronizes. */
h1w_status h1w_capacitance_from_host(h1w_ctx* ctx, int32_t m, const double* J_host, double* J_dev);

/* Starts the row-batch copies of J_host (page-locked HOST, m x N) into J_dev (DEVICE)
 * on the context's copy stream and returns at once, so that the copy of the next
 * system's J runs while the current system is solved; the next
 * h1w_capacitance_from_host(ctx, m, J_host, J_dev) with the same three arguments then
 * waits only for the rows that have not yet arrived, batch by batch. The copies are
 * ordered after the work already queued on the context's stream. J_dev must not be read
 * by a later call before that capacitance (e.g. it must not be the J of the capacitance
 * that the next h1w_pcg uses); J_host must stay valid and unchanged until that
 * capacitance returns. At most two copy sets are pending at a time (double buffering):
 * H1W_ESTATE otherwise, or when another pending copy targets J_dev. No counterpart in the
 * paper (its data never leave the host). */
h1w_status h1w_prefetch_J(h1w_ctx* ctx, int32_t m, const double* J_host, double* J_dev);

/* Per-row-batch timeline of the last h1w_capacitance_from_host, in ms from the start of
 * its line H (negative when a prefetched copy began earlier): copy_begin/end of the batch's
 * rows on the copy stream, cycle_begin/end of its conversion and V-cycles on the
 * context's stream (cycle_begin waits for copy_end). *nbatch receives the batch count;
 * the arrays (any may be NULL) receive min(cap, *nbatch) entries; rows = the batch sizes. */
h1w_status h1w_get_copy_profile(const h1w_ctx* ctx, int32_t cap, int32_t* nbatch, int32_t* rows,
                                float* copy_begin_ms, float* copy_end_ms, float* cycle_begin_ms,
                                float* cycle_end_ms);

/* z = P^-1 r with P = alpha L-hat + J^T J, evaluated by the Woodbury formula
 * of Sec. 3.2: z = alpha^-1 [ L-hat^-1 r - alpha^-1 H C^-1 H^T r ].
 * r and z have N entries and must not overlap. */
h1w_status h1w_apply_prec(h1w_ctx* ctx, const double* r, double* z);

/* q = alpha (K + M) p + J^T (J p) (the matrix-free system operator; J^T J is
 * never formed). p and q have N entries and must not overlap. */
h1w_status h1w_apply_op(h1w_ctx* ctx, const double* p, double* q);

/* x = L-hat^-1 b for nrhs right-hand sides stored contiguously (b[r * N + p]);
 * one V-cycle each, batched. b and x must not overlap. */
h1w_status h1w_vcycle(h1w_ctx* ctx, int32_t nrhs, const double* b, double* x);

/* Gauss-Newton right-hand side of Eq. 2.9 scaled by beta, with the mass term:
 * b = -alpha (K + M) dm - J^T d, where dm = m - m_ref (N entries) and
 * d = g_m - g_obs (m entries, DEVICE). Uses the J of the last h1w_capacitance. */
h1w_status h1w_gn_rhs(h1w_ctx* ctx, const double* dm, const double* d, double* b);

/* Preconditioned conjugate gradients for the system above from x0 = 0,
 * stopping when ||r_k||_2 <= rtol ||b||_2 (the Euclidean criterion of Sec. 4)
 * on the recursively updated residual; the true residual b - A x is then
 * recomputed in FP64 and, if it fails the test, the iteration restarts from
 * it (at most max_restarts times). Vectors and scalars of the iteration are
 * FP64; on FV grids with mg_arith = 0 the passes over J and H inside the
 * iteration read double-float copies (about 48 bits), while the exit test
 * uses the caller's FP64 J. info may be NULL. Synchronizes. Returns
 * H1W_ENOTCONV when maxit is reached first (x holds the last iterate). */
h1w_status h1w_pcg(h1w_ctx* ctx, const double* b, double* x, double rtol, int32_t maxit,
                   h1w_info* info);

/* h1w_pcg with b and x in page-locked HOST memory (cudaHostAlloc'ed or registered, N
 * entries each): b is read and x written by kernels through the device's view of that
 * memory, so the solve queues no copy-engine work on the context's stream. (A host copy
 * queued there behind a large h1w_prefetch_J copy made the stream's following work wait
 * for all of that copy.) The solve runs on the context's own buffers. H1W_EINVAL if either
 * pointer is not page-locked host memory the device can address. Synchronizes. */
h1w_status h1w_pcg_host(h1w_ctx* ctx, const double* b_host, double* x_host, double rtol, int32_t maxit,
                        h1w_info* info);

/* Copies the capacitance matrix C and its lower Cholesky factor L (m x m,
 * row-major, DEVICE) into caller buffers (either may be NULL). */
h1w_status h1w_capacitance_factors(h1w_ctx* ctx, double* C, double* L);

/* Lines H, C, chol and PCG (as h1w_capacitance followed by h1w_pcg) for `count`
 * independent systems, each with its own context, set up on its own stream (not
 * the legacy default stream, which would serialise them). System i takes
 * m[i] measurements with J[i] (borrowed, as in h1w_capacitance), right-hand
 * side b[i] and solution x[i] (DEVICE). Up to `threads` host threads (<= 0:
 * 8) work through the systems concurrently, so that the kernels of small systems
 * overlap on the GPU. info and status (may be NULL) get count entries.
 * Returns H1W_OK when every system converged, else the first failing status; the
 * failing context's h1w_last_error has the reason. The paper solves one system
 * at a time and has no counterpart. Synchronizes. */
h1w_status h1w_solve_batch(h1w_ctx* const* ctxs, int32_t count, const int32_t* m, const double* const* J,
                           const double* const* b, double* const* x, double rtol, int32_t maxit,
                           int32_t threads, h1w_info* info, h1w_status* status);

/* The same as h1w_solve_batch (lines H, C, chol and PCG for `count` independent systems,
 * each with its own context on its own distinct stream, precond = 0), but as ONE CUDA
 * graph: every system's capacitance and its device-driven PCG loop (a conditional while
 * node, as pcg_mode = 0) are captured as parallel branches of a single graph, which is
 * launched once, so the GPU schedules all systems' kernels together with no host thread
 * and no host round trip per iteration. The graph is kept and replayed while the
 * contexts, m, J, b, x, rtol and maxit are the same as in the previous call (it is
 * captured again otherwise). A system whose recursive residual met rtol but whose true
 * residual did not continues with h1w_pcg's restarts. Returns H1W_OK when every system
 * converged, else the first failing status (that context's h1w_last_error has the
 * reason). Synchronizes. No counterpart in the paper (it solves one system at a time). */
h1w_status h1w_solve_batch_graph(h1w_ctx* const* ctxs, int32_t count, const int32_t* m, const double* const* J,
                                 const double* const* b, double* const* x, double rtol, int32_t maxit,
                                 h1w_info* info, h1w_status* status);

/* Autotuner of the batched V-cycle: for this grid and m measurements, sets up a context
 * for each candidate rhs_block (8 .. 256, at most m; every other option from `base`, which
 * may be NULL for the defaults), times one batch of V-cycles on the device with CUDA
 * events (line H's cycle, double-float path), and writes `base` with the smallest
 * rhs_block whose time per right-hand side is within 5 % of the fastest (the cycle's
 * buffers grow with the block) to *out; *ms_per_rhs (may be NULL) gets its time. The
 * result is cached in the process per (discretization, grid, m, smoother), so later calls
 * return at once. The workspace (DEVICE, 256-byte aligned, h1w_autotune_workspace_size
 * bytes) is scratch for the candidate contexts; stream as in h1w_setup. Paths without a
 * batched double-float cycle (m = 0, mg_arith = 1, precond = 1) return `base` untimed.
 * Synchronizes. No counterpart in the paper. */
size_t h1w_autotune_workspace_size(const h1w_grid* grid, int32_t m, const h1w_options* base);
h1w_status h1w_autotune(const h1w_grid* grid, int32_t m, const h1w_options* base, void* workspace, size_t ws_bytes,
                        void* stream, h1w_options* out, float* ms_per_rhs);

/* Phase times and launch counts of the last h1w_capacitance / h1w_pcg. */
h1w_status h1w_get_timings(const h1w_ctx* ctx, h1w_timings* out);

/* Number of multigrid levels and the grid size of level `level` (n[3]). */
h1w_status h1w_level_info(const h1w_ctx* ctx, int32_t level, int32_t* nlevels, int32_t* n);

/* q = alpha (K + M) p + J^T (J p), like h1w_apply_op, for callers that cannot
 * allocate device memory: code whose memory belongs to another allocator (a
 * framework's caching pool or a fixed arena) and that must not call
 * cudaMalloc itself, since cudaMalloc synchronizes the device and takes
 * memory outside that budget. The paper has no counterpart; it is a service
 * of this library. No context and no workspace: the grid (fine level only)
 * is passed directly, and the scratch (partial sums of J p, J p itself and
 * the Q1 element coefficients) lives in one file-scope __device__ array of
 * 2^20 doubles (8 MiB) that every GPU loading this library holds until the
 * process exits. Calls needing more scratch than that, i.e.
 *   32*ceil(ceil(N/4096)*m/32) + 32*ceil(max(m,1)/32) + [Q1] 6*(nx+ny)
 * doubles, return H1W_EINVAL; use h1w_setup with a workspace for those.
 * The call allocates nothing (no cudaMalloc, cudaFree or allocating library
 * routine). The first call on each device, with that device current, looks
 * up the array's device address once; make that first call before any
 * stream capture. All calls on a device share the one array, and it keeps
 * the last call's contents (every value is written before it is read, so
 * nothing needs clearing): calls that overlap on the GPU, e.g. on two
 * streams, race and must be serialized by the caller. Arguments: grid as in
 * h1w_setup; J (m x N row-major), p, q (N entries) are DEVICE pointers of
 * the current device, p and q distinct; stream is a cudaStream_t (NULL =
 * legacy default stream). Asynchronous; errors of the launch are returned,
 * with text in h1w_last_error(NULL). */
h1w_status h1w_apply_op_static(const h1w_grid* grid, int32_t m, const double* J, const double* p,
                               double* q, void* stream);

/* ---- Direct solve (the paper's Gauss-Newton step with an exact inverse) --------
 *
 * The comparison variant of Sec. 3.1 for small grids: x = (alpha (K + M) + J^T J)^-1 b
 * with the J of the last h1w_capacitance, by forming the N x N matrix densely in FP64
 * and factorizing it with the library's blocked Cholesky (the algorithm "Gauss-Newton
 * with direct solver" uses a dense factorization in place of the iterative solve).
 * The workspace (DEVICE, 256-byte aligned) holds the matrix: h1w_direct_workspace_size
 * bytes, 0 when N exceeds H1W_DIRECT_MAX_N (the triangular solves keep x in one
 * block's shared memory). b, x: DEVICE, N entries, may coincide. H1W_ENOTSPD when a
 * pivot is not positive. Synchronizes. */
#define H1W_DIRECT_MAX_N 6144

size_t h1w_direct_workspace_size(const h1w_ctx* ctx);
h1w_status h1w_solve_direct(h1w_ctx* ctx, const double* b, double* x, void* workspace, size_t ws_bytes);

/* ---- ERT forward model and Jacobian (Sec. 4.1, Eqs. 4.1-4.5) ------------------
 *
 * On the context's H1W_FV_CELL grid, with conductivity sigma = exp(m) per cell:
 * -div(sigma grad u) = f, face conductance G_k 2 s_a s_b / (s_a + s_b) between
 * neighbours along axis k (G_k = face area / centre distance), u = 0 on the
 * box faces marked Dirichlet (the paper's gamma_D; a ghost at half a cell,
 * conductance 2 G_k s_a) and zero flux on the others. Electrode e injects a unit
 * current into cell cell[e]; its pole field is u_e = A^-1 e_{cell[e]}.
 * Measurement i with electrodes abmn[i] = (A, B, M, N), any of them -1 for "at
 * infinity" (the paper's B electrode of the pole-dipole survey), is
 *     g_i = k_i (v(cell[M]) - v(cell[N])),  v = u_A - u_B      (Eqs. 4.3, 4.5),
 * and the Jacobian J = dg/dm of Eq. 4.4 in its discrete form is
 *     J_ic = -k_i w^T (dA/dm_c) v,  w = u_M - u_N  (reciprocity),
 * i.e. the exact derivative of the discrete g. */
#define H1W_ERT_MAX_ELECTRODES 128

typedef struct {
  int32_t n_e;              /* electrodes, 1..H1W_ERT_MAX_ELECTRODES */
  const int32_t* cell;      /* HOST [n_e]: level-0 cell index under each electrode */
  int32_t m;                /* measurements (>= 0) */
  const int32_t* abmn;      /* HOST [m][4]: electrode indices A, B, M, N (-1 = at infinity) */
  const double* k;          /* HOST [m]: geometric factors k_i (Eq. 4.5) */
  uint32_t dirichlet;       /* bit f marks box face f Dirichlet, f = 0..5: x-, x+, y-, y+, z-, z+;
                               at least one bit (the operator must be definite) */
} h1w_survey;

/* Bytes of device workspace (256-byte aligned) that h1w_forward and h1w_adjoint
 * need for n_e electrodes and m measurements on this context's grid: about
 * (4 FP64 + 5 FP32) vectors per electrode, the coefficients of every level and
 * m N / 32 partial sums for h1w_ert_jvp.
 * 0 for invalid input or a context that is not H1W_FV_CELL. */
size_t h1w_ert_workspace_size(const h1w_ctx* ctx, int32_t n_e, int32_t m);

/* Pole fields and measurements for the log-conductivity logsigma (N, DEVICE).
 * U (DEVICE, [n_e][N], caller-owned) receives the fields u_e, g (DEVICE, [m])
 * the measurements. The fields are solved together by PCG in FP64 to
 * ||e_c - A u_e||_2 <= rtol (unit sources), preconditioned by two FP32 V-cycles
 * on the same operator over the context's hierarchy, from u_e = 0 or, with
 * H1W_FORWARD_WARM_START, from the fields already in U (e.g. those of the previous
 * Gauss-Newton iterate). The survey's host arrays
 * are copied before the call returns. info (may be NULL): iterations, and the
 * worst field's FP64 true and recursive residuals. H1W_ENOTCONV when maxit
 * iterations do not reach rtol (U holds the iterates), H1W_ENOTSPD when the
 * coarsest operator fails its Cholesky factorization. Synchronizes. */
#define H1W_FORWARD_WARM_START 1u  /* flags: start PCG from the fields already in U (else from 0) */

h1w_status h1w_forward(h1w_ctx* ctx, const h1w_survey* survey, const double* logsigma, double* U, double* g,
                       void* workspace, size_t ws_bytes, double rtol, int32_t maxit, uint32_t flags,
                       h1w_info* info);

/* The Jacobian from the fields U of h1w_forward (same survey and logsigma):
 * J (DEVICE, [m][N] row-major, may be NULL) receives every row, and JTr
 * (DEVICE, [N], may be NULL) receives J^T r for r (DEVICE, [m]), formed without
 * storing J. At least one of J, JTr. Uses the workspace of h1w_forward (its
 * fields are not touched). Synchronizes. */
h1w_status h1w_adjoint(h1w_ctx* ctx, const h1w_survey* survey, const double* logsigma, const double* U,
                       const double* r, double* JTr, double* J, void* workspace, size_t ws_bytes);

/* Jp (DEVICE, [m]) = J p for p (DEVICE, [N]), formed from the fields U of h1w_forward
 * without storing J: each entry J_ic is formed from the face jumps of the pole fields,
 * as in h1w_adjoint, and reduced over the cells in a fixed order. With the J^T r of
 * h1w_adjoint it applies the Gauss-Newton operator's data term J^T J from n_e fields
 * instead of m rows. Synchronizes. */
h1w_status h1w_ert_jvp(h1w_ctx* ctx, const h1w_survey* survey, const double* logsigma, const double* U,
                       const double* p, double* Jp, void* workspace, size_t ws_bytes);

/* ---- Gauss-Newton step (Algorithm "Gauss-Newton with iterative solver") --------
 *
 * One pass of the algorithm's loop on an ERT model: evaluate g_m and J_m at m
 * (h1w_forward, h1w_adjoint), solve the linearized system
 *     (alpha (K + M) + J^T J) dm = -alpha (K + M)(m - m_ref) - J^T (g_m - g_obs)
 * with the Laplace-Woodbury PCG (h1w_capacitance, h1w_gn_rhs, h1w_pcg), and
 * update m := m + dm. Every step runs in this library's kernels.
 * m (DEVICE, N) is updated in place; m_ref (DEVICE, N) and g_obs (DEVICE,
 * survey->m) are inputs; U ([n_e][N]), J ([m][N]) and g ([m]) receive the
 * fields, Jacobian and measurements at the incoming m (DEVICE); scratch
 * (DEVICE) holds 3 N + m doubles; ert_ws is the workspace of h1w_forward.
 * survey->m must not exceed the context's m_max. rtol_fwd and rtol are the
 * forward and GN PCG tolerances; maxit bounds both; fwd_flags goes to h1w_forward
 * (H1W_FORWARD_WARM_START once U holds the previous iterate's fields). Synchronizes. */
typedef struct {
  int32_t fwd_iters;     /* PCG iterations of the forward solve */
  int32_t gn_iters;      /* PCG iterations of the GN solve */
  double misfit;         /* ||g_m - g_obs||_2 at the incoming m */
  double rel_res_true;   /* the GN solve's FP64 true relative residual */
  double step_norm;      /* ||dm||_2 */
} h1w_gn_info;

h1w_status h1w_gn_step(h1w_ctx* ctx, const h1w_survey* survey, const double* g_obs, const double* m_ref,
                       double* m, double* U, double* J, double* g, double* scratch, void* ert_ws,
                       size_t ert_ws_bytes, double rtol_fwd, double rtol, int32_t maxit, uint32_t fwd_flags,
                       h1w_gn_info* info);

/* ---- Line chol on a caller's matrix, and failure-path testing -------------------
 *
 * h1w_cholesky: A = L L^T in place for a symmetric positive definite n x n matrix A
 * (DEVICE, row-major, FP64), with the blocked kernels of line chol (Algorithm "MINRES
 * with the Laplace-Woodbury preconditioner") that factor the capacitance matrix: on
 * return the lower triangle holds L and the strict upper triangle is zero. Runs on the
 * context's stream and synchronizes. H1W_ENOTSPD (with text) when a pivot is not
 * positive, i.e. A is not numerically positive definite; A then holds a partial factor. */
#define H1W_CHOLESKY_MAX_N 16384

h1w_status h1w_cholesky(h1w_ctx* ctx, int32_t n, double* A);

/* h1w_inject_stall: for testing the failure path of the bounded device waits, without a
 * GPU fault. kind H1W_STALL_CAP_GEMM makes the copy warp of the tensor-core capacitance
 * GEMM issue no copies, so that the waits of its MMA and epilogue warps run out and
 * h1w_capacitance returns H1W_ETIMEOUT; H1W_STALL_PREC_SOLVE makes the first block of the
 * cooperative C^-1 solve inside the preconditioner publish no result (m > 32 needed), so
 * that the waits of the other blocks run out and h1w_pcg / h1w_apply_prec report
 * H1W_ETIMEOUT (with maxit small, since PCG then iterates on a broken preconditioner).
 * wait_limit_ns sets the limit of every bounded wait of this context (0: the default of
 * one second; at most 60 s). H1W_STALL_NONE restores normal operation; the context stays
 * usable after a timeout (h1w_capacitance must be called again, since a timed-out call
 * leaves no valid capacitance). No counterpart in the paper. */
enum { H1W_STALL_NONE = 0, H1W_STALL_CAP_GEMM = 1, H1W_STALL_PREC_SOLVE = 2 };

h1w_status h1w_inject_stall(h1w_ctx* ctx, int32_t kind, int64_t wait_limit_ns);

/* Changes h1w_options.pcg_mode of a live context (0 device-driven graph, 1 host loop). */
h1w_status h1w_set_pcg_mode(h1w_ctx* ctx, int32_t mode);

/* Text of the last error on this context (ctx = NULL: the last error of
 * h1w_setup on this thread). Never NULL. */
const char* h1w_last_error(const h1w_ctx* ctx);

/* Releases the host-side context. The workspace stays owned by the caller. */
void h1w_destroy(h1w_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* H1W_H */
