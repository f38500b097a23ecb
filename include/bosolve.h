/*
 * bosolve.h - C ABI of the GPU (sm_103a) CPR-FGMRES solver for the Newton
 * Jacobians of fully implicit three-phase black-oil simulation.
 *
 * The problem (paper Sec. 3.1, Alg. 1): given the Jacobian A and the
 * right-hand side b(x^l) of one Newton step, find dx with
 *     || b - A dx ||_2 <= tol * || b ||_2.
 * A is block sparse with 3x3 blocks (paper Sec. 3.2, Eq. for the block
 * structure of A): one block row per cell of a structured nx x ny x nz grid
 * (paper Sec. 3.3), 7-point two-point-flux stencil.  Unknown 3c+k of a
 * vector is (p, Sw, Sg)[k] of cell c = i + nx (j + ny k); row r of a block is
 * the (oil, water, gas)[r] conservation equation (paper Sec. 2.1, Eq. 3).
 *
 * Solver: restarted flexible GMRES, right preconditioned by CPR-FPF (paper
 * Alg. 2) built on the Quasi-IMPES decoupled matrix (paper Sec. 3.2):
 * red-black block ILU(0) as the local solver R, an aggregation AMG V-cycle
 * on the pressure block A_pp.
 *
 * Conventions for every call:
 *  - Return value: a bo_status (0 = BO_OK, negative = error).  No call
 *    aborts the process or poisons the CUDA context on bad input.
 *  - Execution: every call is ordered on the context's CUDA stream.  Calls
 *    that return results to the host (bo_prec_setup, bo_solve, the
 *    *_levels query) synchronise that stream.
 *  - Memory: `mem` arguments say whether a pointer is host (BO_MEM_HOST) or
 *    device (BO_MEM_DEVICE) memory of the context's device.  The library
 *    copies matrix inputs into memory it owns; vectors passed to spmv /
 *    apply / solve stay owned by the caller.
 *  - Thread safety: one context, matrix or preconditioner must not be used
 *    from two host threads at once.
 */
#ifndef BOSOLVE_H
#define BOSOLVE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bo_ctx bo_ctx;
typedef struct bo_mat bo_mat;
typedef struct bo_prec bo_prec;

typedef enum {
  BO_OK = 0,
  BO_ERR_ARG = -1,           /* bad argument (NULL, size, unsupported option)   */
  BO_ERR_CUDA = -2,          /* a CUDA runtime call failed                       */
  BO_ERR_OOM = -3,           /* device allocation failed                         */
  BO_ERR_PATTERN = -4,       /* input pattern is not the grid's 7-point stencil  */
  BO_ERR_NONFINITE = -5,     /* NaN or Inf in matrix values or right-hand side   */
  BO_ERR_BREAKDOWN = -6,     /* singular pivot in decoupling, ILU or AMG         */
  BO_ERR_NOT_CONVERGED = -7, /* maxit reached; x holds the last iterate          */
  BO_ERR_TIMEOUT = -8        /* a device-side loop cap was hit                   */
} bo_status;

enum { BO_MEM_HOST = 0, BO_MEM_DEVICE = 1 };
/* arithmetic of the preconditioner (and of bo_mat_spmv's matrix values) */
/* Preconditioner / reduced-copy precision.  BO_PREC_FP32: the preconditioner
 * stores and computes in FP32 (mixed precision inside FP64 FGMRES).
 * BO_PREC_BF16: the preconditioner stores its decoupled matrix, ILU pivot
 * inverses and AMG coefficients in BF16 and computes in FP32; for
 * bo_mat_spmv, a BF16 copy of the values with FP32 sums. */
enum { BO_PREC_FP64 = 0, BO_PREC_FP32 = 1, BO_PREC_BF16 = 2 };
/* How bo_solve issues the kernels of each Arnoldi column: one launch per
 * kernel on the stream, or one CUDA-graph launch per column (captured on
 * first use and replayed; no per-column SpMV timing then). */
enum { BO_LAUNCH_STREAM = 0, BO_LAUNCH_GRAPH = 1, BO_LAUNCH_BATCH_GRAPH = 2 };
/* stages of the preconditioner that bo_prec_apply can run on their own */
enum {
  BO_STAGE_CPR = 0,           /* z = CPR(D_QI^{-1} r): the preconditioner FGMRES uses */
  BO_STAGE_ILU = 1,           /* z = R^{-1} r, R = red-black block ILU(0) of D_QI^{-1} A */
  BO_STAGE_AMG = 2,           /* z = Pi_p AMG(A_pp)^{-1} Pi_r r                         */
  BO_STAGE_CPR_DECOUPLED = 3, /* z = CPR(r), Alg. 2 on an already decoupled r          */
  BO_STAGE_ARNOLDI_SPMV = 4   /* z = A r by FGMRES's own Arnoldi product: r split into
                                 two floats per entry (48 significant bits), the split
                                 copy of A, FP32 instructions (see bo_solve)           */
};

/* Structured grid (paper Sec. 3.3).  nx must be even (the red-black layout
 * pairs neighbouring cells of a grid row); ncontinua must be 1 for a bo_mat
 * and 2 for a bo_dp (dual porosity). */
typedef struct {
  int32_t nx, ny, nz;
  double dx, dy, dz;
  int32_t ncontinua;
} bo_grid;

typedef struct {
  int32_t precision;      /* BO_PREC_FP64, BO_PREC_FP32 or BO_PREC_BF16         */
  int32_t amg_nu1;        /* red-black Gauss-Seidel pre-sweeps  (default 2)      */
  int32_t amg_nu2;        /* post-sweeps (default 2)                             */
  double amg_overcorr;    /* coarse correction scale s: x += s P x_c (default 1.3) */
  int32_t amg_coarse_max; /* coarsest level size, <= 128 (default 128)          */
  int32_t decoupling;     /* BO_DECOUPLE_QI (default) or BO_DECOUPLE_ABF          */
} bo_prec_opts;

/* Decoupling operator D of the CPR (paper Sec. 3.2, D^{-1} A x = D^{-1} b).
 * BO_DECOUPLE_QI: Quasi-IMPES, the pressure row of each cell becomes
 *   row_o - (a_{o,Sw}/a_{w,Sw}) row_w - (a_{o,Sg}/a_{g,Sg}) row_g (where that
 *   leaves a non-positive pressure pivot, the cell takes the ABF row).
 * BO_DECOUPLE_ABF: Alternate Block Factorization, D = the block diagonal of
 *   A.  Only the pressure row of D^{-1} A enters the AMG stage, and block
 *   ILU(0) commutes with a block-diagonal left scaling (the factors of
 *   D^{-1} A are those of A scaled row-blockwise), so the library applies
 *   row 0 of each A_ii^{-1} to the pressure row and leaves the other rows:
 *   the preconditioner equals the CPR of the fully ABF-scaled system. */
enum { BO_DECOUPLE_QI = 0, BO_DECOUPLE_ABF = 1 };

typedef struct {
  double tol;             /* relative to ||b||_2 (paper Alg. 1 criterion)         */
  int32_t restart;        /* m of FGMRES(m), 1..64 (default 30)                   */
  int32_t maxit;          /* total iteration cap (default 500)                    */
  int32_t x0_is_zero;     /* 1: ignore x on entry and start from 0                */
  int32_t mem;            /* BO_MEM_DEVICE (default) or BO_MEM_HOST for b and x   */
  int32_t profile;        /* 1: time the Arnoldi SpMV launches with CUDA events   */
} bo_solve_opts;

typedef struct {
  int32_t status;         /* as returned                                          */
  int32_t iters;          /* FGMRES iterations                                    */
  int32_t restarts;       /* completed cycles                                     */
  double true_rel_res;    /* ||b - A x|| / ||b|| recomputed in FP64 at exit       */
  double est_rel_res;     /* last Arnoldi estimate                                */
  double solve_ms;        /* host wall time of the call                           */
  int32_t spmv_launches;  /* profile = 1: Arnoldi SpMV launches timed             */
  double spmv_ms;         /* profile = 1: their summed CUDA-event time            */
} bo_solve_info;

const char* bo_status_str(int status);
/* Fill defaults: FP64, nu1 = nu2 = 2, overcorr 1.3, coarse_max 128 / tol 1e-8,
 * restart 30, maxit 500, device pointers. */
void bo_prec_opts_default(bo_prec_opts* o);
void bo_solve_opts_default(bo_solve_opts* o);

/* Context on CUDA device `device`, ordering work on `cuda_stream`: a
 * cudaStream_t of that device, cudaStreamLegacy ((void*)1) for the legacy
 * default stream, or NULL for a new non-blocking stream owned by the
 * context.  The context must outlive the matrices made with it. */
int bo_ctx_create(int device, void* cuda_stream, bo_ctx** out);
/* Lifetimes are reference counted: a matrix holds its context, a
 * preconditioner its matrix, a dual-porosity system and a network their
 * context.  A *_destroy call drops the caller's reference; the object is
 * freed (after synchronising its stream; an owned stream is destroyed) when
 * the last reference goes, so objects may be destroyed in any order.
 * BO_ERR_ARG for NULL. */
int bo_ctx_destroy(bo_ctx* ctx);

/* Jacobian from BSR arrays (paper Sec. 3.3 matrix of rows; Sec. 3.2 block
 * structure): nbrows = nx ny nz block rows, rowptr[nbrows+1], col[nnzb],
 * val[9 nnzb] row-major 3x3 blocks.  Every block row must hold exactly the
 * diagonal and the existing 7-point neighbours (any order).  Errors:
 * BO_ERR_PATTERN for any other pattern, BO_ERR_NONFINITE for NaN/Inf. */
int bo_mat_create_bsr(bo_ctx* ctx, const bo_grid* grid, int32_t nbrows, int64_t nnzb,
                      const int32_t* rowptr, const int32_t* col, const double* val,
                      int mem, bo_mat** out);
/* Jacobian from scalar CSR with interleaved unknowns (row 3c+r, column
 * 3c'+k): nrows = 3 nx ny nz.  Entries outside the 7-point block pattern
 * give BO_ERR_PATTERN; duplicates are summed; missing entries are zero. */
int bo_mat_create_csr(bo_ctx* ctx, const bo_grid* grid, int32_t nrows, int64_t nnz,
                      const int32_t* rowptr, const int32_t* col, const double* val,
                      int mem, bo_mat** out);
/* New values on the pattern given at create (the next Newton Jacobian):
 * val[9 nnzb] (BSR) or val[nnz] (CSR) in the order of the arrays given at
 * create, host or device per mem, copied.  Invalidates the reduced-precision
 * copies; preconditioners on A keep their old values until bo_prec_update.
 * BO_ERR_NONFINITE for NaN/Inf (the matrix then holds the new values and must
 * not be solved with); BO_ERR_ARG for NULL or a bad mem. */
int bo_mat_update_values(bo_mat* A, const double* val, int mem);
/* y = alpha A x + beta y (paper Sec. 3.3 first basic operation); x, y
 * device vectors of length 3 nx ny nz.  precision BO_PREC_FP64: the values
 * as split pairs of floats (48 significant bits, the copy the solver's
 * Arnoldi product reads), x split the same way on load, products and sums in
 * split arithmetic, so |y - exact| <= 2e-13 (|A| |x|)_i (before alpha and
 * beta); a matrix with a value outside the split form's range [2^-120, 2^126]
 * uses its FP64 values and FP64 products instead.  BO_PREC_FP32 /
 * BO_PREC_BF16: a reduced-precision copy of the values (made on first use
 * after each value update), x rounded to FP32 on load, products and sums in
 * FP32, y written in FP64 (the reduced-storage matrix form of the
 * mixed-precision path).  beta = 0 never reads y.  x and y on a 16-byte
 * boundary (as cudaMalloc and framework allocations are) take the tiled
 * kernels; otherwise the FP64 values with FP64 products are used whatever
 * the precision. */
int bo_mat_spmv(bo_mat* A, double alpha, const double* x, double beta, double* y, int precision);
/* BO_ERR_ARG for NULL; see bo_ctx_destroy for lifetimes. */
int bo_mat_destroy(bo_mat* A);

/* Decoupling, ILU(0) factorisation and AMG hierarchy for the current values
 * of A (paper Sec. 3.2).  The preconditioner keeps a pointer to A.
 * BO_ERR_BREAKDOWN: zero saturation pivot in Quasi-IMPES, singular ILU
 * pivot block, zero AMG diagonal or singular coarsest matrix. */
int bo_prec_setup(bo_mat* A, const bo_prec_opts* opts, bo_prec** out);
/* Recompute all preconditioner values after bo_mat_update_values (same
 * options, no reallocation).  Errors as bo_prec_setup; on error P must be
 * updated again before it is used.  Synchronises. */
int bo_prec_update(bo_prec* P);
/* z = stage(r), r and z device vectors of length 3 nx ny nz (FP64), owned by
 * the caller; stage one of BO_STAGE_* (else BO_ERR_ARG).  Uses P's Krylov
 * workspace: not while a solve with P is in flight.  Synchronises. */
int bo_prec_apply(bo_prec* P, int stage, const double* r, double* z);
/* y = (D_QI^{-1} A) x in FP64, device vectors of length 3 nx ny nz (paper
 * Sec. 3.2 decoupled system).  Uses P's Krylov workspace.  Synchronises. */
int bo_prec_spmv_decoupled(bo_prec* P, const double* x, double* y);
/* AMG level sizes: writes up to cap triples (nx, ny, nz), returns the level
 * count (or a negative status). */
int bo_prec_amg_levels(bo_prec* P, int32_t* dims, int cap);
/* Synchronises P's stream and frees its workspace; drops P's reference on
 * its matrix.  BO_ERR_ARG for NULL. */
int bo_prec_destroy(bo_prec* P);
/* Launch mode of P's solves (BO_LAUNCH_STREAM default, BO_LAUNCH_GRAPH,
 * BO_LAUNCH_BATCH_GRAPH).  Graph mode captures the kernels of each Arnoldi
 * column once per restart length and replays them; the graphs are rebuilt
 * after a change of restart length or of the learned coarse space.  Batch
 * graph mode applies to bo_solve_batched when every system of the batch has
 * it (and no rate-controlled wells): the systems run their FGMRES cycles in
 * lockstep, Arnoldi column j of all of them captured as one CUDA graph (one
 * branch per pool stream) and launched once per column for the whole batch;
 * the two most recent batches' graphs are kept for reuse.  A single solve
 * in that mode runs as in stream mode.  No counterpart in the paper: a
 * launch-overhead measure for batches of small systems. */
int bo_prec_set_launch_mode(bo_prec* P, int mode);
/* Tile parameters of the per-kernel form of P's AMG V-cycle, the form its
 * CUDA-graph launch modes run (captured graphs cannot hold cooperative
 * launches): `cells` level-0 Gauss-Seidel cells per thread (1, 2 or 4, all
 * of a thread's loads issued before its stores) and `threads` per block
 * (128, 256 or 512) for every per-kernel AMG launch.  The V-cycle is the
 * same whatever the shape.  Captured graphs are rebuilt after a change.
 * Default 1 and 256; BO_ERR_ARG for another value.  No counterpart in the
 * paper: a tile choice the batch autotuner makes. */
int bo_prec_set_amg_tile(bo_prec* P, int cells, int threads);

/* New values for many systems at once: for each r, the values val[r]
 * (host or device per mem; NULL keeps the matrix's values) go into P[r]'s
 * matrix as bo_mat_update_values does, then P[r] is refreshed as
 * bo_prec_update does, the systems spread over the stream pool, with one
 * synchronisation for the whole batch instead of two per system.  Each P[r]
 * needs its own matrix.  Returns the first error found (pattern, non-finite
 * value or singular pivot), after all systems were processed. */
int bo_update_batched(bo_prec* const* P, int nreal, const double* const* val, int mem);

/* Streams bo_solve_batched spreads its systems over (1..16, default 16). */
int bo_set_batch_streams(int n);

typedef struct {
  int32_t launch_mode;   /* chosen BO_LAUNCH_* */
  int32_t streams;       /* chosen stream-pool width */
  double best_ms;        /* wall time of the chosen configuration's batch */
  int32_t from_cache;    /* 1: taken from the cache without timing */
  double trial_ms[9];    /* stream x {4, 8, 16}, graph x {4, 8, 16}, batch graph x {4, 8, 16} */
  int32_t amg_cells;     /* chosen tile of the per-kernel AMG form (bo_prec_set_amg_tile) */
  int32_t amg_threads;
  double tile_ms[5];     /* graph forms only: (cells, threads) = (2, 256), (4, 256), (1, 128),
                            (2, 128), (1, 512) with the chosen form and width; 0 otherwise */
} bo_tune_result;

/* Autotuner for bo_solve_batched (no counterpart in the paper).  Times the
 * caller's batch (same arguments as bo_solve_batched; x is overwritten,
 * solves start from zero) under every launch mode (stream, graph, batch
 * graph) and stream-pool width of 4, 8 and 16, then, when a graph form wins,
 * under five more tiles of the per-kernel AMG form with that form and width, two passes each (the first untimed), applies the fastest to
 * all P and to the pool, and records it in the JSON file cache_path (NULL:
 * no cache) under a key of the batch's shape (count, total and largest cell
 * counts as powers of two, FP32 preconditioners, restart).  With an entry
 * for the key already present it applies that entry without timing.  Returns
 * BO_ERR_ARG if the cache cannot be written. */
int bo_autotune_batched(bo_prec* const* P, int nreal, const double* const* b, double* const* x,
                        const bo_solve_opts* opts, const char* cache_path, bo_tune_result* out);
/* Learned coarse space (no counterpart in the paper; an addition to the
 * CPR preconditioner of Sec. 3.3, Alg. 2).  dp: device array of nx ny nz
 * doubles in natural cell order, a predicted pressure update; the grid is
 * cut into tiles of tx x ty x tz cells (partial tiles at the far faces) and
 * Z holds dp restricted to each tile as one column.  E = Z^T A~_pp Z, with
 * A~_pp the quasi-IMPES-decoupled pressure block, is formed and inverted in
 * FP64 now and again on every bo_prec_update; after each AMG V-cycle on a
 * pressure residual f the pressure correction gains Z E^{-1} Z^T f (also in
 * the BO_STAGE_AMG stage of bo_prec_apply).  dp is copied; NULL removes the
 * space.  BO_ERR_ARG if a tile size is < 1 or there are more than 128
 * tiles; BO_ERR_BREAKDOWN if E is singular (the space is then removed).
 * Synchronises. */
int bo_prec_set_coarse_space(bo_prec* P, const double* dp, int tx, int ty, int tz);
/* The same coarse space built straight from a network prediction: dp[c] =
 * scale * pred[c][0], pred [nx ny nz][4] FP32 on the device (natural order,
 * channel 0 the pressure update in the network's normalisation), so the
 * caller does no arithmetic on the prediction.  NULL removes the space;
 * BO_ERR_ARG also for a non-finite scale; otherwise as
 * bo_prec_set_coarse_space. */
int bo_learned_coarse_space(bo_prec* P, const float* pred, double scale, int tx, int ty, int tz);
/* Learned initial guess (no counterpart in the paper): x0[3c + k] =
 * scale[k] pred[c][k] for k < ncomp (1..3), 0 for the other components,
 * from a network prediction pred [nx ny nz][4] FP32 (device); natural
 * order.  Falls back to x0 = 0 (and *used = 0) unless ||b - A x0|| < ||b||,
 * so the guess never starts a solve further from the solution than the zero
 * guess does (both norms reduced in FP64 in P's own workspace, any grid
 * size).  b, x0: device, 3 nx ny nz doubles.  Uses P's Krylov workspace: not
 * while a solve with P is in flight.  Synchronises. */
int bo_learned_guess(bo_prec* P, const double* b, const float* pred, const double* scale, int ncomp, double* x0,
                     int* used);

/* Solve A x = b with FGMRES(m) + CPR to ||b - A x|| <= tol ||b|| (paper
 * Alg. 1 step "find dx").  b, x: length 3 nx ny nz, device or host memory
 * per opts->mem; x holds the initial guess unless x0_is_zero.  On
 * BO_ERR_NOT_CONVERGED (maxit reached, or a whole restart cycle reduced the
 * residual by less than 1%) x holds the last iterate and info is filled.
 * b = 0 returns x = 0.  info may be NULL.
 * Precision: the Krylov basis, Gram-Schmidt (second pass), updates and the
 * true residual that decides convergence are FP64.  The Arnoldi product
 * A z_j uses a copy of A split into two floats per value (48 significant
 * bits for |a| >= 2^-74, 24 below), and the preconditioned vectors z_j are
 * stored the same way; a matrix with a value outside [2^-120, 2^126] makes
 * the product use the FP64 matrix instead.  The split vectors keep FP32's
 * exponent range: a system scaled so that z_j = M^{-1} v_j (|v_j| = 1)
 * leaves that range overflows and the solve returns BO_ERR_BREAKDOWN. */
int bo_solve(bo_prec* P, const double* b, double* x, const bo_solve_opts* opts, bo_solve_info* info);
/* Solve A x = b with BiCGSTAB (van der Vorst 1992) right preconditioned by
 * the same CPR as bo_solve: the solver of the paper's scalability
 * experiments (Sec. 3.3 solver list, Sec. 4).  Same arguments, tolerance rule
 * (||b - A x|| <= tol ||b|| on the recomputed FP64 residual) and info as
 * bo_solve; opts->restart is ignored (it only sizes the workspace shared
 * with bo_solve).  One iteration applies the preconditioner twice.  When a
 * scalar of the recurrence vanishes the iteration restarts from the true
 * residual; BO_ERR_BREAKDOWN if it vanishes right after such a restart.  No
 * residual history is recorded. */
int bo_solve_bicgstab(bo_prec* P, const double* b, double* x, const bo_solve_opts* opts, bo_solve_info* info);
/* Solve nreal independent systems A_r x_r = b_r at once (an ensemble of
 * realisations, possibly of different grid sizes; each P[r] a distinct
 * preconditioner on the same device).  The solves run concurrently on a
 * pool of streams driven by one host thread, each exactly as bo_solve
 * would run it (same kernels, same results).  infos: nreal entries or
 * NULL.  Returns BO_OK or the first failing status; each info holds its
 * own.  Synchronises before returning. */
int bo_solve_batched(bo_prec* const* P, int nreal, const double* const* b, double* const* x,
                     const bo_solve_opts* opts, bo_solve_info* infos);
/* Estimated relative residuals of the last bo_solve with P, one per
 * iteration, into host memory buf[cap]; returns how many were written (at
 * most cap), or BO_ERR_ARG for a NULL P or a NULL buf with cap > 0. */
int bo_prec_residual_history(bo_prec* P, double* buf, int cap);

/* state += dx on the device in FP64 (paper Alg. 1, x^l = x^{l-1} + dx):
 * state, dx device arrays of n doubles owned by the caller, in the solver's
 * natural interleaved order.  n = 0 does nothing; BO_ERR_ARG for NULL or
 * n < 0.  Ordered on the context's stream; does not synchronise. */
int bo_newton_update(bo_ctx* ctx, double* state, const double* dx, int64_t n);

/* Diagnostics (no counterpart in the paper): the number of CUDA kernels this
 * library has launched in the process so far. */
int64_t bo_kernel_launches(void);

/* Residual without device allocation (no counterpart in the paper).  For
 * callers that must not call cudaMalloc when they check a residual: a
 * framework's caching allocator may hold nearly all device memory, and
 * cudaMalloc / cudaFree synchronise the whole device, which a serving loop
 * or a caller that allocates only at start-up cannot afford.
 *   r = b - A x and norms[0] = ||b - A x||_2, norms[1] = ||b||_2, in FP64;
 *   b, x, r: device vectors of length 3 nx ny nz (natural interleaved order);
 *   norms: device array of 2 doubles.  All are owned by the caller.
 *   r must not overlap b or x (each thread reads x at its six neighbours
 *   while others write r): BO_ERR_ARG if it does.
 * Scratch lives in an array compiled into the library (256 KB per device
 * that loads it, held until the process exits), shared by every call on the
 * device: calls that overlap on the GPU race on it.  The first call on each
 * device looks up that array's device address, so make it before any
 * stream capture.  Grids of more than 4,194,304 cells give BO_ERR_ARG.
 * Ordered on the context's stream; does not synchronise. */
int bo_mat_residual_noalloc(bo_mat* A, const double* b, const double* x, double* r, double* norms);

/* ---------------------------------------------------------------------------
 * The black-oil model on the device and the inexact Newton method (paper
 * Sec. 2.1 Eq. 3 with its closure relations, Sec. 2.3 Eq. 4, Sec. 3.1
 * Alg. 1).  The residual of cell c and component (oil, water, gas) is
 *   R = V / (5.615 dt) [M(x) - M(x^n)] - sum of face fluxes - well rates,
 * M_w = phi Sw / Bw, M_o = phi So / Bo, M_g = phi (Sg / Bg + Rs So / Bo);
 * face fluxes T lambda_up (Phi_b - Phi_a) per phase with two-point
 * transmissibilities T = 0.001127 A 2 / (h / k_a + h / k_b), Corey curves and
 * Stone II oil relative permeability, phase-potential upwinding, potentials
 * p - rho D / 144; wells at fixed bottom-hole pressure with the cell's phase
 * mobilities (producers) or total mobility (water injectors).  No-flow outer
 * boundary.  b = -R(x), A = dR/dx (exact derivatives).  Units: ft, psi, mD,
 * cp, day, stb, Mscf.  Unknowns (p, Sw, Sg) per cell, interleaved, natural
 * cell order; depth grows with k.
 * ------------------------------------------------------------------------- */
typedef struct bo_model bo_model;

/* Fluid, rock and saturation-function constants of the model (the paper gives
 * none for synthetic cases): Bw = bw0 (1 - cw (p - pref)), Bo = bo0 + dbo
 * (p - pref), Rs = rs0 + drs (p - pref) Mscf/stb, Bg = bg0 - dbg (p - pref)
 * rb/Mscf, viscosities in cp, stock-tank densities in lb/ft^3, porosity
 * phi0 (1 + cr (p - pref)); Corey end points swc, sorw, sorg, sgc and
 * exponents nw, now, ng, nog; gravity 1 (hydrostatic terms) or 0. */
typedef struct {
  double pref;
  double bw0, cw, muw;
  double bo0, dbo, rs0, drs, muo;
  double bg0, dbg, mug;
  double rhow_sc, rhoo_sc, rhog_sc;
  double cr;
  double swc, sorw, sorg, sgc;
  double nw, now, ng, nog;
  double gravity;
} bo_fluid;

enum { BO_FORCING_FIXED = 0, BO_FORCING_EW1 = 1, BO_FORCING_EW2 = 2, BO_FORCING_EW3 = 3 };
enum { BO_NEWTON_MAX_STEPS = 64 };

typedef struct {
  double eps;          /* stop when ||b(x^l)|| < eps; 0: eps = eps_rel ||b(x^0)||      */
  double eps_rel;      /* (default 1e-8)                                              */
  int32_t forcing;     /* BO_FORCING_*: the three choices of Sec. 3.1, or fixed theta  */
  double theta_fixed;  /* BO_FORCING_FIXED: theta of every step (default 1e-2)         */
  double theta_max;    /* theta_0, and the upper clip of every theta (default 0.1)     */
  double theta_min;    /* lower clip (default 1e-10)                                   */
  double gamma, beta;  /* the third choice: theta = gamma (||b_new|| / ||b_old||)^beta  */
  int32_t maxit;       /* Newton steps, at most BO_NEWTON_MAX_STEPS (default 20)       */
  int32_t restart;     /* FGMRES restart of the linear solves (default 30)             */
  int32_t lin_maxit;   /* iteration cap of each linear solve (default 1000)            */
} bo_newton_opts;

typedef struct {
  int32_t status;                            /* as returned                      */
  int32_t iters;                             /* Newton steps taken               */
  int32_t converged;                         /* ||b(x)|| < eps at exit           */
  int32_t lin_total;                         /* linear iterations in all steps   */
  double bnorm[BO_NEWTON_MAX_STEPS + 1];     /* ||b(x^l)||, l = 0 .. iters       */
  double theta[BO_NEWTON_MAX_STEPS];         /* forcing term of step l           */
  int32_t lin_iters[BO_NEWTON_MAX_STEPS];    /* FGMRES iterations of step l      */
  double lin_rel_res[BO_NEWTON_MAX_STEPS];   /* ||b - A dx|| / ||b|| of step l   */
} bo_newton_info;

/* Defaults: eps 0 with eps_rel 1e-8, the third forcing term with gamma 0.9,
 * beta 2, theta in [1e-10, 0.1], 20 steps, restart 30, 1000 linear its. */
void bo_newton_opts_default(bo_newton_opts* o);

/* The model of one reservoir on ctx's device.  Host arrays of nx ny nz
 * values (natural order): permeabilities kx, ky, kz (mD, > 0), reference
 * porosity phi0 (> 0), cell-centre depth (ft).  nperf perforations: cell
 * perf_cell[e], well type perf_type[e] (0 water injector, 1 producer),
 * bottom-hole pressure perf_bhp[e] (psi) at reference depth perf_dref[e],
 * and well index perf_wi[e] (the Peaceman index of the completion, an input
 * like the permeability).  Copied; grid rules as for bo_mat_create_bsr.
 * BO_ERR_ARG for a bad size, a non-positive permeability or porosity, a
 * perforation outside the grid.  Holds a reference on ctx.  Synchronises. */
int bo_model_create(bo_ctx* ctx, const bo_grid* grid, const bo_fluid* fluid, const double* kx, const double* ky,
                    const double* kz, const double* phi0, const double* depth, int32_t nperf,
                    const int32_t* perf_cell, const int32_t* perf_type, const double* perf_bhp,
                    const double* perf_dref, const double* perf_wi, bo_model** out);
int bo_model_destroy(bo_model* M);
/* Residual and Jacobian at state x (device, 3 nx ny nz doubles, (p, Sw, Sg)
 * interleaved) with previous time level xn and time step dt (days): b =
 * -R(x) into b (device, 3 nx ny nz; NULL: not copied out), the Jacobian values
 * into val (device, 9 nnzb doubles in the BSR order of the 7-point pattern:
 * rows in cell order, columns -z, -y, -x, diag, +x, +y, +z as they exist;
 * NULL: not copied out), ||b||_2 into *bnorm (host; NULL: not computed).
 * BO_ERR_BREAKDOWN if a cell's porosity or formation volume factor is not
 * positive at x.  Synchronises. */
int bo_model_assemble(bo_model* M, const double* x, const double* xn, double dt, double* b, double* val,
                      double* bnorm);
/* The inexact Newton method (Alg. 1) for one time step: from x (device, in:
 * the initial guess x^0, out: the last iterate), while ||b(x^l)|| >= eps:
 * assemble on the device, put the Jacobian into P's matrix and refresh P
 * (as bo_mat_update_values and bo_prec_update), solve A dx = b with FGMRES and
 * P to ||b - A dx|| <= theta_l ||b|| from a zero guess, x += dx, and compute
 * the next theta from the chosen forcing term of Sec. 3.1 (the second with
 * the absolute value of its difference), clipped to [theta_min, theta_max];
 * theta_0 = theta_max.  P must be set up on a matrix of the model's grid and
 * context.  Returns BO_OK when converged, BO_ERR_NOT_CONVERGED after maxit
 * steps (x then holds the last iterate), or the first error of an assembly,
 * setup or solve.  info (may be NULL) records every step.  No saturation
 * chopping: the method as stated. */
int bo_newton_solve(bo_model* M, bo_prec* P, double* x, const double* xn, double dt, const bo_newton_opts* opts,
                    bo_newton_info* info);

/* ---------------------------------------------------------------------------
 * Dual-porosity systems (paper Sec. 2.1, the dual-porosity model: fracture
 * and matrix continua per cell with a transfer term between them).
 *
 * Input: a BSR matrix of nbrows = 2 nx ny nz block rows (3x3, row-major,
 * columns (p, Sw, Sg)); block row c < N is the fracture node of cell c with
 * its 7-point fracture neighbours and column N + c; block row N + c is the
 * matrix node of cell c with exactly the columns c and N + c (any order
 * within a row).  Vectors have 6N doubles, the fracture nodes' (p, Sw, Sg)
 * first.  grid->ncontinua must be 2; other rules as for bo_mat_create_bsr.
 *
 * The matrix unknowns are eliminated exactly per cell (they couple only to
 * their own fracture node): S = A_ff - A_fm A_mm^{-1} A_mf is a 7-point
 * system on the fracture nodes, solved by the single-porosity CPR-FGMRES;
 * x_m = A_mm^{-1} (b_m - A_mf x_f) is recovered afterwards.  Convergence is
 * judged on the full system's FP64 residual ||b - A x|| / ||b||.
 * ------------------------------------------------------------------------- */
typedef struct bo_dp bo_dp;

/* Copies the pattern and values (host or device per mem), checks the
 * pattern (BO_ERR_PATTERN), forms S and A_mm^{-1} (BO_ERR_BREAKDOWN on a
 * singular A_mm, BO_ERR_NONFINITE on NaN/Inf).  Holds a reference on ctx.
 * Synchronises. */
int bo_dp_create(bo_ctx* ctx, const bo_grid* grid, int32_t nbrows, int64_t nnzb, const int32_t* rowptr,
                 const int32_t* col, const double* val, int mem, bo_dp** out);
/* New values on the same pattern; S changes in place, so a preconditioner on
 * it needs bo_prec_update afterwards.  Synchronises. */
int bo_dp_update_values(bo_dp* dp, const double* val, int mem);
/* The condensed fracture system S (owned by dp, valid until bo_dp_destroy):
 * set up the preconditioner on it with bo_prec_setup. */
bo_mat* bo_dp_fracture_matrix(bo_dp* dp);
/* Solve A x = b (device vectors of 6N doubles) to ||b - A x|| <= tol ||b||
 * with P set up on bo_dp_fracture_matrix(dp): condense, CPR-FGMRES on S,
 * recover the matrix unknowns, check the full residual in FP64 and refine
 * (up to two more passes) if rounding left it above tol.  info sums the
 * passes' iterations and reports the full system's true_rel_res; returns
 * BO_OK or BO_ERR_NOT_CONVERGED (x then holds the last iterate). */
int bo_dp_solve(bo_dp* dp, bo_prec* P, const double* b, double* x, const bo_solve_opts* opts, bo_solve_info* info);
/* Solve nreal dual-porosity systems at once (an ensemble of dual-porosity
 * realisations; no counterpart in the paper): every system condensed onto
 * its fracture nodes, the condensed systems solved together as
 * bo_solve_batched does (P[r] set up on bo_dp_fracture_matrix(dp[r])), the
 * matrix unknowns recovered, and each full FP64 residual checked; a system
 * that rounding left above tol is solved again alone as bo_dp_solve does.
 * b, x: device arrays of 6 N_r doubles.  infos (may be NULL) per system;
 * returns BO_OK or the first failing status.  Synchronises. */
int bo_dp_solve_batched(bo_dp* const* dp, bo_prec* const* P, int nreal, const double* const* b, double* const* x,
                        const bo_solve_opts* opts, bo_solve_info* infos);
int bo_dp_destroy(bo_dp* dp);

/* ---------------------------------------------------------------------------
 * Two-phase oil-water systems (paper Sec. 2.2: per cell the unknowns
 * (p_o, S_w) and the (oil, water) conservation equations; 2x2 blocks on the
 * 7-point pattern, rules as for bo_mat_create_bsr with 4 values per block,
 * row-major).  Vectors hold 2N doubles, (p_o, S_w) of cell c at 2c, 2c+1.
 *
 * The system runs on the three-unknown layout: each block padded to 3x3
 * with a unit diagonal for a third unknown that nothing else touches (its
 * component stays zero in every vector), so every CPR stage is the 2x2
 * stage (see bo_prec_opts.decoupling for Quasi-IMPES or ABF).  The padded
 * matrix stores 9 values per block where a native 2x2 layout would store 4.
 * ------------------------------------------------------------------------- */
typedef struct bo_ow bo_ow;

/* Copies pattern and values (host or device per mem); BO_ERR_PATTERN /
 * BO_ERR_NONFINITE as bo_mat_create_bsr.  Holds a reference on ctx.
 * Synchronises. */
int bo_ow_create(bo_ctx* ctx, const bo_grid* grid, int32_t nbrows, int64_t nnzb, const int32_t* rowptr,
                 const int32_t* col, const double* val, int mem, bo_ow** out);
/* New 2x2 values on the same pattern (a preconditioner on bo_ow_matrix
 * needs bo_prec_update afterwards).  Synchronises. */
int bo_ow_update_values(bo_ow* w, const double* val, int mem);
/* The padded matrix (owned by w, valid until bo_ow_destroy): set up the
 * preconditioner on it with bo_prec_setup. */
bo_mat* bo_ow_matrix(bo_ow* w);
/* y = alpha A x + beta y, device vectors of 2N doubles (FP64 product).
 * Synchronises. */
int bo_ow_spmv(bo_ow* w, double alpha, const double* x, double beta, double* y);
/* Solve A x = b (device vectors of 2N doubles; opts->mem must be
 * BO_MEM_DEVICE) with P set up on bo_ow_matrix(w): CPR-FGMRES, or
 * BiCGSTAB (the solver of the paper's oil-water scalability runs).  Status
 * and info as bo_solve / bo_solve_bicgstab. */
int bo_ow_solve(bo_ow* w, bo_prec* P, const double* b, double* x, const bo_solve_opts* opts, bo_solve_info* info);
int bo_ow_solve_bicgstab(bo_ow* w, bo_prec* P, const double* b, double* x, const bo_solve_opts* opts,
                         bo_solve_info* info);
int bo_ow_destroy(bo_ow* w);

/* ---------------------------------------------------------------------------
 * Rate-controlled wells (paper Sec. 2.3: a well under a fixed water, oil or
 * liquid rate has its bottom-hole pressure p_h as an unknown and one
 * constraint equation, the sum of its perforations' rates equal to the
 * target).  The Newton system takes the bordered block form of Sec. 3.2,
 *
 *     [ A     A_pw ] [x  ]   [b  ]
 *     [ A_wp  A_ww ] [x_w] = [b_w],
 *
 * A the reservoir matrix (a bo_mat), and per perforation e of well v in cell
 * c: apw[3e + r] = the derivative of cell c's equation r with respect to
 * p_h of v (column v of A_pw, rows 3c..3c+2), awp[3e + u] = the derivative
 * of v's constraint with respect to unknown u of cell c (row v of A_wp);
 * aww[v] = the derivative of v's constraint with respect to its own p_h
 * (A_ww is diagonal: a constraint involves only its own well).  Vectors of
 * the bordered system hold 3N + W doubles: the cells' (p, Sw, Sg), then the
 * W well unknowns.
 *
 * The solve eliminates the wells exactly (Schur complement
 * S = A - A_pw A_ww^{-1} A_wp on the reservoir unknowns), runs CPR-FGMRES on
 * S with the preconditioner's well coupling corrected by the Woodbury
 * identity (exact with respect to the CPR of A), and recovers
 * x_w = A_ww^{-1} (b_w - A_wp x).  Convergence is judged on the bordered
 * system's residual ||[b; b_w] - A_b [x; x_w]|| / ||[b; b_w]||.
 * ------------------------------------------------------------------------- */
typedef struct bo_wells bo_wells;

/* The border's structure on matrix A: nwells (1..128) wells, nperf (>= 0)
 * perforations with host arrays perf_cell[e] (natural cell index) and
 * perf_well[e] (0..nwells-1, non-decreasing: perforations grouped by well).
 * A cell may be perforated once (BO_ERR_ARG otherwise).  Holds a reference
 * on A.  Synchronises. */
int bo_wells_create(bo_mat* A, int32_t nwells, int32_t nperf, const int32_t* perf_cell, const int32_t* perf_well,
                    bo_wells** out);
/* The border's values (host or device per mem): apw, awp of 3 nperf
 * doubles, aww of nwells.  BO_ERR_NONFINITE on NaN/Inf, BO_ERR_BREAKDOWN
 * where aww[v] == 0.  Synchronises. */
int bo_wells_update_values(bo_wells* w, const double* apw, const double* awp, const double* aww, int mem);
/* 1 (default): the preconditioner carries the Woodbury correction of the
 * well coupling (set up at the first solve after a change of the well
 * values or of the preconditioner: nwells applications of the CPR); 0: the
 * plain CPR of A (more iterations, no setup). */
int bo_wells_set_coupling(bo_wells* w, int mode);
/* y = alpha A_b x + beta y on device vectors of 3N + W doubles (FP64; the
 * cell rows by bo_mat_spmv's FP64 product).  Synchronises. */
int bo_wells_spmv(bo_wells* w, double alpha, const double* x, double beta, double* y);
/* Solve the bordered system (device vectors of 3N + W doubles, opts->mem
 * must be BO_MEM_DEVICE) with P set up on w's matrix.  A nonzero initial
 * guess (opts->x0_is_zero == 0) is refined by a correction solve.  info
 * reports the bordered system's true_rel_res.  Returns BO_OK,
 * BO_ERR_NOT_CONVERGED (x holds the last iterate), or the status of a
 * failed setup.  Synchronises. */
int bo_solve_bordered(bo_prec* P, bo_wells* w, const double* b, double* x, const bo_solve_opts* opts,
                      bo_solve_info* info);
int bo_wells_destroy(bo_wells* w);

/* ---------------------------------------------------------------------------
 * Learned Newton update.  No counterpart in the paper: an addition of this
 * library that feeds the Krylov solve of Sec. 3 a predicted initial guess
 * and a predicted coarse space; the architecture is this library's choice.
 *
 * A 3D convolutional network on the reservoir grid: an input convolution
 * (16 -> 32 channels, ReLU), 6 residual blocks of two 32 -> 32 convolutions
 * (ReLU; the second adds the block input before its ReLU) and an output
 * convolution (32 -> 16, linear).  Every convolution is 3x3x3 with 'same'
 * zero padding.  Output channel 0 is the predicted Newton pressure update dp
 * of each cell, channels 1..2 optionally (dSw, dSg), in the caller's
 * normalisation.
 *
 * Layouts (all device memory owned by the caller unless noted):
 *   activations / inputs: BF16 bit patterns (uint16), NDHWC:
 *     [batch][nz][ny][nx][C], voxel v = x + nx (y + ny z) (the solver's cell
 *     index); the network input has C = 16 (features zero-padded);
 *   weights: BF16 [27][Cout][Cin], tap t = 9 (dz+1) + 3 (dy+1) + (dx+1)
 *     (cross-correlation: output v reads input v + (dx, dy, dz));
 *   biases, gradients of activations, predictions: FP32;
 *   predictions / targets: FP32 [batch][V][4] (channel 3 unused).
 * Arithmetic: BF16 x BF16 products with FP32 accumulation on the tensor
 * cores; hidden activations are stored in BF16; the loss is accumulated in
 * FP64.  Every call is ordered on the context's stream.
 * ------------------------------------------------------------------------- */
typedef struct bo_cnn bo_cnn;

/* Network for grids of nx x ny x nz voxels and up to max_batch samples;
 * weights He-normal from `seed` (the second convolution of each block and the
 * output convolution scaled by 0.1), biases zero.  Holds a reference on ctx.
 * BO_ERR_ARG if max_batch nx ny nz > 2^31.  Synchronises. */
int bo_cnn_create(bo_ctx* ctx, int nx, int ny, int nz, int max_batch, uint64_t seed, bo_cnn** out);
int bo_cnn_destroy(bo_cnn* net);
/* Number of FP32 parameters: per layer 27 Cout Cin weights then Cout biases. */
int64_t bo_cnn_param_count(const bo_cnn* net);
/* Copy the FP32 master parameters (or the gradients of the last backward
 * pass) to / from HOST memory of at least bo_cnn_param_count floats;
 * set_params also refreshes the BF16 copy.  Synchronise. */
int bo_cnn_get_params(bo_cnn* net, float* host, int64_t cap);
int bo_cnn_set_params(bo_cnn* net, const float* host, int64_t count);
int bo_cnn_get_grads(bo_cnn* net, float* host, int64_t cap);
/* pred[batch][V][4] = network(x); x: [batch][V][16] BF16. */
int bo_cnn_forward(bo_cnn* net, const uint16_t* x, int batch, float* pred);
/* Forward pass, loss = (1 / (batch V)) sum_v mask_v sum_{k < nout}
 * (pred[v][k] - target[v][k])^2 (mask NULL: all ones; 1 <= nout <= 4) and
 * the backward pass into the network's gradient buffer.  *loss (host, may be
 * NULL) receives the loss; a non-NULL loss synchronises. */
int bo_cnn_backward(bo_cnn* net, const uint16_t* x, const float* target, const float* mask, int nout, int batch,
                    double* loss);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected) on the
 * FP32 master weights with the last gradients; refreshes the BF16 copy. */
int bo_cnn_adam_step(bo_cnn* net, float lr);

/* Single convolutions (the network's layers; also what the parity tests
 * check).  Supported (cin, cout): forward (16, 32), (32, 32), (32, 16) as
 * used by the network; modes by the non-NULL outputs:
 *   y only, relu = 1           : y = ReLU(conv(x) + bias (+ residual)) BF16;
 *   y and yf, relu = 0         : y = conv(x) + bias in BF16 and yf[v][0..3] =
 *                                channels 0..3 in FP32 (cout = 16 only);
 *   yf only, relu = 0          : yf[v][co] = conv(x) + bias in FP32.
 * backward_data: dx[v][ci] = sum_t,co dy[v - off(t)][co] w[t][co][ci] (FP32),
 *   dy BF16 [batch][V][cout];
 * backward_weights: dw[t][co][ci] = sum_v dy[v][co] x[v + off(t)][ci] and
 *   db[co] = sum_v dy[v][co] (FP32); dy FP32 [batch][V][cout] is rounded to
 *   BF16 for the products.
 * backward_data and backward_weights allocate and free scratch and
 * synchronise.  BO_ERR_ARG on an unsupported (cin, cout) or mode. */
int bo_conv3d_forward(bo_ctx* ctx, int nx, int ny, int nz, int batch, int cin, int cout, const uint16_t* x,
                      const uint16_t* w, const float* bias, const uint16_t* residual, int relu, uint16_t* y,
                      float* yf);
int bo_conv3d_backward_data(bo_ctx* ctx, int nx, int ny, int nz, int batch, int cin, int cout, const uint16_t* dy,
                            const uint16_t* w, float* dx);
int bo_conv3d_backward_weights(bo_ctx* ctx, int nx, int ny, int nz, int batch, int cin, int cout, const uint16_t* x,
                               const float* dy, float* dw, float* db);
/* Convolution engine for the 32 -> 32 layers (forward and data gradient;
 * process-wide): 0 = mma.sync kernel, 1 = tcgen05 kernel (tensor memory
 * accumulator, TMA-fetched tiles; the default).  The other layers always use
 * mma.sync. */
int bo_set_conv_engine(int engine);
/* How the AMG V-cycle is launched (process-wide); every form computes the
 * same V-cycle of paper Sec. 3.2's pressure AMG stage:
 * 2 (the default) = levels 0 and 1 in two cooperative launches, a down leg
 *   and an up leg whose blocks meet at grid-wide barriers between the
 *   Gauss-Seidel half sweeps, around one thread-block-cluster launch (up to
 *   16 blocks, hardware cluster barriers) for all coarser levels, the
 *   levels of at most 4096 cells in one of its blocks;
 * 1 = the cooperative legs smooth every multi-block level, around one
 *   block for the levels of at most 4096 cells;
 * 0 = one kernel per half sweep, restriction and prolongation.
 * Inside stream capture (CUDA-graph launch mode) the per-kernel form is used
 * whatever the setting, and a form the device refuses falls back to it.  A
 * grid barrier that waits too long ends the launch and the solve returns
 * BO_ERR_TIMEOUT.  BO_ERR_ARG for another mode. */
int bo_set_amg_cooperative(int on);
/* Polls of a grid barrier of the cooperative AMG legs before it gives up
 * (process-wide; read at each V-cycle launch).  0 restores the default,
 * 2^22 polls of about 30 ns.  A lower limit makes a barrier give up while
 * other blocks are still on their way: the launch then ends early and the
 * solve returns BO_ERR_TIMEOUT with x holding the last iterate; the next
 * solve starts clean.  No counterpart in the paper: it exists so the bounded
 * waits' error path can be exercised without hanging a GPU. */
int bo_set_amg_barrier_spins(uint32_t spins);
/* Gram-Schmidt form of the Arnoldi step (CGS2): 1 (default) three passes
 * over the basis, the first update fused with the second coefficient pass;
 * 0 four separate passes.  The same arithmetic; process-wide. */
int bo_set_gs_fused(int on);
/* BO_ERR_TIMEOUT if a tcgen05 convolution gave up waiting on one of its
 * barriers since the last call (its output is then incomplete), else BO_OK;
 * clears the flag.  Synchronises the device. */
int bo_tc_status(void);

#ifdef __cplusplus
}
#endif
#endif /* BOSOLVE_H */
