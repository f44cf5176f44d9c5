/*
 * pmg.h -- C-ABI of the GB300 ILUT-smoothed p-multigrid solver for Galerkin
 * IgA discretisations of Poisson's equation (and the paper's
 * convection-diffusion-reaction benchmark).
 *
 * Method: Tielen, Moeller, Goeddeke, Vuik, "A p-multigrid method enhanced with
 * an ILUT smoother and its comparison to h-multigrid methods within
 * Isogeometric Analysis" (arXiv 1901.01685).  The linear system is
 * A_{h,p} u_{h,p} = f_{h,p} of Sec. 2 (Eq. los); the solver is the V-cycle of
 * Sec. 3 (two-grid correction scheme applied recursively down to p = 1), with
 * the ILUT smoother of Sec. 3 "Smoother", the lumped L2-projection transfers
 * of Sec. 3 "Prolongation and restriction" and an h-multigrid coarse solve at
 * p = 1; the stopping rule of Sec. 5 (relative residual, divergence above 1e10).
 *
 * Conventions (all entry points):
 *  - Every call returns a pmg_status; the library never aborts, traps or
 *    exits.  On failure pmg_last_error() returns a thread-local message.
 *  - Vectors are FP64, interior degrees of freedom only (boundary DOFs are
 *    eliminated, Sec. 5), numbered lexicographically with the first
 *    parametric direction fastest, 0-based.
 *  - "_dev" pointers are CUDA device pointers owned by the caller; "_host"
 *    pointers are host memory owned by the caller.  `stream` is a
 *    cudaStream_t passed as void* (NULL = legacy default stream).
 *  - The library allocates no device memory.  The hierarchy is copied into
 *    a caller-provided device arena (pmg_upload) and each solve uses a
 *    caller-provided device workspace (pmg_workspace_create); a workspace
 *    for several right-hand sides also holds a small pinned host buffer.
 *  - A handle's data is immutable after pmg_upload and may be shared by
 *    concurrent solves that use different workspaces; only its kernel choice
 *    changes (pmg_autotune, pmg_set_kernels), never while a solve uses it.
 *    A workspace serves one solve at a time.
 */
#ifndef PMG_H_
#define PMG_H_

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PMG_OK = 0,
  PMG_ERR_ARG = 1,        /* invalid argument, size or alignment */
  PMG_ERR_OOM = 2,        /* host allocation failed, or a caller buffer is too small */
  PMG_ERR_ZERO_PIVOT = 3, /* ILUT met a zero pivot during setup */
  PMG_ERR_DIVERGED = 4,   /* relative residual above 1e10 (Sec. 5) */
  PMG_ERR_MAXITER = 5,    /* max_iter V-cycles without reaching rel_tol */
  PMG_ERR_TIMEOUT = 6,    /* a bounded device-side wait expired; results invalid */
  PMG_ERR_CUDA = 7,       /* a CUDA runtime call failed */
  PMG_ERR_BUSY = 8,       /* slot call while a cycle is pending, or load into an active slot */
  PMG_ERR_STATE = 9       /* call out of order (e.g. solve before upload) */
} pmg_status;

/* Benchmarks of Sec. 2: 1 quarter annulus (Poisson), unit square (Poisson),
 * 4 unit cube (Poisson), 2 unit square with the convection-diffusion-reaction
 * coefficients D = [[1.2, -0.7], [-0.4, 0.9]], v = (0.4, -0.2), R = 0.3
 * (non-symmetric operator; the P1 levels rediscretise the same equation). */
typedef enum { PMG_QUARTER_ANNULUS = 0, PMG_UNIT_SQUARE = 1, PMG_UNIT_CUBE = 2, PMG_CDR_SQUARE = 3 } pmg_domain;

/* Manufactured solution used for the load vector and the Dirichlet data.
 * PMG_U_SINPROD: u = sin(pi x) sin(pi y) [sin(pi z)];
 * PMG_U_PAPER_B1: benchmark 1 of Sec. 2, u = -(x^2+y^2-1)(x^2+y^2-4) x y^2
 * (quarter annulus only). */
typedef enum { PMG_U_SINPROD = 0, PMG_U_PAPER_B1 = 1 } pmg_exact;

/* Residual projection (Sec. 3 and App. A): indirect p -> p-1 -> ... -> 1, or
 * direct p -> 1. */
typedef enum { PMG_PROJ_INDIRECT = 0, PMG_PROJ_DIRECT = 1 } pmg_projection;

typedef struct {
  double drop_tol;    /* ILUT tolerance tau; default 1e-12 (Sec. 3 "Smoother") */
  double fill_factor; /* ILUT fill factor m; default 1 (Sec. 3 "Smoother") */
  int nu_pre;         /* pre-smoothing steps nu_1; default 1 (Sec. 5) */
  int nu_post;        /* post-smoothing steps nu_2; default 1 (Sec. 5) */
  int projection;     /* pmg_projection; default PMG_PROJ_INDIRECT */
  int coarse_cycles;  /* h-multigrid V-cycles per coarse solve; default 2 (Sec. 3) */
  int exact;          /* pmg_exact; default PMG_U_SINPROD */
  int transfer_mass;  /* mass matrix of the L2-projection transfers (Sec. 3, App. B):
                         PMG_MASS_LUMPED (default, the paper's choice) or
                         PMG_MASS_CONSISTENT (single-vector solves only) */
} pmg_options;

/* Transfer mass matrix (Sec. 3 "Prolongation and restriction", App. B):
 * lumped (row sums, a diagonal) or consistent (solved exactly through its
 * tensor-product structure: one banded Cholesky solve per grid line and
 * direction). */
enum { PMG_MASS_LUMPED = 0, PMG_MASS_CONSISTENT = 1 };

#define PMG_MAX_LEVELS 16

typedef struct {
  int dim;                              /* 2 or 3 */
  int p, log2_inv_h;                    /* degree and h = 2^-log2_inv_h */
  int nlevels;                          /* ILUT-smoothed levels (degrees p .. 2, or p only) */
  int degree[PMG_MAX_LEVELS];           /* degree of level l (level 0 = p) */
  int n[PMG_MAX_LEVELS];                /* interior unknowns of level l */
  long long nnz_A[PMG_MAX_LEVELS];      /* non-zeros of A_l */
  long long nnz_L[PMG_MAX_LEVELS];      /* non-zeros of the strict lower ILUT factor */
  long long nnz_U[PMG_MAX_LEVELS];      /* non-zeros of the upper ILUT factor incl. diagonal */
  long long nnz_P[PMG_MAX_LEVELS];      /* non-zeros of the transfer matrix below level l */
  int depth_L[PMG_MAX_LEVELS];          /* critical path (wavefronts) of the L solve */
  int depth_U[PMG_MAX_LEVELS];          /* critical path of the U solve */
  int nhlevels;                         /* P1 h-multigrid levels incl. the coarsest */
  int n_h[PMG_MAX_LEVELS];              /* unknowns per P1 level */
  long long nnz_h[PMG_MAX_LEVELS];      /* non-zeros per P1 operator */
  int depth_gs[PMG_MAX_LEVELS];         /* critical path of a lexicographic GS sweep */
  size_t device_bytes;                  /* arena size pmg_upload needs */
  double setup_ms_assembly, setup_ms_ilut, setup_ms_transfer, setup_ms_hmg;
  double cycle_bytes;                   /* algorithmic DRAM bytes of one V-cycle */
  double cycle_flops;                   /* floating-point operations of one V-cycle */
  /* kernel variant of each solve (0 windowed line-pipelined, 1 ring, 2 lines
   * per CTA, 3 chain and producers on clusters of two CTAs a line), two bits each.
   * tune_p[l]: single-vector forward, backward; batched FP64 forward,
   * backward; batched FP32 forward, backward (2 bits each, bits 0-11); then
   * the chain configuration of the clustered kernel for the forward and the
   * backward solve (3 bits each, bits 12-14 and 15-17; 0..7: producer sums
   * enter the chain in groups of 1, 2, 4, 8 rows one line per cluster, then
   * groups of 2 / 4 rows with two lines per cluster, 2 / 4 rows with four
   * lines per cluster).  tune_h[j]: single-vector forward, backward sweep
   * (variant 2 there: the wavefront sweep over grid lines of a 2D P1 level);
   * batched forward, backward sweep (2 bits each, bits 0-7); chain
   * configuration of the forward and the backward sweep (3 bits each, bits
   * 8-10 and 11-13). */
  int tune_p[PMG_MAX_LEVELS];
  int tune_h[PMG_MAX_LEVELS];
} pmg_info_t;

typedef struct pmg_hierarchy_s* pmg_handle;
typedef struct pmg_workspace_s* pmg_ws;

/* Fills `opt` with the paper's settings (tau = 1e-12, m = 1, nu1 = nu2 = 1,
 * two coarse h-MG cycles) and indirect projection.  PMG_ERR_ARG if opt is NULL. */
pmg_status pmg_default_options(pmg_options* opt);

/* Builds the hierarchy on the host (Sec. 2 assembly with p+1 Gauss points per
 * direction, Sec. 3 ILUT factors, lumped L2-projection transfers, p = 1
 * h-multigrid levels down to h = 2^-3).  No GPU work.  domain: pmg_domain;
 * p in [2, 8]; log2_inv_h in [3, 12] (<= 6 for the cube).  opt may be NULL
 * (defaults).  *out receives a handle owned by the caller (pmg_destroy).
 * Errors: PMG_ERR_ARG, PMG_ERR_OOM, PMG_ERR_ZERO_PIVOT. */
pmg_status pmg_setup(int domain, int p, int log2_inv_h, const pmg_options* opt, pmg_handle* out);

/* Sizes, non-zeros, solve depths, setup times and per-cycle algorithmic bytes. */
pmg_status pmg_info(pmg_handle h, pmg_info_t* info);

/* Copies the hierarchy into `arena_dev` (caller-owned device memory of at least
 * info.device_bytes bytes, 256-byte aligned) on `stream`, then synchronises the
 * stream.  The arena must stay valid until pmg_destroy.  Errors: PMG_ERR_ARG
 * (size or alignment), PMG_ERR_CUDA. */
pmg_status pmg_upload(pmg_handle h, void* arena_dev, size_t bytes, void* stream);

/* Copies the assembled load vector f (interior, Dirichlet lift applied,
 * Sec. 2 Eq. los) into f_host (n[0] doubles). */
pmg_status pmg_rhs(pmg_handle h, double* f_host);

/* Device bytes a workspace for up to max_rhs simultaneous right-hand sides needs. */
pmg_status pmg_workspace_bytes(pmg_handle h, int max_rhs, size_t* bytes);

/* Creates a workspace in caller-owned device memory `mem_dev` (>= the size from
 * pmg_workspace_bytes, 256-byte aligned); initialises it on `stream`.
 * *out is owned by the caller (pmg_ws_destroy).  PMG_ERR_ARG for max_rhs > 1
 * on a hierarchy set up with PMG_MASS_CONSISTENT transfers. */
pmg_status pmg_workspace_create(pmg_handle h, int max_rhs, void* mem_dev, size_t bytes,
                                void* stream, pmg_ws* out);

/* Stand-alone p-multigrid solve (Sec. 5): u = u0, then V-cycles until
 * ||f - A u||_2 / ||f - A u0||_2 < rel_tol, at most max_iter cycles.
 * f_dev, u0_dev: inputs (n[0] doubles, device).  u_dev: output (device, may
 * alias u0_dev).  *iters: cycles done.  hist_host[i] (i < min(iters, hist_cap)):
 * relative residual after cycle i+1.  Blocks until the solve is finished.
 * Errors: PMG_ERR_DIVERGED, PMG_ERR_MAXITER (iters and history still written),
 * PMG_ERR_TIMEOUT, PMG_ERR_CUDA, PMG_ERR_STATE. */
pmg_status pmg_solve(pmg_handle h, pmg_ws ws, const double* f_dev, const double* u0_dev,
                     double rel_tol, int max_iter, double* u_dev, int* iters,
                     double* hist_host, int hist_cap, void* stream);

/* As pmg_solve with host buffers: copies f_host and u0_host to the workspace,
 * solves, copies the solution back to u_host (all on `stream`). */
pmg_status pmg_solve_host(pmg_handle h, pmg_ws ws, const double* f_host, const double* u0_host,
                          double rel_tol, int max_iter, double* u_host, int* iters,
                          double* hist_host, int hist_cap, void* stream);

/* BiCGSTAB (van der Vorst 1992) with the p-multigrid V-cycle as right
 * preconditioner: each preconditioner application is one V-cycle with zero
 * initial guess, two per iteration (Sec. 5, "p-Multigrid as a
 * preconditioner", Table 5).  Arguments, buffers and ownership as pmg_solve;
 * the stopping test (relative residual < rel_tol) uses the recursively updated
 * residual after the half step and after the full step, and an exit at the
 * half step counts the iteration in progress; res_hist_host gets one relative
 * residual per iteration.  Errors: as pmg_solve; a breakdown (r-hat . r = 0)
 * returns PMG_ERR_DIVERGED. */
pmg_status pmg_solve_bicgstab(pmg_handle h, pmg_ws ws, const double* f_dev, const double* u0_dev, double rel_tol,
                              int max_iter, double* u_dev, int* iters, double* res_hist_host, int hist_cap,
                              void* stream);

/* Precision of the batched solve's inner V-cycle: FP64; FP32 arithmetic with
 * FP32 factors; FP32 arithmetic with the ILUT factors' values stored as FP16
 * or as BF16 (widened to FP32 on load). */
enum { PMG_PREC_FP64 = 0, PMG_PREC_MIXED = 1, PMG_PREC_MIXED_FP16 = 2, PMG_PREC_MIXED_BF16 = 3 };

/* Batched stand-alone solves of nrhs right-hand sides with one hierarchy.
 * Each right-hand side follows the iteration u <- u + C(f - A u) of Sec. 5, C
 * being one V-cycle with zero initial guess (the same affine map as the
 * V-cycle of pmg_solve), until its own relative residual is below rel_tol (it
 * is then frozen) or it diverges (> 1e10).  precision: PMG_PREC_FP64 runs the
 * whole cycle in FP64; PMG_PREC_MIXED runs the residual-to-correction cycle on
 * levels q >= 2 in FP32 (SpMV, triangular solves, transfers) inside the FP64
 * defect-correction loop; the outer residual, the update of u and the p = 1
 * coarse correction stay FP64.  F_dev, U0_dev, U_dev: nrhs x n[0] doubles,
 * right-hand side k contiguous at offset k*n[0] (device).  The workspace must
 * have been created with max_rhs >= max(nrhs, 2) (batched buffers); the solve
 * runs on the workspace's continuous-batching slots (pmg_slots_*), releasing
 * all of them before and after, so slot work in progress on it is cancelled.
 * iters_host[k]: cycles of right-hand side k; hist_host (may be NULL):
 * max_iter x nrhs relative residuals, row = cycle.  On a non-default stream
 * with profiling off, the cycles after the first are replayed as one CUDA
 * graph.  Blocks until done.  Errors: PMG_ERR_ARG,
 * PMG_ERR_MAXITER / PMG_ERR_DIVERGED (results still written), PMG_ERR_TIMEOUT,
 * PMG_ERR_CUDA. */
pmg_status pmg_solve_batched(pmg_handle h, pmg_ws ws, int nrhs, const double* F_dev, const double* U0_dev,
                             double rel_tol, int max_iter, int precision, double* U_dev, int* iters_host,
                             double* hist_host, void* stream);

/* Continuous batching (the paper has no counterpart).  The max_rhs slots of a
 * workspace (created with max_rhs >= 2) are filled, iterated and drained
 * independently, so right-hand sides can join and leave a running batch
 * between V-cycles.  Every slot follows exactly the iteration of
 * pmg_solve_batched; its result depends neither on the other slots nor on
 * when it was loaded.  All slot calls of one workspace go to one stream and
 * do not block, except pmg_slots_wait.
 *
 * pmg_slots_load: copies n right-hand sides and initial guesses (device,
 *   right-hand side k contiguous at offset k*n[0]) into slots slot0..slot0+n-1
 *   (none of them active), computes their initial residual norms and makes
 *   them active (a slot with a zero initial residual is reported converged
 *   with 0 cycles after the next cycle's wait).
 * pmg_slots_cycle: one V-cycle (precision as in pmg_solve_batched; replayed
 *   as a CUDA graph on a non-default stream) for every active slot, then each
 *   one's stopping test
 *   (relative residual < rel_tol: converged; > 1e10: diverged).  A no-op when
 *   no slot is active.
 * pmg_slots_wait: when the last cycle has finished (at once if
 *   blocking), sets *ready = 1 and copies per slot (arrays of max_rhs entries,
 *   each may be NULL) the last relative residual, the state (0 free, 1 active,
 *   2 converged, 3 diverged) and the cycles done; otherwise *ready = 0.
 * pmg_slots_read: copies the current solutions of n slots out (device,
 *   stream-ordered).
 * pmg_slots_release: frees n slots (an active slot is cancelled).
 * Errors: PMG_ERR_ARG, PMG_ERR_BUSY (load / cycle / release while a cycle
 * has not been waited for, or load into an active slot),
 * PMG_ERR_TIMEOUT (reported by pmg_slots_wait), PMG_ERR_CUDA. */
pmg_status pmg_slots_load(pmg_handle h, pmg_ws ws, int slot0, int n, const double* F_dev, const double* U0_dev,
                          void* stream);
pmg_status pmg_slots_cycle(pmg_handle h, pmg_ws ws, int precision, double rel_tol, void* stream);
pmg_status pmg_slots_wait(pmg_handle h, pmg_ws ws, int blocking, int* ready, double* relres_host, int* state_host,
                          int* iters_host);
pmg_status pmg_slots_read(pmg_handle h, pmg_ws ws, int slot0, int n, double* U_dev, void* stream);
pmg_status pmg_slots_release(pmg_handle h, pmg_ws ws, int slot0, int n, void* stream);

/* Kernel autotuner (the paper has no counterpart): times every available
 * kernel variant of each triangular solve and Gauss-Seidel sweep of the
 * hierarchy on the current device, single-vector and (if the workspace holds
 * several right-hand sides) batched in both precisions, with the workspace's
 * buffers as scratch, and keeps the fastest for later solves on this handle.
 * The variants compute the same operation with a different order of
 * floating-point summation.  Blocks until done.  Not to be called while
 * another solve uses the handle.  Errors: PMG_ERR_ARG, PMG_ERR_STATE,
 * PMG_ERR_TIMEOUT, PMG_ERR_CUDA. */
pmg_status pmg_autotune(pmg_handle h, pmg_ws ws, void* stream);

/* Sets the kernel variant of every solve by hand, in the packing of
 * pmg_info_t.tune_p / tune_h (arrays of nlevels / nhlevels ints): single-vector
 * solves take 0, 1 or 3, single-vector sweeps 0..3, batched ones 1 or 2;
 * chain configurations 0..7.  The hierarchy must be uploaded.  Errors: PMG_ERR_ARG (a variant out of
 * range; nothing changed), PMG_ERR_STATE. */
pmg_status pmg_set_kernels(pmg_handle h, const int* tune_p, const int* tune_h);

/* Single steps of the cycle, for checking each one on its own.  `level` is a
 * p-level index (0 = degree p) for the first group and a P1 level index
 * (0 = h) for the second.  x, b: inputs; y: output (device).  Sizes follow
 * the level (coarse side = next level down).
 *   PMG_OP_RESIDUAL     y = b - A_l x                     (Eq. smooth, Eq. res)
 *   PMG_OP_SMOOTH       y = x + U^{-1} L^{-1} (b - A_l x) (Eq. inverse)
 *   PMG_OP_LSOLVE       y = L^{-1} b   (unit lower factor)
 *   PMG_OP_USOLVE       y = U^{-1} b
 *   PMG_OP_RESTRICT     y = (M^L_c)^{-1} P^T x  (coarse side)   (Eq. restriction)
 *   PMG_OP_PROLONG_ADD  y = b + (M^L_l)^{-1} P x (x coarse)     (Eq. prolongation)
 *   PMG_OP_COARSE_SOLVE y = coarse_cycles h-MG V-cycles on A_{h,1} y = b from 0
 *   PMG_OP_VCYCLE       y = one V-cycle at level l applied to (x, b)
 *   PMG_OP_GS_FWD       y = one forward lexicographic Gauss-Seidel sweep (P1 level)
 *   PMG_OP_GS_BWD       y = one backward sweep
 *   PMG_OP_HMG_VCYCLE   y = one h-MG V-cycle at P1 level `level` applied to (x, b) */
enum {
  PMG_OP_RESIDUAL = 0, PMG_OP_SMOOTH = 1, PMG_OP_LSOLVE = 2, PMG_OP_USOLVE = 3,
  PMG_OP_RESTRICT = 4, PMG_OP_PROLONG_ADD = 5, PMG_OP_COARSE_SOLVE = 6, PMG_OP_VCYCLE = 7,
  PMG_OP_GS_FWD = 8, PMG_OP_GS_BWD = 9, PMG_OP_HMG_VCYCLE = 10
};
pmg_status pmg_apply(pmg_handle h, pmg_ws ws, int op, int level, const double* x_dev,
                     const double* b_dev, double* y_dev, void* stream);

/* Host copy of a setup matrix in CSR (for checks).  which: 0 A_l, 1 L_l, 2 U_l
 * (with diagonal), 3 unscaled P between level l and the next coarser level
 * (rows: level l), 4 A of P1 level l.  Call with rp == NULL to get sizes. */
pmg_status pmg_export_csr(pmg_handle h, int which, int level, int* nrows, int* ncols,
                          long long* nnz, int* rp, int* ci, double* v);

/* Lumped mass (interior) of p-level l, or of V_{h,1} when l == nlevels. */
pmg_status pmg_export_lumped(pmg_handle h, int level, double* out_host);

/* L2 error against the manufactured solution of the degree-p solution given by
 * its interior coefficients (host), boundary values from the Dirichlet lift. */
pmg_status pmg_l2_error(pmg_handle h, const double* u_host, double* err);

/* Kernel classes for the per-workspace launch statistics. */
enum {
  PMG_K_RESIDUAL = 0,     /* r = f - A u on a p-level */
  PMG_K_TRANSFER = 1,     /* restriction / prolongation SpMV between p-levels */
  PMG_K_LSOLVE = 2,       /* forward substitution with the ILUT factor L */
  PMG_K_USOLVE = 3,       /* backward substitution with U (and u += e) */
  PMG_K_GS = 4,           /* Gauss-Seidel sweep on a P1 level */
  PMG_K_P1 = 5,           /* P1 residual and canonical transfers */
  PMG_K_COARSE = 6,       /* dense coarsest solve */
  PMG_K_NORM = 7,         /* residual norm and stopping test */
  PMG_NKERN = 8
};

typedef struct {
  double ms[PMG_NKERN];          /* summed CUDA-event time per class (profiling on) */
  long long launches[PMG_NKERN]; /* launches per class (profiling on) */
  double bytes[PMG_NKERN];       /* summed algorithmic DRAM bytes per class (profiling on) */
  long long total_launches;      /* all kernel launches issued through this workspace */
  long long graph_launches;      /* V-cycles replayed as one CUDA graph (counted in total_launches by their kernels) */
} pmg_stats_t;

/* Turns per-launch CUDA-event timing on (enable != 0) or off for `ws`.  Events
 * are recorded on the launch stream around every kernel; their times are
 * collected when the call that issued them synchronises. */
pmg_status pmg_ws_profile(pmg_ws ws, int enable);

/* Copies the statistics of `ws` into *out; clears them if reset != 0. */
pmg_status pmg_ws_stats(pmg_ws ws, pmg_stats_t* out, int reset);

/* Allocation-free forward substitution y = L^{-1} b for a strict lower CSR
 * matrix L with implied unit diagonal (the ILUT factor layout of
 * pmg_export_csr, which = 1).  The paper has no counterpart: this entry point
 * exists for callers that cannot allocate device memory -- code confined to a
 * memory pool or arena sized up front, plug-ins whose host application owns
 * all device allocations, or loops that must not allocate once running.  It
 * calls no cudaMalloc, cudaFree or allocating library routine: the kernel's
 * scratch (per-row ready flags, row counter, error word) lives in one fixed
 * device array of this library, present on every GPU that loads it until the
 * process exits, which limits n to 1,048,576 rows (4 MiB of scratch).
 *   n: rows; rp_dev (n+1), ci_dev, v_dev: CSR arrays of L on the device, columns
 *   ascending, all < their row (a column outside [0, row) is not checked and
 *   gives undefined results); ci_dev and v_dev must be non-null even when L
 *   has no entries; b_dev: right-hand side; y_dev: output (may not alias
 *   b_dev).  All device memory is owned by the caller.
 * The first call on a device looks up the array's device address (with that
 * device current); make that first call before any stream capture.  Every call
 * shares the one array and clears the part it uses; calls whose work overlaps
 * on the GPU (other streams, other host threads) race on it and must be
 * serialised by the caller.  Blocks until the solve on `stream` is finished.
 * Errors: PMG_ERR_ARG (n above the limit, or null pointers), PMG_ERR_TIMEOUT,
 * PMG_ERR_CUDA. */
pmg_status pmg_lsolve_noalloc(int n, const int* rp_dev, const int* ci_dev, const double* v_dev,
                              const double* b_dev, double* y_dev, void* stream);

pmg_status pmg_ws_destroy(pmg_ws ws);
pmg_status pmg_destroy(pmg_handle h);

/* Message of the last failed call on this thread ("" if none). */
const char* pmg_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* PMG_H_ */
