/*
 * r3mg.h — C ABI of the B300 (sm_103a) R-tree algebraic-geometric multilevel
 * preconditioned conjugate-gradient solver.
 *
 * Method: R3MG-C ("a high-order algebraic-geometric multilevel preconditioner
 * for continuous finite element discretizations").  Support points are
 * partitioned by an R-tree into axis-aligned boxes (Section 3; Section 4,
 * point-based agglomeration); on each box the tensor space Q^{p'} is
 * interpolated at the points the box owns, giving a sparse prolongation P
 * (Section 4; Section 5, eq. (localinterpolation)); the level operators are
 * inherited, A_{l+1} = P^T A_l P (Section 1, Section 4); one V-cycle with a
 * Chebyshev-Jacobi smoother (Section 5, Remark on the smoother; Section 6)
 * preconditions CG (Section 4, Section 6).  The coarsest level is solved by
 * a dense Cholesky factorisation (the paper uses a sparse direct solver).
 *
 * Conventions for every entry point
 *   - Status codes only; nothing throws or exits across this boundary.  On
 *     failure r3mg_last_error() describes the cause.
 *   - "host" pointers are ordinary CPU memory; "device" pointers are CUDA
 *     global memory on the current device.  Inputs are borrowed for the call
 *     only (copied or reformatted); outputs go to caller buffers.
 *   - Vectors use the caller's numbering of the free DoFs; the tree order
 *     used internally is never exposed except by r3mg_partition.
 *   - All device work is enqueued on `stream` (a cudaStream_t, NULL = legacy
 *     default stream).  Calls that return host values synchronise it.
 *   - A hierarchy owns all its device memory until r3mg_destroy.  A
 *     hierarchy is not thread-safe: calls on one hierarchy must not overlap.
 */
#ifndef R3MG_H
#define R3MG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct r3mg_hierarchy r3mg_hierarchy;

typedef enum {
  R3MG_OK = 0,
  R3MG_E_ARG = 1,          /* invalid argument, malformed CSR, non-finite input */
  R3MG_E_CUDA = 2,         /* a CUDA runtime call failed */
  R3MG_E_OOM = 3,          /* device or host allocation failed */
  R3MG_E_DEPTH = 4,        /* bisection tree too shallow for the requested levels */
  R3MG_E_UNISOLVENT = 5,   /* a box's points cannot carry Q^{p'} (Section 4, Remark on (m, M)) */
  R3MG_E_NOT_SPD = 6,      /* non-positive diagonal or Cholesky pivot */
  R3MG_E_NOCONV = 7,       /* PCG reached maxit */
  R3MG_E_BREAKDOWN = 8,    /* p^T A p <= 0 or non-finite CG scalar */
  R3MG_E_LIMIT = 9,        /* an internal size limit was exceeded (e.g. window > 65535 points) */
  R3MG_E_TIMEOUT = 10      /* a bounded device wait expired */
} r3mg_status;

typedef struct {
  int leaf_size;        /* maximum fine points per level-1 box; must be >= (pprime+1)^dim */
  int pprime;           /* coarse polynomial degree p' >= 0 (0 = Nicolaides space, Section 1) */
  int levels;           /* L >= 2 levels counting the fine level (the paper's "lvls") */
  int cheb_degree;      /* Chebyshev degree k >= 1 (Section 6: 3) */
  int sweeps;           /* pre- and post-smoothing sweeps (Section 6: 2) */
  int lanczos_steps;    /* Lanczos steps for lambda_max(D^-1 A_l) (Section 6) */
  double eig_safety;    /* upper interval end = eig_safety * Ritz estimate (1.1) */
  double eig_ratio;     /* lower interval end = upper / eig_ratio (30) */
  int precision;        /* 0: FP64 V-cycle inside FP64 PCG; 1: FP32 V-cycle inside FP64 flexible CG */
  int group_lanes;      /* lanes per matrix row in the level kernels (4, 8, 16, 32); 0 = automatic */
  uint64_t seed;        /* splitmix64 seed of the Lanczos start vectors (level l uses seed + l) */
  int kernel_form;      /* level operator kernel: 0 = autotuned at setup (each level times the
                           register- and TMA-streamed kernels over lanes-per-row and CTA sizes
                           and keeps the fastest), 1 = register-streamed, 2 = TMA-streamed
                           where a box fits the shared memory */
} r3mg_params;

/* Fill `p` with the defaults: leaf 64, p' 1, 3 levels, degree 3, 2 sweeps,
 * 10 Lanczos steps, 1.1, 30, FP64, automatic lanes, seed 0x5EED, automatic kernel form. */
void r3mg_default_params(r3mg_params* p);

/*
 * Host-only R-tree bisection of n points (Section 3, Definition of the
 * R-tree; Section 4, point-based agglomeration), read as a balanced,
 * bulk-loaded bisection tree: depth D = smallest t with ceil(n/2^t) <=
 * leaf_size; every node is split at ceil(|S|/2) after ordering its points by
 * (x_a, x_{a+1}, ..., original index), a = axis of the longest MBR extent
 * (ties to the smaller axis).  Needs no GPU.
 *   coords_host: n*dim doubles, row-major (point i at coords[i*dim .. i*dim+dim-1]).
 *   perm_out (host, n): perm_out[k] = caller index of the k-th point in tree order.
 *   leaf_offsets_out (host, 2^D + 1 entries, may be NULL): start of each leaf in tree order.
 *   depth_out (may be NULL): D.
 * Errors: R3MG_E_ARG (n < 1, dim not 2/3, leaf < 2, non-finite coordinate),
 *         R3MG_E_DEPTH (D - dim*(levels-2) < 0).
 */
r3mg_status r3mg_partition(int64_t n, int dim, const double* coords_host, int leaf_size, int levels,
                           int64_t* perm_out, int64_t* leaf_offsets_out, int* depth_out);

/*
 * The row groups of the block kernels' grouped fine level (block form 20; rows whose stored
 * column lists are equal share each gathered slice of the right-hand sides), computed on the
 * host from a windowed per-row layout.  Needs no GPU.  Within each box, rows with equal index
 * lists form runs; a run, in increasing row order, is cut into groups of 8 rows, then 4, 2 and 1.
 *   row_ptr (n+1, host): row r's window indices are idx[row_ptr[r] .. row_ptr[r+1]), row_ptr[0] = 0.
 *   box_row (nbox+1, host): box B holds rows box_row[B] .. box_row[B+1]-1 (0 to n, non-decreasing).
 *   idx (host, row_ptr[n] entries; may be NULL when that is 0): 16-bit window indices.
 *   counts_out (4): the number of groups of 8, 4, 2 and 1 rows.
 *   rows_out (n, int32): every row once, the groups of 8 first, then of 4, 2 and 1; within a
 *     size, boxes in order; within a group, increasing rows.
 * Errors: R3MG_E_ARG (null pointer, n < 0 or >= 2^31, nbox < 1, bad offsets), R3MG_E_OOM.
 */
r3mg_status r3mg_group_rows(int64_t n, const int64_t* row_ptr, int64_t nbox, const int64_t* box_row,
                            const uint16_t* idx, int64_t* counts_out, int32_t* rows_out);

/*
 * Build the hierarchy for the free-DoF system A (CSR, host memory) whose
 * support points are coords_host (n x dim, host).  Performs the partition
 * and the symbolic analysis on the host, then on the device: the P values
 * (box Q^{p'} basis at owned points, Section 4), the Galerkin products
 * A_{l+1} = P^T A_l P (Sections 1, 4), Lanczos estimates of
 * lambda_max(D_l^{-1} A_l) (Section 6) and the coarsest Cholesky factor.
 *   rowptr_host (n+1, int64), colidx_host (nnz, int32, 0-based), vals_host (nnz):
 *     a symmetric matrix with a positive diagonal stored in every row;
 *     column order inside a row is free.
 *   params: see r3mg_params; NULL = defaults.
 *   out: receives the hierarchy (NULL on failure).
 * Errors: R3MG_E_ARG, R3MG_E_DEPTH, R3MG_E_UNISOLVENT, R3MG_E_NOT_SPD,
 *         R3MG_E_LIMIT, R3MG_E_OOM, R3MG_E_CUDA.  The stream is synchronised.
 */
r3mg_status r3mg_setup(int64_t n, int dim, const double* coords_host, const int64_t* rowptr_host,
                       const int32_t* colidx_host, const double* vals_host, const r3mg_params* params,
                       void* stream, r3mg_hierarchy** out);

/*
 * Host-only cell-based agglomeration (Section 4): the bisection rule of r3mg_partition applied
 * to cells (node MBR = union of the cells' MBRs; split key = the cell's MBR centre
 * (m_a, m_{a+1}, ..., cell index); leaf_size counts cells, >= 2), then the level-1 agglomerates,
 * visited in order, each take every support point of their cells that no earlier one took
 * (the paper's three-step ownership procedure).  A point's level-l box is the level-l ancestor
 * of its level-1 owner; a box's MBR is the union of its cells' MBRs.  Needs no GPU.
 *   cell_ptr_host (ncells+1, int64), cell_pts_host (cell_ptr[ncells], int64): the support
 *     points of every cell in the caller's numbering; an entry < 0 is a point not in the
 *     system (an eliminated Dirichlet node).  A cell's MBR is taken over its points in the
 *     system; cells without any take no part.
 *   perm_out (n): caller index of the k-th point in tree order (by owner, then caller index).
 *   box_offsets_out (2^D + 1, may be NULL): start of each level-1 box in tree order.
 *   box_lo_out, box_hi_out (2^D * dim each, may be NULL): level-1 box MBRs.
 * Errors: R3MG_E_ARG (bad sizes, an index >= n, a point in no cell, no valid cell),
 *         R3MG_E_DEPTH.
 */
r3mg_status r3mg_partition_cells(int64_t n, int dim, const double* coords_host, int64_t ncells,
                                 const int64_t* cell_ptr_host, const int64_t* cell_pts_host, int leaf_size, int levels,
                                 int64_t* perm_out, int64_t* box_offsets_out, double* box_lo_out, double* box_hi_out,
                                 int* depth_out);

/* As r3mg_setup with cell-based agglomeration (r3mg_partition_cells) in place of the point
 * bisection; leaf_size counts cells.  Everything after the partition (P on the agglomerates'
 * boxes, Galerkin levels, smoother, solves) is the same.  Additional error: R3MG_E_UNISOLVENT
 * when a late agglomerate is left with fewer than (p'+1)^d points. */
r3mg_status r3mg_setup_cells(int64_t n, int dim, const double* coords_host, const int64_t* rowptr_host,
                             const int32_t* colidx_host, const double* vals_host, int64_t ncells,
                             const int64_t* cell_ptr_host, const int64_t* cell_pts_host, const r3mg_params* params,
                             void* stream, r3mg_hierarchy** out);

/*
 * Batched setup: nprob independent problems (uneven sizes allowed), each with its own R-tree
 * partition, transfers, Galerkin levels, smoother intervals and coarsest factor, stored as one
 * block-diagonal hierarchy so that every V-cycle step of all problems is one kernel launch.
 * The paper solves one problem at a time; batching is a serving extension of the same method.
 *   n[k], coords_host[k], rowptr_host[k], colidx_host[k], vals_host[k]: problem k, as in
 *   r3mg_setup (host memory; each problem in its own 0-based numbering).
 * Vectors of batched calls are the problems' vectors concatenated in order (problem 0 first).
 * All problems share params (dim, p', leaf size, levels ...).  The TMA kernel form is not used.
 * Errors: as r3mg_setup; the message names the failing problem.
 */
r3mg_status r3mg_batch_setup(int nprob, int dim, const int64_t* n, const double* const* coords_host,
                             const int64_t* const* rowptr_host, const int32_t* const* colidx_host,
                             const double* const* vals_host, const r3mg_params* params, void* stream,
                             r3mg_hierarchy** out);

/*
 * Solve every problem of a batched hierarchy: PCG with the FP64 V-cycle, flexible CG with the FP32
 * V-cycle, per-problem scalars and stop tests (||r_k|| <= rtol ||b_k||).  After a host-launched
 * start, the iteration loop of all problems runs as ONE CUDA graph launch whose conditional
 * WHILE node repeats a batched iteration until every problem has stopped.
 *   b_dev, x_dev: device, concatenated (sum of n) doubles; x in = x0, out = solution.
 *   iters_out, relres_out (host, nprob): per-problem iterations and true relative residuals.
 * Errors: R3MG_E_NOCONV (some problem reached maxit), R3MG_E_BREAKDOWN, R3MG_E_CUDA.
 */
r3mg_status r3mg_batch_pcg(r3mg_hierarchy* h, const double* b_dev, double* x_dev, double rtol, int maxit,
                           int* iters_out, double* relres_out, void* stream);

/* Number of problems and their row offsets on level l (row_off_host: nprob + 1 entries). */
r3mg_status r3mg_batch_offsets(const r3mg_hierarchy* h, int level, int* nprob_out, int64_t* row_off_host);

/*
 * Replace the matrix values (same pattern as at setup, CSR order, device
 * memory, nnz doubles) and redo every numeric setup step: P is unchanged,
 * the Galerkin levels, smoother intervals and coarsest factor are rebuilt.
 * Errors: R3MG_E_NOT_SPD, R3MG_E_CUDA.  The stream is synchronised.
 */
r3mg_status r3mg_update_values(r3mg_hierarchy* h, const double* vals_dev, void* stream);

/*
 * z = M^{-1} r: one V-cycle (Section 4) applied to r (device, n doubles,
 * caller numbering); z (device, n doubles) may not alias r.  Uses the
 * precision chosen at setup (an FP32 V-cycle converts r to FP32 and z back).
 * Asynchronous: no host synchronisation.
 */
r3mg_status r3mg_vcycle(r3mg_hierarchy* h, const double* r_dev, double* z_dev, void* stream);

/*
 * Solve A x = b with CG preconditioned by one V-cycle per iteration
 * (Section 4, Section 6).  FP64 V-cycle: Hestenes-Stiefel PCG.  FP32 V-cycle:
 * flexible CG (Notay) with FP64 vectors, dot products and scalars.
 * Stops when ||b - A x||_2 <= rtol ||b||_2 (the recursive residual, confirmed
 * by an FP64 recomputation of the true residual before returning success).
 *   b_dev (device, n), x_dev (device, n): in = initial guess, out = solution.
 *   iters_out: completed updates of x; relres_out: final ||r||/||b||.
 * Errors: R3MG_E_NOCONV (maxit reached; x holds the last iterate),
 *         R3MG_E_BREAKDOWN, R3MG_E_CUDA, R3MG_E_ARG (batched hierarchy: use r3mg_batch_pcg).
 *         Synchronises the stream.
 */
r3mg_status r3mg_pcg(r3mg_hierarchy* h, const double* b_dev, double* x_dev, double rtol, int maxit,
                     int* iters_out, double* relres_out, void* stream);

/* As r3mg_pcg with b_host / x_host in host memory: the host->device copy of b
 * and x0 and the device->host copy of x happen inside the call. */
r3mg_status r3mg_pcg_host(r3mg_hierarchy* h, const double* b_host, double* x_host, double rtol, int maxit,
                          int* iters_out, double* relres_out, void* stream);

/*
 * Several right-hand sides at once (Section 6's PCG, run per column): m <= 16 systems
 * A x_c = b_c on one hierarchy, every level operator reading the matrix once for all columns
 * (block vectors of M = 4, 8 or 16 columns, row-interleaved inside the library; unused columns
 * are zero).  Each column has its own CG scalars and stopping test ||b_c - A x_c|| <=
 * rtol ||b_c|| (confirmed by an FP64 true residual); converged columns stop updating while the
 * others continue.  Precision as in r3mg_pcg (FP64 PCG, or FP32 V-cycle inside FP64 FCG).
 *   b_dev, x_dev (device): m vectors of n doubles each, vector c at offset c*n, caller numbering;
 *   x_dev in = initial guesses, out = solutions.
 *   iters_out[m]: completed updates of each column; relres_out[m]: final ||r_c|| / ||b_c||.
 * Errors: R3MG_E_ARG (m outside 1..16, null pointer, batched hierarchy), R3MG_E_NOCONV (some
 * column reached maxit; x holds the last iterates), R3MG_E_BREAKDOWN, R3MG_E_CUDA, R3MG_E_OOM.
 * Synchronises the stream.  The library allocates the block vectors at the first call (and
 * again when the column count class changes) and keeps them until r3mg_destroy.
 */
r3mg_status r3mg_pcg_multi(r3mg_hierarchy* h, int m, const double* b_dev, double* x_dev, double rtol, int maxit,
                           int* iters_out, double* relres_out, void* stream);

/* One V-cycle (Section 4) on m <= 16 vectors at once: z_c = M^{-1} r_c, in the hierarchy's
 * V-cycle precision.  r_dev, z_dev: m x n doubles (vector c at offset c*n), caller numbering.
 * Asynchronous on the stream. */
r3mg_status r3mg_vcycle_multi(r3mg_hierarchy* h, int m, const double* r_dev, double* z_dev, void* stream);

/* y_c = A_l x_c for m <= 16 vectors with the block kernel: fp32 = 0 uses the FP64 values,
 * fp32 = 1 the FP32 V-cycle values (hierarchies built with precision 1, levels below the
 * coarsest only, else R3MG_E_ARG; inputs are rounded to FP32, outputs widened).  x_dev, y_dev: m x n_l doubles, vector c at offset c*n_l,
 * level numbering as in r3mg_level_apply.  Asynchronous. */
r3mg_status r3mg_level_apply_multi(r3mg_hierarchy* h, int level, int m, int fp32, const double* x_dev, double* y_dev,
                                   void* stream);

/* Block-kernel configuration of level l (fp32 = 0: FP64 blocks, 1: FP32 V-cycle blocks), tuned
 * by timing at the first block call: slots = 2, 4 or 8 entry slots per row (window gathered
 * through L1), 0 = coarse-level kernel with the box window staged in shared memory, 1 = coarse-
 * level kernel with the window staged and the block rows streamed into shared memory by the
 * copy engine (cp.async.bulk, bounded mbarrier waits: R3MG_E_TIMEOUT if one expires), 3 =
 * coarse-level FP32 kernel on the tensor cores through mma.sync (8 or 16 columns; TF32
 * head/tail splitting keeps FP32 accuracy), 5 = coarse-level FP32 kernel on the 5th-generation
 * tensor cores (tcgen05.mma into a TMEM accumulator, operands staged in shared memory; 16
 * columns, boxes of at most 32 rows, the same TF32 head/tail splitting; its mbarrier waits are
 * bounded as set by r3mg_set_wait_limit and an expiry gives R3MG_E_TIMEOUT), 6 = the same
 * product warp-specialised with the A operand in TMEM (tcgen05.st) and both operands fed by
 * cp.async.bulk six chunks ahead (one CTA per SM; same limits and wait bounds as 5), 10 +
 * slots (12, 14, 18) = fine-level flat row sweep on global column indices (built once, 4 bytes
 * per stored entry), 20 = fine level in groups of rows with equal column lists (Q_p: the DoFs
 * interior to one cell, face or edge; groups of 8, 4, 2 and 1 rows of one box, the column list
 * stored once and the values entry-major, so one gathered slice of X serves the whole group;
 * built once on first use, its values gathered again after r3mg_update_values), -1 = not tuned
 * yet.  The setter pins one choice (R3MG_E_ARG for an invalid or untuned combination). */
r3mg_status r3mg_block_config(r3mg_hierarchy* h, int level, int fp32, int* slots);
r3mg_status r3mg_set_block_config(r3mg_hierarchy* h, int level, int fp32, int slots);

/*
 * y = A_l x on level l, FP64, in level numbering (level 0: caller numbering
 * of the free DoFs; level l >= 1: coarse DoF box*b + q, boxes numbered left
 * to right in the tree).  x_dev, y_dev: device, n_l doubles.  Asynchronous.
 */
r3mg_status r3mg_level_apply(r3mg_hierarchy* h, int level, const double* x_dev, double* y_dev, void* stream);

/*
 * The coarsest-level solve of the V-cycle on its own: z = A_{L-1}^{-1} r with the explicit
 * inverse formed at setup from the dense Cholesky factor (the paper's coarse direct solve,
 * Section 6, read as a dense Cholesky), FP64.  r_dev, z_dev: device, n_{L-1} doubles in
 * coarsest-level numbering (box * b + q); no aliasing.  Asynchronous.
 * Errors: R3MG_E_ARG (null pointer, batched hierarchy), R3MG_E_CUDA.
 */
r3mg_status r3mg_coarse_solve(r3mg_hierarchy* h, const double* r_dev, double* z_dev, void* stream);

/*
 * One level-operator product in a chosen precision: y = A_l x with the level kernel chosen for
 * that precision (the kernel the V-cycle runs).  fp32 = 0 is r3mg_level_apply (FP64 values);
 * fp32 = 1 uses the FP32 values of the FP32 V-cycle (Section 4's level operators stored in
 * single precision): x is rounded to FP32 (round to nearest), the row sums run in FP32 with FP32
 * accumulation, y is widened to FP64 exactly.  x_dev, y_dev: device, n_l doubles, level
 * numbering as in r3mg_level_apply.  The level's V-cycle vectors serve as scratch, so this call
 * must not overlap a V-cycle or solve on the same hierarchy.  Asynchronous.
 * Errors: R3MG_E_ARG (fp32 = 1 on an FP64 hierarchy or on the coarsest level), R3MG_E_CUDA.
 */
r3mg_status r3mg_level_apply_prec(r3mg_hierarchy* h, int level, int fp32, const double* x_dev, double* y_dev,
                                  void* stream);

/*
 * One fused Chebyshev-Jacobi step of the smoother (Section 5, Remark on the smoother; Section 6;
 * Saad's Algorithm 12.1 with the Jacobi preconditioner D_l^{-1}) on a smoothed level l < L-1, in
 * the hierarchy's V-cycle precision and with the kernel the V-cycle uses:
 *   x' = x + d;   r' = r - A_l d;   d' = a d + c D_l^{-1} r'.
 * x_dev, r_dev, d_dev (device, n_l doubles, level numbering; level 0 = caller numbering) are
 * read, rounded to the V-cycle precision; x_out, r_out, d_out (device, n_l doubles) receive the
 * results widened to FP64; a and c are rounded to the V-cycle precision.  Outputs may alias
 * inputs.  Uses the level's V-cycle vectors as scratch (no overlap with a V-cycle or solve on
 * the same hierarchy).  Asynchronous.  Errors: R3MG_E_ARG (coarsest level, batched hierarchy).
 */
r3mg_status r3mg_level_cheb_step(r3mg_hierarchy* h, int level, const double* x_dev, const double* r_dev,
                                 const double* d_dev, double a, double c, double* x_out, double* r_out,
                                 double* d_out, void* stream);

/* The coarsest solve of r3mg_coarse_solve in a chosen precision: fp32 = 1 applies the FP32
 * copy of the explicit inverse that the FP32 V-cycle uses (r rounded to FP32, FP32 GEMV with
 * FP32 accumulation, z widened), fp32 = 0 is r3mg_coarse_solve.  Errors: R3MG_E_ARG (fp32 = 1
 * on an FP64 or batched hierarchy).  Asynchronous. */
r3mg_status r3mg_coarse_solve_prec(r3mg_hierarchy* h, int fp32, const double* r_dev, double* z_dev, void* stream);

/*
 * Stop test of r3mg_pcg, r3mg_pcg_host and r3mg_pcg_multi (per column):
 *     ||r_k||_2 <= max(rtol ||b||_2, atol, reduction ||r_0||_2),   r_0 = b - A x_0,
 * confirmed on the FP64 true residual.  The defaults atol = reduction = 0 leave the relative
 * test; rtol = 0 with atol = 1e-9 and reduction = 1e-6 is the paper's rule (Section 6: stop when
 * the absolute residual norm falls below 1e-9 or the residual has dropped by six orders).
 * Kept on the hierarchy until changed.  Batched solves keep the relative test.
 * Errors: R3MG_E_ARG (negative or non-finite value).
 */
r3mg_status r3mg_set_stop_rule(r3mg_hierarchy* h, double atol, double reduction);

/*
 * Condition-number estimate of the last solve (the "Cond." column of the paper's tables,
 * Section 6: the condition number estimated by PCG).  The solve keeps its CG coefficients
 * alpha_j, beta_j on the device (the first 1024 of each; a restart from the true residual
 * begins a new sequence); this call builds the Lanczos tridiagonal T (T_jj = 1/alpha_j +
 * beta_{j-1}/alpha_{j-1}, T_{j,j+1} = sqrt(beta_j)/alpha_j) on the host and returns its extreme
 * eigenvalues (Sturm bisection), estimates of those of M^{-1} A.  For flexible CG (FP32
 * V-cycle) beta is taken with the sign flipped, which is the PCG beta when the preconditioner is
 * fixed, so the estimate then holds to the FP32 V-cycle's accuracy.
 *   column < 0: the last r3mg_pcg / r3mg_pcg_host; column >= 0: that column of the last
 *   r3mg_pcg_multi.  cond_out = lmax / lmin (1 when no iteration ran), lmin_out, lmax_out
 *   (0 when none), steps_out = size of T.  Any output may be NULL.  Synchronises.
 * Errors: R3MG_E_ARG (no such column, batched hierarchy), R3MG_E_CUDA.
 */
r3mg_status r3mg_cond_estimate(r3mg_hierarchy* h, int column, double* cond_out, double* lmin_out, double* lmax_out,
                               int* steps_out);

/*
 * Mesh statistics of the paper's tables (Section 6, table legend): H_out = the largest diameter
 * (Euclidean length of the MBR diagonal) of a coarsest-level box; h_out = the largest distance
 * between two support points coupled by a stored entry of A, which is the largest element
 * diameter over the elements whose vertices are unknowns (two points share a stored entry
 * exactly when they share an element); ratio_out = H / h.  ritz_out (levels entries, may be
 * NULL): the Lanczos Ritz value of D_l^{-1} A_l on every smoothed level (the upper Chebyshev
 * interval end is eig_safety times it), 0 on the coarsest.  Batched hierarchies: maxima over
 * the problems.  Host-only; never fails on a valid hierarchy.
 */
r3mg_status r3mg_stats(r3mg_hierarchy* h, double* H_out, double* h_out, double* ratio_out, double* ritz_out);

/*
 * Transfer operator between levels l and l+1 (0 <= l < L-1) as a CSR matrix of n_l rows and
 * n_{l+1} columns (Section 4): l = 0 is P_0 (rows in the caller's numbering, row i has the b
 * columns box(i)*b + q, q = 0..b-1, value phi_{box(i),q}(x_i)); l >= 1 is the injection P~_l
 * (row (c, q') has the columns parent(c)*b + q, value phi_{parent(c),q}(xi_{c,q'})).  The
 * pattern is structural: exactly b entries per row, columns ascending, zeros kept.
 *   rowptr_host (n_l + 1, required), cols_host (n_l * b, may be NULL), vals_host (n_l * b, FP64,
 *   may be NULL; reading values synchronises the stream).  n_l from r3mg_info.
 * Errors: R3MG_E_ARG, R3MG_E_CUDA.
 */
r3mg_status r3mg_get_transfer_pattern(r3mg_hierarchy* h, int level, int64_t* rowptr_host, int32_t* cols_host,
                                      double* vals_host);

/*
 * Galerkin operator A_l (1 <= l < L, Sections 1 and 4) as a CSR matrix in coarse numbering
 * (row and column (B, q) = B*b + q): row (B, q') holds, for every neighbour box of B in
 * ascending order (r3mg_get_level_pattern), the b columns of that box in ascending order; the
 * dense b x b blocks are stored whole (structural zeros kept), FP64 values.
 *   rowptr_host (n_l + 1, required); cols_host, vals_host (rowptr[n_l] entries each, may be
 *   NULL: call once with both NULL to size them).  Reading values synchronises the stream.
 * Errors: R3MG_E_ARG, R3MG_E_CUDA, R3MG_E_OOM.
 */
r3mg_status r3mg_get_level_matrix(r3mg_hierarchy* h, int level, int64_t* rowptr_host, int32_t* cols_host,
                                  double* vals_host);

/*
 * Expiry report of the bounded device waits.  The copy-engine-streamed kernels (the TMA level
 * kernel form and the streamed coarse block kernel) give every mbarrier wait an iteration limit;
 * on expiry a kernel raises a flag on the hierarchy and returns.  r3mg_pcg, r3mg_pcg_host and
 * r3mg_pcg_multi read the flag before returning; calls that return without synchronising
 * (r3mg_vcycle, r3mg_level_apply, r3mg_level0_apply_noalloc, ...) leave it for the next of those
 * or for this call, which synchronises, returns R3MG_E_TIMEOUT if the flag was raised since the
 * last check (and clears it), else R3MG_OK.  Callers that replay captured graphs check here.
 */
r3mg_status r3mg_device_status(r3mg_hierarchy* h, void* stream);

/*
 * Form of the coarsest solve (the paper's direct coarse solve, Section 6, read as a dense
 * Cholesky factorisation A_c = L L^T): mode 0 (default) applies the explicit inverse
 * A_c^{-1} = L^{-T} L^{-1} formed at setup (one GEMV, every row in parallel); mode 1 runs forward
 * and back substitution with L (the textbook solve; a chain of dependent 32-row blocks, one CTA
 * per substitution, solution in shared memory).  Applies to the V-cycle (both precisions) and to
 * r3mg_coarse_solve / r3mg_coarse_solve_prec.  Drops captured graphs; synchronises.
 * Errors: R3MG_E_ARG (mode 1 on a batched hierarchy), R3MG_E_LIMIT (mode 1 when the coarsest
 * level holds more than 26,880 rows, beyond one CTA's shared memory).
 */
r3mg_status r3mg_set_coarse_mode(r3mg_hierarchy* h, int mode);

/*
 * Execution of r3mg_batch_pcg's iteration loop on a batched hierarchy.  mode 0 (default): one
 * CUDA graph launch whose conditional WHILE node repeats a batched iteration, each V-cycle step,
 * transfer, dot and update of all problems being one kernel.  mode 1: one persistent cooperative
 * kernel (captured in a CUDA graph when the driver allows it) runs the whole loop: its CTAs, all
 * resident at once, walk the same phases in the same order of rounding, separated by a grid
 * barrier whose waits are bounded (r3mg_set_wait_limit; on expiry the kernel returns and the
 * solve reports R3MG_E_TIMEOUT), and skip the work of problems that have stopped.  Every
 * problem's iterates are the same in both modes.  Level kernels run in the register form with the
 * lanes per row tuned for each level.  mode 2 (the default of a batched hierarchy): automatic --
 * the first solve runs mode 0 and the second mode 1, each timed with CUDA events per iteration of
 * the loop, and later solves take the faster (mode 0 alone beyond 8 levels); since both give the
 * same iterates, the choice changes no result; setting mode 2 again restarts the measurement.  Errors: R3MG_E_ARG (not a batched hierarchy, mode
 * outside 0..2), R3MG_E_LIMIT (mode 1 with more than 8 levels).
 */
r3mg_status r3mg_set_batch_mode(r3mg_hierarchy* h, int mode);

/* The batched loop's mode setting (0, 1, 2), the form the last solve used (0 or 1), and the
 * per-iteration loop times measured by the automatic mode (ms; -1 where not measured yet).
 * Any output may be NULL. */
r3mg_status r3mg_get_batch_mode(const r3mg_hierarchy* h, int* mode, int* used, float* ms_graph, float* ms_persistent);

/*
 * Limit of the bounded mbarrier waits of the copy-engine-streamed kernels on this hierarchy:
 * cycles = clock64 cycles per wait (0 = the default, about one second at 2 GHz; at most 4e9).
 * The same limit bounds the grid-barrier waits of the persistent batched solve.
 * withhold_first_copy = 1 is the library's test of the expiry path: CTA 0 of the TMA level
 * kernel announces its first descriptor copy on its mbarrier but never issues it, so that wait
 * runs out; the kernel then raises the flag, waits (bounded) for the copies it did issue, and
 * returns, and r3mg_device_status reports R3MG_E_TIMEOUT.  In the persistent batched solve CTA 0
 * withholds its arrival at the first grid barrier, so every CTA's wait runs out and the solve
 * returns R3MG_E_TIMEOUT.  0 in normal use.  Drops captured graphs; synchronises.
 * Errors: R3MG_E_ARG.
 */
r3mg_status r3mg_set_wait_limit(r3mg_hierarchy* h, long long cycles, int withhold_first_copy);

/*
 * Self-test of the bounded-wait mechanism, on the current device: one CTA waits on an mbarrier
 * phase whose arrival announces 16 bytes that no copy delivers, so the wait runs out after
 * limit_cycles (1 .. 4e9) clock64 cycles; the kernel records the expiry, invalidates the
 * barrier and returns with nothing in flight.  expired_out (may be NULL) = 1 when it ran out.
 * Returns R3MG_E_TIMEOUT when the wait expired (the expected outcome; the context stays
 * usable), R3MG_OK if it somehow completed, R3MG_E_ARG, R3MG_E_OOM or R3MG_E_CUDA otherwise.
 * Allocates and frees one int of device memory; synchronises the stream.
 */
r3mg_status r3mg_wait_selftest(long long limit_cycles, int* expired_out, void* stream);

/*
 * As r3mg_setup with the CSR arrays in device memory (rowptr_dev n+1 int64, colidx_dev nnz
 * int32, vals_dev nnz doubles; coords stay host).  The library reads the arrays back to the
 * host on `stream` (the partition and the symbolic analysis are host work) and then proceeds as
 * r3mg_setup.  Errors: as r3mg_setup.
 */
r3mg_status r3mg_setup_device(int64_t n, int dim, const double* coords_host, const int64_t* rowptr_dev,
                              const int32_t* colidx_dev, const double* vals_dev, const r3mg_params* params,
                              void* stream, r3mg_hierarchy** out);

/* Level sizes: n_out[l] rows, nnz_out[l] stored values (padding excluded),
 * nbox_out[l] boxes (level 0: number of level-1 boxes), lam_out[l] upper
 * Chebyshev interval end (0 on the coarsest level).  Arrays hold `levels`
 * entries; any may be NULL. */
r3mg_status r3mg_info(const r3mg_hierarchy* h, int* levels_out, int* depth_out, int64_t* n_out, int64_t* nnz_out,
                      int64_t* nbox_out, double* lam_out);

/* box_of_point_host (n, host): level-l box of every fine point, caller numbering, 1 <= l < L. */
r3mg_status r3mg_get_agglomerates(const r3mg_hierarchy* h, int level, int64_t* box_of_point_host);

/* Block adjacency of A_l (l >= 1; level 1 derives from A's structure):
 * nbr_ptr_host (nbox_l + 1), nbr_host (nbr_ptr[nbox_l]) sorted per box.
 * Call once with nbr_host = NULL to read nbr_ptr only. */
r3mg_status r3mg_get_level_pattern(const r3mg_hierarchy* h, int level, int64_t* nbr_ptr_host, int64_t* nbr_host);

/* Values of A_l (l >= 1), FP64, host: for box B, neighbour slot s (as in
 * r3mg_get_level_pattern), the b x b block at
 * vals_host[(nbr_ptr[B] + s) * b * b + q' * b + q] = A_l[(B,q'), (nbr_s, q)]. Synchronises. */
r3mg_status r3mg_get_level_blocks(r3mg_hierarchy* h, int level, double* vals_host);

/* P values: level 0: p_host (n x b, caller numbering) row i = phi_{box(i),q}(x_i);
 * level l >= 1: p_host (nbox_l x b x b), block c = P~[(c,q'), (parent(c), q)]. Synchronises. */
r3mg_status r3mg_get_prolongation(r3mg_hierarchy* h, int level, double* p_host);

/*
 * Instrumentation.  r3mg_profile_enable(h, 1) records a pair of CUDA events on the
 * library's internal stream (the stream the kernels run on) around every level-operator
 * launch of subsequent r3mg_pcg calls: kind 0 = the CG product A p (FP64 fine level),
 * kind 1 + l = the fused Chebyshev-Jacobi steps on level l (the V-cycle graph is
 * recaptured with event-record nodes).  Enabling or disabling resets the totals and the
 * kernel launch counter.  Synchronises the stream.
 */
r3mg_status r3mg_profile_enable(r3mg_hierarchy* h, int on);

/* Totals for one kind since r3mg_profile_enable: summed event time (ms), number of
 * launches timed, the kind's algorithmic bytes per launch (stored nonzeros x (value +
 * index bytes) + 8 bytes per row pointer + each vector read or written once), and the
 * number of kernels launched by solve-path calls.  Any output may be NULL.  Synchronises. */
r3mg_status r3mg_profile_read(r3mg_hierarchy* h, int kind, double* total_ms, int64_t* count, double* bytes_per_launch,
                              int64_t* kernel_launches);

/* Level-operator kernel chosen for level l and precision (fp32 = 0: FP64, 1: FP32):
 * form 0 = register-streamed, 1 = TMA-streamed, 2 = register-streamed persistent with a
 * double-buffered window, 3 = register-streamed with a bulk L2 prefetch of each box's matrix
 * slice, 4 = symmetric block form (coarse FP32 levels: only the upper blocks are streamed, each
 * used for both of its products), 5 = register-streamed with a software-pipelined row loop
 * (the next chunk of matrix entries is in flight while the current one is consumed), 6 = form 5
 * with the L2 prefetch, 7 = symmetric block form with each box's upper slice requested at once
 * by one bulk copy into shared memory (cp.async.bulk on an mbarrier; slices larger than the
 * stage are read as in form 4; bounded wait as set by r3mg_set_wait_limit, R3MG_E_TIMEOUT on
 * expiry); lanes per matrix row (form 7: resident CTAs per SM, 1..8); threads per CTA;
 * the autotuner's measured time of one launch (0 when not tuned).  Any output may be NULL. */
r3mg_status r3mg_kernel_config(const r3mg_hierarchy* h, int level, int fp32, int* form, int* lanes, int* threads,
                               float* tuned_ms);

/*
 * y = A x on the fine level (the product of r3mg_level_apply with level 0), without any
 * device allocation.  For callers that cannot call cudaMalloc when they apply the operator:
 * code recording its own CUDA graph by stream capture (an allocation cannot be captured and
 * would break the capture), and latency-critical or memory-budgeted loops that forbid the
 * allocator after start-up.  The paper has no counterpart; this is a library service.
 *   x_dev, y_dev: device, n doubles, caller numbering (as r3mg_level_apply); no aliasing.
 * Scratch: a static 16 MiB device array inside the library (two vectors of 2^20 doubles),
 * loaded with the library on every GPU that uses it and kept until the process exits.
 * Limits: n <= 2^20 (1,048,576 DoFs), else R3MG_E_LIMIT and nothing is launched (y untouched).
 * Set-up: r3mg_setup / r3mg_batch_setup look up the array's device address
 * (cudaGetSymbolAddress) on the hierarchy's device and keep it on the hierarchy, so this call
 * itself needs no set-up step.  Nothing in the scratch needs clearing: every call overwrites
 * the n entries it reads.  A bounded-wait expiry of the TMA kernel form (if the fine level uses
 * it) is reported by r3mg_device_status, not by this call.  All calls share the one array, which keeps the last call's contents, so calls
 * whose work overlaps on the GPU (other streams, other threads, other hierarchies on the
 * same device) race and must be serialised by the caller.  Asynchronous on `stream`.
 * Errors: R3MG_E_ARG, R3MG_E_LIMIT, R3MG_E_CUDA.
 */
r3mg_status r3mg_level0_apply_noalloc(r3mg_hierarchy* h, const double* x_dev, double* y_dev, void* stream);

/*
 * Sampled outer product on the stored pattern of A:  out[k] = alpha * lam[i] * u[j] for every
 * stored entry k = (i, j) of the CSR given to r3mg_setup, in that CSR's order.  With
 * alpha = -1, lam the adjoint solution (A lam = dL/du; A is symmetric so the same hierarchy
 * solves it) and u the solution, this is dL/dA on the pattern (the gradient of a loss of
 * u = A^{-1} b with respect to the stored values).  The paper has no adjoint; this serves
 * differentiation through the solve.
 *   lam_dev, u_dev: device, n doubles (caller numbering); out_dev: device, nnz doubles.
 * Asynchronous.  Errors: R3MG_E_ARG, R3MG_E_CUDA.
 */
r3mg_status r3mg_sampled_outer(r3mg_hierarchy* h, const double* lam_dev, const double* u_dev, double alpha,
                               double* out_dev, void* stream);

/* Pin the level-operator kernel of level l and precision (fp32 = 1 needs an FP32 V-cycle):
 * form 0..7 as reported by r3mg_kernel_config, lanes in {4, 8, 16, 32} (also 2 on the FP64 fine
 * level's register forms; 1..8 resident CTAs per SM for form 7), threads per CTA in {128, 256}
 * for the register forms, {96, 128} for form 4 (96: one thread per four-column group of a 27-row
 * box's 380-column upper window), 128 for form 7 and {256, 512, 1024} for the TMA form.  Replays a configuration chosen earlier (reproducible timing
 * and profiling).  Errors: R3MG_E_ARG for an unsupported combination.  Synchronises. */
r3mg_status r3mg_set_kernel_config(r3mg_hierarchy* h, int level, int fp32, int form, int lanes, int threads);

/* As r3mg_set_kernel_config, with the FP64 register kernels' unroll depth: 0 = default
 * (2 steps of 4 entries in flight per lane), 4 = four steps (FP64 only). */
r3mg_status r3mg_set_kernel_config2(r3mg_hierarchy* h, int level, int fp32, int form, int lanes, int threads, int unroll);

/* The unroll depth chosen for level l and precision (0 = default, 4). */
r3mg_status r3mg_kernel_unroll(const r3mg_hierarchy* h, int level, int fp32, int* unroll);

/*
 * Device characterisation for the FP64 roofline: the sustained FP64 FMA rate and the FP64
 * tensor-core (mma.sync m8n8k4) rate of the current GPU, in TFLOP/s (2 flops per FMA).  Each is
 * timed with CUDA events over one launch of 8 independent FMA (or 4 independent mma) chains per
 * thread on 8 CTAs of 256 threads per SM, after one warm-up launch.  The FP64 level kernels do
 * one FMA per 8-10 bytes of matrix stream, so on a GPU whose FP64 rate is low next to its memory
 * bandwidth these rates, not HBM, bound them.  Allocates and frees a small device buffer;
 * synchronises the stream.  Errors: R3MG_E_CUDA, R3MG_E_OOM.
 */
r3mg_status r3mg_measure_fp64_rates(double* fma_tflops, double* mma_tflops, void* stream);

/* Message of the last failure on h (or of the last failed r3mg_setup /
 * r3mg_partition in this thread when h is NULL).  Never NULL. */
const char* r3mg_last_error(const r3mg_hierarchy* h);

/* Free all device and host memory of h (NULL is a no-op). */
void r3mg_destroy(r3mg_hierarchy* h);

#ifdef __cplusplus
}
#endif
#endif
