/*
 * kkt.h -- C interface of the fixed-pattern KKT refactorization library.
 *
 * The library factors a sequence of sparse matrices that share one sparsity
 * pattern while their values change at every interior-point iteration
 * (arXiv 2306.14337, Sec. 2, Eq. 4 and the remark after it: all K_k have the
 * same pattern, so work on the pattern should be reused).  It follows the
 * paper's three phases (Sec. 4): a host-side analysis once per pattern, then
 * for every value set a numeric refactorization with the same pivot sequence
 * (Sec. 4 "refactorization", Sec. 5), triangular solves, and iterative
 * refinement (Sec. 5.1).  Everything after the analysis runs in this
 * library's CUDA kernels on one GPU; the host only launches them.
 *
 * Conventions shared by all calls
 *   - Indices are int32, values float64.  The matrix is given in compressed
 *     sparse row form (row_ptr[n+1], col_idx[nnz]) with strictly increasing
 *     column indices in every row; values are in the same order.
 *   - "_dev" pointers are device pointers on the context's device; the
 *     caller owns them, keeps them valid until the stream reaches the call,
 *     and may reuse them afterwards.  "_host" pointers are host memory.
 *   - The context owns the factors and every workspace buffer; all of it is
 *     allocated by kkt_analyze (Sec. 5.1: buffers allocated once and reused).
 *   - Calls that take a stream are asynchronous on that stream (NULL = the
 *     legacy default stream) unless stated otherwise.  Conditions found on
 *     the device (perturbed pivots, non-finite values, a wait that ran out)
 *     accumulate in a device status word read by kkt_status_sync.  Errors
 *     found on the host return at once and launch nothing.
 *   - Calls on one context must be ordered on one stream; a context is not
 *     safe for concurrent use from several host threads.
 */
#ifndef KKT_H
#define KKT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct kkt_ctx kkt_ctx;
typedef void *kkt_stream; /* a cudaStream_t */

typedef enum {
    KKT_OK = 0,
    KKT_ERR_ARG = 1,            /* invalid argument (null pointer, size, option) */
    KKT_ERR_PATTERN = 2,        /* unsorted / duplicate / out-of-range index, n <= 0 */
    KKT_ERR_ALLOC = 3,          /* host or device allocation failed */
    KKT_ERR_CUDA = 4,           /* a CUDA runtime call failed */
    KKT_ERR_NONFINITE = 5,      /* a value or a computed pivot was NaN or infinite */
    KKT_ERR_NOT_CONVERGED = 6,  /* refinement did not reach tol in max_it solves;
                                   the caller may re-analyze (Sec. 5.1) */
    KKT_ERR_TIMEOUT = 7,        /* a bounded device wait ran out; results invalid */
    KKT_ERR_STATE = 8,          /* call out of order (e.g. solve before refactor),
                                   or a device call on a host-only context */
    KKT_ERR_INTERNAL = 9,       /* a device-side consistency check failed */
    KKT_WARN_PERTURBED = 100    /* success, but some pivots were perturbed */
} kkt_status;

enum { KKT_ORDER_AMD = 0, KKT_ORDER_NATURAL = 1, KKT_ORDER_USER = 2 };
enum { KKT_REFINE_CLASSIC = 0, KKT_REFINE_FGMRES = 1, KKT_REFINE_AUTO = 2, KKT_REFINE_FGMRES_JACOBI = 3 };

typedef struct {
    int factor_fp32;        /* 0: factors and triangular solves in FP64;
                               1: in FP32 (residual, update, pivot test stay FP64) */
    int equilibrate;        /* 1: power-of-two symmetric scaling s_i = 2^-floor(floor(log2 r_i)/2),
                               r_i = max_j |a_ij|, recomputed at every refactorization */
    int ordering;           /* KKT_ORDER_*: approximate minimum degree on A + A^T
                               (Sec. 5.2), identity, or user_perm */
    const int *user_perm;   /* ordering == USER: host array, perm[new] = old, length n;
                               copied during kkt_analyze */
    int refine_mode;        /* KKT_REFINE_*: classic (Sec. 5.1 x += K^-1 (r - K x)),
                               FGMRES with the LU solve as right preconditioner and
                               CGS2 (Sec. 5.1), or classic switching to FGMRES when an
                               iteration fails to halve the scaled residual, or
                               FGMRES whose preconditioner replaces the two
                               triangular solves by jacobi_sweeps Jacobi sweeps each
                               (Sec. 6: iterative approximate triangular solves) */
    int fgmres_restart;     /* Krylov basis size (default 20) */
    int max_refine;         /* default limit on solves in kkt_refine (20, Sec. 5.3) */
    double tol;             /* default scaled-residual target (1e-14, Sec. 5.3) */
    double pivot_tau_rel;   /* perturbation threshold relative to max|A'|; 0 selects
                               1e-14 (FP64 factors) or 2^-24 (FP32 factors) */
    long long spin_limit;   /* polls before a device wait gives up (KKT_ERR_TIMEOUT) */
    int device;             /* CUDA device ordinal; -1 = host-only analysis (no CUDA
                               call at all; only the kkt_get_* / export calls work) */
    int max_batch;          /* capacity of the batched calls, fixed at analysis */
    int cta_warps;          /* warps per CTA of the persistent kernels (1..8; 0 = 8);
                               the single-system triangular solves use twice as many */
    int refactor_ctas;      /* CTAs of the refactorization (0 = all that fit at once) */
    int solve_ctas;         /* CTAs of the single-system triangular solves (0 = one per
                               SM); every CTA must fit on the device at once */
    size_t update_map_budget; /* bytes allowed for the refactorization's update maps
                                 (relative positions of every multiply-add; 0 = 1 GiB);
                                 over budget the kernel searches each row instead */
    int trace;              /* 1: record per work item claim/completion times on the
                               device (see kkt_export_trace) */
    int poll_ns_max;        /* backoff cap (ns) of a waiting lane; one lane per warp
                               polls, doubling its sleep from 32 ns (0 = 128 ns) */
    int unpublished_row;    /* failure-detection testing only (-1 = off): the
                               refactorization never publishes this row (numbered
                               like kkt_export_symbolic), so the rows that depend on
                               it exhaust spin_limit and report KKT_ERR_TIMEOUT */
    int refactor_big_warps; /* warps per CTA of the refactorization that own a
                               shared-memory row for the rows longer than 1,024
                               entries (k > 0: k, at most half the CTA, as far as
                               shared memory allows; 0 = none: such rows work in
                               global scratch, the faster choice where measured) */
    int symmetric;          /* 1: the values are symmetric (A = A^T, as the KKT matrices
                               of Eq. 4); the refactorization then computes A' = L D L^T
                               (Sec. 3 inertia, Sec. 5.3 MA57's form): row i's multipliers
                               l(i,d) = u(d,i)/u(d,d) come from rows below it, only its
                               U part is reduced (half the flops of LU), the factors are
                               stored as for LU, and kkt_inertia reports the pivot signs.
                               Only A's upper triangle is read.  Needs the update maps
                               (else the LU refactorization runs, same factors in exact
                               arithmetic).  Batched and queued calls use LU. */
    int jacobi_sweeps;      /* sweeps per triangular factor of KKT_REFINE_FGMRES_JACOBI
                               (default 8) */
    const int *user_row_perm; /* NULL, or a host array of n rows: the context then
                               factors Q A, whose row j is row user_row_perm[j] of A
                               (copied during analysis; see kkt_analyze_values) */
    int dense_block;        /* dense root block (Sec. 4, supernodal methods: dense
                               blocks where the factor is dense): the last k rows of
                               the elimination order are stored as a full k x k block
                               of the factor (explicit zeros where the fill pattern has
                               none) and, after the sparse rows, factored by a blocked
                               dense LU with the same fixed pivots and perturbation
                               test.  -1: none; 0 (default): the largest trailing
                               block of at most 2,048 rows whose pattern is at least
                               80% full, if it has 96 rows or more; k > 0: k rows.
                               The block is the top of one path of the elimination
                               tree (each row the parent of the one before), so k is
                               capped at that path's length (the forward levels of
                               the tree).  The exported pattern (kkt_export_symbolic)
                               then holds the whole block; its entries outside the
                               fill pattern of the oracle's definition are exactly
                               zero.  Used by kkt_refactor; the batched and queued
                               refactorizations treat the block's rows as sparse rows. */
    int refactor_row_cap;   /* entries of the shared-memory row buffer of each warp of
                               the single-system refactorization (0: the longest row,
                               at most 1,024); longer rows work in global memory.  A
                               larger buffer fits fewer warps on an SM. */
    double refine_auto_ratio; /* refine mode auto: classic steps continue while each
                               lowers the scaled residual to at most this fraction of
                               the previous one, then FGMRES takes over (0: 0.5; must
                               be below 1) */
    int solve_far_blocks;   /* triangular solves: a row of a long task (one run by a
                               whole CTA) whose sources in its own task lie more than
                               this many 32-row blocks back -- at least 32 of them --
                               has their sum computed by a partner CTA of the task,
                               which streams those entries on another SM as the
                               task's CTA publishes the rows; the task's CTA then
                               reads only the last blocks' entries of such a row.
                               0: 2 blocks; -1: off. */
    int solve_far_ctas;     /* partner CTAs of the single-system solves, given to the
                               long tasks with the most far entries (0: 8; -1: none;
                               at most a third of the CTAs left after the long tasks) */
} kkt_options;

typedef struct {
    int n;                  /* dimension */
    long long nnz_a;        /* stored entries of the user pattern */
    long long nnz_sym;      /* entries of A + A^T + I */
    long long nnz_lu;       /* entries of combined L+U (diagonal once) */
    int n_levels;           /* levels of the refactorization / forward solve */
    int n_levels_u;         /* levels of the backward solve */
    int max_row;            /* longest row of L+U */
    double flops_refactor;  /* sum over pivots d of |L(:,d)| (1 + 2 |U(d,:)|) */
    double bytes_refactor;  /* compulsory bytes of one refactorization */
    double bytes_solve;     /* compulsory bytes of one forward + backward solve */
    double bytes_spmv;      /* compulsory bytes of one residual */
    size_t device_bytes;    /* device memory held by the context */
    int grid_ctas;          /* CTAs of the refactorization */
    int solve_ctas;         /* CTAs of the single-system triangular solves */
    int warps_per_cta;      /* of the refactorization and the batched kernels */
    int last_refine_iters;  /* solves used by the last kkt_refine */
    double last_omega;      /* scaled residual after the last kkt_refine */
    int factor_fp32;
    long long kernel_launches; /* CUDA kernels this context has launched so far */
    long long update_map_entries; /* 0 when the update maps are not built */
    int n_tasks;            /* longest-path tasks of the triangular solves */
    int max_task;           /* rows in the longest task */
    int refactor_big_warps; /* warps per CTA of the refactorization that take the
                               rows longer than 1,024 entries (0: no such rows) */
    int refactor_big_cap;   /* row capacity (entries) of those warps' shared memory */
    int dense_rows;         /* rows of the dense root block (0: none) */
    int refactor_row_cap;   /* row buffer entries of the refactorization's warps */
    int solve_far_rows;     /* rows of long solve tasks whose far sources in their own
                               task a partner CTA sums (forward phase) */
    int solve_far_ctas;     /* partner CTAs of the single-system solves */
} kkt_stats;

typedef struct {
    int iters;              /* solves with the factors used */
    int converged;          /* 1 if omega <= tol */
    double omega;           /* final scaled residual */
    double omega_hist[64];  /* omega before each solve and after the last (first 64) */
    int n_hist;
} kkt_refine_info;

/* Fill *opt with the defaults listed above (AMD, equilibration on, FP64). */
void kkt_default_options(kkt_options *opt);

/* Human-readable name of a status code (static storage). */
const char *kkt_status_string(kkt_status s);

/* Text of the last host-detected error on the calling thread ("" if none);
 * valid until the next call on that thread. */
const char *kkt_last_error(void);

/*
 * Analyze a pattern once (Sec. 4 symbolic phase; Sec. 5.2 preprocessing:
 * symmetric fill-reducing ordering of A + A^T, symbolic LU, reused for every
 * later value set).  Host only; then copies the index structures to the device
 * once (Sec. 5: data moves to the GPU once) and allocates all workspace.
 *   n, row_ptr[n+1], col_idx[nnz]: host CSR, sorted and unique per row.
 *   opt: NULL for defaults.
 *   out: receives the new context (NULL on failure).
 * Missing diagonal entries are added as structural zeros.  Errors:
 * KKT_ERR_PATTERN for a malformed pattern, KKT_ERR_ARG for a bad option or
 * user permutation, KKT_ERR_ALLOC / KKT_ERR_CUDA.
 */
kkt_status kkt_analyze(int n, const int *row_ptr, const int *col_idx,
                       const kkt_options *opt, kkt_ctx **out);

/*
 * Value-aware analysis (Sec. 5.2: MC64 matching before the fill-reducing
 * ordering; Sec. 5.1: a pivot sequence chosen on the values of the first
 * system).  A row permutation Q is computed from values_host (nnz float64 in
 * CSR order): a perfect matching of the nonzeros that maximizes the product
 * of the matched |a_ij| (the weighted bipartite matching MC64 solves), so Q A
 * has a nonzero diagonal with the largest product; options.user_row_perm, when
 * set, is used instead.  The pattern of Q A is then analyzed as by
 * kkt_analyze, and the context factors Q A with diagonal pivots: KKT matrices
 * without regularization, whose zero diagonal blocks give zero pivots in the
 * pattern-only analysis, get nonzero ones.  Every call keeps the caller's
 * numbering of A (values in A's CSR order, b, x, g, lambda, dA); the library
 * applies Q at the boundary.  The exports describe Q A (kkt_export_row_perm
 * gives Q).  Batched and queued calls are not available on such a context.
 * The matching is recomputed only by a new analysis: when refinement returns
 * KKT_ERR_NOT_CONVERGED the caller may analyze again on the current values
 * (the paper's re-analysis policy, Sec. 5.1).  Errors: as kkt_analyze;
 * KKT_ERR_PATTERN when A has no perfect matching (structurally singular).
 */
kkt_status kkt_analyze_values(int n, const int *row_ptr, const int *col_idx, const double *values_host,
                              const kkt_options *opt, kkt_ctx **out);

/* The row permutation of the context: row j of the factored matrix is row
 * row_of_col[j] of A (the identity without one).  row_of_col: host, n ints. */
kkt_status kkt_export_row_perm(const kkt_ctx *ctx, int *row_of_col);

/* Release everything the context holds.  NULL is allowed. */
void kkt_destroy(kkt_ctx *ctx);

/*
 * Numeric refactorization with the fixed pivot sequence (Sec. 4
 * refactorization; Sec. 5.2: fill A's values into the combined L+U storage,
 * then factor).  values_dev: nnz float64 in the CSR order given to analyze.
 * The context keeps the pointer: residuals of later kkt_refine calls read the
 * original matrix from it, so it must stay valid and unchanged until the next
 * kkt_refactor.  Perturbed pivots (|p| below tau, Sec. 5 static-pivot
 * reading) are counted in the device status word.
 */
kkt_status kkt_refactor(kkt_ctx *ctx, const double *values_dev, kkt_stream stream);

/* x = A^-1 b with the current factors (permute/scale fused, Sec. 5.2).
 * b_dev, x_dev: n float64; they may not alias. */
kkt_status kkt_solve(kkt_ctx *ctx, const double *b_dev, double *x_dev, kkt_stream stream);

/*
 * Approximate solve with the current factors by Jacobi sweeps instead of
 * substitution (Sec. 6: iterative approximation of the triangular solves;
 * Anzt, Chow and Dongarra 2015).  With L = I + L_s and U = D + U_s:
 *   w_0 = c, w_{k+1} = c - L_s w_k;  z_0 = D^-1 w, z_{k+1} = D^-1 (w - U_s z_k),
 * `sweeps` sweeps each, c = S P b and x = S P^T z (transpose = 1: the same on
 * A'^T = U^T L^T).  Every sweep is one parallel sparse product with no
 * dependency chain; the result equals the exact solve once sweeps reaches
 * the number of levels minus one, and is an approximation (a preconditioner
 * for FGMRES) below that.  b_dev, x_dev: n float64, not aliased.
 */
kkt_status kkt_solve_jacobi(kkt_ctx *ctx, const double *b_dev, double *x_dev, int sweeps, int transpose,
                            kkt_stream stream);

/* lam = A^-T g with the same factors (A'^T = U^T L^T).  g_dev, lam_dev: n float64. */
kkt_status kkt_solve_transpose(kkt_ctx *ctx, const double *g_dev, double *lam_dev,
                               kkt_stream stream);

/*
 * Iterative refinement (Sec. 5.1) of x_dev (in/out, n float64) for A x = b
 * until omega = ||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf) <= tol or
 * max_it solves were used (tol <= 0 / max_it < 0 select the context's
 * defaults).  The residual is FP64 on the original A.  Reads omega on the host
 * once per iteration, so this call synchronizes the stream.  info (host, may
 * be NULL) receives the history.  Returns KKT_ERR_NOT_CONVERGED when the
 * target was missed.
 */
kkt_status kkt_refine(kkt_ctx *ctx, const double *b_dev, double *x_dev, double tol,
                      int max_it, kkt_refine_info *info, kkt_stream stream);

/* Same for the transposed system A^T lam = g. */
kkt_status kkt_refine_transpose(kkt_ctx *ctx, const double *g_dev, double *lam_dev,
                                double tol, int max_it, kkt_refine_info *info,
                                kkt_stream stream);

/*
 * Gradient of x = A^-1 b: dA_k = -lam[row_k] * x[col_k] for every stored
 * entry k of the user pattern (nnz float64, CSR order); the gradient of b is
 * lam itself.  lam_dev, x_dev: n float64.
 */
kkt_status kkt_adjoint_gather(kkt_ctx *ctx, const double *lam_dev, const double *x_dev,
                              double *dA_dev, kkt_stream stream);

/* Synchronize the stream, read and clear the device status word.  Returns
 * KKT_ERR_INTERNAL, KKT_ERR_TIMEOUT, KKT_ERR_NONFINITE, KKT_WARN_PERTURBED or KKT_OK;
 * *n_perturbed (may be NULL) receives the count of perturbed pivots. */
kkt_status kkt_status_sync(kkt_ctx *ctx, kkt_stream stream, int *n_perturbed);

/*
 * Inertia of A from the last refactorization (options.symmetric = 1): the
 * numbers of positive and negative pivots of A' = L D L^T (Sec. 3: the
 * inertia an interior method checks; Sylvester's law of inertia makes them
 * those of A, since A' = S P A P^T S is congruent to A).  n_perturbed: pivots
 * replaced by +-tau in that refactorization (counted with the sign they got):
 * A is then singular or nearly so in the pivot test's sense.  Synchronizes
 * the stream.  KKT_ERR_STATE without options.symmetric or before a
 * refactorization.  Any pointer may be NULL.
 */
kkt_status kkt_inertia(kkt_ctx *ctx, kkt_stream stream, int *n_pos, int *n_neg, int *n_perturbed);

/* Sizes, byte and flop counts of the analysis (host, no synchronization). */
kkt_status kkt_get_stats(const kkt_ctx *ctx, kkt_stats *stats);

/*
 * Copy the analysis to host arrays (sizes from kkt_get_stats):
 *   perm[n] (new -> old), lu_row_ptr[n+1], lu_col_idx[nnz_lu] (pattern of
 *   combined L+U of the permuted matrix, row-wise, sorted),
 *   level[n], level_u[n] (forward and backward level of every permuted row).
 * Everything is numbered by perm, the ordering given (KKT_ORDER_USER) or
 * computed; internally the rows are also relabelled by a postorder of the
 * elimination tree, which changes neither the fill nor the levels.
 * Any pointer may be NULL to skip that array.
 */
kkt_status kkt_export_symbolic(const kkt_ctx *ctx, int *perm, int *lu_row_ptr,
                               int *lu_col_idx, int *level, int *level_u);

/*
 * Rows of the dense root block (options.dense_block; Sec. 4 on supernodal
 * dense blocks), numbered like kkt_export_symbolic, in their elimination
 * order: rows[0 .. dense_rows-1] (dense_rows from kkt_get_stats; nothing is
 * written when it is 0).  The exported pattern is the fill pattern of the
 * ordering plus every (rows[a], rows[b]).  Host only.  KKT_ERR_ARG for a
 * NULL context, or NULL rows when the block is not empty.
 */
kkt_status kkt_export_dense_rows(const kkt_ctx *ctx, int *rows);

/*
 * Checkpoint and resume of the analysis (Sec. 4 and Sec. 5.2: one symbolic
 * analysis serves every later system; a saved one lets a new run skip it).
 * kkt_save_analysis writes a self-contained image of everything the analysis
 * computed -- ordering, fill pattern, levels, maps, solve tasks, and the row
 * permutation of a value-aware context -- ending in a 64-bit checksum: with
 * buf NULL it only stores the size needed in *size; otherwise cap must be at
 * least that size.  kkt_load_analysis creates a context from such an image
 * with the given options (their ordering, user_perm and user_row_perm are
 * ignored: the image fixes them; the update maps are those of the image) and
 * allocates and uploads as kkt_analyze does.  An image whose checksum,
 * version or array sizes do not match returns KKT_ERR_ARG.  The image must
 * come from kkt_save_analysis of this library version.
 */
kkt_status kkt_save_analysis(const kkt_ctx *ctx, void *buf, size_t cap, size_t *size);
kkt_status kkt_load_analysis(const void *buf, size_t size, const kkt_options *opt, kkt_ctx **out);

/* Copy the current factor values (float64, in the lu_col_idx order of
 * kkt_export_symbolic; L strictly below the diagonal, U on and above it) to
 * out_dev (nnz_lu float64). */
kkt_status kkt_export_factors(kkt_ctx *ctx, double *out_dev, kkt_stream stream);

/*
 * Device trace of the most recent launch of one phase (options.trace = 1):
 * phase 0 refactorization (work item = row, numbered like kkt_export_symbolic), 1 forward solve,
 * 2 backward solve, 3 transposed forward, 4 transposed backward (work item =
 * task in claim order, followed by the long tasks that ran on a CTA each, in
 * decreasing length), 5 the dense root block's LU (work item = tile task in
 * claim order: per step the diagonal tile, the L and U tiles, the updates).  out_host receives 2 words per item, the %globaltimer
 * value (ns) at claim and at completion; *n_items the number of items copied.
 * Synchronizes the device.
 */
kkt_status kkt_export_trace(kkt_ctx *ctx, int phase, unsigned long long *out_host, long long max_items,
                            long long *n_items);

/* Copy the current scaling s (n float64, original indexing) to out_dev. */
kkt_status kkt_export_scaling(kkt_ctx *ctx, double *out_dev, kkt_stream stream);

/*
 * Batched same-pattern systems (configuration option max_batch >= B).  All
 * arrays are batch innermost: entry k of system s at k * B + s for values
 * (nnz x B), entry i of system s at i * B + s for vectors (n x B).  Work
 * items are (row or task, system) pairs, claimed in topological order with
 * every system of a row or task together; one warp runs the single-system
 * body on one pair, the row's entries across its lanes, so a warp's loads
 * step through one system's entries B values apart (not coalesced across the
 * batch: a warp per row of 4 adjacent systems, 8 lanes each, was measured
 * slower on the 10,000-bus x 64 case).  The B systems' independent
 * dependency chains run side by side and fill the GPU that one system leaves
 * idle.  Refinement is classic (Sec. 5.1) and stops when every system reaches
 * tol; omega_host (B doubles, may be NULL) receives each system's scaled
 * residual and *iters the solves used.
 */
kkt_status kkt_batch_refactor(kkt_ctx *ctx, int B, const double *values_dev, kkt_stream stream);
kkt_status kkt_batch_solve(kkt_ctx *ctx, int B, const double *b_dev, double *x_dev, kkt_stream stream);
kkt_status kkt_batch_solve_transpose(kkt_ctx *ctx, int B, const double *g_dev, double *lam_dev,
                                     kkt_stream stream);
kkt_status kkt_batch_refine(kkt_ctx *ctx, int B, const double *b_dev, double *x_dev, double tol,
                            int max_it, double *omega_host, int *iters, kkt_stream stream);
kkt_status kkt_batch_refine_transpose(kkt_ctx *ctx, int B, const double *g_dev, double *lam_dev,
                                      double tol, int max_it, double *omega_host, int *iters,
                                      kkt_stream stream);
/* Factor values of one system of the last batched refactorization, in the
 * order of kkt_export_factors. */
kkt_status kkt_batch_export_factors(kkt_ctx *ctx, int sys, double *out_dev, kkt_stream stream);

/*
 * Uneven batch: several contexts with different patterns (same device and
 * factor precision) processed together.  Work items (system, row) and
 * (system, task) are ordered by elimination level across systems and claimed
 * from one device counter, so each phase (refactorization, forward and
 * backward solve) is one persistent launch over all systems.
 *
 * kkt_queue_run: for every system k, refactor with values[k], solve into
 * x[k] from b[k], then n_refine classic refinement steps; if omega_dev is not
 * NULL (m doubles on the device) it receives each system's scaled residual.
 * The whole sequence is recorded once into a CUDA graph and replayed; it is
 * recorded again when any pointer or n_refine changes.  The arrays of
 * pointers are host arrays of m device pointers.  The contexts keep the
 * factors for later single-system calls.
 * kkt_queue_solve_transpose: lam[k] = A_k^-T g[k] with the current factors.
 * kkt_queue_set_launch: warps per CTA (1..8) and CTA count of the persistent
 * kernels (0 = defaults), used by the autotuner.
 */
typedef struct kkt_queue kkt_queue;
kkt_status kkt_queue_create(kkt_ctx *const *ctxs, int m, kkt_queue **out);
void kkt_queue_destroy(kkt_queue *q);
kkt_status kkt_queue_set_launch(kkt_queue *q, int cta_warps, int ctas);
/* Tile choice of the queue's solves, used by the autotuner: how many of the
 * queue's longest solve tasks (at most 48, longest first; -1 = all of them)
 * run on a whole CTA each (with 8 warps per CTA), the others as warp items.
 * The captured graph is recorded again at the next kkt_queue_run. */
kkt_status kkt_queue_set_tiles(kkt_queue *q, int cta_tasks);
kkt_status kkt_queue_run(kkt_queue *q, const double *const *values, const double *const *b,
                         double *const *x, int n_refine, double *omega_dev, kkt_stream stream);
kkt_status kkt_queue_solve_transpose(kkt_queue *q, const double *const *g, double *const *lam,
                                     kkt_stream stream);
kkt_status kkt_queue_status_sync(kkt_queue *q, kkt_stream stream, int *n_perturbed);

/*
 * Measured fused multiply-add throughput of the device (TFLOP/s, 2 flops per
 * FMA) in FP64 (fp64 = 1) or FP32 (fp64 = 0): every thread of 8 CTAs of 256
 * per SM runs eight independent FMA chains; the best of five timed launches.
 * The paper has no counterpart; it supplies the arithmetic roofline against
 * which the benchmark states the refactorization's rate.  Synchronizes the
 * device and allocates a small output buffer.  Errors: KKT_ERR_ARG,
 * KKT_ERR_CUDA (text in kkt_last_error()).
 */
kkt_status kkt_probe_fma_tflops(int device, int fp64, double *tflops);

/*
 * Scaled residual without any device allocation and without a context.
 *
 * The paper has no counterpart of this call; it exists for callers that cannot
 * call cudaMalloc where they need the residual: programs that give their whole
 * device-memory budget to their own pool allocator at start-up (a hidden
 * allocation would fail or break the budget), and loops that cannot afford the
 * device-wide synchronization that allocating and freeing can cause.  Such
 * callers may not be able to create a kkt_ctx either, since kkt_analyze
 * allocates.
 *
 * Computes rho = b - A x (FP64, same per-row arithmetic as kkt_refine) and
 *   out_dev[0] = omega = ||rho||_inf / (||A||_inf ||x||_inf + ||b||_inf)
 *                (+infinity when any entry of x, b, rho or A is NaN or infinite),
 *   out_dev[1..4] = ||rho||_inf, ||x||_inf, ||b||_inf, ||A||_inf.
 *   n, row_ptr_dev[n+1], col_idx_dev[nnz], values_dev[nnz]: the matrix in CSR
 *   on the current device; b_dev, x_dev, rho_dev: n float64; out_dev: 5 float64.
 * Asynchronous on stream, on the calling thread's current device.
 *
 * Its only scratch is a fixed 4 MiB array compiled into the library (one
 * partial result per 32 rows), so n may not exceed 4,194,304: larger n returns
 * KKT_ERR_ARG and launches nothing.  A GPU commits the array when the library's
 * device code is loaded on it -- with CUDA's lazy loading, at the latest during
 * the first call on that device -- and keeps it until the process exits.  That
 * first call also looks up the array's device address (once per device, with
 * the device current), so make it before any stream capture.  All calls on a
 * device share the array and it keeps the last call's contents; calls that
 * overlap on the GPU race on it, so order them on one stream.  Failures set
 * the text of kkt_last_error().
 */
kkt_status kkt_scaled_residual_noalloc(int n, const int *row_ptr_dev, const int *col_idx_dev,
                                       const double *values_dev, const double *b_dev,
                                       const double *x_dev, double *rho_dev, double *out_dev,
                                       kkt_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* KKT_H */
