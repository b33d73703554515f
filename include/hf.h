/*
 * hf.h -- C ABI of the GB300 hybrid sparse factorization.
 *
 * Method: A. Suzuki, "A hybrid factorization algorithm for sparse matrix with
 * mixed precision arithmetic" (arXiv 2208.01907).
 *   Sec. 2      diagonal scaling K = Q Kbar Q with diag(K) in {-1, 0, 1}
 *   Sec. 2.1-2.2 LDL^T with symmetric 1x1 pivoting and threshold postponing
 *               along a nested-dissection tree; split Lambda = Lambda_1 + Lambda_2
 *   Alg. 1      K11 X12 = K12 by an iterative solver preconditioned with the
 *               lower-precision factor; S22 = K22 - K21 X12 in higher precision;
 *               S22 factorized with symmetric (1x1 / 2x2) pivoting
 *   Alg. 2      block forward / backward substitution
 *   Sec. 3.5    block GCR ("Algorithm 5")
 *
 * Conventions for every entry point:
 *   - Indices are 0-based.  Matrices are square, structurally symmetric and
 *     numerically symmetric (the LDL^T form of Sec. 4.1), or J times a symmetric
 *     matrix with the row signs J declared by hf_set_row_signs (the unsymmetric
 *     LDU form [A B^T; -B delta D] of Sec. 4.2).  CSR rows are sorted by column
 *     and every row stores its diagonal entry (it may be 0).
 *   - "device" pointers are CUDA global-memory addresses on the current device;
 *     "host" pointers are ordinary process memory.  The caller owns every
 *     buffer it passes; the library never frees or retains caller pointers
 *     beyond the call.
 *   - Device work is stream-ordered on hf_opts.cuda_stream (NULL = legacy
 *     default stream).  Calls that return host-visible results synchronise
 *     that stream before returning.
 *   - Return value: HF_OK (0) or one of the HF_ERR_* codes below.  On error the
 *     context stays valid and keeps its previous state unless stated.
 *   - A context is not thread-safe.
 */
#ifndef HF_H
#define HF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  HF_OK = 0,
  HF_ERR_ARG = 1,            /* invalid argument (null pointer, negative size, ...) */
  HF_ERR_STATE = 2,          /* call order violated, e.g. hf_schur before hf_factorize */
  HF_ERR_PATTERN = 3,        /* CSR unsorted, index out of range, pattern not symmetric,
                                or a row without its diagonal entry */
  HF_ERR_NUMERIC = 4,        /* NaN / Inf in the input values */
  HF_ERR_NOT_CONVERGED = 5,  /* block GCR hit gcr_maxit; results usable, see hf_info */
  HF_ERR_TIMEOUT = 6,        /* a bounded device-side wait expired */
  HF_ERR_CUDA = 7,           /* a CUDA runtime call failed */
  HF_ERR_OOM = 8,            /* device memory allocation failed */
  HF_ERR_CAPACITY = 9        /* a front outgrew the panel kernels' shared memory: with
                                the rows postponed into it, more than about 25,000 rows
                                (FP32 factor); a smaller tau postpones fewer rows */
};

/* Precision forms (Table 1 columns). */
enum {
  HF_PREC_MIXED = 0,   /* FP32 factor + FP64 block GCR / S22 / dense LDL^T: Alg. 1 */
  HF_PREC_FP64 = 1,    /* plain FP64 factor, S22 taken from the FP64 factor ("double") */
  HF_PREC_FP32 = 2     /* FP32 factor, S22 from the FP32 factor ("single") */
};

typedef struct hf_ctx hf_ctx;   /* opaque; owns every device buffer it allocates */

typedef struct {
  double tau;            /* postponing threshold tau > 0 (Sec. 2.2); default 1e-2 */
  int    n_enlarge;      /* entries moved into the hard part (Sec. 2.2, "n = 4"); default 4 */
  int    precision;      /* HF_PREC_*; default HF_PREC_MIXED */
  double gcr_tol;        /* block GCR stop: max_k |r_k|/|b_k| <= gcr_tol; default 1e-14 */
  int    gcr_maxit;      /* block GCR iteration limit; default 40 */
  double kernel_eps;     /* null pivot of S22 if |pivot| <= max(kernel_eps * scale, noise), scale =
                            max(max|pivot|, max|diag K22|), noise = 100 x the estimated error of
                            S22; default 1e-10 */
  double kernel_gap;     /* minimum ratio gap that separates null pivots; default 1e4 */
  int    nd_leaf;        /* dissection stops when a set has <= nd_leaf unknowns; default 256 */
  int    nd_levels;      /* if > 0, force the number of tree levels m (Sec. 2.2); default 0 */
  int    delay_cap;      /* initial capacity for postponed rows per front; default 256
                            (grown and retried automatically when exceeded) */
  int    panel;          /* pivots per panel of the front factorization; default 64 */
  void*  cuda_stream;    /* cudaStream_t; NULL = default stream */
  int    fp64_gemm;      /* FP64 Grams and block updates of block GCR: 0 = emulated on the BF16
                            tensor cores with exact slice products (FP64 accuracy normwise, i.e.
                            relative to the largest entries of each column; hf_schur and hf_solve
                            run a block GCR that stagnates above gcr_tol again with the FP64
                            units, counted in hf_info.gcr_restarts), 1 = FP64 units; default 0 */
  int    trailing;       /* trailing updates of the FP32 factor: 0 = tensor cores for the tree
                            levels whose largest front has >= 256 rows (exact 3 x BF16 split of
                            FP32, six products, FP32 accumulation in TMEM; FP32 SIMT for the
                            smaller levels), 1 = FP32 SIMT everywhere; default 0; the FP64 form
                            always uses FP64 SIMT */
  int    null_test;      /* 0 = postpone on the ratio test of Sec. 2.2 alone (the paper's rule);
                            1 = also postpone a candidate on its own when its diagonal is below
                            tau times the magnitude of the terms it was formed from (|K_ii| plus
                            the accumulated |l_ik|^2 |d_k|), a cancellation test that is not in the
                            paper; default 0 */
  int    spin_limit;     /* polls of a bounded device wait of the triangular sweeps (a block waiting
                            for a diagonal block another block solves) before the wait gives up and
                            the call returns HF_ERR_TIMEOUT; 0 = the built-in limit (2^22 polls with
                            sleeps, seconds); default 0 */
} hf_opts;

typedef struct {
  int64_t L;              /* order of K */
  int64_t N;              /* #Lambda_1 */
  int64_t M;              /* #Lambda_2 */
  int64_t n_lambda0;      /* #Lambda_0 (postponed along the tree) */
  int64_t nnz_factor;     /* entries of the stored lower factor (all fronts) */
  int64_t n_nodes;        /* dissection tree nodes (2^m - 1) */
  int32_t levels;         /* m */
  int32_t kernel_dim;     /* detected dimension of ker(S22) (Sec. 3, rank revealing) */
  int32_t gcr_iters;      /* block GCR iterations of the last hf_schur */
  int32_t solve_iters;    /* block GCR iterations of the last hf_solve */
  double  gcr_relres;     /* max column |R|/|B| reached by the last hf_schur */
  double  solve_relres;   /* same for the last hf_solve */
  double  factor_flops;   /* dense LDL^T flops of the fronts actually factorized */
  int64_t front_bytes;    /* device bytes of the front arena */
  int32_t delay_retries;  /* times the delay capacity had to be grown */
  int32_t precision;      /* form used */
  double  trailing_flops; /* algorithmic flops of the trailing (Schur) updates of the fronts:
                             sum over panels of 2 x width x (lower-triangle entries updated) */
  int64_t solve_factor_entries; /* factor entries one forward (or backward) sweep of the K11
                             solve reads */
  /* which code paths the last calls took (for tests and profiles): */
  int32_t panel_cluster;  /* largest thread-block cluster of the pivoted panel (CTAs per front) */
  int32_t panel_global;   /* tree levels whose largest front ran the global-memory panel */
  int32_t sweep_blocks;   /* largest number of 64-row diagonal blocks of one front in the sweeps */
  int32_t ldlt_kernel;    /* S22 LDL^T of the last hf_schur: 0 none (M = 0), 1 one cluster with S22
                             in distributed shared memory, 2 cooperative grid, 3 one block */
  int32_t gcr_restarts;   /* block GCR runs since the last hf_schur began (its own and those of the
                             hf_solve calls after it) that stagnated above gcr_tol with the
                             emulated FP64 products and were run again with the native ones */
} hf_info;

/* Kernel classes of the profile (hf_get_profile). */
enum {
  HF_PROF_SCALE = 0, HF_PROF_ASSEMBLE, HF_PROF_PANEL, HF_PROF_TRAILING, HF_PROF_LAMBDA,
  HF_PROF_TRSV_FWD, HF_PROF_TRSV_BWD, HF_PROF_SPMM, HF_PROF_GRAM, HF_PROF_BLOCK_UPDATE,
  HF_PROF_SCHUR, HF_PROF_DENSE_LDLT, HF_PROF_VECTOR,
  /* the launches around the classes above, kept apart so that each class above is one kernel:
     panel_swap = the row interchanges applied after a level's panels, sweep_io = gathers and
     scatters of the solve vectors around each sweep level, tc_prep = operand preparation of
     the tensor-core products (exponents, slices and split-K reductions of the emulated FP64
     products; the BF16 split of the panel for the tensor-core trailing update),
     diag_inverse = the inverses of the factor's 64 x 64 diagonal blocks for the sweeps;
     panel_global = the panels of the levels that take the global-memory panel kernel
     (panel = the cluster panel) */
  HF_PROF_PANEL_SWAP, HF_PROF_SWEEP_IO, HF_PROF_TC_PREP, HF_PROF_DIAG_INV, HF_PROF_PANEL_GLOBAL, HF_NPROF
};

/* Fill *opts with the defaults listed above.  Returns HF_ERR_ARG if opts is NULL. */
int hf_default_opts(hf_opts* opts);

/*
 * Changes opts.spin_limit of an existing context (the other options are fixed at
 * hf_analyze).  limit >= 0; 0 restores the built-in limit.  Takes effect at the next call
 * that runs a triangular sweep.  A wait that gave up voids the solves of the current
 * factor (HF_ERR_TIMEOUT from every later solve) until the next hf_factorize.
 * Errors: HF_ERR_ARG (null ctx, negative limit).
 */
int hf_set_spin_limit(hf_ctx* ctx, int limit);

/* Human-readable name of an HF_* code (static string). */
const char* hf_error_string(int code);

/*
 * Analysis (Sec. 2.2, Fig. 1): nested-dissection bisection tree of 2^m - 1 index
 * sets Lambda_l, elimination tree, front row structures and assembly maps.
 * Host only: touches no GPU.
 *   L       order of K (> 0)
 *   rowptr  host, L+1 entries, CSR row pointers of the pattern
 *   col     host, rowptr[L] entries, column indices (sorted per row)
 *   coords  host, nullable, L x dim row-major coordinates of the unknowns; when
 *           given the bisection is geometric, otherwise graph based (BFS levels)
 *   dim     1..3 when coords is given
 *   opts    host, nullable (defaults)
 *   out     receives a new context (free with hf_free)
 * Errors: HF_ERR_ARG, HF_ERR_PATTERN.
 */
int hf_analyze(int64_t L, const int64_t* rowptr, const int32_t* col, const double* coords,
               int dim, const hf_opts* opts, hf_ctx** out);

/*
 * Numeric factorization, Alg. 1 step 1 (Sec. 2.1-2.2): scales Kbar (Sec. 2), factorizes
 * the fronts in the precision of opts.precision with symmetric max-|diag| pivoting and
 * threshold postponing (tau), refactorizes the postponed set Lambda_0 and enlarges the
 * hard part by n_enlarge.  Re-callable with new values for the same pattern.
 *   vals  device, rowptr[L] doubles: the values of Kbar in the CSR order given to
 *         hf_analyze.  Read during the call only.
 *   tau   threshold (> 0); overrides opts.tau for this and later calls.
 * On return the split (N, M, Lambda_2) is known on the host (one small D2H copy).
 * Errors: HF_ERR_ARG, HF_ERR_NUMERIC, HF_ERR_CUDA, HF_ERR_OOM, HF_ERR_CAPACITY.
 */
int hf_factorize(hf_ctx* ctx, const double* vals, double tau);

/*
 * LDU form with row signs (Sec. 2.1 writes the rank-1 update with the pivot's column
 * and row separately; the Stokes matrix [A B^T; -B delta D] of Sec. 4.2 is unsymmetric).
 * Declares Kbar = J S with J = diag(sign) and S symmetric, as for [A B^T; -B delta D]
 * = diag(I, -I) [A B^T; B -delta D].  Every Schur complement of J S is J times that of
 * S, so the pivots, postponed sets, Lambda_2, X12 and the solution of Kbar x = b are
 * those of S with the right-hand side J b.  The next hf_factorize therefore factorizes
 * K = J Q Kbar Q (= Q S Q) and hf_solve scales b by J Q; the getters (factor, X12, S22,
 * its LDL^T, Q^-1) describe that K, whose S22 is J_2 times the Schur complement of
 * Q Kbar Q.  The kernel basis is that of Kbar.
 *   sign  host, L entries, each +1 or -1, copied before the call returns; NULL clears
 *         the signs (Kbar symmetric again).
 * The values given to hf_factorize must make J Kbar symmetric; the library does not
 * check it.  Invalidates an earlier factorization (hf_factorize must run again).
 * Errors: HF_ERR_ARG (null ctx, an entry other than +1 / -1), HF_ERR_CUDA, HF_ERR_OOM.
 */
int hf_set_row_signs(hf_ctx* ctx, const int8_t* sign);

/*
 * Schur generation, Alg. 1 steps 2-5: for HF_PREC_MIXED, X12 = K11^-1 K12 by block GCR
 * (Sec. 3.5) in FP64 preconditioned by the FP32 factor, S22 = K22 - K21 X12 in FP64;
 * for the other forms S22 is taken from the factor.  Then S22 is factorized in FP64
 * by LDL^T with complete symmetric pivoting (Bunch-Parlett, 1x1 / 2x2 blocks), which puts
 * the null pivots last, and its kernel dimension is detected.
 * Errors: HF_ERR_STATE, HF_ERR_NOT_CONVERGED (results still usable), HF_ERR_CUDA, HF_ERR_OOM,
 * HF_ERR_TIMEOUT (a bounded wait of a tensor-core product or of a triangular sweep gave
 * up: the results are not valid; a sweep timeout persists until the next hf_factorize).
 */
int hf_schur(hf_ctx* ctx);

/*
 * Solve Kbar x = b, Alg. 2 (block forward/backward substitution; the K11 solve by the
 * same block GCR for HF_PREC_MIXED).  Kernel pivots of S22 are treated as zero, so for
 * singular Kbar and consistent b the particular solution is returned.
 *   nrhs     number of right-hand sides (>= 1)
 *   b, ldb   device, column-major L x nrhs, leading dimension ldb >= L
 *   x, ldx   device, column-major L x nrhs output, ldx >= L (may not alias b)
 * Errors: HF_ERR_STATE, HF_ERR_ARG, HF_ERR_NOT_CONVERGED, HF_ERR_CUDA, HF_ERR_OOM,
 * HF_ERR_TIMEOUT (as for hf_schur).
 */
int hf_solve(hf_ctx* ctx, int nrhs, const double* b, int64_t ldb, double* x, int64_t ldx);

/*
 * The lower-precision solve of Sec. 3.1-3.2, W = Q^-1 R with Q the factor of K11 (Eq. 1),
 * on m vectors of the scaled unknowns (K = Q_s Kbar Q_s): R is cast to the factor's
 * precision, solved by forward / diagonal / backward substitution, and cast back.
 *   m     number of vectors (>= 1)
 *   R, W  device, row-major L x m (the m entries of an unknown contiguous); rows of
 *         Lambda_2 are ignored in R and set to zero in W.  W may not alias R.
 * The FP32 forms run each tree level of the forward and backward substitution as one
 * launch whose blocks wait (bounded) for the diagonal blocks they read; a wait that gives
 * up is reported as HF_ERR_TIMEOUT (sticky until the next hf_factorize).
 * Errors: HF_ERR_STATE (before hf_factorize), HF_ERR_ARG, HF_ERR_CUDA, HF_ERR_OOM,
 * HF_ERR_TIMEOUT.
 */
int hf_precond(hf_ctx* ctx, int m, const double* R, double* W);

/*
 * The two dense products of the block GCR of Sec. 3.5 (Alg. 5) on their own, computed
 * the way the iteration computes them (FP64-accurate BF16 tensor-core products when
 * hf_opts.fp64_gemm == 0, native FP64 kernels otherwise), with ctx's stream and
 * scratch; ctx is any context from hf_analyze (no factorization needed).
 *   hf_gram_fp64:   G = scale * A^T B;  A: L x ma, B: L x mb (device, row-major),
 *                   G: ma x mb (device, row-major, overwritten).
 *   hf_update_fp64: Y = (Yinit ? Yinit : Y) + sgn * A C;  A, Y, Yinit: L x m, C: m x m
 *                   (device, row-major); Y may not alias A or C; Yinit may be Y or NULL.
 * Both synchronise the stream before returning.
 * Errors: HF_ERR_ARG (sizes), HF_ERR_OOM, HF_ERR_CUDA, HF_ERR_TIMEOUT (a bounded
 * tensor-core wait gave up; the output is not valid).
 */
int hf_gram_fp64(hf_ctx* ctx, int64_t L, int ma, int mb, const double* A, const double* B, double* G, double scale);
int hf_update_fp64(hf_ctx* ctx, int64_t L, int m, const double* A, const double* C, double* Y, const double* Yinit,
                   double sgn);

/*
 * The iterations on K11 X = B compared in the paper (Sec. 3.3-3.5, Fig. 2), each with the
 * lower-precision factor Q of hf_factorize as preconditioner, on the scaled unknowns:
 *   method 0  block GCR on all m columns at once (Alg. 5; what hf_schur uses)
 *   method 1  GCR one column at a time (Alg. 4)
 *   method 2  iterative refinement (Alg. 3: x0 = Q^-1 b, then x += Q^-1 (b - K11 x))
 *   m        number of columns (>= 1)
 *   B, X     device, row-major L x m (the m entries of an unknown contiguous); the rows of
 *            Lambda_2 must be zero in B and are zero in X.  X is overwritten.
 *   maxit    iterations at most (>= 1); stop when max_k |r_k| / |b_k| <= opts.gcr_tol
 *   hist     host, maxit + 1 doubles or NULL: hist[n] = max_k |r_k| / |b_k| after n
 *            iterations (hist[0]: after x0 = Q^-1 b); entries past *iters are untouched
 *   iters    host, iterations done (or NULL)
 * Errors: HF_ERR_STATE (before hf_factorize), HF_ERR_ARG, HF_ERR_NOT_CONVERGED (X and
 * hist still valid), HF_ERR_CUDA, HF_ERR_OOM, HF_ERR_TIMEOUT.
 */
int hf_k11_iterate(hf_ctx* ctx, int method, int m, const double* B, double* X, int maxit, double* hist, int* iters);

/*
 * hf_precond without any device allocation (the paper has no counterpart; this is a
 * deployment variant).  For callers that must not allocate device memory while they
 * run: a process whose device memory is owned by another allocator (a framework's
 * caching pool that reserved it), a real-time loop where cudaMalloc's implicit device
 * synchronisation is not acceptable, or a host thread that may not grow the context's
 * buffers.  It computes exactly what hf_precond computes (same kernels, same arguments
 * and layout: R, W device, row-major L x m), but its scratch (the per-front solve
 * vectors and the precision-cast copies) lives in one file-scope device array of
 * 64 MiB that every GPU loading the library holds until the process exits.
 *  - Limits: rejects with HF_ERR_ARG any call whose scratch exceeds 64 MiB, i.e.
 *    (4 or 8) * m4 * (front rows of all fronts) + (12 or 8) * L * m bytes, m4 = m rounded
 *    up to a multiple of 4, plus 8 bytes per (64-row diagonal block, 64-column tile) for
 *    the sweeps' tickets and flags, rounded.
 *  - The first call on a device looks up the array's device address (with that device
 *    current); make that first call before any stream capture.  Call with the device of
 *    the hf_factorize that built the context current.
 *  - Every call on a device shares the array and leaves its contents behind; the solve
 *    writes every value it reads before reading it and clears the sweeps' tickets and
 *    flags (cudaMemsetAsync) before each sweep.  Two calls whose GPU work overlapped
 *    would race on the array.  Within one process the entry point prevents that: it
 *    holds a library lock from its start until it has synchronised its stream, so
 *    concurrent host callers run one after another.
 *  - Allocates nothing: no cudaMalloc / cudaFree / allocating library call.  Profiling
 *    events are not recorded for this call.
 * Errors: HF_ERR_ARG (bad argument or scratch above the limit), HF_ERR_STATE (before
 * hf_factorize), HF_ERR_CUDA, HF_ERR_TIMEOUT (as for hf_precond).
 */
int hf_precond_noalloc(hf_ctx* ctx, int m, const double* R, double* W);

/*
 * Adjoint of the solve with respect to the matrix values.  For x = Kbar^-1 b and an
 * objective J(x), with lam = Kbar^-T dJ/dx (for a symmetric Kbar, i.e. without row
 * signs, lam comes from hf_solve with the same factor), dJ/dKbar_ij = -sum_r lam_i^r x_j^r for every stored
 * entry (i, j).  Writes that gradient in CSR order (the order given to hf_analyze).
 *   nrhs       number of columns of x and lam (>= 1)
 *   x, ldx     device, column-major L x nrhs, ldx >= L
 *   lam, ldl   device, column-major L x nrhs, ldl >= L
 *   grad_vals  device, rowptr[L] doubles (overwritten)
 * Errors: HF_ERR_ARG, HF_ERR_STATE (before hf_factorize), HF_ERR_CUDA.
 */
int hf_values_adjoint(hf_ctx* ctx, int nrhs, const double* x, int64_t ldx, const double* lam, int64_t ldl,
                      double* grad_vals);

/*
 * The split of Alg. 1 step 1 (host outputs, any may be NULL):
 *   pivot_order  L entries: the elimination order Pi (Lambda_1 in order Pi_1, then
 *                Lambda_2 ascending)
 *   lambda2      M entries, ascending
 *   info         summary
 */
int hf_get_split(hf_ctx* ctx, int32_t* pivot_order, int32_t* lambda2, hf_info* info);

/* Summary of the last calls (host output). */
int hf_get_info(hf_ctx* ctx, hf_info* info);

/*
 * The dissection tree (Sec. 2.2), nodes in elimination order (children first):
 *   parent    n_nodes entries, index of the parent node, -1 for the root (host)
 *   set_ptr   n_nodes+1 entries; set_idx[set_ptr[t] .. set_ptr[t+1]) = Lambda_t (host)
 *   set_idx   L entries (host)
 * Call with all three NULL to only read info->n_nodes through hf_get_info.
 */
int hf_get_tree(hf_ctx* ctx, int32_t* parent, int64_t* set_ptr, int32_t* set_idx);

/*
 * Pivot decisions of the last hf_factorize (host outputs):
 *   node_ptr   n_nodes+2 entries; pivots of node t (elimination order) are
 *              piv[node_ptr[t] .. node_ptr[t+1]) in the order chosen; entry
 *              n_nodes is the refactorization of Lambda_0
 *   piv        (number of eliminated indices) entries, original indices
 *   moved      n_enlarge entries (fewer if fewer pivots exist): the indices moved
 *              into Lambda_2 by the enlargement, in elimination order
 *   n_moved    receives their count
 */
int hf_get_pivots(hf_ctx* ctx, int64_t* node_ptr, int32_t* piv, int32_t* moved, int32_t* n_moved);

/*
 * Candidate order of every front after the factorization, to replay its decisions:
 *   node_ptr  n_nodes+2 entries; cand[node_ptr[t] .. node_ptr[t+1]) are the pivot candidates
 *             of node t (Lambda_t; entry n_nodes is the Lambda_0 stage) in final front order
 *   cand      original indices (host)
 *   counts    2*(n_nodes+1) entries (k_t, nact_t): cand[0, k) were eliminated in that order,
 *             cand[k, nact) were postponed by the ratio test, cand[nact, end) were postponed one
 *             at a time by the null-pivot test (the first one skipped is last)
 */
int hf_get_pivot_events(hf_ctx* ctx, int64_t* node_ptr, int32_t* cand, int32_t* counts);

/*
 * The lower-precision factor of K11 (Eq. 1), for checking: column j of L for pivot
 * piv[j] (same order as hf_get_pivots).  Host outputs:
 *   col_ptr  (#pivots + 1) entries
 *   row_idx  col_ptr[#pivots] entries: original row indices (strictly later pivots
 *            and postponed rows, Lambda_2 rows included)
 *   val      same count, values of L (unit diagonal not stored), as double
 *   d        #pivots entries, the pivots
 * Call with row_idx = val = NULL to get only col_ptr (sizes).
 */
int hf_get_factor(hf_ctx* ctx, int64_t* col_ptr, int32_t* row_idx, double* val, double* d);

/*
 * Results of hf_schur (device outputs, FP64):
 *   x12  L x M row-major (ldx12 >= M): X12 in original row indices, zero on Lambda_2 rows
 *   s22  M x M row-major, rows/cols in ascending Lambda_2 order
 */
int hf_get_x12(hf_ctx* ctx, double* x12, int64_t ldx12);

/*
 * Kernel basis of K-bar (mixed form, after hf_schur; Sec. 3: the null pivots of the S22
 * LDL^T carry the kernel of K).  For each of the info.kernel_dim null pivot directions v
 * of the S22 factorization, n2 = P Lf^-T v is a null vector of S22 and
 * Q [-X12 n2 ; n2] (Lambda_2 rows from n2, the others from -X12 n2, unscaled by Q) is a
 * null vector of K-bar.  basis: device, L x kernel_dim column-major, ldb >= L (not
 * normalised, not orthogonalised).  HF_ERR_STATE before hf_schur or for the FP64 / FP32
 * forms (no X12 is kept there); nothing is written when kernel_dim = 0.
 */
int hf_get_kernel_basis(hf_ctx* ctx, double* basis, int64_t ldb);
int hf_get_s22(hf_ctx* ctx, double* s22);

/*
 * LDL^T factors of S22 (complete symmetric pivoting; host outputs, M entries each, M*M for lf):
 *   perm   row order: P^T S22 P = Lf D Lf^T with row i of the factor = S22 row perm[i]
 *   lf     M x M row-major unit lower triangular Lf
 *   dblk   M entries: 1 = 1x1 block start, 2 = 2x2 block start, 0 = second row of a 2x2
 *   dval   M x 2 row-major: [d_ii, d_i,i+1] (the 2x2 off-diagonal for a 2x2 start)
 *   null   M entries: 1 where the pivot magnitude was declared null (kernel)
 */
int hf_get_s22_factor(hf_ctx* ctx, int32_t* perm, double* lf, int32_t* dblk, double* dval, int32_t* null_piv);

/*
 * Tracing.  Kernel launches are always counted per class.  With hf_profile(ctx, 1) every
 * launch is also bracketed by CUDA events recorded on the context's stream; hf_get_profile
 * synchronises that stream, returns per class the summed device time (ms, HF_NPROF
 * entries), the launch count, and the algorithmic flops and bytes of those launches (what
 * the operation must compute and move: e.g. 2 N M^2 for an N x M by M x M block update,
 * the factor entries read by a triangular sweep) since the last call, and resets them.
 * Any output may be NULL.  hf_profile_name gives the class names (static strings).
 */
int hf_profile(hf_ctx* ctx, int enable);
int hf_get_profile(hf_ctx* ctx, double* ms, int64_t* launches, double* flops, double* bytes);
const char* hf_profile_name(int cls);

/*
 * Batched form: the same step on n independent systems (distinct contexts, each from its
 * own hf_analyze), run concurrently.  A pool of host worker threads takes the contexts
 * in order; a context created with cuda_stream = NULL runs on the worker's own
 * non-blocking stream for the duration of the call, otherwise on its own stream.  Every
 * context's work is complete when the call returns.  The per-system semantics are those
 * of hf_factorize / hf_schur / hf_solve on the same context (Alg. 1 and 2 per system,
 * each with its own tau and its own Lambda_2); systems do not interact.
 *   ctxs      n distinct contexts
 *   vals_dev  n device pointers (K values of system i, CSR order of its pattern)
 *   b_dev, x_dev  n device pointers: right-hand sides / solutions (as hf_solve), with
 *             leading dimensions ldb[i], ldx[i] (NULL: system i's L)
 *   status    optional, n entries: the HF_* status of each system
 * Returns HF_OK if every system succeeded, else the first non-OK status in index order
 * (HF_ERR_ARG for NULL or repeated contexts, nothing run).  Workers: HF_BATCH_WORKERS
 * environment variable (default 8).
 */
int hf_factorize_batched(hf_ctx* const* ctxs, int n, const double* const* vals_dev, double tau, int32_t* status);
int hf_schur_batched(hf_ctx* const* ctxs, int n, int32_t* status);
int hf_solve_batched(hf_ctx* const* ctxs, int n, int nrhs, const double* const* b_dev, const int64_t* ldb,
                     double* const* x_dev, const int64_t* ldx, int32_t* status);

/* Release every device and host buffer of the context.  NULL is ignored. */
void hf_free(hf_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* HF_H */
