/*
 * hif.h -- C ABI of the GB300 (sm_103a) HIF-IE library.
 *
 * The library factors the dense matrix of a discretized integral equation
 * (Sec. 1, Eq. (1.1); Sec. 3.1, Eq. (3.1))
 *
 *      A = diag(a) + diag(b) K diag(c),     K_ij = G(|x_i - x_j|) w_j   (i != j),
 *                                          K_ii = integral of G over the cell of x_i,
 *
 * with G the Laplace kernel of Eq. (1.4) (kernel_id 0: -log(r)/(2 pi) in 2D,
 * kernel_id 1: 1/(4 pi r) in 3D), by the hierarchical interpolative
 * factorization HIF-IE (Sec. 4, Algorithms 4.1 and 4.2, with the second-kind
 * modifications of Sec. 4.4 and, for symmetric A, the one-sided proxy
 * matrices of Sec. 5), and applies the factorization F ~ A and its inverse
 * in factored form (Eqs. (4.1), (4.2)).  The cell of DOF i is the
 * square/cube of volume w_i centred at x_i; its self term is the exact
 * integral in closed form.
 *
 * Conventions common to every call
 *  - Pointers: arrays may live in host memory or in device memory of the
 *    current CUDA device; the library inspects each pointer and copies host
 *    arrays to the device itself.  The caller keeps ownership of every array
 *    it passes; the handle copies what it keeps.
 *  - Points are N x dim, row-major (x_0, y_0[, z_0], x_1, ...), FP64.
 *  - Vectors are FP64, column-major N x nrhs with leading dimension ld >= N.
 *  - Work is issued on the stream given in hif_options (NULL = legacy default
 *    stream); every call returns after its results are complete.
 *  - Errors are returned as hif_status, never thrown.  On failure *out is
 *    set to NULL and nothing is leaked.  A handle is not thread-safe.
 */
#ifndef HIF_H
#define HIF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hif_handle_s* hif_handle;

typedef enum {
    HIF_OK = 0,
    HIF_EINVAL = 1,      /* bad argument (size, pointer, option)               */
    HIF_ENOMEM = 2,      /* device or host allocation failed                   */
    HIF_ESINGULAR = 3,   /* zero pivot in an elimination block (Lemma 2.1)     */
    HIF_ENUMERIC = 4,    /* NaN/Inf produced or met in the inputs              */
    HIF_ECUDA = 5,       /* a CUDA runtime call failed                         */
    HIF_ETIMEOUT = 6,    /* a bounded device-side wait gave up                 */
    HIF_ENOTCONV = 7     /* iterative refinement / GMRES missed its tolerance  */
} hif_status;

typedef struct {
    int dim;                /* 2 or 3                                                      */
    int leaf_occupancy;     /* max DOFs per finest cell; sets the depth L (default 64)     */
    int second_kind;        /* 1: Sec. 4.4 modifications (rho_g tolerance, split groups)   */
    int precision;          /* 0: FP64 factorization, 1: FP32 factorization                */
    int fractional_levels;  /* 1: HIF-IE (cells + edges[/faces]); 0: RSF (cells only)      */
    int skip_levels;        /* skip the fractional sublevels of the first skip_levels levels */
    int proxy_points;       /* number of proxy points P (64 in 2D, 512 in 3D, Sec. 3.3)    */
    double proxy_radius;    /* proxy radius in units of the cell width (1.5, Sec. 3.3)     */
    const double* proxy_dirs; /* P x dim unit vectors (host or device); NULL = 2D circle   */
    double fp32_tol_floor;  /* FP32 factorization: local ID tolerance >= this (2^-17)      */
    double root_lo[3];      /* root box lower corner; used when root_width > 0            */
    double root_width;      /* <= 0: bounding cube of the DOF cells                        */
    void* stream;           /* cudaStream_t                                                */
    int direct_precision;   /* direct sum on uniform grids: 0 = paired FP32 (~2^-48 relative),
                               1 = FP64, 2 = tensor cores on exact 8-bit digits (~2^-55 of
                               max|K| max|x| per term, FP64 class sums; default);
                               other point sets always use FP64                          */
    int use_graphs;         /* capture the sweeps of each (operation, nrhs) in a CUDA graph
                               and replay it (default 1)                                   */
    int autotune;           /* time the candidate CTA sizes of every sublevel's sweep after
                               the factorization and keep the fastest (the sweep's
                               arithmetic does not depend on it); in FP32 factorizations
                               also time 16 and 32 rows per fold chunk for every box-width
                               bucket on its first sighting in the process and keep the
                               faster (default 1)                                         */
    int symmetric;          /* 1 (default): when b == c and all weights are equal, A is
                               symmetric and the one-sided proxy matrix Y'_c = [A_{cN,c};
                               Y_{cE,c}] is compressed (Sec. 5; same ID, half the rows);
                               0: always the full Y_c of Eq. (3.3)                        */
    double wavenumber;      /* kernel_id 2: the wavenumber k of (i/4) H_0^(1)(k r) (> 0)     */
    int ldl;                /* 1 (default): when the symmetric shortcut applies, factor the
                               diagonal blocks B_rr by LDL with 1 x 1 symmetric pivots and
                               keep X only (Y = X^T; Sec. 5); a block whose pivot fails the
                               Bunch-Kaufman 1 x 1 test falls back to LU. 0: always LU   */
} hif_options;

typedef struct {
    int64_t N;
    int dim;
    int levels;             /* L                                                           */
    int sublevels;          /* skeletonization sublevels actually run                      */
    int64_t top_size;       /* |s_L|                                                       */
    int64_t factor_bytes;   /* m_f: bytes held by the factors (T, L, D, U, X, Y, top LU)   */
    int64_t skeletons[64];  /* per sublevel: sum of skeleton sizes                         */
    int64_t redundant[64];  /* per sublevel: sum of redundant sizes                        */
    int64_t boxes[64];      /* per sublevel: number of non-empty boxes                     */
    int kinds[64];          /* per sublevel: 0 cell, 1 face, 2 edge                        */
    int max_box[64];        /* per sublevel: largest |c|                                   */
    double factor_seconds;  /* wall time of hif_factor                                     */
    double flops;           /* algorithmic FP work of the factorization: per box 2 m n^2
                               for the QR fold of the m x n proxy matrix, and 6 k^2 r +
                               6 k r^2 + 2 r^3 / 3 for the Lemma 2.4 blocks, the LU of
                               Lemma 2.1, X, Y and the Schur update; 4 |s_L|^3 / 3 for the
                               top block                                                  */
    double kernel_evals;    /* kernel evaluations spent on the proxy matrices Y_c          */
    int64_t proxy_rows;     /* rows of all proxy matrices compressed (Y_c or Y'_c)         */
    int symmetric_problems; /* problems whose A was symmetric and compressed through Y'_c  */
    int64_t ldl_boxes;      /* eliminated boxes factored by LDL (Sec. 5), top blocks included */
    int64_t ldl_fallbacks;  /* LDL boxes refactored by LU after a pivot failed the 1x1 test */
} hif_stats_t;

/* Defaults for dimension dim (2 or 3): occupancy 64, second_kind 1, FP64,
 * fractional levels on, proxy 64 points (2D) / 512 (3D) at radius 1.5,
 * fp32_tol_floor 2^-17, bounding-cube root box, default stream, direct sums
 * on the tensor cores (direct_precision 2), graph-replayed and autotuned
 * sweeps, symmetric shortcut and LDL on. */
hif_status hif_options_default(int dim, hif_options* opt);

/*
 * hif_factor -- HIF-IE of A (Algorithm 4.1 for dim 2, Algorithm 4.2 for dim 3).
 *   points   N x dim collocation points (row-major)
 *   weights  N cell volumes w_j (quadrature weights of Eq. (3.1))
 *   a, b, c  N samples of the coefficient functions of Eq. (1.1)
 *   kernel_id 0 (2D log kernel) or 1 (3D 1/r kernel), must match dim
 *   eps      base relative precision of the interpolative decompositions (>= 0)
 *   opt      options (NULL = hif_options_default(2))
 *   out      receives the handle (NULL on failure)
 * Errors: HIF_EINVAL on bad sizes/options, HIF_ENOMEM, HIF_ESINGULAR when an
 * elimination block B_rr (Lemma 2.4) or the top block is singular,
 * HIF_ENUMERIC on non-finite input or results, HIF_ECUDA.
 */
hif_status hif_factor(const double* points, int64_t N, const double* weights,
                      const double* a, const double* b, const double* c,
                      int kernel_id, double eps, const hif_options* opt, hif_handle* out);

/*
 * One problem of a batch: the arrays of hif_factor for one integral equation.
 */
typedef struct {
    const double* points;   /* N x dim, row-major */
    int64_t N;
    const double* weights;
    const double* a;
    const double* b;
    const double* c;
} hif_problem;

/*
 * hif_factor_batched -- HIF-IE of `count` independent problems in one handle.
 * Every problem gets its own tree; the boxes of the same sublevel (counted
 * from the leaves) of all problems are skeletonized in the same kernel
 * launches (Sec. 3.1: boxes of one level are independent).  The handle's
 * operator is block diagonal: vectors are the concatenation of the problems'
 * vectors in the order given (problem q at rows off_q .. off_q + N_q - 1,
 * off_q = N_0 + ... + N_{q-1}), and every call below acts on all problems at
 * once.  hif_solve_refined with method 0 judges the residual problem by
 * problem and column by column.  Options and errors as for hif_factor.
 */
hif_status hif_factor_batched(int count, const hif_problem* problems, int kernel_id, double eps,
                              const hif_options* opt, hif_handle* out);

/* y = F x  (Eq. (4.1) first line; generalized FMM).  x, y: N x nrhs, ld >= N. */
hif_status hif_apply(hif_handle h, const double* x, double* y, int64_t nrhs, int64_t ld);
/* y = F^T x: the transpose of Eq. (4.1)'s product, every factor transposed
 * and the order reversed (Sec. 3.1: the transposes of the unit-triangular
 * factors are unit-triangular with the off-diagonal block transposed).
 * x, y: N x nrhs, ld >= N. */
hif_status hif_apply_transpose(hif_handle h, const double* x, double* y, int64_t nrhs, int64_t ld);
/* x = F^{-1} b  (Eq. (4.1) second line; direct solver / preconditioner). */
hif_status hif_solve(hif_handle h, const double* b, double* x, int64_t nrhs, int64_t ld);
/* x = F^{-T} b: Eq. (4.1)'s inverse transposed, i.e. the adjoint solve
 * (Sec. 3.1 inverts each factor by negating its off-diagonal block; the
 * transpose keeps that form).  b, x: N x nrhs, ld >= N. */
hif_status hif_solve_transpose(hif_handle h, const double* b, double* x, int64_t nrhs, int64_t ld);

/*
 * hif_matvec -- y = A x (trans = 0) or y = A^T x (trans = 1) by direct
 * summation over all N^2 pairs, exactly the operator the handle factored
 * (A = diag(a) + diag(b) K diag(c) of Eq. (1.1) discretized as in Sec. 3.1,
 * Eq. (3.1): same quadrature, same self terms), with FP64 inputs and
 * outputs; the operator the refinement and GMRES of Sec. 5 apply.  On a
 * full uniform grid the sum is a convolution with an FP64 table; it is
 * accumulated in FP64 (direct_precision = 1), in paired FP32 with
 * error-free transformations, good to ~2^-48 relative per operation
 * (direct_precision = 0), or on the tensor cores from exact signed 8-bit
 * digits of table and sources with integer class sums (direct_precision = 2;
 * HIF_ETIMEOUT if a pipeline wait in the kernel expired).  x, y: N x nrhs,
 * ld >= N.
 */
hif_status hif_matvec(hif_handle h, int trans, const double* x, double* y,
                      int64_t nrhs, int64_t ld);

/*
 * hif_matvec_digits -- hif_matvec with the tensor-core sum limited to the
 * digit classes 0..classes-1 (classes = 4, 5 or 6; 8 is hif_matvec itself): the
 * pairs of table digit s and source digit t with s + t < classes, the shorter
 * sums that hif_solve_refined's method 0 takes for residuals that do not
 * decide convergence (Sec. 5 refinement; the full sum decides).  Dropped
 * pairs are below (classes + 1) 2^(-2 - 8 classes) x 16 max|K| max|c x| per
 * term, of mean zero over the terms: relative errors of y are ~6e-9
 * (classes 4), ~2e-11 (classes 5) and ~1e-13 (classes 6) on the 2D
 * log-kernel grid with Gaussian sources.  Problems
 * without the tensor-core sum (direct_precision != 2, or points not on a full
 * grid) compute their one sum.  HIF_EINVAL for other class counts.
 */
hif_status hif_matvec_digits(hif_handle h, int trans, int classes, const double* x, double* y,
                             int64_t nrhs, int64_t ld);

/*
 * hif_solve_refined -- solve A u = f (trans = 0) or A^T u = f (trans = 1) to
 * relative residual |f - A u| / |f| <= tol per column, with F^{-1} as right
 * preconditioner: method 0 = iterative refinement u += F^{-1}(f - A u),
 * method 1 = right-preconditioned restarted GMRES(20) with modified
 * Gram-Schmidt (Sec. 5).  Residuals use hif_matvec (FP64 direct sum); with
 * the tensor-core sum, method 0 computes the residuals that do not decide
 * convergence by the short sums of hif_matvec_digits: the first residual
 * with 5 classes (FP32 factorization) or 6 (FP64), a later one, while its
 * predicted size is above 10 tol, with the fewest classes whose estimated
 * error (a bound on the sum's relative error per unit of the grid table's
 * spread max|T| sqrt(#T) / |T|_2, times that spread, times |b K c u| / |f|)
 * stays below 0.05 tol and 1e-4 of the residual; none when tol < 1e-11 or
 * HIF_SHORT_RESIDUAL=0.  Every residual at or below tol, at maxit, or whose
 * error estimate misses that bound is recomputed in full.
 *   iters   (may be NULL) receives the largest iteration count over columns
 *   relres  (may be NULL) receives the largest final relative residual
 * Returns HIF_ENOTCONV (with u holding the last iterate) when maxit is reached.
 */
hif_status hif_solve_refined(hif_handle h, int trans, const double* f, double* u,
                             int64_t nrhs, int64_t ld, double tol, int maxit, int method,
                             int* iters, double* relres);

/*
 * hif_adjoint_gradients -- the coefficient part of the adjoint method for a
 * loss L(u) with A u = f (A = diag(a) + diag(b) K diag(c)): given the solution
 * u and the adjoint solution lam = A^{-T} dL/du (N x nrhs each, column-major,
 * leading dimension ld, host or device), writes the N-vectors
 *   grad_a = -sum_col lam .* u,
 *   grad_b = -sum_col lam .* (K (c .* u)),     K (c u)   = (F u - a u) / b,
 *   grad_c = -sum_col u .* (K^T (b .* lam)),   K^T (b l) = (F^T lam - a lam) / c,
 * with the factorization's fast apply F standing in for A (accurate to e_a);
 * dL/df = lam itself.  Outputs are host or device arrays of N doubles.
 * HIF_EINVAL when some b_i or c_i is zero.  Not a step of the paper: the
 * solver's adjoint for gradient-based use.
 */
hif_status hif_adjoint_gradients(hif_handle h, const double* u, const double* lam, int64_t nrhs, int64_t ld,
                                 double* grad_a, double* grad_b, double* grad_c);

/*
 * hif_error_estimates -- the a posteriori operator errors of Sec. 5 by power
 * iteration on E^T E: norms[0] ~ |A|, norms[1] ~ |A - F| and
 * norms[2] ~ |I - A F^{-1}| (2-norms), so e_a = norms[1] / norms[0] and
 * e_s = norms[2].  Each run starts from v0 / |v0| (N values, host or device;
 * the paper uses a standard uniform random vector), takes w = E v,
 * u = E^T w, the estimate sqrt(|u|) and v = u / |u|, and stops when the
 * estimate moved by at most rtol of itself (the paper: 1e-2) or after maxit
 * steps.  A is applied by the direct sum of hif_matvec, F by the factored
 * form.  For a batched handle the operators are block diagonal and each norm
 * is the largest over the problems.
 *   iters   (may be NULL) receives the three step counts
 * Returns HIF_ENOTCONV (norms still filled) when a run reached maxit, and
 * HIF_EINVAL for a zero or non-finite v0.
 */
hif_status hif_error_estimates(hif_handle h, const double* v0, double rtol, int maxit,
                               double* norms, int* iters);

/*
 * hif_eliminated_dofs -- the DOFs eliminated at one sublevel: the redundant
 * sets of the skeletonized boxes (Lemma 2.4), box by box, each in ascending
 * order within its column groups, as 0-based indices into the handle's DOFs.
 * Sublevels 0 .. hif_stats().sublevels - 1 are the skeletonization
 * sublevels; sublevel hif_stats().sublevels is the top block s_L.  With
 * out == NULL only *count is written; otherwise out (host or device) must
 * hold cap >= *count ints.  HIF_EINVAL for a sublevel out of range.
 */
hif_status hif_eliminated_dofs(hif_handle h, int sublevel, int* out, int64_t cap, int64_t* count);

/* Factorization statistics (Sec. 5 columns |s_L|, m_f, t_f and ranks per sublevel). */
hif_status hif_stats(hif_handle h, hif_stats_t* st);

/* Releases every resource the handle owns: the factors of Eq. (4.1) (T, L,
 * D, U, X, Y per box and the top block's LU of Sec. 3.1, level L), the
 * Schur-complement interaction store and the work buffers.  NULL is
 * accepted.  Waits for the handle's stream first; always returns HIF_OK. */
hif_status hif_destroy(hif_handle h);

/* Static, human-readable name of a status code.  Error reporting of this
 * library; the paper has no counterpart. */
const char* hif_status_string(hif_status s);

/* Detail of the last failure on the calling thread (file:line and the CUDA
 * error text when the failure came from the runtime); empty if none.  Error
 * reporting of this library; the paper has no counterpart. */
const char* hif_last_error(void);

/* Number of CUDA kernels the library has launched in this process so far
 * (all handles, all threads); callers difference it around a region.  For
 * measurement; the paper has no counterpart. */
uint64_t hif_kernel_launches(void);

/* Device time of the tensor-core direct-sum kernel (direct_precision = 2),
 * for measurement: while enabled, every launch of the full digit set (not the
 * short sums of hif_matvec_digits) is bracketed by a pair of CUDA events on
 * its own stream.  Each call returns in *ms the summed event time
 * and in *launches the number of launches recorded since the previous call
 * (either pointer may be NULL), synchronizing on the recorded events, and
 * then sets recording on (enable != 0) or off.  Process-wide; not
 * thread-safe against concurrent direct sums.  The paper has no counterpart. */
hif_status hif_kernel_timing(int enable, double* ms, int64_t* launches);

/* One kernel family of hif_kernel_profile. */
typedef struct {
    const char* name;       /* static name of the kernel family                         */
    int64_t ranges;         /* timed ranges (one launch or one launch group each)        */
    double ms;              /* summed CUDA-event time of those ranges                    */
    double flops;           /* algorithmic flops of the work in them (0: byte-bound)     */
    double bytes;           /* algorithmic bytes of the work in them (0: flop-bound)     */
} hif_profile_entry;

/* Per-kernel-family device time, for measurement: while enabled, the launches
 * of the factorization kernels, the sweeps (one range per whole sweep of an
 * operation) and the direct sums are bracketed by CUDA events on their
 * stream, with the algorithmic work counted from the sizes of the run
 * (per box 2 m n^2 flops for the QR fold of an m x n proxy matrix; QR to
 * rank k plus T = R1^{-1} R2 for the ID; 6 k^2 r + 6 k r^2 + 2 r^3/3 for an
 * elimination; for a large-box pivot step the bytes of the columns it
 * reads and writes; for a sweep the factor and vector bytes it moves; 2 N^2
 * flops per right-hand side for a direct sum).  Each call writes the sums
 * since the previous call into out[0 .. min(cap, *count)) (either may be
 * NULL), synchronizing on the recorded events, and then turns recording on
 * (enable != 0) or off.  Ranges on a stream being captured into a graph are
 * not recorded.  Process-wide; the paper has no counterpart. */
hif_status hif_kernel_profile(int enable, hif_profile_entry* out, int cap, int* count);

/*
 * hif_kernel_block -- entries A_ij = a_i delta_ij + b_i K_ij c_j (Eq. (3.1))
 * for i in rows[0..nr), j in cols[0..nc), written column-major to
 * out (nr x nc, leading dimension ldo >= nr).  All arrays on the device or all
 * on the host.  Entries are generated on demand (Sec. 3.1: A is never stored).
 */
hif_status hif_kernel_block(const double* points, int64_t N, int dim, const double* weights,
                            const double* a, const double* b, const double* c, int kernel_id,
                            const int32_t* rows, int64_t nr, const int32_t* cols, int64_t nc,
                            double* out, int64_t ldo, void* stream);

/*
 * hif_id_batched -- interpolative decompositions of `count` independent
 * matrices by column-pivoted Householder QR (Sec. 2.2, Lemma 2.2) with
 * adaptive rank: k = number of pivots with |R_jj| > tol[i] |R_11|.
 * The index and tolerance arrays (off, m, n, tol, poff, toff) are read on
 * the host and must be host memory; mats, k, perm and T may be host or device.
 *   mats    column-major m[i] x n[i] blocks at offsets off[i] (FP64)
 *   tol     per-matrix relative tolerance
 *   k       out: rank per matrix
 *   perm    out: n[i] column indices per matrix at poff[i]: skeletons in pivot
 *           order, then redundant columns in ascending order
 *   T       out: k[i] x (n[i]-k[i]) column-major at toff[i] (room for n[i]^2/4
 *           doubles must be reserved)
 * The pivot is the remaining column of largest 2-norm (ties: lowest index);
 * norms are recomputed exactly after each step.
 */
hif_status hif_id_batched(int count, const double* mats, const int64_t* off,
                          const int32_t* m, const int32_t* n, const double* tol,
                          int32_t* k, int32_t* perm, const int64_t* poff,
                          double* T, const int64_t* toff, void* stream);

/* One product of hif_gemm_batched_f32. */
typedef struct {
    const float* A;         /* device, column-major                                      */
    const float* B;         /* device, column-major                                      */
    float* C;               /* device, column-major, m x n                               */
    int64_t lda, ldb, ldc;  /* leading dimensions (>= the stored rows, >= 1)             */
    int32_t m, n, k;        /* op(A) is m x k, op(B) k x n                               */
    int32_t trans_a;        /* 0: op(A) = A (m x k stored); 1: op(A) = A^T (k x m stored) */
    int32_t trans_b;        /* 0: op(B) = B (k x n stored); 1: op(B) = B^T (n x k stored) */
    float alpha;
    int32_t beta;           /* 0: C = alpha op(A) op(B); 1: C += alpha op(A) op(B)       */
} hif_gemm_problem;

/*
 * hif_gemm_batched_f32 -- the dense contractions of the large-box elimination
 * of the FP32 factorization, exposed for testing and reuse: the products of
 * Lemma 2.4 (B_sr = A_sr - A_ss T, B_rr = A_rr - T^T B_sr - A_rs T,
 * B_rs = A_rs - T^T A_ss) and the Schur update -X Z of the skeleton block
 * (Sec. 3.1, Eq. (3.2)) are products of this form.  For every problem,
 *     C = beta C + alpha op(A) op(B)
 * on the tcgen05 tensor cores: FP32 values are split into three BF16 pieces
 * and the six piece products of weight >= 2^-16 are accumulated in FP32, so
 * the result has FP32 accuracy (error ~ k 2^-24 max|a| max|b|).  Problems run
 * concurrently and must not write overlapping C.  `problems` is a host array
 * (copied by the call); the matrices are device arrays.  Returns HIF_EINVAL
 * for negative sizes, NULL pointers where a product needs them, leading
 * dimensions too small or beta not 0 / 1; HIF_ETIMEOUT if a bounded wait of
 * the kernel ran out (C then undefined).  Synchronizes `stream`.
 */
hif_status hif_gemm_batched_f32(int count, const hif_gemm_problem* problems, void* stream);

/*
 * hif_id_batched_noalloc -- the batched interpolative decomposition of
 * hif_id_batched for callers that must not allocate device memory: services
 * that reserve their device memory once at start-up and may not fail on an
 * allocation later (a fixed memory budget), and callers that may not call
 * cudaMalloc or cudaFree at all because those calls can synchronize the
 * whole device and stall the work of other streams.  This entry point has
 * no counterpart in the paper; it calls no cudaMalloc, cudaFree or
 * allocating library routine.  It does wait for its own stream (below).
 *
 * Arguments, results and the rank rule are those of hif_id_batched, except
 * that every array must already live in device memory (HIF_EINVAL otherwise).
 * The QR work space is one fixed array in device memory that every GPU which
 * loads the library keeps until the process exits: about 8 MiB of matrix
 * copies plus 32 KiB of offsets.  Limits: at most 4096 matrices, at most 1024
 * columns per matrix, and sum over matrices of (m|1)*n <= 1,048,576 doubles;
 * larger inputs are rejected with HIF_EINVAL (hif_last_error says why) and
 * leave the outputs untouched; a later call within the limits is not
 * affected by a refused one.
 *
 * The first call on a device looks up that device's address of the array;
 * make that first call before any stream capture.  All calls share the one
 * array and it keeps the last call's contents; calls that overlap on the GPU
 * (different streams, different threads) race on it.  The call reads a
 * status word back from the array and returns after its results are
 * complete on `stream` (it synchronizes that stream, not the device).
 */
hif_status hif_id_batched_noalloc(int count, const double* mats, const int64_t* off,
                                  const int32_t* m, const int32_t* n, const double* tol,
                                  int32_t* k, int32_t* perm, const int64_t* poff,
                                  double* T, const int64_t* toff, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* HIF_H */
