/*
 * kep.h - C ABI of the GB300 k-th eigenpair library.
 *
 * Problem (Section 1, Eq. 1.1): A x = lambda B x with n x n sparse symmetric A and symmetric
 * positive definite B sharing one sparsity pattern (Section 4.1); eigenvalues ascending,
 * k 1-based.  The library's hot path is the numeric phase of the sparse LDL^T factorization
 * P Q (A - sigma B) Q^T P^T = L D L^T (Algorithm 1', the factorization step), which gives the
 * Sylvester inertia count nu_sigma(A, B) = nu_0(D, I) (Section 2.1) and the shifted solves of
 * the shift-and-invert Lanczos stage (Eq. 2.5).
 *
 * Conventions for every call:
 *  - All floating point is IEEE double (FP64).  Integers are int64_t unless stated.
 *  - Inputs are caller-owned and only read.  kep_analyze copies what it needs; after it returns
 *    the caller may free its arrays.  Outputs go to caller-allocated buffers.
 *  - The context owns every device allocation it makes (factors, fronts, workspaces) and frees
 *    them in kep_destroy.  One context serves one host thread at a time; it is not thread-safe.
 *  - Errors are returned as kep_status codes; nothing aborts, traps or throws across the ABI.
 *    After an error the context stays usable unless the code is KEP_ERR_CUDA.
 *  - ptr_kind selects where a vector argument lives: KEP_HOST (pageable or pinned host memory;
 *    the call copies in and out and synchronises) or KEP_DEVICE (device memory on the context's
 *    device; the call is ordered on the context's stream and synchronises before returning).
 */
#ifndef KEP_H
#define KEP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct kep_ctx kep_ctx;

typedef enum {
  KEP_OK = 0,
  KEP_ERR_INVALID = 1,        /* bad argument: null pointer, index out of range, duplicate entry */
  KEP_ERR_NOT_SPD = 2,        /* B is not positive definite (its inertia at 0 is not (0, 0, n)) */
  KEP_ERR_SINGULAR = 3,       /* an exact zero pivot: sigma is an eigenvalue; inertia still filled */
  KEP_ERR_NOT_CONVERGED = 4,  /* an iteration hit its limit */
  KEP_ERR_CLUSTER = 5,        /* Algorithm 3 could not validate the interval (clustered/multiple) */
  KEP_ERR_POOL = 6,           /* delayed pivots exceeded the front slack (internal re-plan failed) */
  KEP_ERR_TIMEOUT = 7,        /* a bounded device-side wait gave up */
  KEP_ERR_CUDA = 8,           /* a CUDA runtime call failed */
  KEP_ERR_NONFINITE = 9,      /* a NaN or Inf appeared in a pivot */
  KEP_ERR_NOMEM = 10          /* device or host allocation failed */
} kep_status;

enum { KEP_HOST = 0, KEP_DEVICE = 1 };

/* kep_analyze flags */
enum {
  KEP_PATTERN_FULL = 0,       /* CSR holds both triangles */
  KEP_PATTERN_LOWER = 1,      /* CSR holds the lower triangle (col <= row) only */
  KEP_ORDER_GRAPH = 2,        /* ignore coords; order by graph breadth-first levels */
  KEP_ORDER_REFINED = 4       /* nested dissection with a search over balanced cuts on every
                                 long axis and minimum-vertex-cover separators (slower analysis,
                                 less fill; see kep_symbolic_info) */
};

/* Inertia of a factored matrix: counts of negative, zero and positive eigenvalues of D, and the
 * number of pivots that were passed from a front to its parent ("delayed"). */
typedef struct {
  int64_t neg, zero, pos, delayed;
} kep_inertia;

/* Symbolic-analysis facts (Section 4.3: #nzf predicts the run time). */
typedef struct {
  int64_t n, nnz;             /* order, stored entries of the full symmetric pattern */
  int64_t nfronts, nlevels;   /* fronts of the assembly tree, tree height + 1 */
  int64_t max_front;          /* largest symbolic front order m */
  int64_t nnz_factor;         /* #nzf: entries of L and D (symbolic, without delays) */
  double flops_factor;        /* multiply-add = 2 flops, symbolic count for one factorization */
  int64_t front_bytes;        /* device bytes of one factor slot's front storage */
  int64_t replans;            /* times the storage was re-planned because delayed pivots overflowed
                                 a front's slack (only the overflowing fronts grow) */
  int64_t cb_bytes;           /* device bytes of the contribution-block arena (the peak of the
                                 level schedule's first-fit placement) */
  int64_t slot_bytes;         /* device bytes one factorization holds: front storage, pivots, D,
                                 solve vectors, contribution blocks and the L21 workspace */
} kep_info;

/* Parameters of Algorithm 4 (Section 3.4) and of the stage-3 iteration. */
typedef struct {
  int64_t m_max;              /* Algorithm 1' stop: nu_u - nu_l <= m_max (paper: 20) */
  double tau_res;             /* Algorithm 3 relative residual 2-norm tolerance (paper: 1e-10) */
  double tau_diff;            /* Algorithm 3 relative difference 2-norm tolerance (paper: 1e-10) */
  int64_t max_lanczos;        /* Algorithm 2 iteration limit */
  int64_t max_si;             /* Algorithm 3 iteration limit */
  const double* start_vectors;/* optional host array of 2n: v_1 (Algorithm 2) then v~_1
                                 (Algorithm 3); NULL draws them from a counter-based generator */
  uint64_t seed;              /* seed of that generator */
  int32_t init;               /* initial interval: KEP_INIT_LANCZOS (Algorithm 2, default) or
                                 KEP_INIT_GERSHGORIN (an interval holding the whole spectrum,
                                 the variant of Section 4.2) */
  int32_t nshift;             /* shifts per Algorithm 1' step: 1 bisection (default), s > 1
                                 multisection into s + 1 equal parts */
  int32_t solve_precision;    /* Algorithm 3's factor and solves: KEP_SOLVE_F64 (default) or
                                 KEP_SOLVE_F32_IR (KEP_SCHUR_FP32 factor, every solve refined in
                                 FP64 to a normwise backward error <= 1e-13; the inertia
                                 factorizations of stages 1-2 stay FP64-accurate) */
  int32_t b_factor;           /* where B's factor (the B-solves of Algorithms 2 and 3) lives:
                                 KEP_BFACTOR_AUTO (default) its own factor slot when a second
                                 factor fits in free device memory, else shared;
                                 KEP_BFACTOR_SHARED the slot of the A - sigma B factorizations
                                 (the largest problems): B is factored once (which also shows it
                                 positive definite), later B-solves that find the slot replaced
                                 run conjugate gradients to a relative residual of 1e-14 and
                                 factor B again only if 500 iterations do not reach it;
                                 KEP_BFACTOR_OWN its own slot always */
  int32_t split;              /* Algorithm 1''s shift rule: KEP_SPLIT_BISECT (default: the paper's
                                 midpoints, or multisection with nshift) or KEP_SPLIT_INTERP (the
                                 interpolating rule of kep_interp_point, one shift per step; the
                                 root-finder variant of Sections 2.1 and 5; nshift must be 1) */
} kep_params;

enum { KEP_INIT_LANCZOS = 0, KEP_INIT_GERSHGORIN = 1 };
enum { KEP_BFACTOR_AUTO = 0, KEP_BFACTOR_SHARED = 1, KEP_BFACTOR_OWN = 2 };
enum { KEP_SOLVE_F64 = 0, KEP_SOLVE_F32_IR = 1 };
enum { KEP_SPLIT_BISECT = 0, KEP_SPLIT_INTERP = 1 };

/* Report of kep_kth_eigenpair. */
typedef struct {
  double lambda;              /* lambda_k */
  double eta;                 /* error bound of Proposition 3 for lambda_k */
  double rel_res;             /* ||(A - lambda B) x||_2 / ||x||_2, computed explicitly */
  double rel_res_normwise;    /* ||A x - lambda B x||_2 / (||A||_inf ||x||_2) */
  double sigma_lo, sigma_hi;  /* interval after Algorithm 1' */
  int64_t nu_lo, nu_hi;       /* its inertia counts */
  double init_lo, init_hi;    /* interval from Algorithm 2 */
  int64_t init_nu_lo, init_nu_hi;
  int64_t n_factor;           /* numeric factorizations (B included) */
  int64_t n_lanczos;          /* Algorithm 2 iterations */
  int64_t n_bisect;           /* Algorithm 1' iterations */
  int64_t n_si_iter;          /* Algorithm 3 iterations */
  int64_t si_iter_bound;      /* first Algorithm 3 iteration with inclusion and disjointness */
  double t_stage[3];          /* seconds spent in stages 1, 2, 3 */
  int64_t n_refine;           /* refinement corrections in Algorithm 3 (KEP_SOLVE_F32_IR) */
  double solve_berr;          /* largest final backward error of those solves */
  int64_t cap_cols;           /* Lanczos basis columns available to Algorithms 2 and 3 (fewer than
                                 max_lanczos / max_si + 2 when device memory is short) */
  double last_res;            /* Algorithm 3's tests at its last iteration: largest residual of the
                                 interval's pairs from the Lanczos relation (Eq. 2.12), */
  double last_diff;           /* largest relative difference (Eq. 3.5; -1 when not formed), */
  double last_res_explicit;   /* largest explicit residual of the last confirmation (0 if none) */
  int32_t restarted;          /* 1 when Algorithm 3 ran a second time with every shifted solve
                                 refined in FP64: the explicit residuals had stopped above tau_res (a
                                 floor set by the solves' rounding) although the Lanczos relation
                                 and the relative differences had converged; n_si_iter then counts
                                 the second run's iterations */
  int32_t reserved;
} kep_report;

void kep_default_params(kep_params* p);

/*
 * kep_analyze - symbolic phase (Section 3.3: "fill-reducing ordering Q and symbolic
 * factorization ... recycled for other shifted matrices"; task (i) of Section 4.3).
 *
 * n        order of A and B (n >= 1).
 * rowptr   n+1 row offsets into colind (int64, rowptr[0] = 0), CSR of the common pattern.
 * colind   column indices (int32, 0 <= c < n); no duplicates within a row.
 * a_val, b_val  values of A and B on that pattern (double, rowptr[n] each).  Both must be
 *          symmetric; with KEP_PATTERN_LOWER only entries with colind <= row are given.
 * flags    KEP_PATTERN_FULL / KEP_PATTERN_LOWER, optionally | KEP_ORDER_GRAPH, | KEP_ORDER_REFINED.
 * coords   optional 3n doubles (x, y, z of the atom owning each row; an ordering hint only).
 * out      receives the new context.
 * Computes the nested-dissection ordering, the assembly tree, front structures and index maps
 * on the host, and uploads them and the values to the current CUDA device.  Errors:
 * KEP_ERR_INVALID for a malformed pattern, KEP_ERR_NOMEM, KEP_ERR_CUDA.
 */
kep_status kep_analyze(int64_t n, const int64_t* rowptr, const int32_t* colind,
                       const double* a_val, const double* b_val, int flags,
                       const double* coords, kep_ctx** out);

/*
 * kep_analyze_hermitian - as kep_analyze for a complex Hermitian pencil (A, B), B positive
 * definite (the pencil of Eq. 1.1 with complex entries, e.g. tight-binding models with Peierls
 * phases).
 *
 * a_val, b_val  complex values on the pattern, interleaved (re, im): 2*rowptr[n] doubles each.
 *          Hermitian: with KEP_PATTERN_FULL the (j, i) entry must be the conjugate of (i, j); with
 *          KEP_PATTERN_LOWER only col <= row is given and the upper triangle is its conjugate.
 *          Diagonal entries must have zero imaginary part.
 * The context holds the real symmetric embedding of order 2n, [[Re A, -Im A], [Im A, Re A]] and
 * likewise for B, which has every eigenvalue of (A, B) twice.  On such a context:
 *  - kep_factor / kep_factor_pencil / kep_factor_multi report the counts of (A, B) (half those of
 *    the embedding); a count that is odd on the embedding (an eigenvalue within rounding of sigma)
 *    is returned as KEP_ERR_SINGULAR;
 *  - kep_solve, kep_solve_refined, kep_spmv and kep_grad take and return complex vectors of order n
 *    interleaved (re, im) (2n doubles each; device pointers 16-byte aligned); kep_kth_eigenpair
 *    takes k <= n and returns x_k interleaved with x^H B x = 1; its start vectors, when given, are
 *    2 * 2n doubles of the embedding;
 *  - kep_set_values takes complex values in this call's layout (diagonal imaginary parts zero);
 *    kep_get_info reports the embedding (order 2n).
 * Errors: as kep_analyze; KEP_ERR_INVALID also for a diagonal entry with an imaginary part.
 */
kep_status kep_analyze_hermitian(int64_t n, const int64_t* rowptr, const int32_t* colind,
                                 const double* a_val, const double* b_val, int flags,
                                 const double* coords, kep_ctx** out);

/*
 * Arithmetic of the deferred Schur update (the update of a front's trailing matrix with a window of
 * up to 256 pivots, Algorithm 1' factorization step).
 *   KEP_SCHUR_FP64      FP64 FMA tiles everywhere.
 *   KEP_SCHUR_EMULATED  (default, min_front = 512) fronts of order >= min_front form the
 *                       update from bf16 tensor-core products of an exact splitting of L and L*D
 *                       into eight 8-bit pieces per entry (column balancing, per-row power-of-two
 *                       scales, exact FP32 level sums, exact int64 combination): as accurate as an
 *                       FP64 update, on the tensor pipe.
 *   KEP_SCHUR_FP32      a reduced-precision factor for kep_solve_refined: fronts of order >=
 *                       min_front take the tensor-core update with four 8-bit pieces per entry
 *                       (10 bf16 products per multiply-add instead of 36; about 31 bits of each
 *                       row's scale), smaller fronts FP32 FMA tiles (pivot blocks and L21 stay
 *                       FP64); backward error near FP32 rounding.  Its inertia is that of a nearby
 *                       matrix, so inertia counts should come from the other modes.
 * Takes effect at the next factorization.  Errors: KEP_ERR_INVALID.
 */
enum { KEP_SCHUR_FP64 = 0, KEP_SCHUR_EMULATED = 1, KEP_SCHUR_FP32 = 2 };
kep_status kep_set_schur_mode(kep_ctx* ctx, int mode, int64_t min_front);

/*
 * kep_set_schur_tile - edge of the tiles of the Schur updates that do not run on the tensor cores
 * (fronts below the tensor-core threshold; FP64, or FP32 in KEP_SCHUR_FP32): 64 (default) or 32.
 * A tile-shape choice with no effect on the result's accuracy, for the autotuner.  Takes effect at
 * the next factorization.  Errors: KEP_ERR_INVALID.
 */
kep_status kep_set_schur_tile(kep_ctx* ctx, int edge);

/* The current Schur settings of ctx (any pointer may be NULL): mode (KEP_SCHUR_*), tensor-core
 * threshold, tile edge. */
kep_status kep_get_schur_config(const kep_ctx* ctx, int* mode, int64_t* min_front, int* tile);

/* Fill *info with the symbolic facts of ctx. */
kep_status kep_get_info(const kep_ctx* ctx, kep_info* info);

/*
 * kep_symbolic_info - the symbolic facts kep_analyze would compute for this pattern (ordering,
 * assembly tree, #nzf and flop count of one factorization; Section 4.3 task (i)), on the host
 * only: no device is needed and nothing is kept.  Arguments as kep_analyze without the values.
 * Errors: KEP_ERR_INVALID for a malformed pattern.
 */
kep_status kep_symbolic_info(int64_t n, const int64_t* rowptr, const int32_t* colind, int flags,
                             const double* coords, kep_info* info);

/*
 * kep_set_stream - order all of ctx's device work on the given cudaStream_t (NULL: the legacy
 * default stream).  The stream must belong to the context's device.
 */
kep_status kep_set_stream(kep_ctx* ctx, void* stream);

/*
 * kep_factor - numeric LDL^T of the permuted A - sigma*B and the inertia count read off D, the
 * factorization step of Algorithm 1' (Section 2.1: Sylvester's law of inertia).
 *
 * The factor stays in ctx for kep_solve until the next kep_factor.  out->neg is nu_sigma(A, B),
 * the number of eigenvalues below sigma.  Returns KEP_ERR_SINGULAR (with *out filled) when an
 * exact zero pivot occurs, i.e. sigma is an eigenvalue; KEP_ERR_NONFINITE on NaN/Inf input.
 */
kep_status kep_factor(kep_ctx* ctx, double sigma, kep_inertia* out);

/*
 * kep_factor_multi - inertia of A - sigmas[i] B for ns shifts (the evaluations of one
 * multisection step of Algorithm 1'); out[i] receives each; the factor of the last shift stays
 * for kep_solve.  Shifts that are eigenvalues (exact zero pivot) keep their counts with
 * zero > 0.  Errors: as kep_factor, KEP_ERR_INVALID for ns < 1 or null pointers.
 */
kep_status kep_factor_multi(kep_ctx* ctx, const double* sigmas, int32_t ns, kep_inertia* out);

/*
 * kep_factor_pencil - as kep_factor for the matrix ca*A + cb*B (kep_factor(sigma) is
 * ca = 1, cb = -sigma; ca = 0, cb = 1 factors B, task (ii) of Section 4.3).
 */
kep_status kep_factor_pencil(kep_ctx* ctx, double ca, double cb, kep_inertia* out);

/*
 * kep_solve - x = (ca*A + cb*B)^{-1} rhs with the last factorization (the solves of Eq. 2.5 and,
 * with the B factor, of Eq. 2.2): x = P^T Q^T L^{-T} D^{-1} L^{-1} Q P rhs.
 *
 * rhs, x   n*nrhs doubles, column-major (column i at offset i*n); may alias.
 * ptr_kind KEP_HOST or KEP_DEVICE for both rhs and x.
 * Returns KEP_ERR_INVALID if no factorization is present, KEP_ERR_SINGULAR if it had a zero pivot.
 */
kep_status kep_solve(kep_ctx* ctx, const double* rhs, double* x, int64_t nrhs, int ptr_kind);

/*
 * kep_solve_refined - x = (ca*A + cb*B)^{-1} b by GMRES-based iterative refinement with the last
 * factor S (typically a KEP_SCHUR_FP32 one) as preconditioner: x_0 = solve(b); each outer step
 * takes r = b - M x in FP64 (sparse products) and runs up to 20 right-preconditioned GMRES steps
 * on M S^{-1} (one solve each), until the normwise backward error
 *   ||b - M x||_inf / (||M||_inf ||x||_inf + ||b||_inf),  ||M||_inf <= |ca| ||A||_inf + |cb| ||B||_inf,
 * is <= tol or max_iter GMRES steps were taken.  One right-hand side (n doubles, ptr_kind memory).
 * The first call allocates a Krylov workspace of 41 n doubles, kept until kep_destroy.
 * *iters (GMRES steps taken) and *berr (final backward error) may be NULL.  Returns
 * KEP_ERR_NOT_CONVERGED if tol was not reached (x holds the last iterate), KEP_ERR_NOMEM if the
 * workspace cannot be allocated, KEP_ERR_INVALID without a valid factor.
 */
kep_status kep_solve_refined(kep_ctx* ctx, const double* rhs, double* x, int ptr_kind, double tol,
                             int32_t max_iter, int32_t* iters, double* berr);

/*
 * kep_spmv - ax = A x and bx = B x (the products of Eqs. 2.2 and 2.5), original numbering.
 * x, ax, bx: n doubles each; ax or bx may be NULL to skip it.
 */
kep_status kep_spmv(kep_ctx* ctx, const double* x, double* ax, double* bx, int ptr_kind);

/*
 * kep_kth_eigenpair - Algorithm 4 (Section 3.4): Algorithm 2 (initial interval from Ritz
 * values), Algorithm 1' (bisection to at most m_max eigenvalues), Algorithm 3 (shift-and-invert
 * Lanczos with modified Ritz vectors x_{i,2}, Proposition 3 bounds, index validation).
 *
 * k        target index, 1 <= k <= n.
 * params   NULL for the paper's settings (m_max 20, tau_res = tau_diff = 1e-10).
 * lambda   receives lambda_k.
 * x        optional host array of n doubles: x_k, B-normalized (x^T B x = 1).
 * report   optional.
 * Returns KEP_ERR_CLUSTER when Algorithm 3 cannot validate the interval within max_si
 * iterations (multiple or clustered eigenvalues, Section 3.4), KEP_ERR_NOT_SPD if B's
 * factorization shows B is not positive definite.  The report is written on errors too, with
 * what the stages reached.
 */
kep_status kep_kth_eigenpair(kep_ctx* ctx, int64_t k, const kep_params* params, double* lambda,
                             double* x, kep_report* report);

/*
 * kep_multisection_points - the shifts of one step of Algorithm 1' on [lo, hi) (host only, no
 * device): nshift = 1 gives the midpoint (lo + hi) / 2 (the paper's bisection); nshift > 1 the
 * points lo + (hi - lo) q / (nshift + 1), q = 1 .. nshift (multisection, the evaluations of one step
 * being independent factorizations).  sigmas: nshift doubles, increasing.  Errors: KEP_ERR_INVALID
 * for nshift < 1, lo >= hi or a null pointer.
 */
kep_status kep_multisection_points(double lo, double hi, int32_t nshift, double* sigmas);

/*
 * kep_multisection_update - the bracket update of one step of Algorithm 1' (host only): given the
 * bracket [*lo, *hi) with *nu_lo < k <= *nu_hi (nu = the inertia count nu_sigma(A, B), Section 2.1)
 * and the counts nus of the first `count` shifts of kep_multisection_points, in increasing order,
 * keep the part [sigma_{q-1}, sigma_q) whose counts bracket k (k 1-based).  The counts may stop at
 * the first one >= k.  Errors: KEP_ERR_INVALID when k is not bracketed, a shift lies outside the
 * bracket or out of order, or the counts decrease with sigma (a non-monotone count means a wrong
 * factorization); the bracket is then left unchanged.
 */
kep_status kep_multisection_update(int64_t k, int32_t count, const double* sigmas, const int64_t* nus,
                                   double* lo, double* hi, int64_t* nu_lo, int64_t* nu_hi);

/*
 * Interpolating shift rule for Algorithm 1' (host only, no device).  Section 2.1 notes that
 * bisection's midpoint may be replaced by another root-finder on the count function nu(sigma)
 * (non-decreasing, integer-valued), and Section 5 that any derivative-free method that keeps the
 * root bracketed locates lambda_k.  This rule is such a method; its output contract is Algorithm
 * 1''s (nu_lo < k <= nu_hi, nu_hi - nu_lo <= m_max), reached in fewer factorizations when the
 * density of eigenvalues is smooth.
 *
 * Each step moves the end farther from k in count: the target count is k - h (lower end) or
 * k - 1 + h (upper end), h = max(1, m_max / 4), and the shift is the linear interpolation of sigma
 * between the ends at their weighted counts w_lo, w_hi, kept (hi - lo) / 2^20 away from both ends.
 * The weights are the true counts, except that an end kept through two consecutive steps has its
 * count distance to k halved (the Illinois modification of regula falsi).  Safeguard: when the
 * count width has not halved over the last three steps, the next shift is the midpoint.
 *
 * The state is caller-allocated; its fields are read-only to the caller (kep_interp_init sets
 * them, kep_interp_update advances them).
 */
typedef struct {
  double lo, hi;              /* the bracket: nu(lo) = nu_lo < k <= nu_hi = nu(hi) */
  int64_t nu_lo, nu_hi;
  double w_lo, w_hi;          /* the ends' counts as the interpolation weighs them */
  int64_t width[4];           /* the last count widths nu_hi - nu_lo, newest at width[nwidth - 1] */
  int32_t nwidth;             /* entries of width in use (at most 4) */
  int32_t last;               /* the end the previous step replaced: +1 upper, -1 lower, 0 none */
  int32_t bisect_next;        /* the next shift is the safeguard's midpoint */
  int32_t reserved;
} kep_interp_state;

/* kep_interp_init - a new state for the bracket [lo, hi) of k.  Errors: KEP_ERR_INVALID unless
 * lo < hi and nu_lo < k <= nu_hi, or for a null pointer. */
kep_status kep_interp_init(int64_t k, double lo, double hi, int64_t nu_lo, int64_t nu_hi, kep_interp_state* st);

/* kep_interp_point - the next shift (strictly inside the bracket).  Errors: KEP_ERR_INVALID for
 * m_max < 1, a bracket that does not hold k, or a null pointer; KEP_ERR_CLUSTER when lo and hi are
 * adjacent doubles (more than m_max eigenvalues within rounding of one value). */
kep_status kep_interp_point(const kep_interp_state* st, int64_t k, int64_t m_max, double* sigma);

/* kep_interp_update - the count nu = nu(sigma) at the shift kep_interp_point gave: the end on
 * sigma's side is replaced and the weights and safeguard advance.  Errors: KEP_ERR_INVALID (state
 * unchanged) when sigma is not strictly inside the bracket or nu lies outside [nu_lo, nu_hi] (a
 * count that is not monotone in sigma means a wrong factorization). */
kep_status kep_interp_update(kep_interp_state* st, int64_t k, double sigma, int64_t nu);

/*
 * kep_set_values - new values of A and B on the pattern given to kep_analyze (same layout:
 * a_val, b_val as there, host arrays; complex interleaved for kep_analyze_hermitian).  The
 * symbolic analysis is kept; the factors of the old values become invalid.  Errors:
 * KEP_ERR_INVALID, KEP_ERR_CUDA.
 */
kep_status kep_set_values(kep_ctx* ctx, const double* a_val, const double* b_val);

/*
 * kep_grad - derivatives of an eigenvalue lambda of A x = lambda B x with respect to the stored
 * values of A and B (Hellmann-Feynman theorem; the paper states the eigenpair problem of
 * Section 2 and has no derivative counterpart): with s = x^T B x,
 *   d_lambda_d_a[e] = lambda_bar * x_i x_j / s,   d_lambda_d_b[e] = -lambda * d_lambda_d_a[e]
 * for every entry e = (i, j) in the layout of kep_analyze's a_val, each entry an independent
 * variable; with KEP_PATTERN_LOWER an off-diagonal entry stands for (i, j) and (j, i) and gets
 * twice that.  x: the eigenvector (any nonzero scaling; n doubles), lambda_bar: the factor the
 * derivatives are multiplied by (the incoming gradient).  Either output may be NULL.  Vectors
 * in ptr_kind memory.  On a Hermitian context (kep_analyze_hermitian) x is complex (interleaved),
 * s = x^H B x, and each output holds 2 doubles per entry: G_ij = lambda_bar * x_i conj(x_j) / s
 * (and -lambda G_ij), so that d lambda = sum Re(conj(G_ij) dM_ij) (doubled for a lower off-diagonal
 * entry).  Errors: KEP_ERR_INVALID (null pointers, x^T B x <= 0), KEP_ERR_NOMEM, KEP_ERR_CUDA.
 */
kep_status kep_grad(kep_ctx* ctx, double lambda, const double* x, double lambda_bar, double* d_lambda_d_a,
                    double* d_lambda_d_b, int ptr_kind);

/*
 * Kernel accounting.  Classes (index into the arrays): 0 assembly (zero, scatter, extend-add),
 * 1 pivot panel, 2 L21 rows, 3 apply, 4 FP64 Schur tiles, 5 inertia reduction, 6 forward solve,
 * 7 backward solve, 8 permutation, 9 SpMV, 10 vector operations of the eigenpair driver,
 * 11 splitting for the tensor-core Schur update, 12 tensor-core Schur update.
 * launches[] always counts every kernel launch of ctx since the last reset.  ms[] sums the
 * CUDA-event time of each launch (events recorded on ctx's stream around the launch) and is
 * filled only while timing is enabled.  flops[] is the algorithmic work counted on the device:
 * class 4 the FP64 multiply-adds x 2 of its updates, class 12 the bf16 tensor-core products x 2
 * it issued; flush_fp64_equivalent_flops is the FP64 update work those products carried out.
 */
#define KEP_NKCLASS 13
typedef struct {
  int64_t launches[KEP_NKCLASS];
  double ms[KEP_NKCLASS];
  double flops[KEP_NKCLASS];
  double flush_fp64_equivalent_flops;
  int64_t total_launches;
} kep_timing;

/* Run each pass of pivot steps of a factorization level (the panel, L21, apply and update
 * launches of up to a few hundred steps) as a CUDA graph captured at its first use and replayed by
 * later factorizations of the same context (1, the default), or as separate launches (0).  The
 * graphs are captured on ctx's stream; with event timing enabled the launches are always issued
 * separately.  Synchronises ctx's stream.  Errors: KEP_ERR_INVALID. */
kep_status kep_set_graphs(kep_ctx* ctx, int enable);

/* Enable (1) or disable (0) per-launch event timing; synchronises ctx's stream. */
kep_status kep_set_timing(kep_ctx* ctx, int enable);

/* Restrict event timing to the classes whose bit is set in mask (bit c: class c; all bits set by
 * default); launch counts and flops are kept for every class.  Synchronises ctx's stream. */
kep_status kep_set_timing_classes(kep_ctx* ctx, unsigned int mask);

/* Copy the counters into *out; reset (1) zeroes them afterwards.  Synchronises ctx's stream. */
kep_status kep_get_timing(kep_ctx* ctx, kep_timing* out, int reset);

/*
 * kep_dense_inertia_noalloc - inertia (neg, zero, pos) of the dense symmetric matrix a - sigma*b,
 * for callers that must not allocate device memory at the point of the call (a framework that
 * owns all device memory through its own pool, a real-time loop that cannot afford cudaMalloc's
 * synchronisation or failure).  The paper has no counterpart: it is a convenience form of the
 * front elimination (Bunch-Kaufman, alpha = (1+sqrt 17)/8) for one small dense pencil, outside the
 * sparse path.
 *
 * n        order, 1 <= n <= 512 (larger n returns KEP_ERR_INVALID).
 * a, b     device pointers, column-major n x n with leading dimension lda >= n; only the lower
 *          triangles are read; caller-owned, not modified.
 * sigma    the shift.
 * stream   cudaStream_t to run on (NULL: legacy default stream); the call synchronises it.
 * out      host array of 3 int64: neg, zero, pos.
 * The working copy lives in a fixed 2 MiB device array reserved by the library on every GPU that
 * loads it, for the life of the process; no allocator is called.  The first call on each device
 * looks up that array's device address, so make the first call on a device before any stream
 * capture.  All calls share the array: calls that overlap on the GPU race and must be serialised
 * by the caller.  Errors: KEP_ERR_INVALID (bad argument or n > 512), KEP_ERR_CUDA.
 */
kep_status kep_dense_inertia_noalloc(int64_t n, const double* a, const double* b, int64_t lda,
                                     double sigma, void* stream, int64_t* out);

/* Release every resource of ctx (NULL is accepted). */
void kep_destroy(kep_ctx* ctx);

/* Static description of a status code. */
const char* kep_status_str(kep_status s);

#ifdef __cplusplus
}
#endif
#endif /* KEP_H */
