/*
 * pthroot.h - C ABI of the GB300 inverse matrix p-th root engine.
 *
 * The library computes A^{-1/p} for a dense symmetric positive definite A (order n, root index p >= 1)
 * with the iteration of Lass, Kuehne and Plessl, "Using Approximate Computing for the Calculation of
 * Inverse Matrix p-th Roots" (arXiv:1703.02283), Sec. 2:
 *
 *     C_{k+1} = ((p + 1) C_k - C_k^{p+1} A) / p                         (Eq. 1)
 *
 * started from C_0 = (||A||_1 ||A||_inf)^{-1} A^T (Eq. 3), which satisfies ||I - C_0^p A||_2 < 1 (Eq. 2),
 * and run until ||I - C_k^p A||_F meets a tolerance. Every iterate is a polynomial in A, hence symmetric
 * and commuting with A; the library evaluates Eq. 1 in an order that yields the same iterates in exact
 * arithmetic (see pr_form) and computes only the upper-triangle tiles of products that are symmetric.
 *
 * Conventions shared by every entry point:
 *  - Matrices are n x n, FP64, row-major, leading dimension n. Because they are symmetric, row- and
 *    column-major storage coincide.
 *  - A matrix pointer may point to device memory or to host memory (pageable or pinned); the library
 *    copies with cudaMemcpyDefault (unified addressing tells the two apart) on the handle's stream.
 *  - A handle owns all of its device memory; the caller's buffers are never retained after a call
 *    returns. One handle may be used by one host thread at a time; distinct handles are independent.
 *  - Work is issued on the CUDA stream given to pr_init (NULL = the legacy default stream). Entry points
 *    that return host values (residuals, stop decisions) synchronise that stream.
 *  - Errors are reported by status code only; the library never exits, never traps on the device and
 *    never throws across the ABI. pr_last_error() gives a text for the last failing call on a handle.
 *  - All work runs in the library's own CUDA kernels on the current device; there is no CPU fallback.
 */
#ifndef PTHROOT_H
#define PTHROOT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pr_handle_s* pr_handle;

/* Status codes. PR_ESTAGNATED, PR_EMAXITER and PR_EINACCURATE are stop reasons, not failures: the handle
 * stays valid and iteration may be resumed (with another precision, for instance). */
typedef enum {
  PR_OK = 0,          /* tolerance met (pr_iterate/pr_solve) or call succeeded                          */
  PR_EINVAL = 1,      /* bad argument: n < 1, p < 1, unknown enum, NULL pointer, non-finite or
                         non-symmetric A, or tol < 0                                                       */
  PR_ENOTSPD = 2,     /* A is not positive definite: a non-positive diagonal entry, or a failed Cholesky
                         factorisation of one of its diagonal blocks of order 64 (principal submatrices of
                         an SPD matrix are SPD)                                                            */
  PR_ENOMEM = 3,      /* device allocation failed                                                        */
  PR_ECUDA = 4,       /* a CUDA runtime call or kernel launch failed                                     */
  PR_EDIVERGED = 5,   /* the residual became NaN or Inf                                                  */
  PR_ESTAGNATED = 6,  /* residual below stag_below stopped halving: the precision floor was reached      */
  PR_EMAXITER = 7,    /* the step budget of this call (or the handle's max_iter) ran out                 */
  PR_ETIMEOUT = 8,    /* a bounded device wait expired; the kernel returned without finishing            */
  PR_EGATE = 9,       /* a PR_C0_POLY guess failed its gate (Eq. 2 or positivity) and pr_options.gate_fallback
                         is 0                                                                              */
  PR_ESTATE = 10,     /* call out of order (e.g. pr_result before any pr_init)                           */
  PR_EUNSUPPORTED = 11, /* precision or form not available for this n / p                                */
  PR_EINACCURATE = 12  /* coupled form: the carried residual ||I - M_k||_F met tol, but the true residual
                          ||I - X_k^p A||_F evaluated at the stop (pr_stats.true_residual) did not. Rounding
                          errors carried in M since M_0 let X drift from the root (Eq. 3's M_0 spans
                          kappa^(p+1)); iterating further does not help. A stop reason: the handle stays valid */
} pr_status;

/* Arithmetic of the matrix products. */
typedef enum {
  PR_FP64 = 0,   /* native FP64 products (DMMA tensor instructions), FP64 accumulation                   */
  PR_EMU64 = 1,  /* FP64-accurate products from exact FP16 digit slices on the tcgen05 tensor cores:
                    every row of an operand is split into S (default 8) balanced base-256 digits with a
                    row exponent; the digit pairs with s + t <= S + 1 are exact FP16 tensor-core
                    products, summed per level s + t exactly in FP32 (drained every 128 terms) and then
                    in 128-bit integers, rounded once to FP64                                          */
  PR_FP32X = 2,  /* split-FP32 products: the first 3 of PR_EMU64's base-256 digit planes (24 bits per row,
                    the significand width of FP32), the 6 exact digit-pair products with s + t <= 4 summed
                    exactly, rounded once to FP64; about FP32 accuracy (2^-25 per term relative to the row and
                    column scales) at 1/6 of PR_EMU64's tensor work                                         */
  PR_BF16 = 3,   /* BF16 operands, FP32 accumulation in TMEM (tcgen05 kind::f16); FP64 master copies     */
  PR_FP8 = 4     /* E4M3 operands with a power-of-two FP32 scale per row (per column of the B operand,
                    the same for symmetric iterates; the largest |x| of a row maps into [128, 256)),
                    round to nearest even from FP64, FP32 accumulation in TMEM (tcgen05 kind::f8f6f4);
                    FP64 master copies, re-quantised before each FP8 product                              */
} pr_precision;

#define PR_NPREC 5 /* number of pr_precision values: arrays indexed by precision have this length */

/* Evaluation order of Eq. 1 (identical iterates in exact arithmetic). */
typedef enum {
  PR_FORM_AUTO = 0,     /* PR_FORM_NS for p = 1, PR_FORM_COUPLED otherwise                                */
  PR_FORM_COUPLED = 1,  /* X_{k+1} = X_k N_k, M_{k+1} = N_k^p M_k, N_k = ((p+1) I - M_k)/p, M_0 = C_0^p A;
                           the residual is ||I - M_k||_F (equal to ||I - X_k^p A||_F in exact arithmetic) */
  PR_FORM_NS = 2,       /* p = 1 only (Sec. 2, Newton-Schulz): C' = 2C - C (A C), residual ||I - A C||_F  */
  PR_FORM_LITERAL = 3   /* Eq. 1 as printed, C^{p+1} A right to left; unstable for ill-conditioned A      */
} pr_form;

/* Initial guess. */
typedef enum {
  PR_C0_EQ3 = 0,       /* Eq. 3: C_0 = A^T / (||A||_1 ||A||_inf)                                         */
  PR_C0_SCALED_I = 1,  /* C_0 = ||A||_1^{-1/p} I; one of the "different possible choices" of Sec. 2       */
  PR_C0_POLY = 2       /* C_0 = ||A||_1^{-1/p} q(A / ||A||_1), q(x) = c_0 + c_1 x + c_2 x^2 + c_3 x^3 with the
                          coefficients of pr_options.c0_coef (e.g. predicted by a pr_mlp from pr_features).
                          A gate checks it: if q <= 0 somewhere on [0, 1.05 rho] (rho: a power-iteration
                          estimate of ||A||_2 / ||A||_1, so C_0 might not be positive definite) or a
                          power-iteration estimate of ||I - C_0^p A||_2 (Eq. 2) is not below gate_max, the
                          handle falls back to Eq. 3 (pr_stats.c0 reports the guess used), or the call
                          returns PR_EGATE when pr_options.gate_fallback is 0                            */
} pr_c0_kind;

/* The custom-precision experiment of Sec. 4.2-4.3 (Fig. 2): numbers with m stored mantissa bits (m + 1
 * significant bits) and FP64's exponent range, rounded to nearest with ties to even. */
typedef enum {
  PR_QUANT_STORAGE = 1,  /* the input A and every stored iterate (C_0 included) are rounded; arithmetic in FP64  */
  PR_QUANT_ARITH = 2     /* A, C_0 and every operation of the iteration: each product term and partial sum of
                            the matrix products (summed in the order k = 0, 1, ..., n - 1), each operation of
                            ((p + 1) C - C^{p+1} A) / p and of the symmetrisation rnd(C + C^T) / 2             */
} pr_quant_mode;

/* Options fixed at pr_init. */
typedef struct {
  int form;            /* pr_form, default PR_FORM_AUTO                                                  */
  int c0;              /* pr_c0_kind, default PR_C0_EQ3                                                  */
  int max_iter;        /* cap on the total number of updates over the handle's life, default 100         */
  double stag_below;   /* stagnation test armed once the previous residual is below this, default 1e-3  */
  double stag_ratio;   /* ... and fires when r_k > stag_ratio * r_{k-1}, default 0.5                      */
  double sym_tol;      /* pr_init rejects A with max|a_ij - a_ji| > sym_tol * max|a_ij|, default 1e-12   */
  int reanchor;        /* coupled form: on a switch to higher precision recompute M = X^p A, default 1  */
  int emu_slices;      /* PR_EMU64 digit planes per operand, 1..8 (0 = the default, 8): S planes keep
                          8S bits per row and cost S (S + 1) / 2 FP16 products per FP64 product         */
  double stag_below_lowp; /* stag_below for the rungs below FP64 accuracy (PR_FP8, PR_BF16, PR_FP32X),
                             whose floor is higher, default 0.5 (below 0.5 every eigencomponent is in the
                             quadratic phase)                                                          */
  double c0_coef[4];   /* PR_C0_POLY coefficients c_0 .. c_3, default (1, 0, 0, 0) (the scaled identity)  */
  double gate_max;     /* PR_C0_POLY gate on ||I - C_0^p A||_2, default 0.9                                */
  int gate_iters;      /* power iterations of the gate, default 30                                         */
  int verify;          /* coupled form: whenever pr_iterate stops on tol, stagnation or its budget, evaluate
                          the true residual ||I - X^p A||_F (p - 1 symmetric products and one full product
                          at the phase's precision) into pr_stats.true_residual, and turn a stop on
                          ||I - M||_F <= tol into PR_EINACCURATE if the true residual exceeds tol; default 1 */
  int gate_fallback;   /* PR_C0_POLY guess failing its gate: 1 (default) use Eq. 3 instead; 0 return PR_EGATE
                          (pr_init then creates no handle; pr_load and pr_set_initial_guess leave Eq. 3's
                          C_0 in the handle)                                                              */
  int emu_tile;        /* digit-slice products (PR_EMU64, PR_FP32X): output tile width. 0 (default) tunes:
                          the first product of each kind (symmetric / full, per precision) times every kernel
                          variant of this order (tiles 128 x 96 or 128 x 48, whole or split over K into two
                          halves when the tiles fill fewer than 4 waves of the SMs) and keeps the fastest; the
                          choice is remembered for the process per (order, kind, digit planes). 96 or 48 fix
                          the width (tiles split by the wave rule). Products are exact integer sums rounded
                          once, the same for every variant; residuals, which add per-tile partial sums, differ
                          in their last bits between widths                                             */
  int quant_bits;      /* 0 (default): off. 1..52: run the custom-precision experiment with this many stored
                          mantissa bits (PR_FORM_LITERAL from Eq. 3's C_0 with PR_FP64 iterations only, else
                          pr_init returns PR_EUNSUPPORTED). The stop test's residual is evaluated in FP64  */
  int quant_mode;      /* pr_quant_mode, default PR_QUANT_STORAGE                                          */
  int block_sparse;    /* 1 (default): products with A at PR_EMU64 / PR_FP32X skip the K steps where the rows
                          of A that a tile reads are zero, when that leaves out at least 1/8 of the steps
                          (A's zero pattern is read at pr_init / pr_load). The steps skipped hold zero digits,
                          so every product is bit-identical to the dense one. 0: never skip              */
} pr_options;

/* Most Newton corrections one pr_refine call applies. */
#define PR_REFINE_MAX_STEPS 16

/* Counters of one handle. */
typedef struct {
  int64_t n;
  int p;
  int form;                 /* the form actually run (never PR_FORM_AUTO)                               */
  int c0;
  int iterations;           /* updates applied so far                                                    */
  int iterations_by_precision[PR_NPREC]; /* indexed by pr_precision                                      */
  int switch_iteration;     /* iteration index at which the precision last changed, -1 if never          */
  int last_precision;       /* precision of the last update, -1 before the first                          */
  int last_stop;            /* pr_status of the last pr_iterate / pr_solve                                */
  double norm_1;            /* ||A||_1 (Eq. 3)                                                            */
  double norm_inf;          /* ||A||_inf (Eq. 3)                                                          */
  double last_residual;     /* the residual of the current iterate (see pr_form)                          */
  int64_t gemms;            /* matrix products issued                                                     */
  double gemm_flops;        /* algorithmic flops of those products: 2 n^3 per full product, n^2 (n + 1)
                               per symmetric one (the n (n + 1) / 2 upper-triangle outputs)              */
  int64_t launches;         /* kernels launched by the library on the handle's stream                     */
  int64_t gemms_timed;      /* products timed with CUDA events (pr_set_timing)                           */
  double gemm_ms;           /* summed event time of the timed products                                     */
  double gemm_flops_timed;  /* algorithmic flops of the timed products                                     */
  int emu_slices;           /* digit planes per operand used by PR_EMU64 (S; S (S + 1) / 2 FP16 products
                               per emulated product)                                                     */
  int64_t gemms_timed_by_precision[PR_NPREC];  /* the timed counters above, split by pr_precision     */
  double gemm_ms_by_precision[PR_NPREC];
  double gemm_flops_by_precision[PR_NPREC];
  double c0_gate;                   /* PR_C0_POLY: the gate's estimate of ||I - C_0^p A||_2, else 0         */
  double true_residual;     /* ||I - C^p A||_F of the iterate at the last stop of pr_iterate: the verified
                               value of the coupled form (pr_options.verify), the tested residual of the
                               Newton-Schulz and literal forms; -1 before the first stop. After a
                               pr_solve_ladder rung guard restored an earlier iterate: that iterate's value */
  int prescale_log2;        /* k: the handle iterates on 2^k A (see pr_load), 0 when A is taken as given   */
  int emu_tile_n[2];        /* PR_EMU64 products, symmetric [0] and full [1]: tile width in use (0: none yet) */
  int emu_tile_split[2];    /* ... and whether their tiles are split over K                               */
  double emu_tune_ms;       /* time the tuner of pr_options.emu_tile spent on trial launches in this handle */
  double emu_variant_ms[2][4]; /* PR_EMU64 products tuned in this handle, symmetric [0] and full [1]: the best
                                  trial time (ms) of each variant, index (width 48 ? 2 : 0) + (split ? 1 : 0),
                                  0 where not tried (the variant does not apply, or the choice was known) */
  int ladder_restores;      /* pr_solve_ladder: rungs whose result was discarded (see pr_solve_ladder)       */
  int refine_steps;         /* Newton corrections kept by pr_refine over the handle's life                     */
  int64_t refine_cg_iterations; /* their conjugate-gradient iterations                                        */
  int refine_len;           /* residuals recorded by the last pr_refine (its corrections kept + 1), 0 before   */
  double refine_residuals[PR_REFINE_MAX_STEPS + 1]; /* ||G(X_k)||_F of the last pr_refine, k = 0 .. refine_len - 1,
                                                       the last one of the iterate it returned (see pr_refine) */
  int refine_cg[PR_REFINE_MAX_STEPS]; /* conjugate-gradient iterations of each correction of the last pr_refine */
  double sparse_keep;       /* block sparsity of the loaded A (pr_options.block_sparse): the fraction of K steps a
                               full product A X keeps, 1 when products with A run dense                       */
  int64_t sparse_products;  /* products with A that skipped K steps                                            */
} pr_stats_t;

/* Fills *opt with the defaults listed above. */
void pr_default_options(pr_options* opt);

/* Creates a handle for A^{-1/p}.
 *   h       out: the new handle (NULL on failure)
 *   A       n*n FP64, row-major, symmetric positive definite; device or host memory; copied, not retained
 *   n       order, n >= 1
 *   p       root index, p >= 1
 *   opt     options (NULL = defaults)
 *   stream  cudaStream_t to issue all work on (NULL = default stream)
 * Computes ||A||_1 and ||A||_inf (Eq. 3), checks A (finite, symmetric within opt->sym_tol, positive
 * diagonal, Cholesky of every diagonal block of order 64), and forms C_0. Synchronises the stream.
 * Eq. 2 for Eq. 3's C_0: the eigenvalues of C_0^p A are lambda^(p+1) / (||A||_1 ||A||_inf)^p <= ||A||_1^(1-p),
 * so for p > 1 a matrix with ||A||_1 ||A||_inf < 1 can violate Eq. 2 (A = 0.1 I, p = 2 gives
 * ||I - C_0^2 A||_2 = 9) and the iteration diverges. Such an A (p > 1 only) is scaled by an exact power of
 * two, A <- 2^k A with ||2^k A||_1 in [1, 2); the handle iterates on 2^k A (its pr_stats norms are those of
 * 2^k A, prescale_log2 = k), pr_result returns 2^(k/p) C = A^{-1/p}, and every residual ||I - C^p (2^k A)||
 * equals the residual of the returned root for A in exact arithmetic.
 * Errors: PR_EINVAL, PR_ENOTSPD, PR_ENOMEM, PR_ECUDA, PR_EGATE (see pr_options.gate_fallback). */
pr_status pr_init(pr_handle* h, const double* A, int64_t n, int p, const pr_options* opt, void* stream);

/* Loads a new A of the same order into an existing handle without reallocating: repeats the checks,
 * norms, C_0 and (coupled form) M_0 of pr_init and clears the iteration state and history. Counters in
 * pr_stats keep accumulating. A: device or host memory, copied. Synchronises the stream.
 * Errors: as pr_init, plus PR_ESTATE for a NULL handle. */
pr_status pr_load(pr_handle h, const double* A);

/* Runs at most max_steps updates of Eq. 1 at the given precision (Sec. 3: low-precision arithmetic for
 * most iterations, precise arithmetic to refine). Before each update the residual r_k of the current
 * iterate is tested: r_k <= tol returns PR_OK; a non-finite r_k returns PR_EDIVERGED; r_{k-1} < stag_below
 * and r_k > stag_ratio * r_{k-1} (both computed in this call) returns PR_ESTAGNATED; an exhausted budget
 * returns PR_EMAXITER. *steps_done (may be NULL) receives the number of updates applied in this call.
 * When a run below FP64 accuracy (PR_FP8, PR_BF16, PR_FP32X) stops because r_k >= r_{k-1} or r_k is not finite,
 * the last update is undone (the iterate, its residual and the counters return to step k-1) and the stop is
 * PR_ESTAGNATED, so that a following precise phase starts from the better iterate.
 * The residual tested is ||I - C_k^p A||_F for the Newton-Schulz and literal forms and the carried
 * ||I - M_k||_F for the coupled form (equal in exact arithmetic). With pr_options.verify the coupled form
 * then evaluates the true residual of the iterate it stops at (pr_stats.true_residual), and a PR_OK whose
 * true residual exceeds tol becomes PR_EINACCURATE.
 * Synchronises the stream once per update to read r_k. */
pr_status pr_iterate(pr_handle h, int max_steps, int precision, double tol, int* steps_done);

/* The stop rule pr_iterate applies to the residual history, as a pure host function (no device work).
 * hist[0..len) are residuals r_0 .. r_k (r_k of the current iterate), prec[0..len) the pr_precision each
 * was computed at; opt NULL = defaults. Returns PR_EDIVERGED if r_k is not finite, PR_OK if r_k <= tol,
 * PR_ESTAGNATED if r_{k-1} and r_k were computed at the same precision and either
 *   (a) r_{k-1} < arm and r_k > stag_ratio * r_{k-1}, arm = stag_below (PR_FP64, PR_EMU64) or
 *       stag_below_lowp (PR_FP8, PR_BF16, PR_FP32X), or
 *   (b) PR_FP8, PR_BF16, PR_FP32X only: r_k >= r_{k-1} (a low-precision floor, or the iteration leaving its
 *       region of convergence because the rounding of the iterate is too coarse for the conditioning of A),
 * and -1 otherwise (continue). The step budget and max_iter are checked by pr_iterate itself. */
int pr_stop_rule(const double* hist, const int* prec, int len, double tol, const pr_options* opt);

/* The precision ladder in one call: up to bulk_steps updates at bulk_precision (stopping early on its
 * floor, i.e. stagnation, or on tol), then updates at final_precision until tol, stagnation or
 * max_iter. bulk_steps = 0 skips the bulk phase; a bulk phase that ends with PR_OK returns at once, one
 * that ends with PR_ESTAGNATED, PR_EMAXITER or PR_EINACCURATE hands over to the final phase. Returns the
 * stop status of the last phase run. */
pr_status pr_solve(pr_handle h, int bulk_precision, int bulk_steps, int final_precision, double tol,
                   int* steps_done);

/* A precision ladder of `count` rungs in one call: rung r runs pr_iterate at precisions[r] with at most
 * max_steps[r] updates (max_steps NULL: no per-rung limit beyond max_iter). A rung that ends with PR_OK
 * returns at once; one that ends with PR_ESTAGNATED (its precision floor), PR_EMAXITER or PR_EINACCURATE
 * hands over to the next rung; any other status is returned. The coupled form re-forms M = X^p A at the
 * higher precision when the level rises (pr_options.reanchor): PR_FP8 < PR_BF16 < PR_FP32X < PR_FP64 =
 * PR_EMU64. Returns the status of the last rung run; *steps_done (may be NULL) receives the updates of all
 * rungs together. pr_stats.iterations_by_precision and switch_iteration record where each rung ended.
 * Rung guard: a low-precision rung (PR_FP8, PR_BF16, PR_FP32X) followed by a higher level, or last in a
 * ladder of several, tests the carried ||I - M||_F, which can keep falling while rounding errors let X drift
 * from M. Before the first such rung and after each, the library evaluates ||I - X^p A||_F with the next
 * rung's products (PR_EMU64 products after the last rung); a rung that leaves
 * it above the best value seen so far is discarded (X returns to that best iterate and M is re-formed from
 * it). A rung after the first that diverges from the iterate the earlier rungs left (a low-precision rung can
 * leave X^p A indefinite while its Frobenius residual fell) runs once more from the starting iterate.
 * pr_stats.ladder_restores counts both kinds. This costs p products per guarded boundary and two n*n FP64
 * buffers, allocated on first use and kept until pr_destroy (PR_ENOMEM if they cannot be).
 * Errors: as pr_iterate, and PR_EINVAL for count < 1, a NULL precisions array or an unknown precision. */
pr_status pr_solve_ladder(pr_handle h, int count, const int* precisions, const int* max_steps, double tol,
                          int* steps_done);

/* ---- Refinement of an approximate root (Sec. 3 and Sec. 5) ------------------------------------------------
 * Sec. 3 and Sec. 5: a result computed with imprecise arithmetic is refined into a precise root in a few
 * additional precise iterations. Eq. 1's own step does that for p = 1 (Newton-Schulz removes any perturbation
 * to first order) but not for p >= 2: the coupled form keeps X_k M_k^{-1/p} fixed and so converges to
 * X_0 (X_0^p A)^{-1/p}, which differs from A^{-1/p} whenever X_0 carries an error that does not commute with A
 * (the rounding errors of a low-precision phase, or those of M_0 = C_0^p A from Eq. 3's C_0, whose eigenvalues
 * span kappa^(p+1)). pr_refine applies Newton's method to the balanced residual
 *     G(X) = I - sym(X^m A X^m'),   m = floor(p/2), m' = p - m,   sym(Y) = (Y + Y^T) / 2,
 * which vanishes at A^{-1/p}. A step solves the linearised equation
 *     sym(dP_m(D) A X^m' + X^m A dP_m'(D)) = G(X),   dP_k(D) = sum_{j<k} X^j D X^(k-1-j),
 * for a symmetric correction D by conjugate gradients (Frobenius inner product, preconditioner R -> sym(X R) / p)
 * and sets X <- X + D. Each step squares the error of X up to a constant, whatever its structure; the
 * solve needs only the accuracy the step is to gain, so its products may be low precision while G(X) is
 * evaluated with FP64-accurate products.
 *   precision        products of G(X) (and of the true residual at the end): PR_EMU64 or PR_FP64 for an
 *                    FP64-accurate root; any pr_precision is accepted
 *   inner_precision  products of the conjugate-gradient solve, any pr_precision (PR_FP32X: about 1e-6 per
 *                    correction; PR_BF16: about 1e-2, more steps but each far cheaper)
 *   max_steps        at most this many corrections, 0 .. PR_REFINE_MAX_STEPS
 *   tol              stop when ||G(X)||_F <= tol
 *   cg_max, cg_tol   the solve stops when ||G - L(D)||_F <= cg_tol ||G||_F or after cg_max >= 1 iterations
 *   steps_done       (may be NULL) corrections kept in this call
 * Before each step ||G(X_k)||_F is evaluated and tested: PR_OK if <= tol; if it is not finite, or not below
 * the previous step's value, the last correction is undone (X returns to the previous iterate) and the stop is
 * PR_EDIVERGED or PR_ESTAGNATED; PR_ESTAGNATED also when the previous value was below stag_below and this one
 * above stag_ratio times it (the precision floor; the iterate is kept); PR_EMAXITER after max_steps
 * corrections. Then the true residual ||I - X^p A||_F of the returned iterate is evaluated with `precision`
 * products into pr_stats.true_residual, and a PR_OK whose true residual exceeds tol becomes PR_EINACCURATE.
 * pr_stats records each step's residual and solve length (refine_residuals, refine_cg). The iteration counters
 * and history of Eq. 1 are not changed; a following pr_iterate re-forms the coupled form's M from the refined X.
 * Works on every form and on the iterate pr_iterate, pr_solve, pr_solve_ladder or pr_set_iterate left.
 * Products per step: 1 (p = 1), 2 (p = 2), 3 (p = 4) or 4 (p = 3) with `precision`; per solve iteration
 * 2, 2, 3 or 4 with `inner_precision`. Uses three n*n FP64 matrices (with their BF16 copies, and digit planes
 * where the products need them) and a copy of X beyond pr_init's, allocated on the first call and kept until
 * pr_destroy (PR_ENOMEM if they cannot be). Synchronises the stream twice per solve iteration.
 * Errors: PR_ESTATE (NULL handle, no matrix), PR_EINVAL (unknown precision, max_steps outside
 * [0, PR_REFINE_MAX_STEPS], tol, cg_tol < 0 or NaN, cg_max < 1), PR_EUNSUPPORTED (the custom-precision
 * experiment, pr_options.quant_bits), PR_ECUDA, PR_ETIMEOUT, PR_ENOMEM. */
pr_status pr_refine(pr_handle h, int precision, int inner_precision, int max_steps, double tol, int cg_max,
                    double cg_tol, int* steps_done);

/* Replaces the handle's iterate by X: n*n FP64 row-major, an approximation of A^{-1/p} for the A the caller
 * gave (device or host memory; copied). For pr_refine of a root known to low precision, e.g. one computed
 * elsewhere or the root of a nearby matrix of a sequence, or to restart Eq. 1 from a chosen C_0. Checks X as
 * pr_init checks A (finite, symmetric within sym_tol, positive diagonal, Cholesky of the diagonal blocks of
 * order 64) and multiplies it by 2^(-k/p) when the handle iterates on 2^k A (pr_stats.prescale_log2).
 * Clears the iteration state, history and counters as pr_set_initial_guess does. Synchronises the stream.
 * Errors: PR_ESTATE (NULL handle, no matrix), PR_EINVAL (X NULL, non-finite or not symmetric), PR_ENOTSPD,
 * PR_ECUDA. */
pr_status pr_set_iterate(pr_handle h, const double* X);

/* True residual ||I - C^p A||_F of the current iterate (Eq. 2 in the Frobenius norm), evaluated with
 * products at the given precision: C^p by symmetric products, then the full product with A.
 * Synchronises the stream. */
pr_status pr_residual(pr_handle h, int precision, double* res_fro);

/* Copies the current iterate C_k (n*n FP64, row-major) to C_out (device or host memory, caller-owned),
 * multiplied by 2^(k/p) when pr_load scaled A by 2^k (pr_stats.prescale_log2), so that C_out approximates the
 * root of the A the caller gave. Synchronises the stream when C_out is host memory. */
pr_status pr_result(pr_handle h, double* C_out);

/* Copies the handle's counters to *out. */
pr_status pr_stats(pr_handle h, pr_stats_t* out);

/* Copies up to cap residuals r_0 .. r_k (one per iterate, in order) to out (host memory) and the
 * number available to *len. */
pr_status pr_history(pr_handle h, double* out, int cap, int* len);

/* One matrix product of the iteration on its own, for testing and timing the product kernels:
 * P = X Y for symmetric n x n FP64 X and Y (device or host memory) that commute, so that X Y is symmetric.
 * sym != 0 computes only the upper-triangle tiles and mirrors them (the iteration's symmetric products);
 * sym == 0 computes every tile. precision PR_FP64 uses FP64 DMMA; PR_BF16 rounds X and Y to BF16 and
 * accumulates in FP32 on the tcgen05 tensor cores; PR_FP8 rounds X 2^-sx_i and Y 2^-sy_j to E4M3 row by
 * row (see PR_FP8) and accumulates in FP32; PR_EMU64 forms the product from 8 balanced base-256 digit
 * planes per operand, exact in FP16, and the 36 digit-plane pairs that reach FP64 accuracy (see PR_EMU64);
 * PR_FP32X uses the first 3 of those planes and their 6 pairs. P: n*n FP64 output (device or host),
 * caller-owned.
 * Allocates and frees temporary device buffers. Synchronises the stream. */
pr_status pr_matmul(int precision, const double* X, const double* Y, int64_t n, int sym, double* P, void* stream);

/* pr_matmul with PR_EMU64 products of `slices` digit planes per operand (1..8; pr_matmul uses 8), for
 * testing every slice count the options allow (pr_options.emu_slices). Errors: as pr_matmul, and
 * PR_EINVAL for slices outside [1, 8]. */
pr_status pr_matmul_emu(int slices, const double* X, const double* Y, int64_t n, int sym, double* P, void* stream);

/* pr_matmul_emu with a chosen work-list variant of the digit-slice kernel (the variants pr_options.emu_tile
 * tunes between): tile_n = 96 or 48 output columns per 128-row tile; split = 1 splits every tile over K into
 * two halves run by different CTAs (orders above 16), 0 never, -1 when the tiles fill fewer of the SMs'
 * waves than the halves would. Every variant gives the same product (exact digit-pair sums, rounded once).
 * Errors: as pr_matmul_emu, and PR_EINVAL for another tile_n or split. */
pr_status pr_matmul_emu_tiled(int slices, int tile_n, int split, const double* X, const double* Y, int64_t n, int sym,
                              double* P, void* stream);

/* ---- Checkpoint and resume ----------------------------------------------------------------------------
 * The state of an iteration as one host byte buffer: the iterate X and, for the coupled form with its
 * product formed, M and N (FP64, and their BF16 copies), the residual history with the precision of each
 * entry, and the counters the stop rule reads. Importing it into a handle that holds the same A (same
 * order, root and form, and the same ||A||_1, ||A||_inf; from pr_init or pr_load) resumes the iteration
 * where the export left it: the iterates that follow are bit-identical to those of the exporting handle.
 * Layout: pr_state_header; hist_len doubles (r_0 ..); hist_len int32 precisions, padded to a multiple of
 * 8 bytes; n_mats FP64 matrices n x n (X, then M, N); n_mats BF16 matrices n x ldl (same order). */
#define PR_STATE_MAGIC 0x5052535441544531ull /* "PRSTATE1" */
#define PR_STATE_VERSION 2                   /* 2: per-precision counters for PR_NPREC precisions */
typedef struct {
  uint64_t magic;
  int64_t n;
  int32_t version;         /* PR_STATE_VERSION */
  int32_t p;
  int32_t form;
  int32_t c0;
  double norm_1;           /* of the A the state belongs to */
  double norm_inf;
  int32_t state_ready;     /* coupled form: M, N and the residual of X are formed */
  int32_t state_level;     /* precision level at which M was formed */
  int32_t lp_stale;        /* the BF16 copies are out of date */
  int32_t iterations;
  int32_t iterations_by_precision[PR_NPREC];
  int32_t switch_iteration;
  int32_t last_precision;
  int32_t hist_len;
  int32_t n_mats;          /* 1 (X) or 3 (X, M, N) */
  int32_t ldl;             /* leading dimension of the BF16 copies */
  int32_t reserved;
  int32_t reserved2;
  double last_residual;
} pr_state_header;

/* *bytes = the size of the state buffer pr_export_state writes now. Errors: PR_ESTATE, PR_EINVAL. */
pr_status pr_state_size(pr_handle h, size_t* bytes);

/* Writes the state into buf (host memory, `bytes` >= pr_state_size). Synchronises the stream.
 * Errors: PR_ESTATE, PR_EINVAL (NULL or short buffer), PR_ECUDA. */
pr_status pr_export_state(pr_handle h, void* buf, size_t bytes);

/* Replaces the handle's iteration state by an exported one. Errors: PR_ESTATE, PR_EINVAL (bad magic or
 * version, short buffer, or a state of another order, root, form or matrix), PR_ECUDA. */
pr_status pr_import_state(pr_handle h, const void* buf, size_t bytes);

/* Exercises the failure path of the library's bounded device waits: launches one kernel that waits on an
 * mbarrier that nothing completes, through the same bounded-wait helper every tcgen05 kernel uses. The
 * wait gives up after its limit (2 s), records its code in a device error word and the kernel returns; the
 * CUDA context stays usable. Returns PR_ETIMEOUT (the expected outcome; *waited_s, if not NULL, receives
 * the device-clock time the wait took), PR_ECUDA if the wait did not run out or a CUDA call failed. */
pr_status pr_selftest_wait(void* stream, double* waited_s);

/* Enables (on != 0) or disables CUDA-event timing of every matrix-product kernel; the summed times
 * appear in pr_stats (gemm_ms, gemms_timed, gemm_flops_timed). Adds two event records per product. */
pr_status pr_set_timing(pr_handle h, int on);

/* ---- Batches: many independent problems solved together ------------------------------------------------
 * A batch holds `count` SPD matrices A_i (orders n_i, roots p_i) and iterates them together: every matrix
 * product stage of an iteration is one launch of the PR_EMU64 tensor-core kernel over the tiles of every
 * matrix taking part in it (matrices packed row-wise with one leading dimension). Per matrix, the forms,
 * the initial guess (Eq. 3 or the scaled identity), the stop rule and the results are those of pr_iterate;
 * a matrix whose stop rule fires leaves the work lists. A solve is one CUDA graph with a device-side loop:
 * work lists, residuals, stop rules and the loop condition are computed on the GPU. */
typedef struct pr_batch_s* pr_batch;

/* Creates a batch. n[i] in [1, 16384], p[i] in [1, 64], A[i]: n[i]*n[i] FP64 row-major, device or host,
 * copied. opt: form must be PR_FORM_AUTO (NULL = defaults). Checks every matrix as pr_init does and, where
 * Eq. 2 needs it (p > 1, ||A||_1 ||A||_inf < 1), scales it by a power of two as pr_load does.
 * Errors: PR_EINVAL, PR_ENOTSPD, PR_ENOMEM, PR_ECUDA. */
pr_status pr_batch_init(pr_batch* b, int count, const int64_t* n, const int* p, const double* const* A,
                        const pr_options* opt, void* stream);

/* Replaces the batch's matrices by A[0..count) of the same orders (device or host, copied; checked as
 * pr_batch_init checks them) and restarts every matrix from its initial guess. Keeps the device memory and
 * the captured solve graph. Errors: PR_ESTATE (b NULL), PR_EINVAL, PR_ENOTSPD, PR_ECUDA. */
pr_status pr_batch_load(pr_batch b, const double* const* A);

/* Iterates every active matrix until its stop rule fires (tol, stagnation, max_iter, divergence), with
 * PR_EMU64 products. iterations[i] and status[i] (a pr_status stop code; may be NULL) receive the outcome
 * per matrix. With pr_options.verify (default) the graph then evaluates, as pr_iterate does, the true
 * residual ||I - X^p A||_F of every coupled-form matrix that stopped on tol, stagnation or max_iter, and a
 * PR_OK whose true residual exceeds tol becomes PR_EINACCURATE (pr_batch_matrix gives the value).
 * The first call captures the solve graph (on a private stream); every call launches it once
 * on the batch's stream and synchronises that stream once, at the end. A call after every matrix has
 * stopped changes nothing. Errors: PR_ESTATE, PR_EINVAL (tol < 0), PR_EUNSUPPORTED (precision other than
 * PR_EMU64), PR_ECUDA, PR_ETIMEOUT (a bounded device wait expired). */
pr_status pr_batch_solve(pr_batch b, int precision, double tol, int* iterations, int* status);

/* Copies the result of matrix i (n[i]*n[i] FP64, row-major) to C_out (device or host), multiplied by
 * 2^(k/p) for a matrix the batch iterated as 2^k A (pr_batch_matrix_t.prescale_log2). */
pr_status pr_batch_result(pr_batch b, int i, double* C_out);

/* Residual history r_0 .. r_k of matrix i (host memory), as pr_history. */
pr_status pr_batch_history(pr_batch b, int i, double* out, int cap, int* len);

/* What the batch knows about matrix i after the last pr_batch_solve. */
typedef struct {
  int64_t n;
  int p;
  int form;              /* PR_FORM_NS (p = 1) or PR_FORM_COUPLED                                          */
  int status;            /* its pr_status stop code, -1 before a solve                                    */
  int iterations;
  double norm_1;         /* ||A||_1 and ||A||_inf of the matrix iterated on (2^k A, see prescale_log2)     */
  double norm_inf;
  int prescale_log2;     /* k: as pr_load, a matrix with p > 1 and ||A||_1 ||A||_inf < 1 is iterated as 2^k A
                            with ||2^k A||_1 in [1, 2) (Eq. 2 for Eq. 3's C_0); pr_batch_result scales back    */
  double true_residual;  /* ||I - C^p A||_F at the stop: for the coupled form the verification after the solve
                            loop (pr_options.verify), for p = 1 the tested residual; -1 if not evaluated        */
} pr_batch_matrix_t;

/* Fills *out for matrix i. Errors: PR_ESTATE (b NULL), PR_EINVAL (bad index, out NULL). */
pr_status pr_batch_matrix(pr_batch b, int i, pr_batch_matrix_t* out);

/* Kernels launched by the batch so far. */
int64_t pr_batch_launches(pr_batch b);

/* Counters of a batch. A "product" is one matrix's share of one stage; its FP64-equivalent algorithmic
 * flops are n^2 (n + 1) for a symmetric product (upper tiles) and 2 n^3 for a full one. The executed
 * tensor-core work is emu_slices (emu_slices + 1) / 2 FP16 digit-pair products of each. */
typedef struct {
  int64_t launches;          /* kernels launched so far (in the solve graph: its prologue, epilogue and every
                                pass of its loop body, whether or not a launch found work) */
  int64_t stages;            /* product launches with work (a graph stage whose list is empty does not count) */
  int64_t products;          /* per-matrix products in those launches */
  double product_flops;      /* their FP64-equivalent algorithmic flops */
  int64_t stages_timed;      /* product launches timed (pr_batch_set_timing) */
  double stage_ms;           /* summed time of the timed launches: first CTA start to last CTA end */
  double stage_flops_timed;  /* FP64-equivalent algorithmic flops of the timed launches */
  int emu_slices;            /* digit planes per operand */
  int tile_n;                /* output columns per tile of the batch's products: pr_options.emu_tile, or the
                                width the tuner at pr_batch_init found faster on the symmetric product A A of
                                every matrix (one launch per width, best of two)                            */
  double tune_ms;            /* time of those trial launches                                               */
} pr_batch_stats_t;

/* Fills *out. Errors: PR_ESTATE (b NULL), PR_EINVAL (out NULL). */
pr_status pr_batch_stats(pr_batch b, pr_batch_stats_t* out);

/* on != 0: add the product launches of the following solves to stages_timed / stage_ms /
 * stage_flops_timed. Each launch folds the device clock (%globaltimer, ns) at the start of its first CTA
 * and at the end of its last into a slot that the solve graph reads back itself. Errors: PR_ESTATE. */
pr_status pr_batch_set_timing(pr_batch b, int on);

/* Text for the last failing call on b (b NULL: the last failing pr_batch_init of this thread). */
const char* pr_batch_last_error(pr_batch b);

/* Frees the batch. b may be NULL. */
pr_status pr_batch_destroy(pr_batch b);

/* ---- The learned initial guess ---------------------------------------------------------------------------
 * Spectral features of the handle's A for predicting a polynomial initial guess:
 * out[k-1] = tr(Ahat^k) / n for k = 1..6 with Ahat = A / ||A||_1, out[6] = ||A||_1, out[7] = ||A||_inf
 * (the norms of the A the caller gave, before any power-of-two scaling of pr_load).
 * The traces come from Ahat, Ahat^2, Ahat^3 (two PR_EMU64 symmetric products) as Frobenius inner products.
 * out: 8 doubles, host memory. Synchronises the stream. */
pr_status pr_features(pr_handle h, double* out);

/* Estimates of the extreme eigenvalues of the caller's A, by `iters` power iterations on the device (each from
 * below): *lam_max = ||A||_2, and *lam_min = ||C||_2^(-p) with C the current iterate (the root the handle
 * returns), which is lambda_min(A) once C has converged to A^{-1/p}. Used to build training labels for the
 * learned guess (the spectral interval of A / ||A||_1). Synchronises the stream.
 * Errors: PR_ESTATE (NULL handle, no matrix), PR_EINVAL (iters < 1, NULL output), PR_ECUDA. */
pr_status pr_spectral_bounds(pr_handle h, int iters, double* lam_min, double* lam_max);

/* Re-forms C_0 from the loaded A with `kind` (PR_C0_EQ3, PR_C0_SCALED_I or PR_C0_POLY; coef: the 4 cubic
 * coefficients for PR_C0_POLY, host memory, else may be NULL) and restarts the iteration from it (history
 * and counts cleared), without re-reading A. PR_C0_POLY is gated exactly as at pr_init; A^2 and A^3
 * computed by pr_features are reused. The handle's options are not changed: a later pr_load forms C_0
 * as pr_init's options say. Errors: PR_ESTATE (NULL handle, no matrix loaded), PR_EINVAL
 * (unknown kind, coef NULL or non-finite for PR_C0_POLY), PR_ECUDA. */
pr_status pr_set_initial_guess(pr_handle h, int kind, const double* coef);

/* A multilayer perceptron 8 -> 64 -> 64 -> 4 (ReLU hidden layers, FP32) on the device, trained with the
 * mean squared error and Adam (beta1 0.9, beta2 0.999, eps 1e-8). Parameters are a flat FP32 vector of
 * PR_MLP_PARAMS: W1 (64 x 8, row-major), b1 (64), W2 (64 x 64), b2 (64), W3 (4 x 64), b3 (4). Inputs X are
 * B x 8, targets T and outputs Y B x 4, row-major, device or host memory, B <= max_batch. */
#define PR_MLP_PARAMS 4996
typedef struct pr_mlp_s* pr_mlp;
pr_status pr_mlp_create(pr_mlp* m, const float* params, int max_batch, void* stream);
pr_status pr_mlp_forward(pr_mlp m, const float* X, int B, float* Y);
/* Loss (host) and its gradient (PR_MLP_PARAMS floats, device or host) at the current parameters. */
pr_status pr_mlp_loss_grad(pr_mlp m, const float* X, const float* T, int B, float* loss, float* grad);
/* One Adam step with learning rate lr on the batch; *loss (host, may be NULL) gets the loss before it. */
pr_status pr_mlp_adam_step(pr_mlp m, const float* X, const float* T, int B, float lr, float* loss);
pr_status pr_mlp_get_params(pr_mlp m, float* params);
pr_status pr_mlp_destroy(pr_mlp m);

/* Largest order accepted by pr_norms_noalloc. */
#define PR_NORMS_NOALLOC_MAX_N 65536

/* ||A||_1 and ||A||_inf (the norms of Eq. 3's initial guess) for callers that cannot allocate device
 * memory. The paper has no counterpart: this entry point exists for code that must not call cudaMalloc or
 * cudaFree, e.g. work issued while a CUDA graph is being captured (allocation calls are not part of a
 * capture), latency-critical paths that cannot afford the synchronisation cudaFree implies, or programs
 * whose device memory is already reserved in full by their own allocator.
 *   A       n*n FP64, row-major, device memory, read only; a NaN entry makes both norms NaN
 *   n       1 <= n <= PR_NORMS_NOALLOC_MAX_N, else PR_EINVAL (nothing is launched)
 *   out     device memory, 2 doubles: out[0] = ||A||_1 (largest absolute column sum),
 *           out[1] = ||A||_inf (largest absolute row sum); written asynchronously on stream
 *   stream  cudaStream_t (NULL = default stream); the call does not synchronise it
 * Scratch: a fixed 1 MiB array in the library's device memory (2 * PR_NORMS_NOALLOC_MAX_N doubles) that
 * every device which loads the library keeps until the process exits. The first call on a device looks up
 * that array's device address (cudaGetSymbolAddress); make that first call before any stream capture
 * begins. The address is kept for the life of the process: after cudaDeviceReset the library must not be
 * called on that device again. All calls on a device share the array and each call overwrites what it
 * uses, so calls that overlap on the GPU (on different streams, or from different threads) race and must
 * be serialised.
 * Allocates nothing: no cudaMalloc, cudaFree or allocating library routine. Errors: PR_EINVAL, PR_ECUDA. */
pr_status pr_norms_noalloc(const double* A, int64_t n, double* out, void* stream);

/* Frees all device memory of the handle. h may be NULL. */
pr_status pr_destroy(pr_handle h);

/* Text describing the last failing call on h; with h NULL, the last failing call of this thread that had
 * no handle (pr_init, pr_matmul, pr_norms_noalloc). */
const char* pr_last_error(pr_handle h);

/* Library version as major*10000 + minor*100 + patch. */
int pr_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PTHROOT_H */
