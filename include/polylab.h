/*
 * polylab.h -- C ABI of the B300-native sparse-monomial engine and the
 * affine-normal direction (libpolylab.so, CUDA kernels for sm_103a).
 *
 * Data model (paper Sec. 2, Table "apisignature"; Sec. 3.2): a polynomial is
 * (vars.id, coef, pow): n unique 64-bit variable ids, an n_terms x n exponent
 * matrix (uint8, row-major) and a coefficient vector (double).  Repeated
 * exponent rows are allowed and mean a sum.
 *
 * Conventions shared by every call
 *   - Pointers documented as DEVICE point to memory of the current CUDA device
 *     and are owned by the caller; pointers documented as HOST are host memory.
 *   - Work is enqueued on `stream` (a cudaStream_t; NULL is the legacy default
 *     stream) and is asynchronous unless a call says it synchronises.
 *   - Scratch memory is taken from the stream-ordered allocator
 *     (cudaMallocAsync/cudaFreeAsync on `stream`) and released before the call
 *     returns, in stream order.
 *   - Every call returns a polylab_status.  Argument and launch errors are
 *     statuses; a call never aborts, traps or exits.  Per-point numerical
 *     failures of the affine-normal direction are flags in polylab_an_info,
 *     not errors.
 *   - A call that fails with POLYLAB_ERR_CUDA leaves the message of the CUDA
 *     error in polylab_last_error() (per thread).
 */
#ifndef POLYLAB_H
#define POLYLAB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* polylab_stream; /* == cudaStream_t */

typedef enum {
  POLYLAB_OK = 0,
  POLYLAB_ERR_INVALID_ARG = 1,   /* null pointer, negative size, bad enum, n mismatch */
  POLYLAB_ERR_EXP_OVERFLOW = 2,  /* a product exponent exceeds 255 */
  POLYLAB_ERR_DUP_VAR_ID = 3,    /* an operand lists one variable id twice */
  POLYLAB_ERR_OOM = 4,           /* scratch or output allocation failed */
  POLYLAB_ERR_CUDA = 5,          /* a CUDA runtime/driver call or launch failed */
  POLYLAB_ERR_TIMEOUT = 6,       /* a bounded device-side wait gave up */
  POLYLAB_ERR_UNSUPPORTED = 7    /* outside this library's stated limits */
} polylab_status;

/* Human-readable name of a status. */
const char* polylab_status_string(polylab_status s);
/* Message of the last CUDA error seen by a call on this thread ("" if none). */
const char* polylab_last_error(void);

/* ------------------------------------------------------------------ data model */

typedef struct {
  int32_t n_vars;           /* n >= 1 */
  const uint64_t* var_ids;  /* HOST, n unique ids (Sec. 3.2 vars.id)            */
  int64_t n_terms;          /* m >= 0                                           */
  const uint8_t* exps;      /* DEVICE, m x n row-major exponents                */
  const double* coef;       /* DEVICE, m coefficients                           */
} polylab_poly;

/* Output of simplify/mul.  The caller sets var_ids (HOST buffer with room for
 * the result's variables: p.n_vars for simplify, a.n_vars + b.n_vars for mul);
 * the call fills n_vars, var_ids, n_terms and sets exps/coef to DEVICE memory
 * obtained from the caller's allocator. */
typedef struct {
  int32_t n_vars;
  uint64_t* var_ids;
  int64_t n_terms;
  uint8_t* exps;            /* n_terms x n_vars row-major, from alloc */
  double* coef;             /* n_terms, from alloc                    */
} polylab_poly_out;

/* Caller-owned output allocation: return `bytes` of DEVICE memory usable in
 * stream order on the call's stream, or NULL on failure (-> POLYLAB_ERR_OOM).
 * Called at most twice per call, never with bytes == 0. */
typedef void* (*polylab_alloc_fn)(size_t bytes, void* ctx);

/* --------------------------------------------------------------- simplify / mul */

/* simplify(p, zeroprec) (Sec. 2, Table "coresemantics"; Sec. 6.3): merge the
 * coefficients of equal exponent rows, drop merged terms with
 * |c| <= zeroprec (zeroprec = 0 drops exact zeros), emit the terms in the
 * engine's canonical monomial order -- total degree, then ascending
 * lexicographic order of the reversed exponent row, the order of Polylab's
 * monolist (Sec. 3.1).  Variables keep the input's order and ids.
 * Exponents of the result are bit-exact; coefficient sums are FP64 in an
 * order of the library's choosing.
 * Synchronises `stream` once (to size the output).
 * Limit: the number of distinct monomials of degree <= max row degree in n
 * variables must be below 2^128 (POLYLAB_ERR_UNSUPPORTED otherwise), and
 * n_terms < 2^31. */
polylab_status polylab_simplify(const polylab_poly* p, double zeroprec, polylab_poly_out* out,
                                polylab_alloc_fn alloc, void* alloc_ctx, polylab_stream stream);

/* a * b (Sec. 2 "mtimes"; Sec. 3.2 alignment): the operands' variable spaces
 * are aligned by id first -- the result's variables are the union of both id
 * sets in ascending id order -- then every pair of terms is expanded
 * (exponents added, coefficients multiplied) and the expansion is simplified
 * as by polylab_simplify.  POLYLAB_ERR_EXP_OVERFLOW if an exponent sum
 * exceeds 255; POLYLAB_ERR_DUP_VAR_ID if an operand repeats an id.
 * Synchronises `stream` once.  Limit: n_terms(a) * n_terms(b) < 2^31. */
polylab_status polylab_mul(const polylab_poly* a, const polylab_poly* b, double zeroprec,
                           polylab_poly_out* out, polylab_alloc_fn alloc, void* alloc_ctx,
                           polylab_stream stream);

/* a + b (Table "coresemantics" "plus"; Sec. 3.2 aligns the variable spaces of
 * operands before they combine): variables aligned by id as for polylab_mul (union in
 * ascending id order), the terms of both operands concatenated and
 * simplified as by polylab_simplify.  Synchronises `stream` once.
 * Limit: n_terms(a) + n_terms(b) < 2^31. */
polylab_status polylab_add(const polylab_poly* a, const polylab_poly* b, double zeroprec,
                           polylab_poly_out* out, polylab_alloc_fn alloc, void* alloc_ctx,
                           polylab_stream stream);

/* a - b (Table "coresemantics" "minus"): as polylab_add with the coefficients
 * of b negated. */
polylab_status polylab_sub(const polylab_poly* a, const polylab_poly* b, double zeroprec,
                           polylab_poly_out* out, polylab_alloc_fn alloc, void* alloc_ctx,
                           polylab_stream stream);

/* p^k for k >= 0 (Table "coresemantics" "mpower"/"prod"; Sec. 6.3 builds p_d^3
 * this way): the product of k copies of p, each partial product simplified
 * as by polylab_mul.  Computed by binary exponentiation (squarings and
 * products of squarings), so the coefficient sums are associated differently
 * from a left-to-right product; k = 0 gives the constant 1 over p's
 * variables.  Intermediates live in stream-ordered library memory; the
 * result goes through `alloc` as for polylab_mul (out->var_ids: p.n_vars
 * entries).  Synchronises `stream` once per partial product.  Errors as
 * polylab_mul (POLYLAB_ERR_EXP_OVERFLOW when a power's exponent exceeds
 * 255); POLYLAB_ERR_INVALID_ARG for k < 0. */
polylab_status polylab_pow(const polylab_poly* p, int32_t k, double zeroprec, polylab_poly_out* out,
                           polylab_alloc_fn alloc, void* alloc_ctx, polylab_stream stream);

/* d p / d x_v for the variable with id `var_id` (Sec. 3.3: term by term,
 * x^a -> a_v x^(a - e_v), terms without x_v vanish), simplified as by
 * polylab_simplify; variables keep p's ids and order.  An id p does not have
 * gives the zero polynomial (n_terms = 0).  Synchronises `stream` once. */
polylab_status polylab_diff(const polylab_poly* p, uint64_t var_id, double zeroprec, polylab_poly_out* out,
                            polylab_alloc_fn alloc, void* alloc_ctx, polylab_stream stream);

/* polylab_simplify for callers that cannot allocate device memory while the
 * call runs -- a host application that reserved all device memory for its own
 * pool up front, or one that runs under a fixed memory budget where a
 * cudaMalloc or cudaMallocAsync could fail or stall at an unpredictable time.
 * The paper has no counterpart of this call; it is an addition of this
 * library.  The result is the same as polylab_simplify's.
 *
 * No device memory is allocated: all scratch lives in one 16 MiB array that
 * the library declares at file scope on the device (every GPU that loads the
 * library holds it until the process exits), and the output goes to buffers
 * the caller passes: out->var_ids (HOST, p->n_vars entries), out->exps
 * (DEVICE, capacity x p->n_vars bytes) and out->coef (DEVICE, capacity
 * doubles).  On return out->n_terms is the number of merged terms.
 * Limits: p->n_terms <= 65,536 and the whole working set (about 100 bytes per
 * term plus 5 bytes per nonzero exponent and 16 (n+1)(D+1) bytes of binomial
 * table, D the largest row degree) must fit in the array; otherwise
 * POLYLAB_ERR_UNSUPPORTED with a message in polylab_last_error().  If the
 * result has more than `capacity` terms, nothing is written, out->n_terms
 * holds the count needed and the status is POLYLAB_ERR_INVALID_ARG.
 * Every call looks up the device address of the array on the current device
 * (cudaGetSymbolAddress) and returns only after all of its work on `stream`
 * has completed, so calls made one after another are ordered on the GPU
 * whatever streams they use.  Calls that run at the same time (from several
 * host threads) share the array and race: serialise them. */
polylab_status polylab_simplify_noalloc(const polylab_poly* p, double zeroprec, polylab_poly_out* out,
                                        int64_t capacity, polylab_stream stream);

/* ------------------------------------------------------------------------ plans */

/* A plan is the device-resident preprocessed form of one polynomial (its term
 * list and, on request, the derived-coefficient matrix of the tensor-core
 * derivative forms).  Creating one synchronises `stream` once; a plan may be
 * passed to any later eval/affine call on the same device and is read-only
 * there.  Passing NULL as the plan makes those calls build a temporary one.
 * Limit of the term list: at most 8 active variables per term and n < 65536
 * (POLYLAB_ERR_UNSUPPORTED otherwise). */
typedef struct polylab_plan polylab_plan;

#define POLYLAB_PLAN_TERMS 0u  /* term list only                         */
#define POLYLAB_PLAN_GEMM  1u  /* also the derived-coefficient matrix    */

polylab_status polylab_plan_create(const polylab_poly* p, uint32_t what, polylab_stream stream,
                                   polylab_plan** plan);
/* Frees the plan's memory after all work already enqueued on `stream`. */
polylab_status polylab_plan_destroy(polylab_plan* plan, polylab_stream stream);
/* Closure-set size K (rows of the derived-coefficient matrix) or -1. */
int64_t polylab_plan_closure_size(const polylab_plan* plan);
/* Shape of a plan's derived-coefficient matrix (plans built with
 * POLYLAB_PLAN_GEMM): closure size K, padded output columns Npad, the number
 * of 64 x 256 BF16 blocks and of 32 x 256 TF32 blocks that hold a nonzero
 * (the tensor-core work one 128-point tile issues).  Any pointer may be NULL.
 * Synchronous (reads a small table back). */
polylab_status polylab_plan_gemm_info(const polylab_plan* plan, int64_t* K, int32_t* Npad,
                                      int64_t* bf16_live_halves, int64_t* tf32_live_tiles);

/* ------------------------------------------------------------ derivatives at points */

typedef enum {
  POLYLAB_FP64 = 0,    /* FP64 throughout (direct per-term sums)                          */
  POLYLAB_TF32X3 = 1,  /* monomial x derived-coefficient contraction on tensor cores,
                          3xTF32 split operands, FP32 accumulation                         */
  POLYLAB_BF16 = 2,    /* same contraction in BF16 with FP32 accumulation, per-column
                          coefficient scaling                                              */
  POLYLAB_FP32 = 3,    /* FP32 direct per-term sums (affine normal: FP32 derivative sums,
                          FP64 Cholesky / log-det / normalisation)                         */
  POLYLAB_F32X2 = 4    /* affine normal, MF_EXACT only: double-word arithmetic (pairs of
                          FP32, ~48 significand bits, on the FP32 pipe) for the term sums,
                          the inverse and W, with FP64 accumulation of the gradient and
                          Hessian sums and the FP64 frame update, Cholesky / log-det and
                          normalisation; held to the FP64 form's error bars             */
} polylab_precision;

/* f, grad f and the Hessian at P points (Sec. 3.3 differentiation and eval;
 * batched).  X: DEVICE, P x n row-major, in the polynomial's variable order.
 * order = 0, 1 or 2 selects which of F, G, H are written.
 * F: DEVICE P; G: DEVICE P x n (order >= 1); H: DEVICE P x n x n, full
 * symmetric matrix (order 2).  Outputs are overwritten.  With POLYLAB_FP64
 * every output agrees with the plain definition within ~1e-15 of the sum of
 * |term contributions|; reduced forms carry their stated error.
 * Asynchronous in every form when `plan` is given (a NULL plan builds a
 * temporary one, which synchronises `stream`).  The tensor-core forms
 * (POLYLAB_TF32X3, POLYLAB_BF16; the plan must be built with
 * POLYLAB_PLAN_GEMM) bound every device-side wait: a wait that gives up --
 * a safety net, not an expected event -- writes NaN to the outputs of its
 * 128-point tile and is reported by the next polylab_eval_check. */
polylab_status polylab_eval_derivs(const polylab_poly* p, const polylab_plan* plan, const double* X,
                                   int64_t P, int32_t order, polylab_precision prec, double* F,
                                   double* G, double* H, polylab_stream stream);

/* Synchronises `stream` and reports whether a bounded wait of a tensor-core
 * polylab_eval_derivs call on the current device gave up since the last
 * check: POLYLAB_ERR_TIMEOUT then (message in polylab_last_error(); the
 * record is cleared), POLYLAB_OK otherwise.  The record is one word per
 * device, shared by every stream and thread. */
polylab_status polylab_eval_check(polylab_stream stream);

/* ------------------------------------------------------------ affine normal (Sec. 5) */

/* Sec. 5 lists three methods: 'mf-exact' (MF-logDet-Exact, the default),
 * 'mf-stochastic' (MF-logDet-Stochastic) and 'ad', the reference route that
 * forms the derivatives literally, the full third-derivative tensor included
 * (POLYLAB_AD: n <= POLYLAB_AD_MAX_N, FP64 only). */
typedef enum { POLYLAB_MF_EXACT = 0, POLYLAB_MF_STOCHASTIC = 1, POLYLAB_AD = 2 } polylab_an_method;
#define POLYLAB_AD_MAX_N 24
typedef enum {
  POLYLAB_PRECOND_JACOBI = 0,  /* |diag(H)| + r of the ambient Hessian, projected      */
  POLYLAB_PRECOND_NONE = 1,
  POLYLAB_PRECOND_MLP = 2      /* learned diagonal-plus-low-rank (needs mlp_weights)   */
} polylab_precond;

/* Options (Sec. 5, Table "affineopts").  Paper defaults: method MF_EXACT,
 * regularization 1e-6, num_probes 8, krylov_tol 1e-4, krylov_maxit 40. */
typedef struct {
  polylab_an_method method;
  double regularization;     /* r: H_T + r I in every tangent solve                 */
  int32_t num_probes;        /* q, stochastic only                                  */
  double krylov_tol;         /* stop when |residual| <= tol |rhs|, stochastic only  */
  int32_t krylov_maxit;      /* stochastic only                                     */
  int32_t assume_nonzero_x;  /* skip the relative zero-gradient check               */
  uint64_t seed;             /* probe generator seed, stochastic only               */
  polylab_precision prec;    /* POLYLAB_FP64, POLYLAB_FP32, or POLYLAB_F32X2 (MF_EXACT) */
  polylab_precond precond;   /* stochastic only                                     */
  const void* mlp_weights;   /* DEVICE, POLYLAB_PRECOND_MLP only                    */
} polylab_an_opts;

void polylab_an_opts_default(polylab_an_opts* o);

#define POLYLAB_FLAG_ZERO_GRAD 1    /* |grad f| = 0 (or relatively negligible)    */
#define POLYLAB_FLAG_NOT_PD 2       /* Cholesky of H_T + r I failed              */
#define POLYLAB_FLAG_KRYLOV_MAXIT 4 /* a Krylov solve stopped at krylov_maxit    */

/* Per-point diagnostics (Sec. 5 "info": gradient norm and work counters). */
typedef struct {
  double grad_norm;
  double logdet;       /* log det(H_T + r I), exact method (NaN for stochastic) */
  int32_t flags;
  int32_t hv_evals;    /* exact: n; stochastic: Krylov iterations + 1           */
  int32_t third_evals; /* exact: n - 1; stochastic: q                           */
  int32_t krylov_iters;
} polylab_an_info;

/* The affine-normal direction at P points (Sec. 5):
 *   e = g/|g|, Q = [Q_T, e], H_T = Q_T^T H Q_T + r I, h = Q_T^T H e,
 *   a_i = tr(H_T^{-1} d_{t_i} H_T), tau = H_T^{-1}(h - |g|/(n+1) a),
 *   D = nu = Q_T tau - e   (the paper's d: nu . e = -1, not unit length).
 * MF_EXACT forms a with the exact trace; MF_STOCHASTIC with a Hutchinson
 * estimate over num_probes probes and preconditioned CG solves; AD from the
 * materialised third-derivative tensor T: a_i = tr(H_T^{-1} Q_T^T S_i Q_T)
 * with S_i = sum_l T(l, :, :) (Q_T)_li, one CTA per point, FP64, every
 * per-point array in shared memory (POLYLAB_ERR_UNSUPPORTED when n >
 * POLYLAB_AD_MAX_N or the arrays do not fit; POLYLAB_ERR_INVALID_ARG unless
 * prec is POLYLAB_FP64).
 * X: DEVICE P x n.  D: DEVICE P x n.  Dunit: DEVICE P x n or NULL (nu/|nu|).
 * info: DEVICE array of P records or NULL.  Flagged points get NaN rows. */
polylab_status polylab_affine_normal(const polylab_poly* p, const polylab_plan* plan, const double* X,
                                     int64_t P, const polylab_an_opts* opts, double* D, double* Dunit,
                                     polylab_an_info* info, polylab_stream stream);

/* ------------------------------------------------- learned preconditioner */

/* A small network mapping per-coordinate Hessian features of a point to a
 * diagonal-plus-low-rank preconditioner Pi (D + U U^T) Pi for the Krylov
 * solves of POLYLAB_MF_STOCHASTIC (this library's addition; the paper uses
 * plain Krylov solves).  Features of coordinate i, with a_i = |H_ii| + r:
 *   [log(a_i), log(sum_{j != i} sum_t |d_i d_j t(x)| + r), x_i, n e_i^2,
 *    log(|g_i| + 1e-30), sum_{j != i} H_ij / a_i, sum_{j != i} H_ij / a_j];
 * network 7 -> 32 (tanh) -> 3; D_i = exp(clip(o_0, -5, 5)) / a_i,
 * U_ik = 0.1 o_k / sqrt(a_i).  Zero output weights reproduce Jacobi.
 * Parameters: POLYLAB_MLP_PARAMS floats (W1 7x32 row-major, b1, W2 32x3, b2).
 * Inference uses a BF16 copy (polylab_mlp_pack) passed as opts.mlp_weights. */
#define POLYLAB_MLP_PARAMS 355
#define POLYLAB_MLP_FEATURES 7
#define POLYLAB_MLP_PROBES 4

int32_t polylab_mlp_param_count(void);
/* W1 uniform in +-1/sqrt(7) and the low-rank outputs' weights (W2 columns
 * 1, 2) uniform in +-0.05, from SplitMix64(seed); everything else 0, so D
 * starts at Jacobi (U = 0 would be a stationary point of the loss).  DEVICE
 * params. */
polylab_status polylab_mlp_init(float* params, uint64_t seed, polylab_stream stream);
/* Training data generated by the method itself at P points: per point,
 * feats (DEVICE P x n x 7), hdiag = H_ii (P x n), e = g/|g| (P x n), and
 * POLYLAB_MLP_PROBES probe pairs z_k = Pi w_k (Rademacher w_k from
 * SplitMix64(seed), probe index p*4 + k, the probe convention of the
 * stochastic method) and y_k = Pi (H + rI) z_k, stored Z, Y (P x n x 4).
 * FP32.  Points with zero gradient are not allowed here. */
polylab_status polylab_mlp_data(const polylab_poly* p, const polylab_plan* plan, const double* X, int64_t P,
                                double regularization, uint64_t seed, float* feats, float* hdiag, float* e,
                                float* Z, float* Y, polylab_stream stream);
/* Mean over points and probes of |Pi (D y + U U^T y) - z|^2 / |z|^2 and its
 * gradient (hand-written backpropagation).  grad: DEVICE 355 floats, loss:
 * DEVICE 1 float, both overwritten. */
polylab_status polylab_mlp_loss_grad(const float* params, int64_t P, int32_t n, const float* feats,
                                     const float* hdiag, const float* e, const float* Z, const float* Y,
                                     double regularization, float* grad, float* loss, polylab_stream stream);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8); m, v: DEVICE 355 floats, zero at step 1. */
polylab_status polylab_mlp_adam(float* params, const float* grad, float* m, float* v, int32_t step, float lr,
                                polylab_stream stream);
/* BF16 copy of the parameters for inference (DEVICE, 355 x 2 bytes). */
polylab_status polylab_mlp_pack(const float* params, void* packed, polylab_stream stream);

/* ------------------------------------------- batched exact directions (one graph) */

/* A batch is a set of polynomials (each with its own n, term list and point
 * set) whose exact affine-normal directions are computed by three stages of
 * persistent kernel launches over all of them (polylab_batch_config; the
 * frame stage may run as one launch per class of n): (polynomial, point)
 * work items are taken from a device counter per launch, most expensive
 * polynomials first, so an uneven batch keeps every SM busy.
 * The stages pass each point's H, W (n x n in the form's precision) and a few
 * vectors through a workspace the batch owns (sum over polynomials of
 * P_i (n_i^2 x 2 x element size + (4 n_i + 8) x 8) bytes).
 * polylab_batch_create uploads the descriptors and allocates the workspace
 * (and builds a term plan for every NULL entry of `plans`; `polys` may then
 * not be NULL), so polylab_batch_run only enqueues the work-counter memsets
 * and the stages' kernels (three to five) on `stream` and may be captured
 * into a CUDA graph and replayed.  Each run overwrites
 * D[i], Dunit[i] (DEVICE P[i] x n_i or NULL) and info[i] (DEVICE P[i] records
 * or NULL) from X[i] (DEVICE P[i] x n_i).  opts->method must be
 * POLYLAB_MF_EXACT; opts->prec POLYLAB_FP64, POLYLAB_FP32 or POLYLAB_F32X2.  The arrays of
 * pointers passed to create are read during the call only. */
typedef struct polylab_batch polylab_batch;

/* Launch configuration.  A run is three stages of persistent launches over the same
 * (polynomial, point) items: the gradient/Hessian term sweep, the frame stage
 * (projected Hessian, FP64 LDL^T, inverse) and the third-derivative sweep with
 * the direction.  threads: frame-stage CTA size (64, 128 or 256 threads per
 * point); ctas_per_sm: cap on resident frame-stage CTAs per SM (0: the
 * occupancy limit); order: 1 = most expensive polynomials first, 0 = as
 * given; term_threads: CTA size of the gradient/Hessian term sweep (64, 128
 * or 256; third_threads, below, sizes the third-derivative sweep). */
typedef struct {
  int32_t threads;
  int32_t ctas_per_sm;
  int32_t order;
  int32_t term_threads;
  /* terms_ctas, third_ctas: caps on resident CTAs per SM of the two term
   * sweeps (0: the occupancy limit). */
  int32_t terms_ctas;
  int32_t third_ctas;
  /* frame_split (0 or 1): the frame stage runs as up to three launches over
   * classes of polynomials by n (n > 40 with `threads` per CTA, 24 < n <= 40
   * and n <= 24 with 64), each sized for its class's largest n and taken in an
   * order of n descending; ctas_per_sm caps the first class only.  0: one
   * launch over all polynomials. */
  int32_t frame_split;
  int32_t third_threads;  /* CTA size of the third-derivative sweep (64, 128 or 256) */
  /* third_split (1..4): the third-derivative sweep as that many launches over
   * ranges of term support sizes ({1..8}; {1..4},{5..8}; {1..4},{5},{6..8};
   * {1..3},{4},{5},{6..8}), each contracting its terms into the point's
   * partial trace term and the last forming the direction: every launch then
   * runs one support size's code at a time on all SMs (instruction-cache
   * locality), at the price of loading W once per launch.  Each range runs as
   * one launch per class of n of the frame stage (n > 40, 24 < n <= 40,
   * n <= 24), each sized for its class's shared memory. */
  int32_t third_split;
} polylab_batch_config;

polylab_status polylab_batch_create(int32_t n_polys, const polylab_poly* polys,
                                    const polylab_plan* const* plans, const double* const* X,
                                    const int64_t* P, const polylab_an_opts* opts, double* const* D,
                                    double* const* Dunit, polylab_an_info* const* info,
                                    polylab_stream stream, polylab_batch** batch);
polylab_status polylab_batch_run(polylab_batch* batch, polylab_stream stream);
/* One stage of a run (0: term sweep, 1: frame stage, 2: third-derivative
 * sweep and directions), for timing the stages separately: a stage reads what
 * the previous stages of an earlier or the same run left in the workspace,
 * so stage s may only be run after stages 0..s-1 have run on the same inputs.
 * POLYLAB_ERR_INVALID_ARG for another stage number. */
polylab_status polylab_batch_run_stage(polylab_batch* batch, int32_t stage, polylab_stream stream);
/* Synchronises `stream` and reports whether any run of this batch gave up a
 * bounded wait (a bulk copy into shared memory that did not complete within
 * two seconds) since the last check: POLYLAB_ERR_TIMEOUT then (the stage is
 * named in polylab_last_error(); the record is cleared, so the batch may run
 * again), POLYLAB_OK otherwise.  The same record carries an internal
 * consistency failure of the term sweep (its list of passes left to the
 * term-by-term kernel overflowed: not reachable with the list's sizing), then
 * reported as POLYLAB_ERR_UNSUPPORTED. */
polylab_status polylab_batch_check(polylab_batch* batch, polylab_stream stream);
polylab_status polylab_batch_get_config(const polylab_batch* batch, polylab_batch_config* cfg);
polylab_status polylab_batch_set_config(polylab_batch* batch, const polylab_batch_config* cfg,
                                        polylab_stream stream);
/* The project's autotuner, stage by stage on this batch (one warm-up and
 * `reps` timed runs per trial, CUDA events on `stream`, synchronising):
 * term_threads in {64,128,256} timed over the gradient/Hessian sweep and
 * third_threads in {64,128,256} and then third_split in {1,2,3} over the
 * third-derivative sweep, then
 * frame_split in {1, 0} x threads in {64,128,256} x ctas_per_sm in
 * {occupancy, 2, 4} timed over the frame stage,
 * then order in {cost order, given order} timed over the whole run.  Keeps
 * the fastest of each step and returns the result
 * (and the mean time of a whole run in ms, if best_ms is not NULL).  The
 * outputs hold the last run's results. */
polylab_status polylab_batch_autotune(polylab_batch* batch, int32_t reps, polylab_stream stream,
                                      polylab_batch_config* chosen, float* best_ms);
polylab_status polylab_batch_destroy(polylab_batch* batch, polylab_stream stream);

/* create + run + destroy in one call. */
polylab_status polylab_affine_normal_batched(int32_t n_polys, const polylab_poly* polys,
                                             const polylab_plan* const* plans, const double* const* X,
                                             const int64_t* P, const polylab_an_opts* opts, double* const* D,
                                             double* const* Dunit, polylab_an_info* const* info,
                                             polylab_stream stream);

/* ----------------------------------------------------- single-precision storage */

/* The paper's precision control (Sec. 3.5: polylab_precision('set','single'),
 * after which new polynomials carry single-precision coefficients and the
 * core operations and affine-normal routes run in single precision; Table
 * "precision" of Sec. 6 compares eval, simplify, mpower, MF-logDet-Exact and
 * MF-logDet-Stochastic in double and single).  Here the precision is a
 * property of the data: polylab_poly_f32 is polylab_poly with FP32
 * coefficients, and each call below is its FP64 namesake with:
 *   engine calls (simplify/mul/add/sub/pow/diff): coefficients read as FP32,
 *     products, negation and merged sums computed in FP32 (sums in an order
 *     of the library's choosing), stored FP32; the zeroprec test compares
 *     |c| of the FP32 sum (exactly widened) with zeroprec; exponents and the
 *     term order are those of the FP64 call, bit for bit;
 *   polylab_plan_create_f32: a plan usable by every call that takes a plan
 *     (the FP32 coefficients are held exactly);
 *   polylab_eval_derivs_f32: the POLYLAB_FP32 direct form (FP32 power
 *     tables, term products and sums) with FP32 points X (P x n) and FP32
 *     outputs F, G, H laid out as in polylab_eval_derivs;
 *   polylab_affine_normal_f32: the POLYLAB_FP32 form of the route in
 *     opts->method (MF_EXACT or MF_STOCHASTIC; opts->prec must be
 *     POLYLAB_FP32) at FP32 points, D and Dunit rounded to FP32; the points
 *     are widened on the device into stream-ordered scratch first.
 * Argument rules, errors and synchronisation are those of the FP64 calls. */
typedef struct {
  int32_t n_vars;
  const uint64_t* var_ids;  /* HOST                    */
  int64_t n_terms;
  const uint8_t* exps;      /* DEVICE, m x n row-major */
  const float* coef;        /* DEVICE, m coefficients  */
} polylab_poly_f32;

typedef struct {
  int32_t n_vars;
  uint64_t* var_ids;
  int64_t n_terms;
  uint8_t* exps;
  float* coef;              /* n_terms, from alloc */
} polylab_poly_out_f32;

polylab_status polylab_simplify_f32(const polylab_poly_f32* p, double zeroprec, polylab_poly_out_f32* out,
                                    polylab_alloc_fn alloc, void* alloc_ctx, polylab_stream stream);
polylab_status polylab_mul_f32(const polylab_poly_f32* a, const polylab_poly_f32* b, double zeroprec,
                               polylab_poly_out_f32* out, polylab_alloc_fn alloc, void* alloc_ctx,
                               polylab_stream stream);
polylab_status polylab_add_f32(const polylab_poly_f32* a, const polylab_poly_f32* b, double zeroprec,
                               polylab_poly_out_f32* out, polylab_alloc_fn alloc, void* alloc_ctx,
                               polylab_stream stream);
polylab_status polylab_sub_f32(const polylab_poly_f32* a, const polylab_poly_f32* b, double zeroprec,
                               polylab_poly_out_f32* out, polylab_alloc_fn alloc, void* alloc_ctx,
                               polylab_stream stream);
polylab_status polylab_pow_f32(const polylab_poly_f32* p, int32_t k, double zeroprec, polylab_poly_out_f32* out,
                               polylab_alloc_fn alloc, void* alloc_ctx, polylab_stream stream);
polylab_status polylab_diff_f32(const polylab_poly_f32* p, uint64_t var_id, double zeroprec,
                                polylab_poly_out_f32* out, polylab_alloc_fn alloc, void* alloc_ctx,
                                polylab_stream stream);
polylab_status polylab_plan_create_f32(const polylab_poly_f32* p, uint32_t what, polylab_stream stream,
                                       polylab_plan** plan);
polylab_status polylab_eval_derivs_f32(const polylab_poly_f32* p, const polylab_plan* plan, const float* X,
                                       int64_t P, int32_t order, float* F, float* G, float* H,
                                       polylab_stream stream);
polylab_status polylab_affine_normal_f32(const polylab_poly_f32* p, const polylab_plan* plan, const float* X,
                                         int64_t P, const polylab_an_opts* opts, float* D, float* Dunit,
                                         polylab_an_info* info, polylab_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* POLYLAB_H */
