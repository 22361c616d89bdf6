// extern "C" entry points: argument checks, temporary plans, dispatch.
#include "common.cuh"

using namespace polylab;

namespace {

// Use the caller's plan or build a temporary term-list plan for this call.
struct PlanRef {
  const polylab_plan* plan = nullptr;
  polylab_plan* owned = nullptr;
  cudaStream_t s;
  explicit PlanRef(cudaStream_t st) : s(st) {}
  ~PlanRef() {
    if (owned) polylab_plan_destroy(owned, (polylab_stream)s);
  }
  polylab_status init(const polylab_poly* p, const polylab_plan* given, uint32_t what) {
    if (given) {
      if (p && (p->n_vars != given->n || p->n_terms != given->m)) return POLYLAB_ERR_INVALID_ARG;
      if ((what & POLYLAB_PLAN_GEMM) && !given->gemm) return POLYLAB_ERR_INVALID_ARG;
      plan = given;
      return POLYLAB_OK;
    }
    PL_TRY(polylab_plan_create(p, what, (polylab_stream)s, &owned));
    plan = owned;
    return POLYLAB_OK;
  }
};

}  // namespace

extern "C" {

polylab_status polylab_eval_derivs(const polylab_poly* p, const polylab_plan* plan, const double* X, int64_t P,
                                   int32_t order, polylab_precision prec, double* F, double* G, double* H,
                                   polylab_stream stream) {
  if (P < 0 || order < 0 || order > 2 || (!p && !plan)) return POLYLAB_ERR_INVALID_ARG;
  if (P > 0 && (!X || !F || (order >= 1 && !G) || (order >= 2 && !H))) return POLYLAB_ERR_INVALID_ARG;
  if (prec < POLYLAB_FP64 || prec > POLYLAB_FP32) return POLYLAB_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const bool gemm = prec == POLYLAB_TF32X3 || prec == POLYLAB_BF16;
  PlanRef pr(s);
  PL_TRY(pr.init(p, plan, gemm ? POLYLAB_PLAN_GEMM : POLYLAB_PLAN_TERMS));
  if (gemm) return eval_gemm(pr.plan, X, P, order, (int)prec, F, G, H, s);
  return eval_direct(pr.plan, X, P, order, prec == POLYLAB_FP32, F, G, H, s);
}

polylab_status polylab_affine_normal(const polylab_poly* p, const polylab_plan* plan, const double* X, int64_t P,
                                     const polylab_an_opts* o, double* D, double* Dunit, polylab_an_info* info,
                                     polylab_stream stream) {
  if (!o || P < 0 || (!p && !plan)) return POLYLAB_ERR_INVALID_ARG;
  if (P > 0 && (!X || !D)) return POLYLAB_ERR_INVALID_ARG;
  if (o->method != POLYLAB_MF_EXACT && o->method != POLYLAB_MF_STOCHASTIC && o->method != POLYLAB_AD)
    return POLYLAB_ERR_INVALID_ARG;
  if (o->prec != POLYLAB_FP64 && o->prec != POLYLAB_FP32) return POLYLAB_ERR_INVALID_ARG;
  if (!(o->regularization >= 0.0)) return POLYLAB_ERR_INVALID_ARG;
  if (o->method == POLYLAB_MF_STOCHASTIC) {
    if (o->num_probes < 1 || o->krylov_maxit < 0 || !(o->krylov_tol >= 0.0)) return POLYLAB_ERR_INVALID_ARG;
    if (o->precond < POLYLAB_PRECOND_JACOBI || o->precond > POLYLAB_PRECOND_MLP) return POLYLAB_ERR_INVALID_ARG;
    if (o->precond == POLYLAB_PRECOND_MLP && !o->mlp_weights) return POLYLAB_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  PlanRef pr(s);
  PL_TRY(pr.init(p, plan, POLYLAB_PLAN_TERMS));
  if (o->method == POLYLAB_MF_EXACT) return affine_exact(pr.plan, X, P, o, D, Dunit, info, s);
  if (o->method == POLYLAB_AD) return affine_ad(pr.plan, X, P, o, D, Dunit, info, s);
  return affine_stochastic(pr.plan, X, P, o, D, Dunit, info, s);
}

}  // extern "C"
