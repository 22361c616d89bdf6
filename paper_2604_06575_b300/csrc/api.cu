// extern "C" entry points: argument checks, temporary plans, dispatch.
#include <algorithm>

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
  template <typename Pub>
  polylab_status init(const Pub* p, const polylab_plan* given, uint32_t what) {
    if (given) {
      if (p && (p->n_vars != given->n || p->n_terms != given->m)) return POLYLAB_ERR_INVALID_ARG;
      if ((what & POLYLAB_PLAN_GEMM) && !given->gemm) return POLYLAB_ERR_INVALID_ARG;
      plan = given;
      return POLYLAB_OK;
    }
    PL_TRY(create(p, what, (polylab_stream)s, &owned));
    plan = owned;
    return POLYLAB_OK;
  }
  static polylab_status create(const polylab_poly* p, uint32_t what, polylab_stream st, polylab_plan** out) {
    return polylab_plan_create(p, what, st, out);
  }
  static polylab_status create(const polylab_poly_f32* p, uint32_t what, polylab_stream st, polylab_plan** out) {
    return polylab_plan_create_f32(p, what, st, out);
  }
};

polylab_status check_an_opts(const polylab_an_opts* o) {
  if (o->method != POLYLAB_MF_EXACT && o->method != POLYLAB_MF_STOCHASTIC && o->method != POLYLAB_AD)
    return POLYLAB_ERR_INVALID_ARG;
  if (o->prec != POLYLAB_FP64 && o->prec != POLYLAB_FP32 &&
      !(o->prec == POLYLAB_F32X2 && o->method == POLYLAB_MF_EXACT))
    return POLYLAB_ERR_INVALID_ARG;
  if (!(o->regularization >= 0.0)) return POLYLAB_ERR_INVALID_ARG;
  if (o->method == POLYLAB_MF_STOCHASTIC) {
    if (o->num_probes < 1 || o->krylov_maxit < 0 || !(o->krylov_tol >= 0.0)) return POLYLAB_ERR_INVALID_ARG;
    if (o->precond < POLYLAB_PRECOND_JACOBI || o->precond > POLYLAB_PRECOND_MLP) return POLYLAB_ERR_INVALID_ARG;
    if (o->precond == POLYLAB_PRECOND_MLP && !o->mlp_weights) return POLYLAB_ERR_INVALID_ARG;
  }
  return POLYLAB_OK;
}

polylab_status run_route(const polylab_plan* plan, const double* X, int64_t P, const polylab_an_opts* o, double* D,
                         double* Dunit, polylab_an_info* info, cudaStream_t s) {
  if (o->method == POLYLAB_MF_EXACT) return affine_exact(plan, X, P, o, D, Dunit, info, s);
  if (o->method == POLYLAB_AD) return affine_ad(plan, X, P, o, D, Dunit, info, s);
  return affine_stochastic(plan, X, P, o, D, Dunit, info, s);
}

// FP32 <-> FP64 copies for the single-precision storage calls
__global__ void widen_kernel(const float* __restrict__ in, int64_t n, double* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (double)in[i];
}
__global__ void narrow_kernel(const double* __restrict__ in, int64_t n, float* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}
unsigned copy_grid(int64_t n) { return (unsigned)std::min<int64_t>(ceil_div(n, 256), (int64_t)num_sms() * 8); }

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
  PL_TRY(check_an_opts(o));
  cudaStream_t s = (cudaStream_t)stream;
  PlanRef pr(s);
  PL_TRY(pr.init(p, plan, POLYLAB_PLAN_TERMS));
  return run_route(pr.plan, X, P, o, D, Dunit, info, s);
}

polylab_status polylab_eval_derivs_f32(const polylab_poly_f32* p, const polylab_plan* plan, const float* X,
                                       int64_t P, int32_t order, float* F, float* G, float* H,
                                       polylab_stream stream) {
  if (P < 0 || order < 0 || order > 2 || (!p && !plan)) return POLYLAB_ERR_INVALID_ARG;
  if (P > 0 && (!X || !F || (order >= 1 && !G) || (order >= 2 && !H))) return POLYLAB_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  PlanRef pr(s);
  PL_TRY(pr.init(p, plan, POLYLAB_PLAN_TERMS));
  return eval_direct_f32(pr.plan, X, P, order, F, G, H, s);
}

polylab_status polylab_affine_normal_f32(const polylab_poly_f32* p, const polylab_plan* plan, const float* X,
                                         int64_t P, const polylab_an_opts* o, float* D, float* Dunit,
                                         polylab_an_info* info, polylab_stream stream) {
  if (!o || P < 0 || (!p && !plan)) return POLYLAB_ERR_INVALID_ARG;
  if (P > 0 && (!X || !D)) return POLYLAB_ERR_INVALID_ARG;
  PL_TRY(check_an_opts(o));
  if (o->method == POLYLAB_AD || o->prec != POLYLAB_FP32) return POLYLAB_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  PlanRef pr(s);
  PL_TRY(pr.init(p, plan, POLYLAB_PLAN_TERMS));
  if (P == 0) return POLYLAB_OK;
  const int64_t len = P * (int64_t)pr.plan->n;
  Scratch scr(s);
  double *Xd = nullptr, *Dd = nullptr, *Dud = nullptr;
  PL_TRY(scr.get(&Xd, (size_t)len));
  PL_TRY(scr.get(&Dd, (size_t)len));
  if (Dunit) PL_TRY(scr.get(&Dud, (size_t)len));
  widen_kernel<<<copy_grid(len), 256, 0, s>>>(X, len, Xd);
  PL_TRY(launch_status("widen_kernel"));
  PL_TRY(run_route(pr.plan, Xd, P, o, Dd, Dud, info, s));
  narrow_kernel<<<copy_grid(len), 256, 0, s>>>(Dd, len, D);
  if (Dunit) narrow_kernel<<<copy_grid(len), 256, 0, s>>>(Dud, len, Dunit);
  return launch_status("narrow_kernel");
}

}  // extern "C"
