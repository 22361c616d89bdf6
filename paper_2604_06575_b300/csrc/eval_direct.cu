// Direct per-term evaluation of f, grad f and the Hessian at a batch of points
// (Sec. 3.3 term-by-term differentiation, evaluated numerically; the FP64 form
// of the batched derivative evaluation).
//
// A CTA owns TP consecutive points.  Thread t works for point t % TP and walks
// the term list with stride blockDim/TP, so every term is read from L2 once
// per CTA and shared by TP points.  Contributions are accumulated in shared
// memory (layout acc[output][point], conflict-free across the TP lanes that
// share a term) with shared-memory atomics; the Hessian is accumulated as its
// upper triangle and mirrored on the way out.  When the accumulators of a
// single point do not fit in shared memory the kernel accumulates straight
// into the zero-initialised global outputs instead.
#include <algorithm>

#include "common.cuh"
#include "terms.cuh"

namespace polylab {

__host__ __device__ __forceinline__ int tri_index(int i, int j, int n) {  // i <= j
  return i * (2 * n - i + 1) / 2 + (j - i);
}

// R: arithmetic type; IO: type of the points and outputs (FP64, or FP32 for
// the single-precision storage calls).
template <typename R, typename IO, int ORDER>
__global__ void __launch_bounds__(256) eval_direct_smem(const Term* __restrict__ terms, int64_t m, int n, int E,
                                                       const IO* __restrict__ X, int64_t P, int TP,
                                                       IO* __restrict__ F, IO* __restrict__ G,
                                                       IO* __restrict__ H) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int E1 = E + 1;
  const int nH = ORDER >= 2 ? n * (n + 1) / 2 : 0;
  const int NO = 1 + (ORDER >= 1 ? n : 0) + nH;
  R* acc = reinterpret_cast<R*>(smem_raw);  // [NO][TP]
  R* pw = acc + (size_t)NO * TP;            // [TP][n][E1]
  const int64_t p0 = (int64_t)blockIdx.x * TP;
  const int tp = (int)std::min<int64_t>(TP, P - p0);

  for (int i = threadIdx.x; i < NO * TP; i += blockDim.x) acc[i] = R(0);
  for (int i = threadIdx.x; i < TP * n; i += blockDim.x) {
    const int p = i / n, v = i - p * n;
    const R x = p < tp ? R(X[(p0 + p) * n + v]) : R(0);
    R* w = pw + (size_t)(p * n + v) * E1;
    R cur = R(1);
    w[0] = cur;
    for (int k = 1; k <= E; ++k) {
      cur = cur * R(x);
      w[k] = cur;
    }
  }
  __syncthreads();

  const int p = threadIdx.x % TP;
  const int lanes = blockDim.x / TP;
  const int tl = threadIdx.x / TP;
  if (tl < lanes && p < tp) {
    const R* mypw = pw + (size_t)p * n * E1;
    for (int64_t t = tl; t < m; t += lanes) {
      const TermRegs tr = load_term(terms, t);
      term_derivs<R, ORDER>(tr, mypw, E1, [&](int kind, int i, int j, R v) {
        int o = kind == 0 ? 0 : kind == 1 ? 1 + i : 1 + n + tri_index(i, j, n);
        atomicAdd(&acc[(size_t)o * TP + p], v);
      });
    }
  }
  __syncthreads();

  for (int i = threadIdx.x; i < tp; i += blockDim.x) F[p0 + i] = (IO)acc[i];
  if (ORDER >= 1)
    for (int i = threadIdx.x; i < tp * n; i += blockDim.x) {
      const int pp = i / n, v = i - pp * n;
      G[p0 * n + i] = (IO)acc[(size_t)(1 + v) * TP + pp];
    }
  if (ORDER >= 2) {
    const int nn = n * n;
    for (int i = threadIdx.x; i < tp * nn; i += blockDim.x) {
      const int pp = i / nn, r = i - pp * nn;
      const int a = r / n, b = r - a * n;
      const int o = 1 + n + (a <= b ? tri_index(a, b, n) : tri_index(b, a, n));
      H[p0 * nn + i] = (IO)acc[(size_t)o * TP + pp];
    }
  }
}

// Fallback for large n: one CTA per point, global atomics into zeroed outputs.
template <typename R, typename IO, int ORDER>
__global__ void __launch_bounds__(256) eval_direct_global(const Term* __restrict__ terms, int64_t m, int n, int E,
                                                         const IO* __restrict__ X, int64_t P,
                                                         IO* __restrict__ F, IO* __restrict__ G,
                                                         IO* __restrict__ H) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int E1 = E + 1;
  R* pw = reinterpret_cast<R*>(smem_raw);
  for (int64_t p = blockIdx.x; p < P; p += gridDim.x) {
    __syncthreads();
    for (int v = threadIdx.x; v < n; v += blockDim.x) {
      const R x = R(X[p * n + v]);
      R cur = R(1);
      pw[v * E1] = cur;
      for (int k = 1; k <= E; ++k) {
        cur = cur * R(x);
        pw[v * E1 + k] = cur;
      }
    }
    __syncthreads();
    for (int64_t t = threadIdx.x; t < m; t += blockDim.x) {
      const TermRegs tr = load_term(terms, t);
      term_derivs<R, ORDER>(tr, pw, E1, [&](int kind, int i, int j, R v) {
        const IO dv = (IO)v;
        if (kind == 0) atomicAdd(&F[p], dv);
        else if (kind == 1) atomicAdd(&G[p * n + i], dv);
        else {
          atomicAdd(&H[(p * n + i) * n + j], dv);
          if (i != j) atomicAdd(&H[(p * n + j) * n + i], dv);
        }
      });
    }
  }
}

template <typename R, typename IO, int ORDER>
static polylab_status launch_direct(const polylab_plan* plan, const IO* X, int64_t P, IO* F, IO* G, IO* H,
                                    cudaStream_t s) {
  const int n = plan->n, E = std::max(plan->max_exp, 1);
  const int nH = ORDER >= 2 ? n * (n + 1) / 2 : 0;
  const size_t NO = 1 + (ORDER >= 1 ? n : 0) + nH;
  const size_t per_point = (NO + (size_t)n * (E + 1)) * sizeof(R);
  const size_t budget = 100 * 1024;  // two CTAs per SM
  int TP = 0;
  for (int cand : {32, 16, 8, 4, 2, 1})
    if (cand * per_point <= budget) {
      TP = cand;
      break;
    }
  if (TP > 0) {
    const size_t smem = TP * per_point;
    auto k = eval_direct_smem<R, IO, ORDER>;
    PL_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k<<<(unsigned)ceil_div(P, TP), 256, smem, s>>>(plan->terms, plan->m, n, E, X, P, TP, F, G, H);
    return launch_status("eval_direct_smem");
  }
  PL_CUDA(cudaMemsetAsync(F, 0, P * sizeof(IO), s));
  if (ORDER >= 1) PL_CUDA(cudaMemsetAsync(G, 0, P * n * sizeof(IO), s));
  if (ORDER >= 2) PL_CUDA(cudaMemsetAsync(H, 0, P * (size_t)n * n * sizeof(IO), s));
  const size_t smem = (size_t)n * (E + 1) * sizeof(R);
  if (smem > 200 * 1024) return POLYLAB_ERR_UNSUPPORTED;
  auto k = eval_direct_global<R, IO, ORDER>;
  PL_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int grid = (int)std::min<int64_t>(P, (int64_t)num_sms() * 8);
  k<<<grid, 256, smem, s>>>(plan->terms, plan->m, n, E, X, P, F, G, H);
  return launch_status("eval_direct_global");
}

polylab_status eval_direct(const polylab_plan* plan, const double* X, int64_t P, int order, bool fp32, double* F,
                           double* G, double* H, cudaStream_t s) {
  if (P == 0) return POLYLAB_OK;
  if (fp32) {
    if (order == 0) return launch_direct<float, double, 0>(plan, X, P, F, G, H, s);
    if (order == 1) return launch_direct<float, double, 1>(plan, X, P, F, G, H, s);
    return launch_direct<float, double, 2>(plan, X, P, F, G, H, s);
  }
  if (order == 0) return launch_direct<double, double, 0>(plan, X, P, F, G, H, s);
  if (order == 1) return launch_direct<double, double, 1>(plan, X, P, F, G, H, s);
  return launch_direct<double, double, 2>(plan, X, P, F, G, H, s);
}

polylab_status eval_direct_f32(const polylab_plan* plan, const float* X, int64_t P, int order, float* F, float* G,
                               float* H, cudaStream_t s) {
  if (P == 0) return POLYLAB_OK;
  if (order == 0) return launch_direct<float, float, 0>(plan, X, P, F, G, H, s);
  if (order == 1) return launch_direct<float, float, 1>(plan, X, P, F, G, H, s);
  return launch_direct<float, float, 2>(plan, X, P, F, G, H, s);
}

}  // namespace polylab
