// The 'ad' route of Sec. 5: the affine-normal direction evaluated literally
// from the derivatives of f, with the full third-derivative tensor formed at
// every point.  It is the paper's transparent reference method for small n;
// MF-logDet-Exact computes the same direction without the tensor.
//
// One CTA per point (grid-stride over the points), FP64 throughout, all
// per-point data in shared memory:
//   1. g, H and T = d^3 f(x) from the term list: a term adds its derivative
//      values (Sec. 3.3: falling factorials of the exponents times the shifted
//      monomial) to the entries with sorted indices i <= j (<= k); the full
//      symmetric H and T are then filled in by symmetry;
//   2. |g| and the zero-gradient test; e = g/|g|; the explicit orthonormal
//      frame Q = I - beta v v^T with v = e + s e_n (s = sign e_n), so Q e_n =
//      -s e and the first m = n-1 columns Q_T span the complement of e;
//   3. H_T = Q_T^T H Q_T + r I and h = Q_T^T H e; Cholesky H_T = L L^T (a
//      pivot that is not positive flags NOT_PD), log det = 2 sum log L_kk,
//      H_T^{-1} column by column;
//   4. for every tangent axis i: the slice S_i = sum_l T(l, :, :) (Q_T)_{li}
//      (the derivative of H along q_i), d_{t_i} H_T = Q_T^T S_i Q_T and
//      a_i = tr(H_T^{-1} d_{t_i} H_T);
//   5. tau = H_T^{-1}(h - |g|/(n+1) a), nu = Q_T tau - e.
// Step 4 costs O(n^4) per point, which is why the route is for small n.
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "terms.cuh"

namespace polylab {

namespace {

constexpr int kAdMaxN = 24;

// Shared-memory layout of one point (offsets in doubles).
struct AdLay {
  int pw, g, H, T, Q, B, S, HT, Hi, e, v, He, h, a, tau, red, total;
};

__host__ __device__ inline AdLay ad_lay(int n, int E1) {
  const int m = n > 0 ? n - 1 : 0;
  AdLay L;
  int o = 0;
  auto take = [&](int count) {
    const int at = o;
    o += (count + 1) & ~1;  // keep every array 16-byte aligned
    return at;
  };
  L.pw = take(n * E1);
  L.g = take(n);
  L.H = take(n * n);
  L.T = take(n * n * n);
  L.Q = take(n * n);
  L.B = take(n * (m > 0 ? m : 1));
  L.S = take(n * n);
  L.HT = take(m * m);
  L.Hi = take(m * m);
  L.e = take(n);
  L.v = take(n);
  L.He = take(n);
  L.h = take(m);
  L.a = take(m);
  L.tau = take(n);
  L.red = take(40);
  L.total = o;
  return L;
}

template <typename T>
__device__ __forceinline__ T ad_warp_sum(T v) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum of one value per thread over the CTA; every thread gets the result.
template <int NT>
__device__ __forceinline__ double ad_block_sum(double v, double* red) {
  constexpr int NW = NT / 32;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  v = ad_warp_sum(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double s = 0.0;
#pragma unroll
  for (int w = 0; w < NW; ++w) s += red[w];
  return s;
}

// Derivative values of one term with exactly K active variables.
// D[q][s] = a_s (a_s - 1) ... (a_s - q + 1) x_s^(a_s - q) (zero when a_s < q);
// the derivative of the term for an index multiset that takes slot s q_s
// times is c * prod_s D[q_s][s] (slots outside the multiset take D[0]).
// Gradient entries are added to g (and their magnitudes to sg), Hessian
// entries to H(va, vb), va <= vb, third derivatives to T(va, vb, vc),
// va <= vb <= vc (a term's variables are in ascending order).
template <int K>
__device__ __forceinline__ void ad_term(const TermRegs& t, const double* __restrict__ pw, int E1, int n,
                                        double* g, double* H, double* T, double& sg) {
  if constexpr (K == 0) {
    return;
  } else {
    double D[4][K];
#pragma unroll
    for (int s = 0; s < K; ++s) {
      const int es = t.exp[s];
      const double* row = pw + t.var[s] * E1;
      double ff = 1.0;  // falling factorial a (a-1) ... (a-q+1), zero once q > a
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        D[q][s] = ff * row[es >= q ? es - q : 0];
        ff *= (double)(es - q);
      }
    }
    const double c = t.coef;
#pragma unroll
    for (int a = 0; a < K; ++a) {
      double val = c;
#pragma unroll
      for (int s = 0; s < K; ++s) val *= D[s == a][s];
      atomicAdd(&g[t.var[a]], val);
      sg += fabs(val);
#pragma unroll
      for (int b = a; b < K; ++b) {
        double hv = c;
#pragma unroll
        for (int s = 0; s < K; ++s) hv *= D[(s == a) + (s == b)][s];
        atomicAdd(&H[t.var[a] * n + t.var[b]], hv);
#pragma unroll
        for (int d = b; d < K; ++d) {
          double tv = c;
#pragma unroll
          for (int s = 0; s < K; ++s) tv *= D[(s == a) + (s == b) + (s == d)][s];
          atomicAdd(&T[(t.var[a] * n + t.var[b]) * n + t.var[d]], tv);
        }
      }
    }
  }
}

__device__ __forceinline__ void ad_term_any(const TermRegs& t, const double* pw, int E1, int n, double* g,
                                            double* H, double* T, double& sg) {
  switch (t.k) {
    case 0: break;
    case 1: ad_term<1>(t, pw, E1, n, g, H, T, sg); break;
    case 2: ad_term<2>(t, pw, E1, n, g, H, T, sg); break;
    case 3: ad_term<3>(t, pw, E1, n, g, H, T, sg); break;
    case 4: ad_term<4>(t, pw, E1, n, g, H, T, sg); break;
    case 5: ad_term<5>(t, pw, E1, n, g, H, T, sg); break;
    case 6: ad_term<6>(t, pw, E1, n, g, H, T, sg); break;
    case 7: ad_term<7>(t, pw, E1, n, g, H, T, sg); break;
    default: ad_term<8>(t, pw, E1, n, g, H, T, sg); break;
  }
}

struct AdArgs {
  const Term* terms;
  int64_t m_terms;
  int n, E1;
  const double* X;
  int64_t P;
  double r;
  int assume_nonzero_x;
  double* D;
  double* Dunit;
  polylab_an_info* info;
};

template <int NT>
__global__ void __launch_bounds__(NT) affine_ad_kernel(AdArgs A) {
  extern __shared__ __align__(16) double sd[];
  const int tid = threadIdx.x;
  const int n = A.n, m = n - 1, nn = n * n, E1 = A.E1;
  const AdLay L = ad_lay(n, E1);
  double* pw = sd + L.pw;
  double* g = sd + L.g;
  double* H = sd + L.H;
  double* T = sd + L.T;
  double* Q = sd + L.Q;    // Q[i * n + j]
  double* B = sd + L.B;    // n x m scratch, B[i * m + j]
  double* S = sd + L.S;    // n x n slice
  double* HT = sd + L.HT;  // m x m, Cholesky factor in its lower triangle
  double* Hi = sd + L.Hi;  // m x m inverse
  double* e = sd + L.e;
  double* v = sd + L.v;
  double* He = sd + L.He;
  double* h = sd + L.h;
  double* av = sd + L.a;
  double* tau = sd + L.tau;
  double* red = sd + L.red;
  __shared__ int s_flag;
  for (int64_t p = blockIdx.x; p < A.P; p += gridDim.x) {
    const double* x = A.X + p * n;
    // ---- 1. powers, zeroed accumulators, term sweep, symmetric fill
    for (int i = tid; i < n; i += NT) {
      const double xi = x[i];
      double cur = 1.0;
      pw[i * E1] = cur;
      for (int k = 1; k < E1; ++k) {
        cur *= xi;
        pw[i * E1 + k] = cur;
      }
      g[i] = 0.0;
    }
    for (int i = tid; i < nn; i += NT) H[i] = 0.0;
    for (int i = tid; i < nn * n; i += NT) T[i] = 0.0;
    __syncthreads();
    double sg = 0.0;
    for (int64_t t = tid; t < A.m_terms; t += NT) ad_term_any(load_term(A.terms, t), pw, E1, n, g, H, T, sg);
    sg = ad_block_sum<NT>(sg, red);  // (its barriers also complete the sweep)
    for (int idx = tid; idx < nn * n; idx += NT) {
      const int l = idx / nn, j = (idx / n) % n, k = idx % n;
      int i0 = l, i1 = j, i2 = k;  // sort the index triple
      if (i0 > i1) { const int q = i0; i0 = i1; i1 = q; }
      if (i1 > i2) { const int q = i1; i1 = i2; i2 = q; }
      if (i0 > i1) { const int q = i0; i0 = i1; i1 = q; }
      if (i0 != l || i1 != j) T[idx] = T[(i0 * n + i1) * n + i2];
    }
    for (int idx = tid; idx < nn; idx += NT) {
      const int i = idx / n, j = idx % n;
      if (i > j) H[idx] = H[j * n + i];
    }
    // ---- 2. gradient norm, zero-gradient test, frame
    double gg = 0.0;
    for (int i = tid; i < n; i += NT) gg += g[i] * g[i];
    const double gn = sqrt(ad_block_sum<NT>(gg, red));
    bool zero = !(gn > 0.0) || !isfinite(gn);
    if (!A.assume_nonzero_x && gn <= 1e-14 * sg) zero = true;
    if (zero) {
      for (int i = tid; i < n; i += NT) {
        A.D[p * n + i] = nan("");
        if (A.Dunit) A.Dunit[p * n + i] = nan("");
      }
      if (tid == 0 && A.info) A.info[p] = polylab_an_info{gn, nan(""), POLYLAB_FLAG_ZERO_GRAD, n, n - 1, 0};
      __syncthreads();
      continue;
    }
    const double en = g[n - 1] / gn;
    const double sgn = en >= 0.0 ? 1.0 : -1.0;
    const double beta = 1.0 / (1.0 + sgn * en);  // 2 / v^T v
    for (int i = tid; i < n; i += NT) {
      e[i] = g[i] / gn;
      v[i] = e[i] + (i == n - 1 ? sgn : 0.0);
    }
    if (tid == 0) s_flag = 0;
    __syncthreads();
    for (int idx = tid; idx < nn; idx += NT) {
      const int i = idx / n, j = idx % n;
      Q[idx] = (i == j ? 1.0 : 0.0) - beta * v[i] * v[j];
    }
    for (int i = tid; i < n; i += NT) {
      double acc = 0.0;
      for (int k = 0; k < n; ++k) acc += H[i * n + k] * e[k];
      He[i] = acc;
    }
    __syncthreads();
    // ---- 3. tangent block, mixed term, Cholesky, log-det, inverse
    for (int idx = tid; idx < n * m; idx += NT) {  // B = H Q_T
      const int i = idx / m, j = idx % m;
      double acc = 0.0;
      for (int k = 0; k < n; ++k) acc += H[i * n + k] * Q[k * n + j];
      B[idx] = acc;
    }
    for (int i = tid; i < m; i += NT) {  // h = Q_T^T H e
      double acc = 0.0;
      for (int k = 0; k < n; ++k) acc += Q[k * n + i] * He[k];
      h[i] = acc;
    }
    __syncthreads();
    for (int idx = tid; idx < m * m; idx += NT) {  // H_T = Q_T^T B + r I
      const int i = idx / m, j = idx % m;
      double acc = 0.0;
      for (int k = 0; k < n; ++k) acc += Q[k * n + i] * B[k * m + j];
      HT[idx] = acc + (i == j ? A.r : 0.0);
    }
    __syncthreads();
    for (int k = 0; k < m; ++k) {  // right-looking Cholesky, lower triangle
      if (tid == 0) {
        const double d = HT[k * m + k];
        if (!(d > 0.0) || !isfinite(d)) s_flag = 1;
        else HT[k * m + k] = sqrt(d);
      }
      __syncthreads();
      if (s_flag) break;
      const double lkk = HT[k * m + k];
      for (int i = k + 1 + tid; i < m; i += NT) HT[i * m + k] /= lkk;
      __syncthreads();
      const int rows = m - k - 1;
      for (int idx = tid; idx < rows * rows; idx += NT) {
        const int i = k + 1 + idx / rows, j = k + 1 + idx % rows;
        if (j <= i) HT[i * m + j] -= HT[i * m + k] * HT[j * m + k];
      }
      __syncthreads();
    }
    if (s_flag) {
      for (int i = tid; i < n; i += NT) {
        A.D[p * n + i] = nan("");
        if (A.Dunit) A.Dunit[p * n + i] = nan("");
      }
      if (tid == 0 && A.info) A.info[p] = polylab_an_info{gn, nan(""), POLYLAB_FLAG_NOT_PD, n, n - 1, 0};
      __syncthreads();
      continue;
    }
    double ld = 0.0;
    for (int k = tid; k < m; k += NT) ld += 2.0 * log(HT[k * m + k]);
    const double logdet = ad_block_sum<NT>(ld, red);
    for (int j = tid; j < m; j += NT) {  // column j of H_T^{-1}: L y = e_j, then L^T z = y, in place
      for (int i = 0; i < m; ++i) {
        double acc = i == j ? 1.0 : 0.0;
        for (int k = 0; k < i; ++k) acc -= HT[i * m + k] * Hi[k * m + j];
        Hi[i * m + j] = acc / HT[i * m + i];
      }
      for (int i = m - 1; i >= 0; --i) {
        double acc = Hi[i * m + j];
        for (int k = i + 1; k < m; ++k) acc -= HT[k * m + i] * Hi[k * m + j];
        Hi[i * m + j] = acc / HT[i * m + i];
      }
    }
    __syncthreads();
    // ---- 4. a_i = tr(H_T^{-1} Q_T^T S_i Q_T), one tangent axis at a time
    for (int i = 0; i < m; ++i) {
      for (int idx = tid; idx < nn; idx += NT) {  // S_i = sum_l T(l, :, :) Q(l, i)
        double acc = 0.0;
        for (int l = 0; l < n; ++l) acc += T[l * nn + idx] * Q[l * n + i];
        S[idx] = acc;
      }
      __syncthreads();
      for (int idx = tid; idx < n * m; idx += NT) {  // B = S_i Q_T
        const int r0 = idx / m, c0 = idx % m;
        double acc = 0.0;
        for (int k = 0; k < n; ++k) acc += S[r0 * n + k] * Q[k * n + c0];
        B[idx] = acc;
      }
      __syncthreads();
      double tr = 0.0;  // sum_{b,c} (H_T^{-1})_{cb} (Q_T^T B)_{bc}
      for (int idx = tid; idx < m * m; idx += NT) {
        const int b = idx / m, c = idx % m;
        double acc = 0.0;
        for (int k = 0; k < n; ++k) acc += Q[k * n + b] * B[k * m + c];
        tr += Hi[c * m + b] * acc;
      }
      tr = ad_block_sum<NT>(tr, red);
      if (tid == 0) av[i] = tr;
    }
    __syncthreads();
    // ---- 5. tau = H_T^{-1}(h - |g|/(n+1) a), nu = Q_T tau - e
    const double kap = gn / (double)(n + 1);
    for (int i = tid; i < m; i += NT) {
      double acc = 0.0;
      for (int k = 0; k < m; ++k) acc += Hi[i * m + k] * (h[k] - kap * av[k]);
      tau[i] = acc;
    }
    __syncthreads();
    double nn2 = 0.0;
    for (int l = tid; l < n; l += NT) {
      double acc = -e[l];
      for (int k = 0; k < m; ++k) acc += Q[l * n + k] * tau[k];
      A.D[p * n + l] = acc;
      nn2 += acc * acc;
    }
    const double nrm = sqrt(ad_block_sum<NT>(nn2, red));
    if (A.Dunit)
      for (int l = tid; l < n; l += NT) A.Dunit[p * n + l] = A.D[p * n + l] / nrm;
    if (tid == 0 && A.info) A.info[p] = polylab_an_info{gn, logdet, 0, n, n - 1, 0};
    __syncthreads();
  }
}

template <int NT>
polylab_status launch_ad(const AdArgs& a, size_t smem, cudaStream_t s) {
  auto k = affine_ad_kernel<NT>;
  PL_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int occ = 0;
  PL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, NT, smem));
  if (occ < 1) return POLYLAB_ERR_UNSUPPORTED;
  const int64_t grid = std::min<int64_t>(a.P, (int64_t)occ * num_sms());
  k<<<(unsigned)grid, NT, smem, s>>>(a);
  return launch_status("affine_ad_kernel");
}

}  // namespace

polylab_status affine_ad(const polylab_plan* plan, const double* X, int64_t P, const polylab_an_opts* o, double* D,
                         double* Dunit, polylab_an_info* info, cudaStream_t s) {
  const int n = plan->n;
  if (n < 1 || n > kAdMaxN) return POLYLAB_ERR_UNSUPPORTED;
  if (o->prec != POLYLAB_FP64) return POLYLAB_ERR_INVALID_ARG;
  if (P == 0) return POLYLAB_OK;
  AdArgs a{};
  a.terms = plan->terms;
  a.m_terms = plan->m;
  a.n = n;
  a.E1 = plan->max_exp + 1;
  a.X = X;
  a.P = P;
  a.r = o->regularization;
  a.assume_nonzero_x = o->assume_nonzero_x;
  a.D = D;
  a.Dunit = Dunit;
  a.info = info;
  const size_t smem = (size_t)ad_lay(n, a.E1).total * sizeof(double);
  int dev = 0, optin = 0;
  PL_CUDA(cudaGetDevice(&dev));
  PL_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  if (smem + 1024 > (size_t)optin) return POLYLAB_ERR_UNSUPPORTED;  // (room for the static shared data)
  if (n <= 8) return launch_ad<64>(a, smem, s);
  if (n <= 16) return launch_ad<128>(a, smem, s);
  return launch_ad<256>(a, smem, s);
}

}  // namespace polylab
