// MF-logDet-Exact affine-normal direction (Sec. 5), one CTA per point.
//
//   phase 1  g, H at x from the term list (shared-memory accumulation)
//   phase 2  e = g/|g|; Householder reflector P = I - beta v v^T with
//            v = e + s e_n (s = sign(e_n)), so P e_n = -s e and the first
//            n-1 columns of P are an orthonormal frame Q_T of e-perp;
//            P H P by a rank-2 update; H_T = (PHP)[0:m,0:m] + r I (m = n-1),
//            h = Q_T^T H e = -s (PHP)[0:m, n-1];
//            Cholesky H_T = L L^T (FP64; failure -> NOT_PD), logdet;
//            M = (H_T)^{-1} = L^{-T} L^{-1};  W = Q_T M Q_T^T = P [M 0; 0 0] P
//   phase 3  c_l = sum_jk d_l d_j d_k f(x) W_jk from the term list; this is
//            a_i = tr(H_T^{-1} d_{t_i} H_T) = (Q_T^T c)_i without ever forming
//            the third-derivative tensor
//   phase 4  tau = M (h - |g|/(n+1) a);  nu = Q_T tau - e = P [tau; 0] - e.
//
// FP32 form (prec = POLYLAB_FP32): the term loops of phases 1 and 3 and the
// triangular inverse run in FP32; the Cholesky factorisation, log-det, tau
// and the normalisation stay FP64.  Matrices live in shared memory when
// 2 n^2 doubles fit, otherwise in a global workspace slice per CTA.
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "terms.cuh"

namespace polylab {

namespace {

template <int NT>
__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = threadIdx.x < NT / 32 ? red[threadIdx.x] : 0.0;
    for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) red[32] = t;
  }
  __syncthreads();
  return red[32];
}

struct SmemLayout {
  size_t off_x, off_g, off_sg, off_e, off_v, off_u, off_w, off_h, off_c, off_t, off_red, off_pw, off_accH,
      off_Wf, off_H, off_M, total;
};

template <typename R>
__host__ __device__ SmemLayout layout(int n, int E1, bool mats_in_smem) {
  SmemLayout L{};
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t r = o;
    o += (bytes + 15) & ~size_t(15);
    return r;
  };
  L.off_x = take(n * 8);
  L.off_g = take(n * 8);
  L.off_sg = take(n * 8);
  L.off_e = take(n * 8);
  L.off_v = take(n * 8);
  L.off_u = take(n * 8);
  L.off_w = take(n * 8);
  L.off_h = take(n * 8);
  L.off_c = take(n * 8);
  L.off_t = take(n * 8);
  L.off_red = take(40 * 8);
  L.off_pw = take((size_t)n * E1 * sizeof(R));
  // FP32 form: separate FP32 accumulators for H and an FP32 copy of W
  L.off_accH = sizeof(R) == 4 ? take((size_t)n * n * 4) : 0;
  L.off_Wf = sizeof(R) == 4 ? take((size_t)n * n * 4) : 0;
  L.off_H = mats_in_smem ? take((size_t)n * n * 8) : 0;
  L.off_M = mats_in_smem ? take((size_t)n * n * 8) : 0;
  L.total = o;
  return L;
}

}  // namespace

template <typename R, int NT>
__global__ void __launch_bounds__(NT) affine_exact_kernel(const Term* __restrict__ terms, int64_t m_terms, int n,
                                                          int E, const double* __restrict__ X, int64_t P, double r,
                                                          int assume_nonzero_x, bool mats_in_smem,
                                                          double* __restrict__ gws, double* __restrict__ D,
                                                          double* __restrict__ Dunit,
                                                          polylab_an_info* __restrict__ info) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int E1 = E + 1;
  const SmemLayout L = layout<R>(n, E1, mats_in_smem);
  double* xs = (double*)(sm + L.off_x);
  double* g = (double*)(sm + L.off_g);
  double* sg = (double*)(sm + L.off_sg);
  double* e = (double*)(sm + L.off_e);
  double* v = (double*)(sm + L.off_v);
  double* u = (double*)(sm + L.off_u);
  double* w = (double*)(sm + L.off_w);
  double* h = (double*)(sm + L.off_h);
  double* c = (double*)(sm + L.off_c);
  double* tv = (double*)(sm + L.off_t);
  double* red = (double*)(sm + L.off_red);
  R* pw = (R*)(sm + L.off_pw);
  double* Hm = mats_in_smem ? (double*)(sm + L.off_H) : gws + (size_t)blockIdx.x * 2 * n * n;
  double* Mm = mats_in_smem ? (double*)(sm + L.off_M) : Hm + (size_t)n * n;
  R* accH = sizeof(R) == 4 ? (R*)(sm + L.off_accH) : (R*)Hm;
  R* Wr = sizeof(R) == 4 ? (R*)(sm + L.off_Wf) : (R*)Mm;
  __shared__ int s_flag;
  __shared__ double s_logdet;
  const int m = n - 1;
  const int tid = threadIdx.x;
  const int nn = n * n;

  for (int64_t p = blockIdx.x; p < P; p += gridDim.x) {
    __syncthreads();
    // ---------------------------------------------------------- phase 1
    for (int i = tid; i < n; i += NT) {
      const double x = X[p * n + i];
      xs[i] = x;
      g[i] = 0.0;
      sg[i] = 0.0;
      c[i] = 0.0;
      R cur = R(1);
      pw[i * E1] = cur;
      for (int k = 1; k <= E; ++k) {
        cur = cur * R(x);
        pw[i * E1 + k] = cur;
      }
    }
    for (int i = tid; i < nn; i += NT) accH[i] = R(0);
    if (tid == 0) {
      s_flag = 0;
      s_logdet = 0.0;
    }
    __syncthreads();
    for (int64_t t = tid; t < m_terms; t += NT) {
      const TermRegs tr = load_term(terms, t);
      term_derivs<R, 2>(tr, pw, E1, [&](int kind, int i, int j, R val) {
        if (kind == 1) {
          atomicAdd(&g[i], (double)val);
          atomicAdd(&sg[i], fabs((double)val));
        } else if (kind == 2) {
          atomicAdd(&accH[i * n + j], val);
        }
      });
    }
    __syncthreads();
    // mirror the upper triangle into a full FP64 matrix
    for (int idx = tid; idx < nn; idx += NT) {
      const int i = idx / n, j = idx - i * n;
      Hm[idx] = (double)(i <= j ? accH[i * n + j] : accH[j * n + i]);
    }
    // ---------------------------------------------------------- phase 2
    double gg = 0.0, ss = 0.0;
    for (int i = tid; i < n; i += NT) {
      gg += g[i] * g[i];
      ss += sg[i] * sg[i];
    }
    const double gn2 = block_sum<NT>(gg, red);
    const double sgn2 = block_sum<NT>(ss, red);
    const double gn = sqrt(gn2);
    bool zero = !(gn > 0.0) || !isfinite(gn);
    if (!assume_nonzero_x && gn <= 1e-14 * sqrt(sgn2)) zero = true;
    if (zero) {
      if (tid == 0 && info) {
        polylab_an_info in{gn, nan(""), POLYLAB_FLAG_ZERO_GRAD, n, n - 1, 0};
        info[p] = in;
      }
      for (int i = tid; i < n; i += NT) {
        D[p * n + i] = nan("");
        if (Dunit) Dunit[p * n + i] = nan("");
      }
      continue;
    }
    const double en = g[n - 1] / gn;
    const double sgn = en >= 0.0 ? 1.0 : -1.0;
    for (int i = tid; i < n; i += NT) {
      e[i] = g[i] / gn;
      v[i] = e[i] + (i == n - 1 ? sgn : 0.0);
    }
    const double vv = 2.0 * (1.0 + sgn * en);
    const double beta = 2.0 / vv;
    __syncthreads();
    // u = H v
    for (int i = tid; i < n; i += NT) {
      double acc = 0.0;
      for (int j = 0; j < n; ++j) acc += Hm[i * n + j] * v[j];
      u[i] = acc;
    }
    __syncthreads();
    double part = 0.0;
    for (int i = tid; i < n; i += NT) part += v[i] * u[i];
    const double gamma = block_sum<NT>(part, red);
    for (int i = tid; i < n; i += NT) w[i] = beta * u[i] - 0.5 * beta * beta * gamma * v[i];
    __syncthreads();
    // P H P = H - v w^T - w v^T
    for (int idx = tid; idx < nn; idx += NT) {
      const int i = idx / n, j = idx - i * n;
      Hm[idx] -= v[i] * w[j] + w[i] * v[j];
    }
    __syncthreads();
    for (int i = tid; i < m; i += NT) h[i] = -sgn * Hm[i * n + (n - 1)];
    for (int i = tid; i < m; i += NT) Hm[i * n + i] += r;
    __syncthreads();
    // Cholesky (lower, in place, leading m x m block, row stride n)
    for (int k = 0; k < m; ++k) {
      if (tid == 0) {
        const double d = Hm[k * n + k];
        if (!(d > 0.0) || !isfinite(d)) {
          s_flag = 1;
        } else {
          const double lk = sqrt(d);
          Hm[k * n + k] = lk;
          s_logdet += 2.0 * log(lk);
        }
      }
      __syncthreads();
      if (s_flag) break;
      const double lk = Hm[k * n + k];
      for (int i = k + 1 + tid; i < m; i += NT) Hm[i * n + k] /= lk;
      __syncthreads();
      const int rem = m - k - 1;
      for (int idx = tid; idx < rem * rem; idx += NT) {
        const int i = k + 1 + idx / rem, j = k + 1 + idx % rem;
        if (j <= i) Hm[i * n + j] -= Hm[i * n + k] * Hm[j * n + k];
      }
      __syncthreads();
    }
    if (s_flag) {
      if (tid == 0 && info) {
        polylab_an_info in{gn, nan(""), POLYLAB_FLAG_NOT_PD, n, n - 1, 0};
        info[p] = in;
      }
      for (int i = tid; i < n; i += NT) {
        D[p * n + i] = nan("");
        if (Dunit) Dunit[p * n + i] = nan("");
      }
      continue;
    }
    // L^{-1}: column j by forward substitution, one thread per column; stored
    // in the upper triangle of Mm transposed (Mm[j*n+i] = Linv[i][j], i >= j)
    for (int j = tid; j < m; j += NT) {
      Mm[j * n + j] = 1.0 / Hm[j * n + j];
      for (int i = j + 1; i < m; ++i) {
        R acc = R(0);
        for (int k = j; k < i; ++k) acc += R(Hm[i * n + k]) * R(Mm[j * n + k]);
        Mm[j * n + i] = -(double)acc / Hm[i * n + i];
      }
    }
    __syncthreads();
    // M = L^{-T} L^{-1}: M_ij = sum_{k >= max(i,j)} Linv[k][i] Linv[k][j]; kept in Hm's
    // space (L is no longer needed), full symmetric, row stride n
    for (int idx = tid; idx < m * m; idx += NT) {
      const int i = idx / m, j = idx - i * m;
      if (j < i) continue;
      R acc = R(0);
      for (int k = j; k < m; ++k) acc += R(Mm[i * n + k]) * R(Mm[j * n + k]);
      Hm[i * n + j] = (double)acc;
    }
    __syncthreads();
    for (int idx = tid; idx < nn; idx += NT) {
      const int i = idx / n, j = idx - i * n;
      double val;
      if (i == n - 1 || j == n - 1) val = 0.0;
      else val = i <= j ? Hm[i * n + j] : Hm[j * n + i];
      Mm[idx] = val;
    }
    __syncthreads();
    // W = P Mt P with Mt = [M 0; 0 0]: u = Mt v, gamma = v.u, w = beta u - beta^2 gamma/2 v
    for (int i = tid; i < n; i += NT) {
      double acc = 0.0;
      for (int j = 0; j < n; ++j) acc += Mm[i * n + j] * v[j];
      u[i] = acc;
    }
    __syncthreads();
    part = 0.0;
    for (int i = tid; i < n; i += NT) part += v[i] * u[i];
    const double gam2 = block_sum<NT>(part, red);
    for (int i = tid; i < n; i += NT) w[i] = beta * u[i] - 0.5 * beta * beta * gam2 * v[i];
    __syncthreads();
    // Hm <- W (full); Mm keeps M (tangent inverse, padded)
    for (int idx = tid; idx < nn; idx += NT) {
      const int i = idx / n, j = idx - i * n;
      const double val = Mm[idx] - (v[i] * w[j] + w[i] * v[j]);
      Hm[idx] = val;
      if (sizeof(R) == 4) Wr[idx] = (R)val;
    }
    __syncthreads();
    // ---------------------------------------------------------- phase 3
    const R* Wuse = sizeof(R) == 4 ? Wr : (const R*)Hm;
    for (int64_t t = tid; t < m_terms; t += NT) {
      const TermRegs tr = load_term(terms, t);
      if (tr.k == 0) continue;
      int deg = 0;
      for (int s = 0; s < tr.k; ++s) deg += tr.exp[s];
      if (deg < 3) continue;
      term_third_contract<R>(tr, pw, E1, [&](int j, int k) { return Wuse[j * n + k]; },
                             [&](int l, R val) { atomicAdd(&c[l], (double)val); });
    }
    __syncthreads();
    // ---------------------------------------------------------- phase 4
    // a = (P c)[0:m] = c - beta v (v.c)
    part = 0.0;
    for (int i = tid; i < n; i += NT) part += v[i] * c[i];
    const double vc = block_sum<NT>(part, red);
    const double wgt = gn / (double)(n + 1);
    for (int i = tid; i < m; i += NT) tv[i] = h[i] - wgt * (c[i] - beta * v[i] * vc);
    __syncthreads();
    // tau = M (h - |g|/(n+1) a) into u[0:m], u[n-1] = 0
    for (int i = tid; i < n; i += NT) {
      double acc = 0.0;
      if (i < m)
        for (int j = 0; j < m; ++j) acc += Mm[i * n + j] * tv[j];
      u[i] = acc;
    }
    __syncthreads();
    part = 0.0;
    for (int i = tid; i < n; i += NT) part += v[i] * u[i];
    const double vt = block_sum<NT>(part, red);
    double nrm = 0.0;
    for (int i = tid; i < n; i += NT) {
      const double nu = u[i] - beta * v[i] * vt - e[i];
      tv[i] = nu;
      nrm += nu * nu;
    }
    const double nn2 = block_sum<NT>(nrm, red);
    const double inv = 1.0 / sqrt(nn2);
    for (int i = tid; i < n; i += NT) {
      D[p * n + i] = tv[i];
      if (Dunit) Dunit[p * n + i] = tv[i] * inv;
    }
    if (tid == 0 && info) {
      polylab_an_info in{gn, s_logdet, 0, n, n - 1, 0};
      info[p] = in;
    }
  }
}

template <typename R, int NT>
static polylab_status launch_exact(const polylab_plan* plan, const double* X, int64_t P, const polylab_an_opts* o,
                                   double* D, double* Dunit, polylab_an_info* info, cudaStream_t s) {
  const int n = plan->n, E = std::max(plan->max_exp, 1);
  SmemLayout Ls = layout<R>(n, E + 1, true);
  const bool in_smem = Ls.total + 1024 <= 200 * 1024;
  SmemLayout L = in_smem ? Ls : layout<R>(n, E + 1, false);
  if (L.total > 200 * 1024) return POLYLAB_ERR_UNSUPPORTED;
  auto k = affine_exact_kernel<R, NT>;
  PL_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total));
  int per_sm = 0;
  PL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, NT, L.total));
  per_sm = std::max(per_sm, 1);
  const int64_t grid = std::min<int64_t>(P, (int64_t)num_sms() * per_sm);
  Scratch scratch(s);
  double* gws = nullptr;
  if (!in_smem) PL_TRY(scratch.get(&gws, (size_t)grid * 2 * n * n));
  k<<<(unsigned)grid, NT, L.total, s>>>(plan->terms, plan->m, n, E, X, P, o->regularization, o->assume_nonzero_x,
                                        in_smem, gws, D, Dunit, info);
  return launch_status("affine_exact_kernel");
}

polylab_status affine_exact(const polylab_plan* plan, const double* X, int64_t P, const polylab_an_opts* o, double* D,
                            double* Dunit, polylab_an_info* info, cudaStream_t s) {
  if (P == 0) return POLYLAB_OK;
  const bool f32 = o->prec == POLYLAB_FP32;
  const int n = plan->n;
  if (n <= 16) return f32 ? launch_exact<float, 64>(plan, X, P, o, D, Dunit, info, s)
                          : launch_exact<double, 64>(plan, X, P, o, D, Dunit, info, s);
  if (n <= 48) return f32 ? launch_exact<float, 128>(plan, X, P, o, D, Dunit, info, s)
                          : launch_exact<double, 128>(plan, X, P, o, D, Dunit, info, s);
  return f32 ? launch_exact<float, 256>(plan, X, P, o, D, Dunit, info, s)
             : launch_exact<double, 256>(plan, X, P, o, D, Dunit, info, s);
}

}  // namespace polylab
