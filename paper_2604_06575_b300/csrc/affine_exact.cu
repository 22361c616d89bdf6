// MF-logDet-Exact affine-normal direction (Sec. 5), one CTA per point, one
// persistent launch for any number of polynomials.
//
//   phase 1  g, H at x from the term list (shared-memory accumulation)
//   phase 2  e = g/|g|; Householder reflector P = I - beta v v^T with
//            v = e + s e_n (s = sign(e_n)), so P e_n = -s e and the first
//            n-1 columns of P are an orthonormal frame Q_T of e-perp;
//            P H P by a rank-2 update; H_T = (PHP)[0:m,0:m] + r I (m = n-1),
//            h = Q_T^T H e = -s (PHP)[0:m, n-1];
//            Cholesky H_T = L L^T in FP64 by one warp (failure -> NOT_PD),
//            log-det; M = (H_T)^{-1} = L^{-T} L^{-1}; W = Q_T M Q_T^T = P [M 0; 0 0] P
//   phase 3  c_l = sum_jk d_l d_j d_k f(x) W_jk from the term list, which is
//            a_i = tr(H_T^{-1} d_{t_i} H_T) = (Q_T^T c)_i without forming the
//            third-derivative tensor
//   phase 4  tau = M (h - |g|/(n+1) a);  nu = Q_T tau - e = P [tau; 0] - e.
//
// R = double: every step in FP64.  R = float (POLYLAB_FP32): term sums, frame
// update, triangular inverse, W and the trace term in FP32; the Cholesky
// factorisation, log-det, tau and normalisation in FP64.
//
// Work items are (polynomial, point) pairs taken from an atomic counter in the
// order of a host-built permutation (most expensive polynomials first), so an
// uneven batch keeps every SM busy in a single launch.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "batch.cuh"
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
  if (threadIdx.x < 32) {
    double t = threadIdx.x < NT / 32 ? red[threadIdx.x] : 0.0;
    for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) red[32] = t;
  }
  __syncthreads();
  return red[32];
}

template <int NT>
__device__ __forceinline__ double2 block_sum2(double a, double b, double* red) {
  for (int o = 16; o; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) {
    red[w] = a;
    red[16 + w] = b;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    double ta = threadIdx.x < NT / 32 ? red[threadIdx.x] : 0.0;
    double tb = threadIdx.x < NT / 32 ? red[16 + threadIdx.x] : 0.0;
    for (int o = 16; o; o >>= 1) {
      ta += __shfl_xor_sync(0xffffffffu, ta, o);
      tb += __shfl_xor_sync(0xffffffffu, tb, o);
    }
    if (threadIdx.x == 0) {
      red[32] = ta;
      red[33] = tb;
    }
  }
  __syncthreads();
  return make_double2(red[32], red[33]);
}

struct Layout {
  size_t x, e, v, h, tv, red, g, sg, c, u, w, pw, Hr, Mr, Ld, total;
};

// Shared-memory layout for one point of an n-variable polynomial with power
// tables up to exponent E1-1.  `mats` false: Hr/Mr/Ld live in global memory.
template <typename R, int NW>
__host__ __device__ Layout exact_layout(int n, int E1, bool mats) {
  Layout L{};
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t r = o;
    o += (bytes + 15) & ~size_t(15);
    return r;
  };
  const size_t m = n > 1 ? n - 1 : 1;
  L.x = take(n * 8);
  L.e = take(n * 8);
  L.v = take(n * 8);
  L.h = take(n * 8);
  L.tv = take(n * 8);
  L.red = take(40 * 8);
  // one replica per warp for the contended vector sums
  L.g = take((size_t)NW * n * sizeof(R));
  L.sg = take((size_t)NW * n * sizeof(R));
  L.c = take((size_t)NW * n * sizeof(R));
  L.u = take(n * sizeof(R));
  L.w = take(n * sizeof(R));
  L.pw = take((size_t)n * E1 * sizeof(R));
  L.Hr = mats ? take((size_t)n * n * sizeof(R)) : 0;
  L.Mr = mats ? take((size_t)n * n * sizeof(R)) : 0;
  // FP32 form: separate FP64 Cholesky storage (packed lower triangle); FP64 form factors in place in Hr
  L.Ld = (mats && sizeof(R) == 4) ? take(m * (m + 1) / 2 * 8) : 0;
  L.total = o;
  return L;
}

// global-memory bytes per CTA when the matrices do not fit in shared memory
template <typename R>
__host__ __device__ size_t exact_gmem(int n) {
  const size_t m = n > 1 ? n - 1 : 1;
  return 2 * (size_t)n * n * sizeof(R) + (sizeof(R) == 4 ? m * (m + 1) / 2 * 8 : 0) + 256;
}

}  // namespace

template <typename R, int NT>
__global__ void __launch_bounds__(NT, sizeof(R) == 4 ? 512 / NT : 1) affine_exact_kernel(const ExactDesc* __restrict__ descs, int n_desc,
                                                          const int64_t* __restrict__ prefix,
                                                          const int* __restrict__ order, int64_t total,
                                                          int* __restrict__ counter, double r,
                                                          int assume_nonzero_x, unsigned char* __restrict__ gws,
                                                          size_t gws_stride) {
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ int64_t s_item;
  __shared__ int s_flag;
  __shared__ double s_logdet;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  constexpr bool kF64 = sizeof(R) == 8;
  constexpr int NW = NT / 32;

  while (true) {
    __syncthreads();
    if (tid == 0) s_item = (int64_t)atomicAdd(counter, 1);
    __syncthreads();
    const int64_t item = s_item;
    if (item >= total) break;
    // locate the polynomial: prefix[] is over polynomials in `order`
    int lo = 0, hi = n_desc;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (prefix[mid] <= item) lo = mid;
      else hi = mid;
    }
    const ExactDesc& pd = descs[order[lo]];
    const int64_t p = item - prefix[lo];
    const int n = pd.n, m = n - 1, nn = n * n, E1 = pd.E + 1;
    const Layout L = exact_layout<R, NW>(n, E1, pd.mats_in_smem);
    double* xs = (double*)(sm + L.x);
    double* e = (double*)(sm + L.e);
    double* v = (double*)(sm + L.v);
    double* h = (double*)(sm + L.h);
    double* tv = (double*)(sm + L.tv);
    double* red = (double*)(sm + L.red);
    R* g = (R*)(sm + L.g);
    R* sg = (R*)(sm + L.sg);
    R* c = (R*)(sm + L.c);
    R* u = (R*)(sm + L.u);
    R* w = (R*)(sm + L.w);
    R* pw = (R*)(sm + L.pw);
    unsigned char* gb = gws + (size_t)blockIdx.x * gws_stride;
    R* Hr = pd.mats_in_smem ? (R*)(sm + L.Hr) : (R*)gb;
    R* Mr = pd.mats_in_smem ? (R*)(sm + L.Mr) : (R*)(gb + (size_t)nn * sizeof(R));
    // FP64 Cholesky storage: in place in Hr (row stride n) for the FP64 form,
    // a packed lower triangle for the FP32 form
    double* Ld = kF64 ? (double*)Hr
                      : (pd.mats_in_smem ? (double*)(sm + L.Ld) : (double*)(gb + 2 * (size_t)nn * sizeof(R)));
    auto LI = [n](int i, int j) { return kF64 ? i * n + j : i * (i + 1) / 2 + j; };
    const double* X = pd.X + p * n;

    // ---------------------------------------------------------- phase 1
    for (int i = tid; i < NW * n; i += NT) {
      g[i] = R(0);
      sg[i] = R(0);
      c[i] = R(0);
    }
    for (int i = tid; i < n; i += NT) {
      const double x = X[i];
      xs[i] = x;
      R cur = R(1);
      pw[i * E1] = cur;
      for (int k = 1; k < E1; ++k) {
        cur = cur * R(x);
        pw[i * E1 + k] = cur;
      }
    }
    for (int i = tid; i < nn; i += NT) Hr[i] = R(0);
    if (tid == 0) {
      s_flag = 0;
      s_logdet = 0.0;
    }
    __syncthreads();
    R gabs = R(0);  // this thread's share of sum |gradient contributions|
    {
      R* gw = g + wid * n;
      for (int64_t t = tid; t < pd.m; t += NT) {
        const TermRegs tr = load_term(pd.terms, t);
        term_derivs<R, 2>(tr, pw, E1, [&](int kind, int i, int j, R val) {
          if (kind == 1) {
            atomicAdd(&gw[i], val);
            gabs += fabs(val);
          } else if (kind == 2) {
            atomicAdd(&Hr[i * n + j], val);
          }
        });
      }
    }
    __syncthreads();
    for (int i = tid; i < n; i += NT) {  // fold the warp replicas into replica 0
      R a = g[i];
      for (int q = 1; q < NW; ++q) a += g[q * n + i];
      g[i] = a;
    }
    for (int idx = tid; idx < nn; idx += NT) {  // mirror the upper triangle
      const int i = idx / n, j = idx - i * n;
      if (i > j) Hr[idx] = Hr[j * n + i];
    }
    // ---------------------------------------------------------- phase 2
    double gg = 0.0;
    for (int i = tid; i < n; i += NT) gg += (double)g[i] * (double)g[i];
    const double2 sums = block_sum2<NT>(gg, (double)gabs, red);
    const double gn = sqrt(sums.x);
    bool zero = !(gn > 0.0) || !isfinite(gn);
    // relative test at the resolution of the form: 1e-14 (FP64), 1e-6 (FP32 sums)
    if (!assume_nonzero_x && gn <= (kF64 ? 1e-14 : 1e-6) * sums.y) zero = true;
    if (zero) {
      if (tid == 0 && pd.info) {
        polylab_an_info in{gn, nan(""), POLYLAB_FLAG_ZERO_GRAD, n, n - 1, 0};
        pd.info[p] = in;
      }
      for (int i = tid; i < n; i += NT) {
        pd.D[p * n + i] = nan("");
        if (pd.Dunit) pd.Dunit[p * n + i] = nan("");
      }
      continue;
    }
    const double en = (double)g[n - 1] / gn;
    const double sgn = en >= 0.0 ? 1.0 : -1.0;
    const double beta = 1.0 / (1.0 + sgn * en);  // 2 / v^T v with v^T v = 2 (1 + s e_n)
    R* vr = sg;  // v in the form's precision (sg is free): no conversions inside n^2 loops
    for (int i = tid; i < n; i += NT) {
      e[i] = (double)g[i] / gn;
      v[i] = e[i] + (i == n - 1 ? sgn : 0.0);
      vr[i] = R(v[i]);
    }
    __syncthreads();
    for (int i = tid; i < n; i += NT) {  // u = H v
      R acc = R(0);
      for (int j = 0; j < n; ++j) acc += Hr[i * n + j] * vr[j];
      u[i] = acc;
    }
    __syncthreads();
    double part = 0.0;
    for (int i = tid; i < n; i += NT) part += v[i] * (double)u[i];
    const double gamma = block_sum<NT>(part, red);
    for (int i = tid; i < n; i += NT) w[i] = R(beta * (double)u[i] - 0.5 * beta * beta * gamma * v[i]);
    __syncthreads();
    for (int idx = tid; idx < nn; idx += NT) {  // P H P = H - v w^T - w v^T
      const int i = idx / n, j = idx - i * n;
      Hr[idx] -= vr[i] * w[j] + w[i] * vr[j];
    }
    __syncthreads();
    for (int i = tid; i < m; i += NT) h[i] = -sgn * (double)Hr[i * n + (n - 1)];
    if constexpr (kF64) {
      for (int i = tid; i < m; i += NT) Hr[i * n + i] += r;
    } else {
      for (int idx = tid; idx < m * m; idx += NT) {
        const int i = idx / m, j = idx - i * m;
        if (j <= i) Ld[LI(i, j)] = (double)Hr[i * n + j] + (i == j ? r : 0.0);
      }
    }
    __syncthreads();
    // Cholesky of the leading m x m block (lower, in place), one warp
    if (wid == 0) {
      double logdet = 0.0;
      bool bad = false;
      for (int k = 0; k < m; ++k) {
        double lk = 0.0, inv = 0.0;
        if (lane == 0) {
          const double d = Ld[LI(k, k)];
          bad = !(d > 0.0) || !isfinite(d);
          if (!bad) {
            lk = sqrt(d);
            inv = 1.0 / lk;
            Ld[LI(k, k)] = lk;
            logdet += 2.0 * log(lk);
          }
        }
        bad = __shfl_sync(0xffffffffu, (int)bad, 0) != 0;
        if (bad) break;
        inv = __shfl_sync(0xffffffffu, inv, 0);
        for (int i = k + 1 + lane; i < m; i += 32) Ld[LI(i, k)] *= inv;
        __syncwarp();
        for (int i = k + 1 + lane; i < m; i += 32) {
          const double lik = Ld[LI(i, k)];
          double* row = Ld + LI(i, 0);
#pragma unroll 4
          for (int j = k + 1; j <= i; ++j) row[j] -= lik * Ld[LI(j, k)];
        }
        __syncwarp();
      }
      if (lane == 0) {
        s_flag = bad ? 1 : 0;
        s_logdet = logdet;
      }
    }
    __syncthreads();
    if (s_flag) {
      if (tid == 0 && pd.info) {
        polylab_an_info in{gn, nan(""), POLYLAB_FLAG_NOT_PD, n, n - 1, 0};
        pd.info[p] = in;
      }
      for (int i = tid; i < n; i += NT) {
        pd.D[p * n + i] = nan("");
        if (pd.Dunit) pd.Dunit[p * n + i] = nan("");
      }
      continue;
    }
    // L in R precision: the FP32 form converts the factor once (into Hr, free now)
    const R* Lr;
    const int lr = n;
    if constexpr (kF64) {
      Lr = (const R*)Ld;
    } else {
      for (int idx = tid; idx < m * m; idx += NT) {
        const int i = idx / m, j = idx - i * m;
        if (j <= i) Hr[i * n + j] = (R)Ld[LI(i, j)];
      }
      __syncthreads();
      Lr = Hr;
    }
    // L^{-1} by forward substitution, one thread per column; stored transposed:
    // Mr[j*n + i] = Linv[i][j] for i >= j.  Reciprocal diagonal first (w is free).
    for (int i = tid; i < m; i += NT) w[i] = R(1) / Lr[i * lr + i];
    __syncthreads();
    for (int j = tid; j < m; j += NT) {
      Mr[j * n + j] = w[j];
      for (int i = j + 1; i < m; ++i) {
        R acc = R(0);
        for (int k = j; k < i; ++k) acc += Lr[i * lr + k] * Mr[j * n + k];
        Mr[j * n + i] = -acc * w[i];
      }
    }
    __syncthreads();
    // M = L^{-T} L^{-1}, upper triangle into Hr (L no longer needed)
    for (int idx = tid; idx < m * m; idx += NT) {
      const int i = idx / m, j = idx - i * m;
      if (j < i) continue;
      R acc = R(0);
      for (int k = j; k < m; ++k) acc += Mr[i * n + k] * Mr[j * n + k];
      Hr[i * n + j] = acc;
    }
    __syncthreads();
    for (int idx = tid; idx < nn; idx += NT) {  // Mr <- [M 0; 0 0], full symmetric
      const int i = idx / n, j = idx - i * n;
      Mr[idx] = (i == n - 1 || j == n - 1) ? R(0) : (i <= j ? Hr[i * n + j] : Hr[j * n + i]);
    }
    __syncthreads();
    for (int i = tid; i < n; i += NT) {  // u = [M 0; 0 0] v
      R acc = R(0);
      for (int j = 0; j < n; ++j) acc += Mr[i * n + j] * vr[j];
      u[i] = acc;
    }
    __syncthreads();
    part = 0.0;
    for (int i = tid; i < n; i += NT) part += v[i] * (double)u[i];
    const double gam2 = block_sum<NT>(part, red);
    for (int i = tid; i < n; i += NT) w[i] = R(beta * (double)u[i] - 0.5 * beta * beta * gam2 * v[i]);
    __syncthreads();
    for (int idx = tid; idx < nn; idx += NT) {  // Hr <- W
      const int i = idx / n, j = idx - i * n;
      Hr[idx] = Mr[idx] - (vr[i] * w[j] + w[i] * vr[j]);
    }
    __syncthreads();
    // ---------------------------------------------------------- phase 3
    {
      R* cw = c + wid * n;
      for (int64_t t = tid; t < pd.m; t += NT) {
        const TermRegs tr = load_term(pd.terms, t);
        int deg = 0;
#pragma unroll
        for (int s2 = 0; s2 < kMaxSupport; ++s2) deg += tr.exp[s2];
        if (deg < 3) continue;
        term_third_contract<R>(tr, pw, E1, [&](int j, int k) { return Hr[j * n + k]; },
                               [&](int l, R val) { atomicAdd(&cw[l], val); });
      }
    }
    __syncthreads();
    for (int i = tid; i < n; i += NT) {
      R a = c[i];
      for (int q = 1; q < NW; ++q) a += c[q * n + i];
      c[i] = a;
    }
    __syncthreads();
    // ---------------------------------------------------------- phase 4
    part = 0.0;
    for (int i = tid; i < n; i += NT) part += v[i] * (double)c[i];
    const double vc = block_sum<NT>(part, red);  // a = (P c)[0:m] = c - beta v (v.c)
    const double wgt = gn / (double)(n + 1);
    for (int i = tid; i < m; i += NT) tv[i] = h[i] - wgt * ((double)c[i] - beta * v[i] * vc);
    __syncthreads();
    double* tau = xs;  // x is no longer needed
    R* tvr = u;          // right-hand side in the form's precision
    for (int i = tid; i < m; i += NT) tvr[i] = R(tv[i]);
    __syncthreads();
    for (int i = tid; i < n; i += NT) {
      R acc = R(0);
      if (i < m)
        for (int j = 0; j < m; ++j) acc += Mr[i * n + j] * tvr[j];
      tau[i] = (double)acc;
    }
    __syncthreads();
    part = 0.0;
    for (int i = tid; i < n; i += NT) part += v[i] * tau[i];
    const double vt = block_sum<NT>(part, red);
    double nrm = 0.0;
    for (int i = tid; i < n; i += NT) {
      const double nu = tau[i] - beta * v[i] * vt - e[i];
      tv[i] = nu;
      nrm += nu * nu;
    }
    const double inv = 1.0 / sqrt(block_sum<NT>(nrm, red));
    for (int i = tid; i < n; i += NT) {
      pd.D[p * n + i] = tv[i];
      if (pd.Dunit) pd.Dunit[p * n + i] = tv[i] * inv;
    }
    if (tid == 0 && pd.info) {
      polylab_an_info in{gn, s_logdet, 0, n, n - 1, 0};
      pd.info[p] = in;
    }
  }
}

// ------------------------------------------------------------------ host side

namespace {

constexpr size_t kSmemCap = 200 * 1024;

template <typename R>
size_t layout_bytes(int n, int E1, bool mats, int threads) {
  if (threads == 64) return exact_layout<R, 2>(n, E1, mats).total;
  if (threads == 128) return exact_layout<R, 4>(n, E1, mats).total;
  return exact_layout<R, 8>(n, E1, mats).total;
}

}  // namespace

template <typename R>
static polylab_status prepare_exact(ExactBatch* b) {
  size_t smem = 0, gstride = 0;
  for (auto& d : b->host_descs) {
    const int E1 = d.E + 1;
    const size_t in = layout_bytes<R>(d.n, E1, true, b->cfg.threads);
    d.mats_in_smem = in <= kSmemCap ? 1 : 0;
    const size_t need = d.mats_in_smem ? in : layout_bytes<R>(d.n, E1, false, b->cfg.threads);
    if (need > kSmemCap) return POLYLAB_ERR_UNSUPPORTED;
    smem = std::max(smem, need);
    if (!d.mats_in_smem) gstride = std::max(gstride, exact_gmem<R>(d.n));
  }
  b->smem = smem;
  b->gws_stride = gstride;
  return POLYLAB_OK;
}

template <typename R, int NT>
static polylab_status launch_exact_t(ExactBatch* b, cudaStream_t s) {
  auto k = affine_exact_kernel<R, NT>;
  PL_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem));
  int per_sm = 0;
  PL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, NT, b->smem));
  per_sm = std::max(1, per_sm);
  if (b->cfg.ctas_per_sm > 0) per_sm = std::min(per_sm, b->cfg.ctas_per_sm);
  const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(b->total, (int64_t)num_sms() * per_sm));
  if (b->gws_stride > 0 && (size_t)grid * b->gws_stride > b->gws_bytes) return POLYLAB_ERR_UNSUPPORTED;
  PL_CUDA(cudaMemsetAsync(b->counter, 0, sizeof(int), s));
  k<<<(unsigned)grid, NT, b->smem, s>>>(b->descs, b->n_desc, b->prefix, b->order, b->total, b->counter,
                                         b->opts.regularization, b->opts.assume_nonzero_x, b->gws, b->gws_stride);
  return launch_status("affine_exact_kernel");
}

polylab_status run_exact_batch(ExactBatch* b, cudaStream_t s) {
  if (b->total == 0) return POLYLAB_OK;
  const bool f32 = b->opts.prec == POLYLAB_FP32;
  const int nt = b->cfg.threads;
  if (f32) {
    if (nt == 64) return launch_exact_t<float, 64>(b, s);
    if (nt == 128) return launch_exact_t<float, 128>(b, s);
    return launch_exact_t<float, 256>(b, s);
  }
  if (nt == 64) return launch_exact_t<double, 64>(b, s);
  if (nt == 128) return launch_exact_t<double, 128>(b, s);
  return launch_exact_t<double, 256>(b, s);
}

polylab_status prepare_exact_batch(ExactBatch* b) {
  return b->opts.prec == POLYLAB_FP32 ? prepare_exact<float>(b) : prepare_exact<double>(b);
}

// Per-point cost estimate used to order the work (expensive polynomials
// first): term work plus the cubic factorisation.
double exact_point_cost(const ExactDesc& d, int max_support) {
  const double k = std::max(1, max_support);
  const double m = d.n - 1;
  return (double)d.m * (k * k + k * k * k / 2.0) + 4.0 * m * m * m / 3.0 * 20.0;
}

polylab_status affine_exact(const polylab_plan* plan, const double* X, int64_t P, const polylab_an_opts* o, double* D,
                            double* Dunit, polylab_an_info* info, cudaStream_t s) {
  if (P == 0) return POLYLAB_OK;
  const polylab_plan* plans[1] = {plan};
  const double* Xs[1] = {X};
  const int64_t Ps[1] = {P};
  double* Ds[1] = {D};
  double* Dus[1] = {Dunit};
  polylab_an_info* infos[1] = {info};
  ExactBatch b;
  PL_TRY(exact_batch_init(&b, 1, plans, Xs, Ps, o, Ds, Dus, infos, s));
  const polylab_status st = run_exact_batch(&b, s);
  exact_batch_release(&b, s);
  return st;
}

}  // namespace polylab
