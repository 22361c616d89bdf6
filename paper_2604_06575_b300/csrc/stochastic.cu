// MF-logDet-Stochastic affine-normal direction (Sec. 5): the trace term a is
// replaced by a Hutchinson estimate over q probes and every tangent solve by
// preconditioned CG, with Hessian-vector products formed matrix-free from the
// term list.
//
// Everything runs in the ambient space on vectors orthogonal to e: with
// Pi = I - e e^T, the tangent system (H_T + r I) y = z of a frame Q_T is the
// system Pi (H + r I) Pi u = Pi w with u = Q_T y, w = Q_T z, and CG on it
// produces the tangent iterates mapped by Q_T (the preconditioner
// Pi D^{-1} Pi corresponds to Q_T^T D^{-1} Q_T), so no frame is formed.
//
// Per point (one CTA):
//   g, |diag H| from the terms; H assembled once into the plan's CSR pattern
//   (each term's K x K block added at its precomputed positions);
//   e = g/|g|; D = |diag H| + r (1 where 0)
//   for each chunk of QC probes:  w_s Rademacher (SplitMix64),
//       b_s = Pi w_s;  PCG:  u_s ~ (Pi (H + rI) Pi)^+ b_s
//       cbar += (1/q) sum_s T(., u_s, b_s)   (term by term, symmetrised)
//   a = Pi cbar;  PCG: u_tau solves Pi (H + rI) Pi u = Pi H e - |g|/(n+1) a
//   nu = u_tau - e
//
// Every Hessian-vector product of the Krylov solves is then a sparse
// matrix times the QC probe columns: QC consecutive threads take one row, a
// thread per probe, and read the row's values and column indices as
// broadcasts and the probe vectors as one contiguous QC-wide load per entry.
//
// R = float (POLYLAB_FP32): HVPs, CG vectors and sums in FP32, the final
// direction and its normalisation in FP64; R = double: FP64 throughout.
#include <algorithm>
#include <cmath>

#include <cuda_bf16.h>

#include "common.cuh"
#include "mlp.cuh"
#include "terms.cuh"

namespace polylab {

namespace {

__device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t k) {
  uint64_t z = seed + (k + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Symmetric k x k Hessian block of one term at one point (slots a, b).
template <typename R, int K>
__device__ __forceinline__ void term_hessian_block(const TermRegs& t, const R* __restrict__ pw, int E1, R* blk) {
  R a0[K], d1[K], d2[K];
#pragma unroll
  for (int s = 0; s < K; ++s) {
    const int es = t.exp[s];
    const R* q = pw + t.var[s] * E1 + es;
    a0[s] = q[0];
    d1[s] = R(es) * q[-1];
    d2[s] = es >= 2 ? R(es * (es - 1)) * q[-2] : R(0);
  }
  R pre[K + 1], suf[K + 1];
  pre[0] = R(1);
#pragma unroll
  for (int s = 0; s < K; ++s) pre[s + 1] = pre[s] * a0[s];
  suf[K] = R(1);
#pragma unroll
  for (int s = K - 1; s >= 0; --s) suf[s] = suf[s + 1] * a0[s];
  const R c = R(t.coef);
#pragma unroll
  for (int s = 0; s < K; ++s) {
    blk[s * K + s] = c * d2[s] * pre[s] * suf[s + 1];
    R mid = R(1);
#pragma unroll
    for (int u = s + 1; u < K; ++u) {
      const R v = c * d1[s] * d1[u] * (pre[s] * mid * suf[u + 1]);
      blk[s * K + u] = v;
      blk[u * K + s] = v;
      mid *= a0[u];
    }
  }
}

// Adds a term's K x K Hessian block into the assembled values at its
// precomputed CSR positions `hp` (wider supports out of line, as in terms.cuh).
template <typename R, int K>
__device__ __forceinline__ void term_assemble_k(const TermRegs& t, const R* __restrict__ pw, int E1,
                                                const int32_t* __restrict__ hp, R* Hv) {
  R blk[K * K];
  term_hessian_block<R, K>(t, pw, E1, blk);
#pragma unroll
  for (int q = 0; q < K * K; ++q) atomicAdd(&Hv[hp[q]], blk[q]);
}
template <typename R, int K>
__device__ __noinline__ void term_assemble_wide(const TermRegs& t, const R* __restrict__ pw, int E1,
                                                const int32_t* __restrict__ hp, R* Hv) {
  term_assemble_k<R, K>(t, pw, E1, hp, Hv);
}

// Y[var_a][s] += sum_b blk[a][b] V[var_b][s] for the QC probes of a chunk
// (4 probes per pass, shared-memory atomics into Y).  V rows are QC apart,
// Y rows QC + 1 apart (an odd stride keeps lanes with different variables on
// different banks).
template <typename R, int K, int QC>
__device__ __forceinline__ void term_hvp(const TermRegs& t, const R* __restrict__ pw, int E1,
                                         const R* __restrict__ V, R* Y, const int* active) {
  R blk[K * K];
  term_hessian_block<R, K>(t, pw, E1, blk);
#pragma unroll 1
  for (int s0 = 0; s0 < QC; s0 += 4) {
    if (!(active[s0] | active[s0 + 1] | active[s0 + 2] | active[s0 + 3])) continue;
    R v[K][4];
#pragma unroll
    for (int b = 0; b < K; ++b)
#pragma unroll
      for (int q = 0; q < 4; ++q) v[b][q] = V[t.var[b] * QC + s0 + q];
#pragma unroll
    for (int a = 0; a < K; ++a) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        R acc = R(0);
#pragma unroll
        for (int b = 0; b < K; ++b) acc += blk[a * K + b] * v[b][q];
        atomicAdd(&Y[t.var[a] * (QC + 1) + s0 + q], acc);
      }
    }
  }
}

template <typename R, int QC>
__device__ __forceinline__ void term_hvp_dispatch(const TermRegs& t, const R* pw, int E1, const R* V, R* Y,
                                                  const int* active) {
  switch (t.k) {
    case 0: break;
    case 1: term_hvp<R, 1, QC>(t, pw, E1, V, Y, active); break;
    case 2: term_hvp<R, 2, QC>(t, pw, E1, V, Y, active); break;
    case 3: term_hvp<R, 3, QC>(t, pw, E1, V, Y, active); break;
    case 4: term_hvp<R, 4, QC>(t, pw, E1, V, Y, active); break;
    case 5: term_hvp<R, 5, QC>(t, pw, E1, V, Y, active); break;
    case 6: term_hvp<R, 6, QC>(t, pw, E1, V, Y, active); break;
    case 7: term_hvp<R, 7, QC>(t, pw, E1, V, Y, active); break;
    default: term_hvp<R, 8, QC>(t, pw, E1, V, Y, active); break;
  }
}

// block-wide sums of QC values per thread; result broadcast to all threads
// (T = the form's precision inside the Krylov iterations: B300's FP64 rate is
// 1/60 of its FP32 rate, and FP32 tree sums over n <= 2000 terms are far more
// accurate than the solver tolerance)
template <int NT, int QC, typename T>
__device__ __forceinline__ void block_sums(T (&v)[QC], T* red) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
  for (int s = 0; s < QC; ++s)
    for (int o = 16; o; o >>= 1) v[s] += __shfl_xor_sync(0xffffffffu, v[s], o);
  __syncthreads();
  if (l == 0)
#pragma unroll
    for (int s = 0; s < QC; ++s) red[w * QC + s] = v[s];
  __syncthreads();
  if (threadIdx.x < QC) {
    T acc = T(0);
    for (int q = 0; q < NT / 32; ++q) acc += red[q * QC + threadIdx.x];
    red[(NT / 32) * QC + threadIdx.x] = acc;
  }
  __syncthreads();
#pragma unroll
  for (int s = 0; s < QC; ++s) v[s] = red[(NT / 32) * QC + s];
  __syncthreads();
}

// Sum over the CTA of one value per thread for the thread's probe
// s = tid % QC (QC a power of two <= 32, NT a multiple of 32): lanes of a warp
// holding the same probe first, then the warps' partials in shared memory.
// Every thread receives its probe's total.
template <int NT, int QC, typename T>
__device__ __forceinline__ T probe_sum(T v, T* red) {
  for (int o = QC; o < 32; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l < QC) red[w * QC + l] = v;
  __syncthreads();
  if (threadIdx.x < QC) {
    T acc = T(0);
    for (int q = 0; q < NT / 32; ++q) acc += red[q * QC + threadIdx.x];
    red[(NT / 32) * QC + threadIdx.x] = acc;
  }
  __syncthreads();
  return red[(NT / 32) * QC + threadIdx.x % QC];
}

// Sum over the CTA of one double per thread, broadcast to every thread.
template <int NT>
__device__ __forceinline__ double block_sum1(double v, double* red) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double acc = 0.0;
  for (int q = 0; q < NT / 32; ++q) acc += red[q];
  __syncthreads();
  return acc;
}

struct StochArgs {
  const Term* terms;
  int64_t m;
  int n, E;
  const double* X;
  int64_t P;
  double r, tol;
  int maxit, q, assume_nonzero_x;
  uint64_t seed;
  int precond;
  const __nv_bfloat16* mlp;  // learned preconditioner weights (BF16), POLYLAB_PRECOND_MLP
  double* D;
  double* Dunit;
  polylab_an_info* info;
  // assembled Hessian: the plan's CSR pattern and per-term block positions
  const int32_t* hrow;
  const int32_t* hcol;
  const int32_t* hpos;
  int64_t hbase[kMaxSupport + 1];
  int64_t koff[kMaxSupport + 2];
  int64_t k3off[kMaxSupport + 1];
  // per CTA: 5 vectors of n*QC R, U (2 n floats) for the learned
  // preconditioner, the HVP output Y (n rows of QC+1 R), then the point's
  // Hessian values and the trace weight Z on the same pattern (hnnz R each,
  // 16-byte aligned)
  unsigned char* gws;
  size_t gws_stride;
  size_t y_off, hval_off;
};

}  // namespace

// MINB: resident CTAs per SM the register budget is sized for (2, or 4 when
// the point's shared memory allows four CTAs: latency hiding then pays for
// a few spilled registers)
template <typename R, int NT, int QC, int MINB>
__global__ void __launch_bounds__(NT, MINB) stochastic_kernel(StochArgs a) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int n = a.n, E1 = a.E + 1, tid = threadIdx.x;
  // shared: power table, vectors g, dg (|diag H|), e, cbar, Dinv; reductions
  R* pw = (R*)sm;
  // per-point vectors in the form's precision (FP32 form: shared memory for n up to ~2000)
  constexpr int YS = QC + 1;  // row stride of Y, the HVP output (global, see below)
  R* g = (R*)(((uintptr_t)(pw + (size_t)n * E1) + 15) & ~(uintptr_t)15);
  R* dg = g + n;
  R* e = dg + n;
  R* cbar = e + n;
  R* Dinv = cbar + n;
  double* red = (double*)(((uintptr_t)(Dinv + n) + 15) & ~(uintptr_t)15);  // (NT/32 + 1) * QC doubles
  __shared__ int s_active[QC];
  __shared__ int s_iters[QC];
  __shared__ double s_bnorm[QC], s_rz[QC], s_rr[QC];
  __shared__ int s_maxed;
  __shared__ float th[kMlpParams];
  const bool use_mlp = a.precond == POLYLAB_PRECOND_MLP;
  if (use_mlp)
    for (int j = tid; j < kMlpParams; j += NT) th[j] = __bfloat162float(a.mlp[j]);

  unsigned char* gb = a.gws + (size_t)blockIdx.x * a.gws_stride;
  const size_t vec = (size_t)n * QC;
  R* Xv = (R*)gb;  // solutions u_s
  R* Rv = Xv + vec;  // residuals
  R* Pv = Rv + vec;  // search directions
  R* Zv = Pv + vec;  // preconditioned residuals
  R* Bv = Zv + vec;  // right-hand sides b_s = Pi w_s
  float* U0 = (float*)(Bv + vec);  // learned low-rank factor, columns 0 and 1
  float* U1 = U0 + n;
  R* Y = (R*)(gb + a.y_off);       // HVP output rows (stride YS) and first-sweep scratch
  R* Hv = (R*)(gb + a.hval_off);  // this point's Hessian values in the CSR pattern
  const int64_t hnnz = a.hrow[n];
  R* Zw = Hv + ((hnnz + 3) & ~int64_t(3));  // trace weight on the same pattern

  for (int64_t p = blockIdx.x; p < a.P; p += gridDim.x) {
    __syncthreads();
    const double* X = a.X + p * n;
    for (int i = tid; i < n; i += NT) {
      const double x = X[i];
      R cur = R(1);
      pw[i * E1] = cur;
      for (int k = 1; k < E1; ++k) {
        cur = cur * R(x);
        pw[i * E1 + k] = cur;
      }
      g[i] = R(0);
      dg[i] = R(0);
      cbar[i] = R(0);
    }
    for (int64_t q = tid; q < hnnz; q += NT) Hv[q] = R(0);
    __syncthreads();
    // gradient, sum of |gradient contributions| (zero test), diag(H) and the
    // off-diagonal |contribution| mass of every row (learned preconditioner, Y[n, 2n))
    for (int i = tid; i < 3 * n; i += NT) Y[i] = R(0);
    __syncthreads();
    double gabs = 0.0;  // this thread's share of sum |gradient contributions|
    for (int64_t t = tid; t < a.m; t += NT) {
      const TermRegs tr = load_term(a.terms, t);
      term_derivs<R, 2>(tr, pw, E1, [&](int kind, int i, int j, R val) {
        if (kind == 1) {
          atomicAdd(&g[i], val);
          gabs += fabs((double)val);
        } else if (kind == 2) {
          if (i == j) {
            atomicAdd(&dg[i], val);
          } else if (use_mlp) {
            atomicAdd(&Y[n + i], (R)fabs((double)val));
            atomicAdd(&Y[n + j], (R)fabs((double)val));
          }
        }
      });
    }
    // assemble H: every term's K x K block at its precomputed CSR positions
    for_support<kMaxSupport>([&](auto kc) {
      constexpr int K = decltype(kc)::value;
      if constexpr (K >= 1) {
        for (int64_t t = a.koff[K] + tid; t < a.koff[K + 1]; t += NT) {
          const TermRegs tr = load_term(a.terms, t);
          const int32_t* hp = a.hpos + a.hbase[K] + (t - a.koff[K]) * (K * K);
          if constexpr (K <= 6) term_assemble_k<R, K>(tr, pw, E1, hp, Hv);
          else term_assemble_wide<R, K>(tr, pw, E1, hp, Hv);
        }
      }
    });
    __syncthreads();
    double gg = 0.0;
    for (int i = tid; i < n; i += NT) gg += (double)g[i] * (double)g[i];
    gg = block_sum1<NT>(gg, red);
    const double gsum = block_sum1<NT>(gabs, red);
    const double gn = sqrt(gg);
    bool zero = !(gn > 0.0) || !isfinite(gn);
    if (!a.assume_nonzero_x && gn <= (sizeof(R) == 8 ? 1e-14 : 1e-6) * gsum) zero = true;
    if (zero) {
      if (tid == 0 && a.info) {
        polylab_an_info in{gn, nan(""), POLYLAB_FLAG_ZERO_GRAD, 0, a.q, 0};
        a.info[p] = in;
      }
      for (int i = tid; i < n; i += NT) {
        a.D[p * n + i] = nan("");
        if (a.Dunit) a.Dunit[p * n + i] = nan("");
      }
      continue;
    }
    for (int i = tid; i < n; i += NT) {
      e[i] = R((double)g[i] / gn);
      const double d = fabs((double)dg[i]) + a.r;
      Dinv[i] = a.precond == POLYLAB_PRECOND_NONE ? R(1) : R(d > 0.0 ? 1.0 / d : 1.0);
      Y[2 * n + i] = R(1.0 / d);  // 1 / a_i for the scaled coupling feature
    }
    if (use_mlp) {  // BF16 weights, FP32 arithmetic
      __syncthreads();
      for (int i = tid; i < n; i += NT) {
        // signed off-diagonal row sums of the assembled Hessian: plain and
        // scaled by 1 / a_j
        R rs = R(0), rsa = R(0);
        for (int q = a.hrow[i]; q < a.hrow[i + 1]; ++q) {
          const int c = a.hcol[q];
          if (c != i) {
            rs += Hv[q];
            rsa += Hv[q] * Y[2 * n + c];
          }
        }
        float f[kMlpF], h[kMlpH], o[kMlpO], D, u0, u1;
        mlp_features(f, (float)dg[i], (float)Y[n + i], (float)X[i], (float)e[i], (float)g[i], n, (float)a.r,
                     (float)rs, (float)rsa);
        mlp_forward(th, f, h, o);
        mlp_factors(o, (float)dg[i], (float)a.r, &D, &u0, &u1);
        Dinv[i] = R(D);
        U0[i] = u0;
        U1[i] = u1;
      }
    }
    if (tid == 0) s_maxed = 0;
    __syncthreads();
    int total_iters = 0;
    const int words = (n + 63) / 64;

    // ---------------------------------------------------------------- PCG
    // Solves Pi (H + rI) Pi u_s = b_s for the `nq` columns present in Bv.
    // Vectors hold QC probe columns per row (element (i, s) at i*QC + s); a
    // thread always handles the same probe s = tid % QC (NT is a multiple of
    // QC), so every per-probe reduction is one value per thread.
    R* redr = (R*)red;
    const int my_s = tid % QC;
    auto project = [&](R* V, int nq, int stride) {  // V_s <- V_s - e (e . V_s); rows `stride` apart
      R d = R(0);
      for (int i = tid; i < (int)vec; i += NT) d += e[i / QC] * V[(i / QC) * stride + my_s];
      d = probe_sum<NT, QC>(d, redr);
      if (my_s < nq)
        for (int i = tid; i < (int)vec; i += NT) V[(i / QC) * stride + my_s] -= e[i / QC] * d;
    };
    // Y[i][s] = sum_j H_ij V[j][s] + shift V[i][s] for the active probes s
    // (QC threads per row, one per probe; rows NT / QC at a time)
    auto spmv = [&](const R* __restrict__ V, R shift) {
      constexpr int RPP = NT / QC;
      const bool on = s_active[my_s] != 0;
      for (int i = tid / QC; i < n; i += RPP) {
        R acc = R(0);
        if (on) {
          int q = a.hrow[i];
          const int q1 = a.hrow[i + 1];
          for (; q + 4 <= q1; q += 4) {
            const int c0 = a.hcol[q], c1 = a.hcol[q + 1], c2 = a.hcol[q + 2], c3 = a.hcol[q + 3];
            const R h0 = Hv[q], h1 = Hv[q + 1], h2 = Hv[q + 2], h3 = Hv[q + 3];
            acc += h0 * V[c0 * QC + my_s] + h1 * V[c1 * QC + my_s] + h2 * V[c2 * QC + my_s] +
                   h3 * V[c3 * QC + my_s];
          }
          for (; q < q1; ++q) acc += Hv[q] * V[a.hcol[q] * QC + my_s];
        }
        Y[i * YS + my_s] = acc + shift * V[i * QC + my_s];
      }
    };
    auto apply_A = [&](const R* V) {  // Y = Pi (H + rI) V (V in e-perp), into shared memory
      spmv(V, R(a.r));
      __syncthreads();
      project(Y, QC, YS);
      __syncthreads();
    };
    auto precondition = [&](int nq) {  // Z = Pi D^{-1} R, or Pi (D + U U^T) R when learned
      if (use_mlp) {
        R u0r = R(0), u1r = R(0);
        for (int i = tid; i < (int)vec; i += NT) {
          u0r += R(U0[i / QC]) * Rv[i];
          u1r += R(U1[i / QC]) * Rv[i];
        }
        u0r = probe_sum<NT, QC>(u0r, redr);
        u1r = probe_sum<NT, QC>(u1r, redr);
        for (int i = tid; i < (int)vec; i += NT) {
          const int row = i / QC;
          Zv[i] = Dinv[row] * Rv[i] + R(U0[row]) * u0r + R(U1[row]) * u1r;
        }
      } else {
        for (int i = tid; i < (int)vec; i += NT) Zv[i] = Dinv[i / QC] * Rv[i];
      }
      __syncthreads();
      project(Zv, nq, QC);
      __syncthreads();
    };
    auto pcg = [&](int nq) {
      for (int i = tid; i < (int)vec; i += NT) {
        Xv[i] = R(0);
        Rv[i] = Bv[i];
      }
      if (tid < QC) {
        s_active[tid] = tid < nq;
        s_iters[tid] = 0;
      }
      __syncthreads();
      precondition(nq);
      for (int i = tid; i < (int)vec; i += NT) Pv[i] = Zv[i];
      R bb = R(0), rz = R(0);
      for (int i = tid; i < (int)vec; i += NT) {
        bb += Bv[i] * Bv[i];
        rz += Bv[i] * Zv[i];
      }
      bb = probe_sum<NT, QC>(bb, redr);
      rz = probe_sum<NT, QC>(rz, redr);
      if (tid < QC) {
        s_bnorm[tid] = sqrt((double)bb);
        s_rz[tid] = rz;
        s_rr[tid] = bb;
      }
      __syncthreads();
      for (int k = 0;; ++k) {
        // convergence test before every iteration: |r_s| <= tol |b_s|
        if (tid < QC && s_active[tid]) {
          if (sqrt(s_rr[tid]) <= a.tol * s_bnorm[tid]) {
            s_active[tid] = 0;
          } else if (k >= a.maxit) {
            s_active[tid] = 0;
            s_maxed = 1;
          }
        }
        __syncthreads();
        int any = 0;
#pragma unroll
        for (int q = 0; q < QC; ++q) any |= s_active[q];
        if (!any) break;
        apply_A(Pv);
        R py = R(0);
        for (int i = tid; i < (int)vec; i += NT) py += Pv[i] * Y[(i / QC) * YS + my_s];
        py = probe_sum<NT, QC>(py, redr);
        // breakdown guard: a probe whose curvature p.Ap is not positive (or not
        // finite) stops here with its current iterate
        if (tid < QC && s_active[tid] && !(py > R(0) && isfinite(py) && isfinite(s_rz[tid]))) s_active[tid] = 0;
        __syncthreads();
        if (s_active[my_s]) {
          const R alpha = R(s_rz[my_s] / (double)py);
          for (int i = tid; i < (int)vec; i += NT) {
            Xv[i] += alpha * Pv[i];
            Rv[i] -= alpha * Y[(i / QC) * YS + my_s];
          }
        }
        __syncthreads();
        precondition(nq);
        R rzn = R(0), rr = R(0);
        for (int i = tid; i < (int)vec; i += NT) {
          const R rv = Rv[i];
          rzn += rv * Zv[i];
          rr += rv * rv;
        }
        rzn = probe_sum<NT, QC>(rzn, redr);
        rr = probe_sum<NT, QC>(rr, redr);
        if (s_active[my_s]) {
          const R beta = R((double)rzn / s_rz[my_s]);
          for (int i = tid; i < (int)vec; i += NT) Pv[i] = Zv[i] + beta * Pv[i];
        }
        __syncthreads();
        if (tid < QC && s_active[tid]) {
          s_rz[tid] = rzn;
          s_rr[tid] = rr;
          s_iters[tid] += 1;
        } else if (tid < QC) {
          s_rr[tid] = rr;
        }
        __syncthreads();
      }
      int it = 0;
#pragma unroll
      for (int q = 0; q < QC; ++q) it += q < nq ? s_iters[q] : 0;
      __syncthreads();
      return it;
    };

    // ----------------------------------------------------- probes, trace term
    for (int s0 = 0; s0 < a.q; s0 += QC) {
      const int nq = min(QC, a.q - s0);
      for (int i = tid; i < (int)vec; i += NT) {
        const int row = i / QC, s = i % QC;
        R w = R(0);
        if (s < nq) {
          const uint64_t k = ((uint64_t)p * a.q + s0 + s) * words + (uint64_t)(row >> 6);
          w = ((splitmix64(a.seed, k) >> (row & 63)) & 1ull) ? R(-1) : R(1);
        }
        Bv[i] = w;
      }
      __syncthreads();
      project(Bv, nq, QC);
      __syncthreads();
      total_iters += pcg(nq);
      // cbar += (1/q) sum_s T(., u_s, b_s): the symmetrised weight
      // Z_jk = (1/2q) sum_s (u_s[j] b_s[k] + u_s[k] b_s[j]) is formed once on
      // the Hessian pattern (every pair a term touches), QC threads per row
      // summing over the probes by shuffles (warp-uniform loops), then each
      // term of degree >= 3 contracts its third derivatives with its block of Z
      {
        const R inv2q = R(0.5 / (double)a.q);
        constexpr int GPW = 32 / QC;  // rows per warp and pass
        const int ls = tid % QC, grp = (tid & 31) / QC;
        for (int base = (tid >> 5) * GPW; base < n; base += (NT / 32) * GPW) {
          const int i = base + grp;
          int q0 = 0, len = 0;
          R xi = R(0), bi = R(0);
          if (i < n) {
            q0 = a.hrow[i];
            len = a.hrow[i + 1] - q0;
            if (ls < nq) {
              xi = Xv[i * QC + ls];
              bi = Bv[i * QC + ls];
            }
          }
          int lmax = len;
          for (int o = QC; o < 32; o <<= 1) lmax = max(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
          for (int k = 0; k < lmax; ++k) {
            const bool ok = k < len;
            const int c = ok ? a.hcol[q0 + k] : 0;
            R v = (ok && ls < nq) ? xi * Bv[c * QC + ls] + Xv[c * QC + ls] * bi : R(0);
            for (int o = QC / 2; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (ok && ls == 0) Zw[q0 + k] = v * inv2q;
          }
        }
      }
      __syncthreads();
      for_support<kMaxSupport>([&](auto kc) {
        constexpr int K = decltype(kc)::value;
        if constexpr (K >= 1) {
          const int32_t* hp = nullptr;
          auto wget = [&](int sa, int sb, int, int) { return Zw[hp[sa * K + sb]]; };
          auto emit = [&](int l, R val) { atomicAdd(&cbar[l], val); };
          for (int64_t t = a.k3off[K] + tid; t < a.koff[K + 1]; t += NT) {
            const TermRegs tr = load_term(a.terms, t);
            hp = a.hpos + a.hbase[K] + (t - a.koff[K]) * (K * K);
            term_third_group<R, K>(tr, pw, E1, wget, emit);
          }
        }
      });
      __syncthreads();
    }
    // ---------------------------------------------------------- tau solve
    // right-hand side Pi (H e) - |g|/(n+1) Pi cbar, one column
    for (int i = tid; i < (int)vec; i += NT) Pv[i] = (i % QC == 0) ? R(e[i / QC]) : R(0);
    if (tid < QC) s_active[tid] = tid == 0;
    __syncthreads();
    spmv(Pv, R(0));  // Y = H e (ambient, column 0)
    __syncthreads();
    const double wgt = gn / (double)(n + 1);
    for (int i = tid; i < (int)vec; i += NT)
      Bv[i] = (i % QC == 0) ? R((double)Y[(i / QC) * YS] - wgt * (double)cbar[i / QC]) : R(0);
    __syncthreads();
    project(Bv, 1, QC);
    __syncthreads();
    total_iters += pcg(1);
    // ---------------------------------------------------------- direction
    double nrm = 0.0;
    for (int i = tid; i < n; i += NT) {
      const double nu = (double)Xv[i * QC] - (double)e[i];
      nrm += nu * nu;
    }
    const double inv = 1.0 / sqrt(block_sum1<NT>(nrm, red));
    for (int i = tid; i < n; i += NT) {
      const double nu = (double)Xv[i * QC] - (double)e[i];
      a.D[p * n + i] = nu;
      if (a.Dunit) a.Dunit[p * n + i] = nu * inv;
    }
    if (tid == 0 && a.info) {
      polylab_an_info in{gn, nan(""), s_maxed ? POLYLAB_FLAG_KRYLOV_MAXIT : 0, total_iters + 1, a.q, total_iters};
      a.info[p] = in;
    }
  }
}

namespace {

template <typename R, int QC>
size_t stoch_smem(int n, int E1, int NT) {
  size_t b = (size_t)n * E1 * sizeof(R);
  b = (b + 15) & ~size_t(15);
  b += 5 * (size_t)n * sizeof(R);
  b = (b + 15) & ~size_t(15);
  b += (size_t)(NT / 32 + 1) * QC * 8;
  return b + 64;
}

template <typename R, int NT, int QC>
polylab_status launch_stoch(const polylab_plan* plan, const double* X, int64_t P, const polylab_an_opts* o, double* D,
                            double* Dunit, polylab_an_info* info, cudaStream_t s) {
  const int n = plan->n, E1 = std::max(plan->max_exp, 1) + 1;
  // the Hessian pattern is a cached part of the plan, built on first use
  PL_TRY(ensure_hessian_pattern(const_cast<polylab_plan*>(plan), s));
  const size_t smem = stoch_smem<R, QC>(n, E1, NT);
  if (smem > 220 * 1024) return POLYLAB_ERR_UNSUPPORTED;
  auto k = 4 * smem <= 200 * 1024 ? stochastic_kernel<R, NT, QC, 4> : stochastic_kernel<R, NT, QC, 2>;
  PL_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  PL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, NT, smem));
  per_sm = std::max(1, per_sm);
  const int64_t grid = std::min<int64_t>(P, (int64_t)num_sms() * per_sm);
  StochArgs a{};
  a.terms = plan->terms;
  a.m = plan->m;
  a.n = n;
  a.E = E1 - 1;
  a.X = X;
  a.P = P;
  a.r = o->regularization;
  a.tol = o->krylov_tol;
  a.maxit = o->krylov_maxit;
  a.q = o->num_probes;
  a.assume_nonzero_x = o->assume_nonzero_x;
  a.seed = o->seed;
  a.precond = o->precond;
  a.mlp = (const __nv_bfloat16*)o->mlp_weights;
  a.D = D;
  a.Dunit = Dunit;
  a.info = info;
  a.hrow = plan->hrow;
  a.hcol = plan->hcol;
  a.hpos = plan->hpos;
  for (int k = 0; k <= kMaxSupport; ++k) a.hbase[k] = plan->hbase[k];
  for (int k = 0; k < kMaxSupport + 2; ++k) a.koff[k] = plan->koff[k];
  for (int k = 0; k < kMaxSupport + 1; ++k) a.k3off[k] = plan->k3off[k];
  a.y_off = ((size_t)5 * n * QC * sizeof(R) + 2 * (size_t)n * sizeof(float) + 15) & ~size_t(15);
  a.hval_off = (a.y_off + (size_t)n * (QC + 1) * sizeof(R) + 15) & ~size_t(15);
  a.gws_stride = (a.hval_off + 2 * (size_t)((plan->hnnz + 3) & ~int64_t(3)) * sizeof(R) + 255) & ~size_t(255);
  Scratch scr(s);
  PL_TRY(scr.get(&a.gws, (size_t)grid * a.gws_stride));
  k<<<(unsigned)grid, NT, smem, s>>>(a);
  return launch_status("stochastic_kernel");
}

}  // namespace

// Training data for the learned preconditioner: per point the features,
// |H_ii| (signed diagonal), e, four probes z_k = Pi w_k (SplitMix64, probe
// index p * 4 + k) and y_k = Pi (H + rI) z_k, all in FP32.
template <int NT>
__global__ void __launch_bounds__(NT) mlp_data_kernel(const Term* __restrict__ terms, int64_t m, int n, int E,
                                                      const double* __restrict__ X, int64_t P, float r,
                                                      uint64_t seed, float* __restrict__ feats,
                                                      float* __restrict__ hdiag, float* __restrict__ E_out,
                                                      float* __restrict__ Z, float* __restrict__ Yg) {
  constexpr int QC = 4;
  extern __shared__ __align__(16) unsigned char sm[];
  const int E1 = E + 1, tid = threadIdx.x;
  float* pw = (float*)sm;
  float* Y = pw + (size_t)n * E1;
  float* g = Y + (size_t)n * (QC + 1);
  float* dg = g + n;
  float* off = dg + n;
  float* rs = off + n;   // sum_{j != i} H_ij
  float* rsa = rs + n;   // sum_{j != i} H_ij / a_j
  double* red = (double*)(((uintptr_t)(rsa + n) + 15) & ~(uintptr_t)15);
  __shared__ int s_all[QC];
  if (tid < QC) s_all[tid] = 1;
  const int words = (n + 63) / 64;
  for (int64_t p = blockIdx.x; p < P; p += gridDim.x) {
    __syncthreads();
    const double* x = X + p * n;
    for (int i = tid; i < n; i += NT) {
      float cur = 1.f;
      pw[i * E1] = cur;
      for (int k = 1; k < E1; ++k) {
        cur *= (float)x[i];
        pw[i * E1 + k] = cur;
      }
      g[i] = dg[i] = off[i] = rs[i] = rsa[i] = 0.f;
    }
    __syncthreads();
    for (int64_t t = tid; t < m; t += NT) {
      const TermRegs tr = load_term(terms, t);
      term_derivs<float, 2>(tr, pw, E1, [&](int kind, int i, int j, float val) {
        if (kind == 1) atomicAdd(&g[i], val);
        else if (kind == 2) {
          if (i == j) atomicAdd(&dg[i], val);
          else {
            atomicAdd(&off[i], fabsf(val));
            atomicAdd(&off[j], fabsf(val));
            atomicAdd(&rs[i], val);
            atomicAdd(&rs[j], val);
          }
        }
      });
    }
    __syncthreads();
    // second sweep once the diagonal is complete: couplings scaled by 1 / a_j
    for (int64_t t = tid; t < m; t += NT) {
      const TermRegs tr = load_term(terms, t);
      term_derivs<float, 2>(tr, pw, E1, [&](int kind, int i, int j, float val) {
        if (kind == 2 && i != j) {
          atomicAdd(&rsa[i], val / (fabsf(dg[j]) + r));
          atomicAdd(&rsa[j], val / (fabsf(dg[i]) + r));
        }
      });
    }
    __syncthreads();
    double gg[QC] = {0.0, 0.0, 0.0, 0.0};
    for (int i = tid; i < n; i += NT) gg[0] += (double)g[i] * (double)g[i];
    block_sums<NT, QC>(gg, red);
    const float ginv = (float)(1.0 / sqrt(gg[0]));
    float* zp = Z + p * (int64_t)n * QC;
    float* yp = Yg + p * (int64_t)n * QC;
    for (int i = tid; i < n; i += NT) {
      const float ei = g[i] * ginv;
      E_out[p * n + i] = ei;
      hdiag[p * n + i] = dg[i];
      mlp_features(feats + (p * (int64_t)n + i) * kMlpF, dg[i], off[i], (float)x[i], ei, g[i], n, r, rs[i],
                   rsa[i]);
      for (int k = 0; k < QC; ++k) {
        const uint64_t key = ((uint64_t)p * QC + k) * words + (uint64_t)(i >> 6);
        zp[i * QC + k] = ((splitmix64(seed, key) >> (i & 63)) & 1ull) ? -1.f : 1.f;
      }
    }
    __syncthreads();
    // z <- Pi z
    double d[QC] = {0.0, 0.0, 0.0, 0.0};
    for (int i = tid; i < n; i += NT)
      for (int k = 0; k < QC; ++k) d[k] += (double)E_out[p * n + i] * zp[i * QC + k];
    block_sums<NT, QC>(d, red);
    for (int i = tid; i < n; i += NT)
      for (int k = 0; k < QC; ++k) zp[i * QC + k] -= (float)(E_out[p * n + i] * d[k]);
    for (int i = tid; i < n * (QC + 1); i += NT) Y[i] = 0.f;
    __syncthreads();
    for (int64_t t = tid; t < m; t += NT) {
      const TermRegs tr = load_term(terms, t);
      term_hvp_dispatch<float, QC>(tr, pw, E1, zp, Y, s_all);
    }
    __syncthreads();
    double dy[QC] = {0.0, 0.0, 0.0, 0.0};
    for (int i = tid; i < n; i += NT)
      for (int k = 0; k < QC; ++k) {
        Y[i * (QC + 1) + k] += r * zp[i * QC + k];
        dy[k] += (double)E_out[p * n + i] * Y[i * (QC + 1) + k];
      }
    block_sums<NT, QC>(dy, red);
    for (int i = tid; i < n; i += NT)
      for (int k = 0; k < QC; ++k) yp[i * QC + k] = Y[i * (QC + 1) + k] - (float)(E_out[p * n + i] * dy[k]);
  }
}

polylab_status affine_stochastic(const polylab_plan* plan, const double* X, int64_t P, const polylab_an_opts* o,
                                 double* D, double* Dunit, polylab_an_info* info, cudaStream_t s) {
  if (P == 0) return POLYLAB_OK;
  if (o->prec == POLYLAB_FP32) return launch_stoch<float, 256, 16>(plan, X, P, o, D, Dunit, info, s);
  return launch_stoch<double, 256, 8>(plan, X, P, o, D, Dunit, info, s);
}

}  // namespace polylab

extern "C" polylab_status polylab_mlp_data(const polylab_poly* p, const polylab_plan* plan, const double* X,
                                           int64_t P, double regularization, uint64_t seed, float* feats,
                                           float* hdiag, float* e, float* Z, float* Y, polylab_stream stream) {
  using namespace polylab;
  if (P < 0 || !X || !feats || !hdiag || !e || !Z || !Y || (!p && !plan)) return POLYLAB_ERR_INVALID_ARG;
  if (P == 0) return POLYLAB_OK;
  cudaStream_t s = (cudaStream_t)stream;
  polylab_plan* owned = nullptr;
  if (!plan) {
    PL_TRY(polylab_plan_create(p, POLYLAB_PLAN_TERMS, stream, &owned));
    plan = owned;
  }
  const int n = plan->n, E = std::max(plan->max_exp, 1);
  const size_t smem = (size_t)n * (E + 1) * 4 + (size_t)n * 5 * 4 + 5 * (size_t)n * 4 + 64 + 16 * 8 * 5;
  polylab_status st = POLYLAB_OK;
  if (smem > 220 * 1024) {
    st = POLYLAB_ERR_UNSUPPORTED;
  } else {
    auto k = mlp_data_kernel<256>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int grid = (int)std::min<int64_t>(P, (int64_t)num_sms() * 2);
    k<<<grid, 256, smem, s>>>(plan->terms, plan->m, n, E, X, P, (float)regularization, seed, feats, hdiag, e, Z, Y);
    st = launch_status("mlp_data_kernel");
  }
  if (owned) polylab_plan_destroy(owned, stream);
  return st;
}
