// Per-term derivative contributions (Sec. 3.3 differentiates term by term):
//   d_i x^a = a_i x^(a - e_i),  d_ij x^a = a_i (a_j - delta_ij) x^(a - e_i - e_j),
//   d_ijk likewise (falling factorials times a shifted monomial).
// Powers come from a per-point table pw[v * (E + 1) + k] = x_v^k built by
// repeated multiplication.  A term reads two entries per active variable, x_v
// and its lowest needed power, and rebuilds the higher powers by the same
// multiplications the table uses (so the values are those of the table):
// shared-memory loads, not arithmetic, bound these sweeps.
#pragma once

#include <type_traits>

#include "common.cuh"
#include "dfloat.cuh"

namespace polylab {

// Load a term into registers: k active slots, variables, exponents.
struct TermRegs {
  double coef;
  int k;
  int var[kMaxSupport];
  int exp[kMaxSupport];
};

__device__ __forceinline__ TermRegs decode_term(uint4 a, uint4 b) {
  TermRegs r;
  r.coef = __hiloint2double((int)a.y, (int)a.x);
  const uint32_t v[4] = {a.z, a.w, b.x, b.y};
  const uint32_t e[2] = {b.z, b.w};
  r.k = 0;
#pragma unroll
  for (int s = 0; s < kMaxSupport; ++s) {
    r.var[s] = (v[s >> 1] >> ((s & 1) * 16)) & 0xffff;
    r.exp[s] = (e[s >> 2] >> ((s & 3) * 8)) & 0xff;
    r.k += r.exp[s] != 0;
  }
  return r;
}

__device__ __forceinline__ TermRegs load_term(const Term* __restrict__ terms, int64_t t) {
  const uint4* p = reinterpret_cast<const uint4*>(terms + t);
  return decode_term(__ldg(p), __ldg(p + 1));
}

// Strided walk t = start, start + stride, ... < m over a term list with the
// next term's 32 bytes loaded one step ahead, so the load latency of the term
// stream overlaps the current term's arithmetic.
struct TermStream {
  const uint4* p;
  int64_t t, m, stride;
  uint4 a, b;
  __device__ __forceinline__ TermStream(const Term* __restrict__ terms, int64_t m_, int64_t start, int64_t stride_)
      : p(reinterpret_cast<const uint4*>(terms)), t(start), m(m_), stride(stride_) {
    if (t < m) {
      a = __ldg(p + 2 * t);
      b = __ldg(p + 2 * t + 1);
    }
  }
  __device__ __forceinline__ bool next(TermRegs& r) {
    if (t >= m) return false;
    const uint4 ca = a, cb = b;
    const int64_t tn = t + stride;
    if (tn < m) {
      a = __ldg(p + 2 * tn);
      b = __ldg(p + 2 * tn + 1);
    }
    r = decode_term(ca, cb);
    t = tn;
    return true;
  }
};

// Value, gradient and upper-triangle Hessian contributions of one term at one
// point, for a term with exactly K active variables (loops fully unrolled).
// `emit(kind, i, j, v)`: kind 0 = f, 1 = g_i, 2 = H_ij (i <= j).
template <typename R, int ORDER, int K, typename Emit>
__device__ __forceinline__ void term_derivs_k(const TermRegs& t, const R* __restrict__ pw, int E1, Emit&& emit) {
  const R c = R(t.coef);
  if constexpr (K == 0) {
    emit(0, 0, 0, c);
  } else {
    R a0[K], d1[K], q2[K];  // x^a, a x^(a-1), x^(a-2) (a >= 2 only) per slot
#pragma unroll
    for (int s = 0; s < K; ++s) {
      const R* row = pw + t.var[s] * E1;
      const int es = t.exp[s];
      const R x = row[1];
      const R q = row[es >= 2 ? es - 2 : 0];
      const R p1 = es >= 2 ? q * x : R(1);
      a0[s] = p1 * x;
      d1[s] = R(es) * p1;
      q2[s] = q;
    }
    R pre[K + 1], suf[K + 1];
    pre[0] = R(1);
#pragma unroll
    for (int s = 0; s < K; ++s) pre[s + 1] = pre[s] * a0[s];
    suf[K] = R(1);
#pragma unroll
    for (int s = K - 1; s >= 0; --s) suf[s] = suf[s + 1] * a0[s];
    emit(0, 0, 0, c * pre[K]);
    if constexpr (ORDER >= 1) {
#pragma unroll
      for (int s = 0; s < K; ++s) {
        const R excl = pre[s] * suf[s + 1];
        emit(1, t.var[s], 0, c * d1[s] * excl);
        if constexpr (ORDER >= 2) {
          const int es = t.exp[s];
          if (es >= 2) emit(2, t.var[s], t.var[s], c * R(es * (es - 1)) * q2[s] * excl);
          R mid = R(1);
#pragma unroll
          for (int u = s + 1; u < K; ++u) {
            emit(2, t.var[s], t.var[u], c * d1[s] * d1[u] * (pre[s] * mid * suf[u + 1]));
            mid *= a0[u];
          }
        }
      }
    }
  }
}

// Largest support size a per-term routine is inlined for.  Terms with more
// active variables are rare; they run out of line so that their register
// demand does not set the budget of the common cases.
template <typename R>
constexpr int kInlineSupport = 6;
// The same for the paths that only points with a near-zero coordinate take:
// double-word code is ~15x larger per operation, so there these stay out of
// line and leave the instruction cache to the common path.
template <typename R>
constexpr int kInlineSupportRare = std::is_same<R, dfloat>::value ? 0 : 6;

template <typename R, int ORDER, int K, typename Emit>
__device__ __noinline__ void term_derivs_wide(const TermRegs& t, const R* __restrict__ pw, int E1, Emit emit) {
  term_derivs_k<R, ORDER, K>(t, pw, E1, emit);
}

// Dispatch on the support size.  Plans keep their term lists sorted by
// support size, so the threads of a warp normally take the same branch.
template <typename R, int ORDER, typename Emit>
__device__ __forceinline__ void term_derivs(const TermRegs& t, const R* __restrict__ pw, int E1, Emit&& emit) {
  switch (t.k) {
    case 0: term_derivs_k<R, ORDER, 0>(t, pw, E1, emit); break;
    case 1: term_derivs_k<R, ORDER, 1>(t, pw, E1, emit); break;
    case 2: term_derivs_k<R, ORDER, 2>(t, pw, E1, emit); break;
    case 3: term_derivs_k<R, ORDER, 3>(t, pw, E1, emit); break;
    case 4: term_derivs_k<R, ORDER, 4>(t, pw, E1, emit); break;
    case 5: term_derivs_k<R, ORDER, 5>(t, pw, E1, emit); break;
    case 6: term_derivs_k<R, ORDER, 6>(t, pw, E1, emit); break;
    case 7: term_derivs_wide<R, ORDER, 7>(t, pw, E1, emit); break;
    default: term_derivs_wide<R, ORDER, 8>(t, pw, E1, emit); break;
  }
}

// c_l += sum_{j,k} d_l d_j d_k (term)(x) * W(j, k) for every l in the support
// of a term with exactly K active variables, W symmetric: `wget(a, b, va, vb)`
// returns W(va, vb) for support slots a, b holding variables va, vb (a caller
// may look W up by variable or by the term's own slots), `emit(l, v)` adds v
// to c_l (l a variable).  The third-derivative tensor of a term
// is symmetric, so each index multiset {a, b, c} of support slots is visited
// once: with D_m[s] = falling(a_s, m) x_s^(a_s - m) its entry is
// prod_s D_{mult_s}[s]; slots outside the multiset contribute D_0 through
// running exclusion products (no division, so zeros in x are safe).
//   {a,b,c} distinct: c_a += 2 T W_bc, c_b += 2 T W_ac, c_c += 2 T W_ab
//   {a,a,b}, a != b:  c_a += 2 T W_ab, c_b += T W_aa
//   {a,a,a}:          c_a += T W_aa
template <typename R, int K, typename WGet, typename Emit>
__device__ __forceinline__ void term_third_contract_k(const TermRegs& t, const R* __restrict__ pw, int E1,
                                                      WGet&& wget, Emit&& emit) {
  R D0[K], D1[K], D2[K], D3[K];
#pragma unroll
  for (int s = 0; s < K; ++s) {
    const int es = t.exp[s];
    const R* row = pw + t.var[s] * E1;
    const R x = row[1];
    const R r3 = row[es >= 3 ? es - 3 : 0];
    const R p2 = es >= 3 ? r3 * x : R(1);  // x^(a-2), a >= 2
    const R p1 = es >= 2 ? p2 * x : R(1);  // x^(a-1)
    D0[s] = p1 * x;
    D1[s] = R(es) * p1;
    D2[s] = es >= 2 ? R(es * (es - 1)) * p2 : R(0);
    D3[s] = es >= 3 ? R(es * (es - 1) * (es - 2)) * r3 : R(0);
  }
  R pre[K + 1], suf[K + 1];
  pre[0] = R(1);
#pragma unroll
  for (int s = 0; s < K; ++s) pre[s + 1] = pre[s] * D0[s];
  suf[K] = R(1);
#pragma unroll
  for (int s = K - 1; s >= 0; --s) suf[s] = suf[s + 1] * D0[s];
  R acc[K];
  R Wd[K];
#pragma unroll
  for (int s = 0; s < K; ++s) {
    acc[s] = R(0);
    Wd[s] = wget(s, s, t.var[s], t.var[s]);
  }
#pragma unroll
  for (int a = 0; a < K; ++a) {
    const int va = t.var[a];
    acc[a] += D3[a] * (pre[a] * suf[a + 1]) * Wd[a];  // {a,a,a}
    R mid_ab = R(1);  // product over slots strictly between a and b
#pragma unroll
    for (int b = a + 1; b < K; ++b) {
      const int vb = t.var[b];
      const R Wab = wget(a, b, va, vb);
      const R ex_ab = pre[a] * mid_ab * suf[b + 1];  // product over slots != a, b
      const R Taab = D2[a] * D1[b] * ex_ab;
      const R Tabb = D1[a] * D2[b] * ex_ab;
      acc[a] += R(2) * Taab * Wab + Tabb * Wd[b];
      acc[b] += Taab * Wd[a] + R(2) * Tabb * Wab;
      R mid_bc = R(1);
#pragma unroll
      for (int cc = b + 1; cc < K; ++cc) {
        const R Tabc = D1[a] * D1[b] * D1[cc] * (pre[a] * mid_ab * mid_bc * suf[cc + 1]);
        acc[a] += R(2) * Tabc * wget(b, cc, vb, t.var[cc]);
        acc[b] += R(2) * Tabc * wget(a, cc, va, t.var[cc]);
        acc[cc] += R(2) * Tabc * Wab;
        mid_bc *= D0[cc];
      }
      mid_ab *= D0[b];
    }
  }
  const R c = R(t.coef);
#pragma unroll
  for (int s = 0; s < K; ++s) emit(t.var[s], c * acc[s]);
}

template <typename R, int K, typename WGet, typename Emit>
__device__ __noinline__ void term_third_contract_wide(const TermRegs& t, const R* __restrict__ pw, int E1, WGet wget,
                                                      Emit emit) {
  term_third_contract_k<R, K>(t, pw, E1, wget, emit);
}

template <typename R, typename WGet, typename Emit>
__device__ __forceinline__ void term_third_contract(const TermRegs& t, const R* __restrict__ pw, int E1, WGet&& wget,
                                                    Emit&& emit) {
  switch (t.k) {
    case 0: break;
    case 1: term_third_contract_k<R, 1>(t, pw, E1, wget, emit); break;
    case 2: term_third_contract_k<R, 2>(t, pw, E1, wget, emit); break;
    case 3: term_third_contract_k<R, 3>(t, pw, E1, wget, emit); break;
    case 4: term_third_contract_k<R, 4>(t, pw, E1, wget, emit); break;
    case 5: term_third_contract_k<R, 5>(t, pw, E1, wget, emit); break;
    case 6: term_third_contract_k<R, 6>(t, pw, E1, wget, emit); break;
    case 7: term_third_contract_wide<R, 7>(t, pw, E1, wget, emit); break;
    default: term_third_contract_wide<R, 8>(t, pw, E1, wget, emit); break;
  }
}

// Gather form of the same contraction, for points where the monomial value
// m = c x^a and 1/x stay normal numbers.  With u_j = a_j / x_j,
//   d_l d_j d_k m = m (a_j a_k - delta_jk a_j)(a_l - delta_lj - delta_lk) / (x_l x_j x_k),
// and grouping the (j, k) of the support by how they meet l,
//   c_l += m u_l [ 2 sum_{j<k; j,k != l} u_j u_k W_jk + sum_{j != l} u_j (u_j - 1/x_j) W_jj
//                + 2 (a_l - 1) / x_l sum_{k != l} u_k W_lk + (a_l - 1)(a_l - 2) / x_l^2 W_ll ].
// Every multiplier is non-negative, so no term cancels another the direct
// contraction would not; the work is K(K+1)/2 lookups of W, O(K^2)
// products and O(K^3) additions instead of a product per index multiset.
// `ix` holds 1/x per variable; wget as above.
template <typename R, int K, typename WGet, typename Emit>
__device__ __forceinline__ void term_third_gather_k(const TermRegs& t, const R* __restrict__ pw, int E1,
                                                   const R* __restrict__ ix, WGet&& wget, Emit&& emit) {
  R m = R(t.coef), xi[K], uk[K], wd[K], gd[K], rs[K], pp[K][K];
#pragma unroll
  for (int q = 0; q < K; ++q) {
    const int v = t.var[q];
    m *= pw[v * E1 + t.exp[q]];
    xi[q] = ix[v];
    uk[q] = R(t.exp[q]) * xi[q];
    wd[q] = wget(q, q, v, v);
    gd[q] = uk[q] * (uk[q] - xi[q]) * wd[q];
    rs[q] = R(0);
  }
#pragma unroll
  for (int j = 0; j < K; ++j) {
#pragma unroll
    for (int k = j + 1; k < K; ++k) {
      const R w = wget(j, k, t.var[j], t.var[k]);
      pp[j][k] = uk[j] * uk[k] * w;
      rs[j] += uk[k] * w;
      rs[k] += uk[j] * w;
    }
  }
#pragma unroll
  for (int l = 0; l < K; ++l) {
    R pairs = R(0), diag = R(0);
#pragma unroll
    for (int j = 0; j < K; ++j) {
      if (j == l) continue;
      diag += gd[j];
#pragma unroll
      for (int k = j + 1; k < K; ++k)
        if (k != l) pairs += pp[j][k];
    }
    const R al = R(t.exp[l]);
    const R bracket = R(2) * pairs + diag + R(2) * (al - R(1)) * xi[l] * rs[l] +
                      (al - R(1)) * (al - R(2)) * xi[l] * xi[l] * wd[l];
    emit(t.var[l], m * uk[l] * bracket);
  }
}

template <typename R, int K, typename WGet, typename Emit>
__device__ __noinline__ void term_third_gather_wide(const TermRegs& t, const R* __restrict__ pw, int E1,
                                                    const R* __restrict__ ix, WGet wget, Emit emit) {
  term_third_gather_k<R, K>(t, pw, E1, ix, wget, emit);
}

template <typename R, int K, typename WGet, typename Emit>
__device__ __forceinline__ void term_third_gather_group(const TermRegs& t, const R* __restrict__ pw, int E1,
                                                       const R* __restrict__ ix, WGet& wget, Emit& emit) {
  if constexpr (K <= 6) term_third_gather_k<R, K>(t, pw, E1, ix, wget, emit);
  else term_third_gather_wide<R, K>(t, pw, E1, ix, wget, emit);
}

// The gather form reduced algebraically.  With u_l = a_l / x_l,
// rs_l = sum_{k != l} u_k W_lk and the pair and diagonal sums written through
// rs (sum_{j<k} u_j u_k W_jk = (1/2) sum_l u_l rs_l, u_l (u_l - 1/x_l) =
// a_l (a_l - 1) / x_l^2), the bracket of the gather form collapses to
//   bracket_l = C - (2 / x_l) q_l,  q_l = rs_l + (a_l - 1) W_ll / x_l,
//   C = sum_j u_j q_j,
// so a term costs K(K+1)/2 lookups of W and O(K^2) products and additions
// with no K x K table.  For a_l = 1 the bracket's (u_l - 1/x_l) rs_l part is
// zero but is formed as a difference here, so the form costs accuracy: it is
// used for the double-word form, whose error bar leaves room for it; the
// FP32 form and the FP64 form (the accuracy reference) keep the
// cancellation-free gather form above.
template <typename R, int K, typename WGet, typename Emit>
__device__ __forceinline__ void term_third_gather_sub_k(const TermRegs& t, const R* __restrict__ pw, int E1,
                                                       const R* __restrict__ ix, WGet&& wget, Emit&& emit) {
  using S = SmallOf<R>;
  R m = R(t.coef), xi[K], rs[K];
#pragma unroll
  for (int q = 0; q < K; ++q) {
    m *= pw[t.var[q] * E1 + t.exp[q]];
    xi[q] = ix[t.var[q]];
    rs[q] = R(0);
  }
#pragma unroll
  for (int j = 0; j < K; ++j) {
#pragma unroll
    for (int k = j + 1; k < K; ++k) {
      const R w = wget(j, k, t.var[j], t.var[k]);
      rs[j] += xi[k] * w * S(t.exp[k]);
      rs[k] += xi[j] * w * S(t.exp[j]);
    }
  }
  R C = R(0);
#pragma unroll
  for (int l = 0; l < K; ++l) {
    const int al = t.exp[l];
    rs[l] += xi[l] * wget(l, l, t.var[l], t.var[l]) * S(al - 1);  // q_l
    C += xi[l] * rs[l] * S(al);
  }
#pragma unroll
  for (int l = 0; l < K; ++l) emit(t.var[l], m * xi[l] * (C - xi[l] * rs[l] * S(2)) * S(t.exp[l]));
}

// The same reduced form in double words, arranged for their cost: u = a/x
// formed once per slot, and rs and C kept as compensated sums.
template <int K, typename WGet, typename Emit>
__device__ __forceinline__ void term_third_gather_dw_k(const TermRegs& t, const dfloat* __restrict__ pw, int E1,
                                                      const dfloat* __restrict__ ix, WGet&& wget, Emit&& emit) {
  dfloat m = dfloat(t.coef), xi[K], u[K], qv[K];
  dw_dot rs[K], C;
#pragma unroll
  for (int q = 0; q < K; ++q) {
    m *= pw[t.var[q] * E1 + t.exp[q]];
    xi[q] = ix[t.var[q]];
    u[q] = xi[q] * (float)t.exp[q];
  }
#pragma unroll
  for (int j = 0; j < K; ++j) {
#pragma unroll
    for (int k = j + 1; k < K; ++k) {
      const dfloat w = wget(j, k, t.var[j], t.var[k]);
      rs[j].add(u[k], w);
      rs[k].add(u[j], w);
    }
  }
#pragma unroll
  for (int l = 0; l < K; ++l) {
    rs[l].add(xi[l] * (float)(t.exp[l] - 1), wget(l, l, t.var[l], t.var[l]));
    qv[l] = rs[l].value();
    C.add(u[l], qv[l]);
  }
  const dfloat Cv = C.value();
#pragma unroll
  for (int l = 0; l < K; ++l) {
    const dfloat xq = xi[l] * qv[l];
    emit(t.var[l], m * u[l] * (Cv - dfloat(2.0f * xq.hi, 2.0f * xq.lo)));  // (x2 exact)
  }
}

template <typename R, int K, typename WGet, typename Emit>
__device__ __noinline__ void term_third_gather_sub_wide(const TermRegs& t, const R* __restrict__ pw, int E1,
                                                        const R* __restrict__ ix, WGet wget, Emit emit) {
  if constexpr (std::is_same<R, dfloat>::value) term_third_gather_dw_k<K>(t, pw, E1, ix, wget, emit);
  else term_third_gather_sub_k<R, K>(t, pw, E1, ix, wget, emit);
}

template <typename R, int K, typename WGet, typename Emit>
__device__ __forceinline__ void term_third_gather_sub_group(const TermRegs& t, const R* __restrict__ pw, int E1,
                                                           const R* __restrict__ ix, WGet& wget, Emit& emit) {
  if constexpr (K > kInlineSupport<R>) term_third_gather_sub_wide<R, K>(t, pw, E1, ix, wget, emit);
  else if constexpr (std::is_same<R, dfloat>::value) term_third_gather_dw_k<K>(t, pw, E1, ix, wget, emit);
  else term_third_gather_sub_k<R, K>(t, pw, E1, ix, wget, emit);
}

// c x^a of one term at one point (any support size).
template <typename R>
__device__ __forceinline__ R term_value(const TermRegs& t, const R* __restrict__ pw, int E1) {
  R v = R(t.coef);
#pragma unroll
  for (int s = 0; s < kMaxSupport; ++s)
    if (t.exp[s]) v *= pw[t.var[s] * E1 + t.exp[s]];
  return v;
}

// Call f(std::integral_constant<int, K>{}) for K = 0..KMAX in order.
template <int KMAX, int K = 0, typename F>
__device__ __forceinline__ void for_support(F&& f) {
  f(std::integral_constant<int, K>{});
  if constexpr (K < KMAX) for_support<KMAX, K + 1>(f);
}

// Per-group entry points: groups up to six active variables inline, wider
// groups out of line (see term_derivs_wide).
template <typename R, int ORDER, int K, typename Emit>
__device__ __forceinline__ void term_derivs_group(const TermRegs& t, const R* __restrict__ pw, int E1, Emit& emit) {
  if constexpr (K <= kInlineSupportRare<R>) term_derivs_k<R, ORDER, K>(t, pw, E1, emit);
  else term_derivs_wide<R, ORDER, K>(t, pw, E1, emit);
}

template <typename R, int K, typename WGet, typename Emit>
__device__ __forceinline__ void term_third_group(const TermRegs& t, const R* __restrict__ pw, int E1, WGet& wget,
                                                 Emit& emit) {
  if constexpr (K <= kInlineSupportRare<R>) term_third_contract_k<R, K>(t, pw, E1, wget, emit);
  else term_third_contract_wide<R, K>(t, pw, E1, wget, emit);
}

}  // namespace polylab
