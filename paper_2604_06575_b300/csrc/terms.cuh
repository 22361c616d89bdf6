// Per-term derivative contributions (Sec. 3.3 differentiates term by term):
//   d_i x^a = a_i x^(a - e_i),  d_ij x^a = a_i (a_j - delta_ij) x^(a - e_i - e_j),
//   d_ijk likewise (falling factorials times a shifted monomial).
// Powers come from a per-point table pw[v * (E + 1) + k] = x_v^k built by
// repeated multiplication.
#pragma once

#include "common.cuh"

namespace polylab {

// Load a term into registers: k active slots, variables, exponents.
struct TermRegs {
  double coef;
  int k;
  int var[kMaxSupport];
  int exp[kMaxSupport];
};

__device__ __forceinline__ TermRegs load_term(const Term* __restrict__ terms, int64_t t) {
  TermRegs r;
  const uint4* p = reinterpret_cast<const uint4*>(terms + t);
  uint4 a = __ldg(p);
  uint4 b = __ldg(p + 1);
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

// Value, gradient and upper-triangle Hessian contributions of one term at one
// point.  `emit(kind, i, j, v)`: kind 0 = f, 1 = g_i, 2 = H_ij (i <= j).
template <typename R, int ORDER, typename Emit>
__device__ __forceinline__ void term_derivs(const TermRegs& t, const R* __restrict__ pw, int E1, Emit&& emit) {
  R a0[kMaxSupport];  // x_v^{a_v}
#pragma unroll
  for (int s = 0; s < kMaxSupport; ++s) a0[s] = s < t.k ? pw[t.var[s] * E1 + t.exp[s]] : R(1);
  R pre[kMaxSupport + 1], suf[kMaxSupport + 1];
  pre[0] = R(1);
#pragma unroll
  for (int s = 0; s < kMaxSupport; ++s) pre[s + 1] = s < t.k ? pre[s] * a0[s] : pre[s];
  suf[kMaxSupport] = R(1);
#pragma unroll
  for (int s = kMaxSupport - 1; s >= 0; --s) suf[s] = s < t.k ? suf[s + 1] * a0[s] : suf[s + 1];
  const R c = R(t.coef);
  emit(0, 0, 0, c * pre[kMaxSupport]);
  if constexpr (ORDER >= 1) {
#pragma unroll
  for (int s = 0; s < kMaxSupport; ++s) {
    if (s < t.k) {
      const int es = t.exp[s];
      const R excl = pre[s] * suf[s + 1];
      const R d1 = R(es) * pw[t.var[s] * E1 + es - 1];
      emit(1, t.var[s], 0, c * d1 * excl);
      if constexpr (ORDER >= 2) {
        if (es >= 2) {
          const R d2 = R(es * (es - 1)) * pw[t.var[s] * E1 + es - 2];
          emit(2, t.var[s], t.var[s], c * d2 * excl);
        }
        R mid = R(1);
#pragma unroll
        for (int u = s + 1; u < kMaxSupport; ++u) {
          if (u < t.k) {
            const int eu = t.exp[u];
            const R d1u = R(eu) * pw[t.var[u] * E1 + eu - 1];
            emit(2, t.var[s], t.var[u], c * d1 * d1u * (pre[s] * mid * suf[u + 1]));
            mid *= a0[u];
          }
        }
      }
    }
  }
  }
}

// c_l += sum_{j,k} d_l d_j d_k (term)(x) * W(j, k) for every l in the support,
// W symmetric: `wget(j, k)` returns W(j, k), `emit(l, v)` adds v to c_l.
// The third-derivative tensor of a term is symmetric, so each index multiset
// {a, b, c} of support slots is visited once: with D[s][m] =
// falling(a_s, m) x_s^(a_s - m) its entry is prod_s D[s][mult_s], where the
// slots outside the multiset contribute D[s][0] through running exclusion
// products (no division, so zeros in x are safe).  Multisets and their
// contributions:
//   {a,b,c} distinct: c_a += 2 T W_bc, c_b += 2 T W_ac, c_c += 2 T W_ab
//   {a,a,b}, a != b:  c_a += 2 T W_ab, c_b += T W_aa
//   {a,a,a}:          c_a += T W_aa
template <typename R, typename WGet, typename Emit>
__device__ __forceinline__ void term_third_contract(const TermRegs& t, const R* __restrict__ pw, int E1, WGet&& wget,
                                                    Emit&& emit) {
  const int k = t.k;
  R D0[kMaxSupport], D1[kMaxSupport], D2[kMaxSupport], D3[kMaxSupport];
#pragma unroll
  for (int s = 0; s < kMaxSupport; ++s) {
    if (s < k) {
      const int es = t.exp[s];
      const R* q = pw + t.var[s] * E1 + es;
      D0[s] = q[0];
      D1[s] = R(es) * q[-1];
      D2[s] = es >= 2 ? R(es * (es - 1)) * q[-2] : R(0);
      D3[s] = es >= 3 ? R(es * (es - 1) * (es - 2)) * q[-3] : R(0);
    } else {
      D0[s] = R(1);
      D1[s] = D2[s] = D3[s] = R(0);
    }
  }
  R pre[kMaxSupport + 1], suf[kMaxSupport + 1];
  pre[0] = R(1);
#pragma unroll
  for (int s = 0; s < kMaxSupport; ++s) pre[s + 1] = pre[s] * D0[s];
  suf[kMaxSupport] = R(1);
#pragma unroll
  for (int s = kMaxSupport - 1; s >= 0; --s) suf[s] = suf[s + 1] * D0[s];
  const R c = R(t.coef);
  R acc[kMaxSupport];
#pragma unroll
  for (int s = 0; s < kMaxSupport; ++s) acc[s] = R(0);
#pragma unroll
  for (int a = 0; a < kMaxSupport; ++a) {
    if (a < k) {
      const int va = t.var[a];
      const R Waa = wget(va, va);
      const R ex_a = pre[a] * suf[a + 1];  // product over slots != a
      acc[a] += D3[a] * ex_a * Waa;        // {a,a,a}
      R mid_ab = R(1);                      // product over slots strictly between a and b
#pragma unroll
      for (int b = a + 1; b < kMaxSupport; ++b) {
        if (b < k) {
          const int vb = t.var[b];
          const R Wab = wget(va, vb);
          const R ex_ab = pre[a] * mid_ab * suf[b + 1];  // product over slots != a, b
          // {a,a,b} and {a,b,b}
          const R Taab = D2[a] * D1[b] * ex_ab;
          const R Tabb = D1[a] * D2[b] * ex_ab;
          acc[a] += R(2) * Taab * Wab + Tabb * wget(vb, vb);
          acc[b] += Taab * Waa + R(2) * Tabb * Wab;
          R mid_bc = R(1);
#pragma unroll
          for (int cc = b + 1; cc < kMaxSupport; ++cc) {
            if (cc < k) {
              const int vc = t.var[cc];
              const R Tabc = D1[a] * D1[b] * D1[cc] * (pre[a] * mid_ab * mid_bc * suf[cc + 1]);
              acc[a] += R(2) * Tabc * wget(vb, vc);
              acc[b] += R(2) * Tabc * wget(va, vc);
              acc[cc] += R(2) * Tabc * Wab;
              mid_bc *= D0[cc];
            }
          }
          mid_ab *= D0[b];
        }
      }
    }
  }
#pragma unroll
  for (int s = 0; s < kMaxSupport; ++s)
    if (s < k) emit(t.var[s], c * acc[s]);
}

}  // namespace polylab
