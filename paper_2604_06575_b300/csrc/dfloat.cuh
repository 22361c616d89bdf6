// Double-word arithmetic on FP32 pairs: a value is hi + lo with |lo| <= ulp(hi)/2,
// about 48 significand bits, computed on the FP32 pipe (B300's FP32 rate is
// ~60x its FP64 rate).  The building blocks are the published error-free
// transformations and double-word algorithms:
//   TwoSum (Knuth, TAOCP vol. 2), FastTwoSum (Dekker 1971), TwoProd by FMA,
//   and the double-word sum, product and product-by-float of Joldes, Muller
//   and Popescu, "Tight and rigorous error bounds for basic building blocks
//   of double-word arithmetic" (ACM TOMS 44, 2017): the accurate sum has
//   relative error <= 3u^2 + 13u^3 and the product <= 5u^2 (u = 2^-24).
// The reciprocal is FP32's correctly rounded reciprocal refined by one Newton
// step in double-word arithmetic.
#pragma once

#include <cmath>
#include <cstdint>

namespace polylab {

struct __align__(8) dfloat {
  float hi, lo;
  dfloat() = default;
  __host__ __device__ constexpr dfloat(float h, float l) : hi(h), lo(l) {}
  __device__ __forceinline__ explicit dfloat(double d) {
    hi = __double2float_rn(d);
    lo = __double2float_rn(d - (double)hi);
  }
  __device__ __forceinline__ explicit dfloat(float f) : hi(f), lo(0.f) {}
  __device__ __forceinline__ explicit dfloat(int i) : hi((float)i), lo(0.f) {}
  __device__ __forceinline__ explicit operator double() const { return (double)hi + (double)lo; }
  __device__ __forceinline__ explicit operator float() const { return hi + lo; }
};

// s + e = a + b exactly (no condition on the magnitudes)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// s + e = a + b exactly when |a| >= |b| (or a = 0)
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}
// p + e = a * b exactly (FMA)
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = __fmul_rn(a, b);
  e = __fmaf_rn(a, b, -p);
}

__device__ __forceinline__ dfloat operator+(dfloat x, dfloat y) {
  float sh, sl, th, tl, vh, vl, zh, zl;
  two_sum(x.hi, y.hi, sh, sl);
  two_sum(x.lo, y.lo, th, tl);
  const float c = __fadd_rn(sl, th);
  fast_two_sum(sh, c, vh, vl);
  const float w = __fadd_rn(tl, vl);
  fast_two_sum(vh, w, zh, zl);
  return {zh, zl};
}
__device__ __forceinline__ dfloat operator-(dfloat x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ dfloat operator-(dfloat x, dfloat y) { return x + (-y); }
__device__ __forceinline__ dfloat operator*(dfloat x, dfloat y) {
  float ch, cl1, zh, zl;
  two_prod(x.hi, y.hi, ch, cl1);
  const float tl0 = __fmul_rn(x.lo, y.lo);
  const float tl1 = __fmaf_rn(x.hi, y.lo, tl0);
  const float cl2 = __fmaf_rn(x.lo, y.hi, tl1);
  fast_two_sum(ch, __fadd_rn(cl1, cl2), zh, zl);
  return {zh, zl};
}
// double-word times float
__device__ __forceinline__ dfloat operator*(dfloat x, float y) {
  float ch, cl1, zh, zl;
  two_prod(x.hi, y, ch, cl1);
  fast_two_sum(ch, __fmaf_rn(x.lo, y, cl1), zh, zl);
  return {zh, zl};
}
__device__ __forceinline__ dfloat& operator+=(dfloat& x, dfloat y) { return x = x + y; }
__device__ __forceinline__ dfloat& operator-=(dfloat& x, dfloat y) { return x = x - y; }
__device__ __forceinline__ dfloat& operator*=(dfloat& x, dfloat y) { return x = x * y; }

// 1/x: r0 = rn(1/hi), then r = r0 + r0 (1 - x r0) with the residual in double words
__device__ __forceinline__ dfloat dw_recip(dfloat x) {
  const float r0 = __frcp_rn(x.hi);
  const dfloat e = dfloat(1.0f, 0.0f) - x * r0;
  float zh, zl;
  fast_two_sum(r0, __fmul_rn(r0, e.hi), zh, zl);
  return {zh, zl};
}
__device__ __forceinline__ dfloat operator/(dfloat x, dfloat y) { return x * dw_recip(y); }

using ::fabs;  // (the overload below must not hide the float and double ones)
__device__ __forceinline__ dfloat fabs(dfloat x) { return x.hi < 0.f ? -x : x; }

// Adds v to the double word *p that concurrent threads update: the high
// words are added by an FP32 atomic whose returned old value gives the exact
// rounding error of that addition (TwoSum of old and v.hi), which goes with
// v.lo into an atomic on the low word.  So the high word plus the low word is
// the exact sum of everything added, up to the low words' own FP32 rounding
// (~2^-48 of the total).  Two native FP32 atomics instead of an FP64 atomic,
// which shared memory implements as a compare-and-swap loop.
__device__ __forceinline__ void atomic_add_dw(dfloat* p, dfloat v) {
  const float old = atomicAdd(&p->hi, v.hi);
  float s, e;
  two_sum(old, v.hi, s, e);
  atomicAdd(&p->lo, __fadd_rn(v.lo, e));
}

// Compensated sum of double words: a float running sum whose additions'
// rounding errors (TwoSum) and the addends' low words gather in one float
// correction (the summation of Ogita, Rump and Oishi, SIAM J. Sci. Comput.
// 26, 2005): about twice the working precision at 8 FP32 operations per
// addend, against 20 for the accurate double-word sum.
struct dw_comp_sum {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(dfloat v) {
    float t, e;
    two_sum(s, v.hi, t, e);
    s = t;
    c = __fadd_rn(c, __fadd_rn(e, v.lo));
  }
  __device__ __forceinline__ dfloat value() const {
    float h, l;
    two_sum(s, c, h, l);
    return {h, l};
  }
};

// Running sum of products m * cf (m a double word, cf a small integer held
// exactly as a float), compensated in the manner of Ogita, Rump and Oishi,
// "Accurate sum and dot product" (SIAM J. Sci. Comput. 26, 2005): the high
// product is split exactly (TwoProd), added to the running float sum exactly
// (TwoSum), and the rounding errors together with the low word's product are
// gathered in one float correction.  About twice the working precision (the
// error is of order n u^2 times the sum of |products|) at 11 FP32 operations
// per product, against 26 for a double-word product and sum.
struct dw_run_sum {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(dfloat m, float cf) {
    float p, ep, t, es;
    two_prod(m.hi, cf, p, ep);
    const float e2 = __fmaf_rn(m.lo, cf, ep);
    two_sum(s, p, t, es);
    s = t;
    c = __fadd_rn(c, __fadd_rn(es, e2));
  }
  __device__ __forceinline__ dfloat value() const {
    float h, l;
    two_sum(s, c, h, l);
    return {h, l};
  }
};

// Compensated dot product of double words: the products of the high words
// split exactly by TwoProd, the cross terms a.hi b.lo + a.lo b.hi folded into
// the product's error, the running float sum split exactly by TwoSum, and
// every error gathered in one float correction (Dot2 of Ogita, Rump and
// Oishi, SIAM J. Sci. Comput. 26, 2005, on double-word operands; the term
// a.lo b.lo, about 2^-48 of the product, is dropped).  12 FP32 operations per
// product, against 17 for a double-word product added to dw_comp_sum and 29
// for a double-word product and accurate sum.
struct dw_dot {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(dfloat a, dfloat b) {
    float p, e, t, es;
    two_prod(a.hi, b.hi, p, e);
    e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
    two_sum(s, p, t, es);
    s = t;
    c = __fadd_rn(c, __fadd_rn(es, e));
  }
  __device__ __forceinline__ dfloat value() const {
    float h, l;
    two_sum(s, c, h, l);
    return {h, l};
  }
};

// Type of a small integer multiplier (an exponent or falling-factorial
// coefficient) in a form's arithmetic: exact as a plain float, and the
// double-word-times-float product is cheaper than a full double-word product.
template <typename R>
struct SmallT {
  using T = R;
};
template <>
struct SmallT<dfloat> {
  using T = float;
};
template <typename R>
using SmallOf = typename SmallT<R>::T;

// warp shuffle of a double word
__device__ __forceinline__ dfloat shfl(dfloat v, int src) {
  return {__shfl_sync(0xffffffffu, v.hi, src), __shfl_sync(0xffffffffu, v.lo, src)};
}

}  // namespace polylab
