// MF-logDet-Exact affine-normal direction (Sec. 5) for a batch of
// (polynomial, point) work items, in three stages of persistent launches
// (the frame stage optionally one launch per class of n) that pass per-point
// data through a device workspace:
//
//   stage 1 (terms)  g = grad f(x) and H = Hess f(x) from the term list,
//                    accumulated in shared memory            -> H, g, sum |g terms|
//   stage 2 (frame)  e = g/|g|; Householder reflector P = I - beta v v^T with
//                    v = e + s e_n (s = sign(e_n)), so P e_n = -s e and the
//                    first m = n-1 columns of P are an orthonormal frame Q_T
//                    of e-perp; P H P by a rank-2 update; H_T = (PHP)[0:m,0:m]
//                    + r I, h = Q_T^T H e = -s (PHP)[0:m, n-1]; LDL^T of H_T in
//                    FP64 (a non-positive pivot flags NOT_PD), log-det;
//                    M = H_T^{-1}; W = Q_T M Q_T^T = P [M 0; 0 0] P
//                                                  -> W, v, e, h, beta, |g|, log-det
//   stage 3 (third)  c_l = sum_jk d_l d_j d_k f(x) W_jk from the term list, so
//                    a_i = tr(H_T^{-1} d_{t_i} H_T) = (Q_T^T c)_i = (P c)_i
//                    without forming the third-derivative tensor;
//                    tau = M (h - |g|/(n+1) a) and, because [M 0; 0 0] = P W P,
//                    nu = Q_T tau - e = W P [h - |g|/(n+1) a; 0] - e.
//
// The two term sweeps are latency bound and run best with many resident CTAs;
// the frame stage is bound by the dependent FP64 factorisation chain.  As
// separate launches each stage gets its own CTA size, register budget and
// shared memory.
//
// R = double: every step in FP64.  R = float (POLYLAB_FP32): term sums, frame
// update, inverse, W and the trace term in FP32; the LDL^T factorisation,
// log-det, the O(n) vectors and the normalisation in FP64.
//
// Work items are taken from one device counter per stage in the order of a
// host-built permutation (most expensive polynomials first), so an uneven
// batch keeps every SM busy.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "async.cuh"
#include "batch.cuh"
#include "common.cuh"
#include "dfloat.cuh"
#include "terms.cuh"

namespace polylab {

namespace {

// Types of a form.  R: the arithmetic of the term sweeps, the frame update
// and the inverse; Acc: the sums of gradient, Hessian and trace-term
// contributions (added atomically in shared memory; H is handed to the
// frame stage in this type); Abs: sums of |contributions| (an error scale
// only).  The double-word form sums into double words by atomic_add_dw.
template <typename R>
struct FormTypes {
  using Acc = R;
  using Abs = R;
};
template <>
struct FormTypes<dfloat> {
  using Acc = dfloat;
  using Abs = float;
};
template <typename R>
using AccOf = typename FormTypes<R>::Acc;
template <typename R>
using AbsOf = typename FormTypes<R>::Abs;

// Sum of products a * b in a form's arithmetic: plain multiply-adds, or for
// double words the compensated sum of the products (17 FP32 operations per
// term instead of 29).
template <typename R>
struct DotAcc {
  R v = R(0);
  __device__ __forceinline__ void add(R a, R b) { v += a * b; }
  __device__ __forceinline__ R value() const { return v; }
};
template <>
struct DotAcc<dfloat> {
  dw_dot c;
  __device__ __forceinline__ void add(dfloat a, dfloat b) { c.add(a, b); }
  __device__ __forceinline__ dfloat value() const { return c.value(); }
};

// the two points' values of one monomial by one vector load (8 or 16 bytes)
__device__ __forceinline__ void load_pair(const float* p, float (&v)[2]) {
  const float2 t = *reinterpret_cast<const float2*>(p);
  v[0] = t.x;
  v[1] = t.y;
}
template <typename R>
__device__ __forceinline__ void load_pair(const R* p, R (&v)[2]) {
  static_assert(sizeof(R) == 8, "8-byte values");
  const uint4 t = *reinterpret_cast<const uint4*>(p);
  v[0] = *reinterpret_cast<const R*>(&t.x);
  v[1] = *reinterpret_cast<const R*>(&t.z);
}

// atomic accumulation into a form's sums
template <typename T>
__device__ __forceinline__ void acc_add(T* p, T v) {
  atomicAdd(p, v);
}
__device__ __forceinline__ void acc_add(dfloat* p, dfloat v) { atomic_add_dw(p, v); }

// Sum of one run of gather records c_r * m_t (the contributions to one
// gradient or Hessian entry) in the form's arithmetic.  Double words use the
// compensated running sum of dfloat.cuh.
template <typename R>
struct RunSum {
  R v = R(0);
  __device__ __forceinline__ void add(R m, SmallOf<R> cf) { v += m * cf; }
  __device__ __forceinline__ AccOf<R> value() const { return AccOf<R>(v); }
};
template <>
struct RunSum<dfloat> : dw_run_sum {};
// |v| in the precision of the zero-gradient scale (a double word's high word)
__device__ __forceinline__ double abs_of(double v) { return fabs(v); }
__device__ __forceinline__ float abs_of(float v) { return fabsf(v); }
__device__ __forceinline__ float abs_of(dfloat v) { return fabsf(v.hi); }

// sum_i a_i / |x_i| over a term's active variables (ix = 1/x): times |c m_t|
// it is the sum of the magnitudes of the term's gradient contributions
// c a_i m_t / x_i, the scale of the zero-gradient test
template <typename R>
__device__ __forceinline__ AbsOf<R> grad_abs_factor(const TermRegs& t, const R* __restrict__ ix) {
  AbsOf<R> s = AbsOf<R>(0);
#pragma unroll
  for (int k = 0; k < kMaxSupport; ++k)
    if (t.exp[k]) s += AbsOf<R>(t.exp[k]) * abs_of(ix[t.var[k]]);
  return s;
}

template <typename T>
__device__ __forceinline__ T shfl_r(T v, int src) {
  return __shfl_sync(0xffffffffu, v, src);
}
__device__ __forceinline__ dfloat shfl_r(dfloat v, int src) { return shfl(v, src); }

// Per-point record of small vectors in the workspace (doubles):
// [0,n) g | [n,2n) v | [2n,3n) e | [3n,4n) h | 4n: sum |g terms| | 4n+1: |g|
// | 4n+2: beta | 4n+3: log-det | 4n+4: status
// per-point record: g, v, e, h (n each), 8 scalars, then the trace term's
// partial sums c (n) carried between the launches of a split third stage
__host__ __device__ inline int64_t vrec(int n) { return 5 * (int64_t)n + 8; }
constexpr double kStOk = 0.0, kStZero = 1.0, kStNotPd = 2.0;

// Elements of a point's n x n slot in the matrix workspaces: n^2 rounded up to
// 16 bytes, so that every slot can move by one bulk copy.
template <typename R>
__host__ __device__ inline int64_t mat_slot(int n) {
  constexpr int q = 16 / sizeof(R);
  return ((int64_t)n * n + q - 1) / q * q;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// next work item of this CTA (uniform across the CTA)
__device__ __forceinline__ int64_t next_item(int* counter, int64_t* s_item) {
  __syncthreads();
  if (threadIdx.x == 0) *s_item = (int64_t)atomicAdd(counter, 1);
  __syncthreads();
  return *s_item;
}

// position of `item` in the permuted polynomial list: prefix[] is over the
// polynomials in work order
__device__ __forceinline__ int find_poly(const int64_t* __restrict__ prefix, int n_desc, int64_t item) {
  int lo = 0, hi = n_desc;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (prefix[mid] <= item) lo = mid;
    else hi = mid;
  }
  return lo;
}

// x_v^k for k < E1, one row per variable
template <typename R, int NT>
__device__ __forceinline__ void power_table(const double* __restrict__ X, int n, int E1, R* pw) {
  for (int i = threadIdx.x; i < n; i += NT) {
    const R x = R(X[i]);
    R cur = R(1);
    pw[i * E1] = cur;
    for (int k = 1; k < E1; ++k) {
      cur = cur * x;
      pw[i * E1 + k] = cur;
    }
  }
}

// LDL^T factorisation of the symmetric positive definite leading m x m block
// in FP64, right-looking, by the whole CTA with one barrier per column.
// col(j)[i] addresses element (i, j), i >= j (consecutive i are consecutive
// doubles).  On return col(j)[i] = l_ij (i > j), dv[k] = d_k, di[k] = 1/d_k.
// Column k+1 is updated and pivoted by warp 0 while the other warps apply
// column k to columns k+2.. (a_ij -= l_ik a_jk, with the unscaled a_jk kept
// in uc), so a step needs no second barrier.  A pivot that is not positive
// and finite sets its flag (the block is not positive definite): pivot c
// writes flag[c & 1] and every thread reads flag[k & 1] after the barrier
// that ends the step which made pivot k, so a flag is never written in the
// step that reads it (warp 0 makes pivot k+1 while a slower warp may still be
// reading pivot k's flag) and every warp leaves at the same step.  The caller
// reads flag[0] | flag[1] after the final barrier.
template <int NT, typename Col>
__device__ __forceinline__ void ldlt_block(int m, Col col, double* __restrict__ uc, double* __restrict__ dv,
                                           double* __restrict__ di, int* flag) {
  static_assert(NT >= 64, "one pivot warp plus at least one update warp");
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (m == 0) return;
  auto pivot = [&](int c) {  // warp 0
    double* cc = col(c);
    const double d = cc[c];
    // positive and finite, tested on the bit pattern (sign clear, not zero,
    // exponent below all-ones) on the integer pipe
    const long long bits = __double_as_longlong(d);
    if (!(bits > 0 && bits < 0x7FF0000000000000ll)) {
      if (lane == 0) flag[c & 1] = 1;
      return;
    }
    const double inv = __drcp_rn(d);
    if (lane == 0) {
      dv[c] = d;
      di[c] = inv;
    }
    double* u = uc + (c & 1) * m;
    for (int i = c + 1 + lane; i < m; i += 32) {
      const double a = cc[i];
      u[i] = a;
      cc[i] = a * inv;
    }
  };
  if (wid == 0) pivot(0);
  __syncthreads();
  for (int k = 0; k + 1 < m; ++k) {
    if (flag[k & 1]) return;
    const double* ck = col(k);
    const double* uk = uc + (k & 1) * m;
    if (wid == 0) {
      double* c1 = col(k + 1);
      const double u1 = uk[k + 1];
      for (int i = k + 1 + lane; i < m; i += 32) c1[i] -= ck[i] * u1;
      __syncwarp();
      pivot(k + 1);
    } else {
      // columns k+2..m-1 of the trailing triangle over the threads of warps
      // 1..NW-1: element q of the triangle listed column by column from the
      // last column (c + 1 rows for column j = m-1-c) sits in the column c
      // with c(c+1)/2 <= q < (c+1)(c+2)/2, found by a square root (exact
      // here: 8q + 1 < 2^14) with a one-step guard, so that consecutive
      // threads take consecutive rows of one column and no thread walks the
      // column boundaries
      constexpr int S = NT - 32;
      const int len = m - k - 2;
      const int T = len * (len + 1) / 2;
      for (int q = tid - 32; q < T; q += S) {
        int c = (int)((__fsqrt_rn(8.f * (float)q + 1.f) - 1.f) * 0.5f);
        c += (c + 1) * (c + 2) / 2 <= q;
        c -= c * (c + 1) / 2 > q;
        const int j = m - 1 - c;
        const int i = j + q - c * (c + 1) / 2;
        col(j)[i] -= ck[i] * uk[j];
      }
    }
    __syncthreads();
  }
}

// The same factorisation in panels of two columns with one barrier per
// panel, for matrices in global memory (large n), where every trailing
// element read and written costs a trip to L2 or DRAM: while warps 1.. apply
// the rank-2 update of panel (k, k+1) to columns k+4.. (a_ij -= l_ik u_jk +
// l_ik+1 u_jk+1), warp 0 applies it to the next panel's columns k+2, k+3 and
// factors them.  Each trailing element is read and written once per two
// columns.  uc holds four unscaled pivot columns.  (In shared memory the
// one-column form is faster: warp 0's pivot chain per barrier doubles here.)
// The flags alternate by panel: pivots c of panel c >> 1 write
// flag[(c >> 1) & 1], read after the barrier that ends their step.
template <int NT, typename Col>
__device__ __forceinline__ void ldlt_block_pairs(int m, Col col, double* __restrict__ uc, double* __restrict__ dv,
                                                 double* __restrict__ di, int* flag) {
  static_assert(NT >= 64, "one pivot warp plus at least one update warp");
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (m == 0) return;
  auto ubuf = [&](int c) { return uc + (c & 3) * m; };
  auto pivot = [&](int c) -> bool {  // warp 0; false when the pivot fails
    double* cc = col(c);
    const double d = cc[c];
    const long long bits = __double_as_longlong(d);
    if (!(bits > 0 && bits < 0x7FF0000000000000ll)) {
      if (lane == 0) flag[(c >> 1) & 1] = 1;
      return false;
    }
    const double inv = __drcp_rn(d);
    if (lane == 0) {
      dv[c] = d;
      di[c] = inv;
    }
    double* u = ubuf(c);
    for (int i = c + 1 + lane; i < m; i += 32) {
      const double a = cc[i];
      u[i] = a;
      cc[i] = a * inv;
    }
    return true;
  };
  // column c1 -= column c0 (rows c1..m-1), then its pivot; warp 0
  auto update_and_pivot = [&](int c0, int c1) -> bool {
    const double* l0 = col(c0);
    const double u = ubuf(c0)[c1];
    double* cc = col(c1);
    for (int i = c1 + lane; i < m; i += 32) cc[i] -= l0[i] * u;
    __syncwarp();
    return pivot(c1);
  };
  if (wid == 0 && pivot(0) && m > 1) update_and_pivot(0, 1);
  __syncthreads();
  for (int k = 0; k + 2 < m; k += 2) {
    if (flag[(k >> 1) & 1]) return;
    const double* l0 = col(k);
    const double* l1 = col(k + 1);
    const double* u0 = ubuf(k);
    const double* u1 = ubuf(k + 1);
    if (wid == 0) {
      for (int c = k + 2; c < k + 4 && c < m; ++c) {
        const double a0 = u0[c], a1 = u1[c];
        double* cc = col(c);
        for (int i = c + lane; i < m; i += 32) cc[i] -= l0[i] * a0 + l1[i] * a1;
      }
      __syncwarp();
      if (pivot(k + 2) && k + 3 < m) update_and_pivot(k + 2, k + 3);
    } else {
      // columns k+4..m-1 of the trailing triangle, placed as in ldlt_block;
      // four elements per thread and round, all loads issued before the
      // stores, so that a thread keeps several memory trips in flight
      constexpr int S = NT - 32, U = 4;
      const int len = m - k - 4;
      const int T = len > 0 ? len * (len + 1) / 2 : 0;
      for (int q0 = tid - 32; q0 < T; q0 += U * S) {
        double* dst[U];
        double val[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int q = q0 + u * S;
          dst[u] = nullptr;
          if (q < T) {
            int c = (int)((__fsqrt_rn(8.f * (float)q + 1.f) - 1.f) * 0.5f);
            c += (c + 1) * (c + 2) / 2 <= q;
            c -= c * (c + 1) / 2 > q;
            const int j = m - 1 - c;
            const int i = j + q - c * (c + 1) / 2;
            dst[u] = col(j) + i;
            val[u] = *dst[u] - (l0[i] * u0[j] + l1[i] * u1[j]);
          }
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (dst[u]) *dst[u] = val[u];
      }
    }
    __syncthreads();
  }
}

struct Bump {
  size_t o = 0;
  __host__ __device__ size_t take(size_t bytes) {
    const size_t r = o;
    o += (bytes + 15) & ~size_t(15);
    return r;
  }
};

// ---------------------------------------------------------------- layouts
// `in_smem` false: the n x n matrices live in global memory instead.

struct Lay1 {
  size_t pw, g, red, ix, gs, mv, H, total;
  size_t pw_step, ix_step, gs_step, mv_step, H_step;  // offset between the two points' arrays
};
// Term sweep of up to `pts` (1 or kTermPoints) points of one polynomial per
// CTA: power tables, gather sums and monomial values (gather form) and H
// slots (in shared memory) per point; the per-warp gradient replicas of the
// term-by-term form are shared (points are swept one after another there).
// `gather`: room for the gather form (1/x, gradient sums, one chunk of
// monomial values)
constexpr int kTermPoints = 2;
static_assert(kTermPoints == 2, "the sweep loads the points' monomial values as pairs");
template <typename R, int NW>
__host__ __device__ Lay1 lay_terms(int n, int E1, bool in_smem, bool gather, int pts = kTermPoints) {
  using Acc = AccOf<R>;
  using Abs = AbsOf<R>;
  Lay1 L{};
  Bump b;
  L.pw_step = ((size_t)n * E1 * sizeof(R) + 15) & ~size_t(15);
  L.pw = b.take(pts * L.pw_step);
  L.red = b.take(kTermPoints * 40 * 8);
  if (!gather) L.g = b.take((size_t)NW * n * sizeof(Acc));  // one replica per warp
  if (gather) {
    L.ix_step = ((size_t)n * sizeof(R) + 15) & ~size_t(15);
    L.gs_step = ((size_t)n * sizeof(Acc) + 15) & ~size_t(15);
    L.ix = b.take(pts * L.ix_step);
    L.gs = b.take(pts * L.gs_step);
    // monomial values of the points of a pass interleaved (value of point q
    // for chunk term t at [t * pts + q]): one vector load per record
    L.mv_step = sizeof(R);
    L.mv = b.take((size_t)pts * kGatherChunk * sizeof(R));
  }
  L.H_step = (size_t)mat_slot<Acc>(n) * sizeof(Acc);
  L.H = in_smem ? b.take(pts * L.H_step) : 0;
  L.total = b.o;
  return L;
}

struct Lay2 {
  size_t e, v, h, dv, di, uc, vr, u, w, Hr, Ld, X, total;
};
// row stride of X = L^{-1}: odd, so that lanes reading rows j, j+1, ... at a
// common column hit different banks
__host__ __device__ inline int x_stride(int m) { return m | 1; }
// 8-byte forms with m <= 64 keep X' = D^{-1/2} L^{-1} in the lower triangle
// (diagonal included) of the factor's own matrix: the factor occupies the
// strict upper triangle (col(j)[i] = Hr[j*n + i], i > j) and the pivots live
// apart, so X'_ij (i >= j) at Hr[i*n + j] overwrites nothing still needed
template <typename R>
__host__ __device__ inline bool x_in_place(int m) { return sizeof(R) == 8 && m <= 64; }
template <typename R>
__host__ __device__ Lay2 lay_frame(int n, bool in_smem) {
  Lay2 L{};
  Bump b;
  const size_t m = n > 1 ? n - 1 : 1;
  L.e = b.take(n * 8);
  L.v = b.take(n * 8);
  L.h = b.take(n * 8);
  L.dv = b.take(m * 8);      // LDL^T pivots d_k
  L.di = b.take(m * 8);      // 1 / d_k
  L.vr = b.take(n * sizeof(R));
  L.u = b.take(n * sizeof(R));
  L.w = b.take(n * sizeof(R));
  // unscaled pivot columns (two buffers; four for the pairs form).  With
  // 8-byte values the two buffers of the shared-memory form live in u and w
  // (2 x 8n bytes >= 2 x 8m), which the factorisation leaves unused: one
  // more CTA per SM at n = 60 (seven instead of six)
  L.uc = (in_smem && sizeof(R) == 8) ? L.u : b.take((in_smem ? 2 : 4) * m * 8);
  if (in_smem) {
    L.Hr = b.take((size_t)mat_slot<R>(n) * sizeof(R));
    // FP32 form: FP64 factor in a packed column-major lower triangle, whose
    // m(m+1)/2 doubles then hold X (m rows of stride m|1 floats); the FP64
    // form factors in place in Hr and keeps X apart
    if (sizeof(R) == 4) {
      L.Ld = L.X = b.take(m * (m + 1) / 2 * 8);
    } else if (!x_in_place<R>((int)m)) {
      L.X = b.take(m * x_stride((int)m) * sizeof(R));
    }
  }
  L.total = b.o;
  return L;
}
// global-memory bytes per CTA when the frame matrices do not fit in shared memory
template <typename R>
size_t frame_gmem(int n) {
  const size_t m = n > 1 ? n - 1 : 1;
  return (size_t)mat_slot<R>(n) * sizeof(R) + (sizeof(R) == 4 ? m * (m + 1) / 2 * 8 : m * x_stride((int)m) * sizeof(R)) + 256;
}

struct Lay3 {
  size_t pw, c, v, e, y, yr, ix, W, total;
};
template <typename R, int NW>
__host__ __device__ Lay3 lay_third(int n, int E1, bool in_smem) {
  Lay3 L{};
  Bump b;
  L.pw = b.take((size_t)n * E1 * sizeof(R));
  L.c = b.take((size_t)NW * n * sizeof(AccOf<R>));  // one replica per warp
  L.v = b.take(n * 8);
  L.e = b.take(n * 8);
  L.y = b.take(n * 8);
  L.yr = b.take(n * sizeof(R));
  L.ix = b.take(n * sizeof(R));
  L.W = in_smem ? b.take((size_t)mat_slot<R>(n) * sizeof(R)) : 0;
  L.total = b.o;
  return L;
}

template <typename R>
struct StageArgs {
  const ExactDesc* descs;
  int n_desc;
  const int64_t* prefix;
  const int* order;
  int64_t item_begin, item_end;  // this launch's range of the work order
  int* counter;
  AccOf<R>* mats_h;  // per point n x n: H (stage 1 -> 2)
  R* mats_w;         // per point n x n: W (stage 2 -> 3)
  double* vecs;
  double r;
  int assume_nonzero_x;
  unsigned char* gws;
  size_t gws_stride;
  int* err;  // set when a bounded wait expires
  int kmin, kmax;  // third stage: the support sizes this launch contracts (all launches of a step cover 1..8)
};

// The gradient/Hessian sweep's list of passes left to its term-by-term
// kernel: (first item, points) pairs, their count and the list's capacity.
// (A parameter of its own: the stage arguments of the frame and third
// kernels keep their size, and with it those kernels' register allocation.)
struct PassList {
  int64_t* pass;
  int* count;
  int cap;
  int pts;  // points per pass of the gather launch (1 or kTermPoints)
};

__device__ __forceinline__ void write_failed(const ExactDesc& pd, int64_t p, int n, double gn, int flag) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    pd.D[p * n + i] = nan("");
    if (pd.Dunit) pd.Dunit[p * n + i] = nan("");
  }
  if (threadIdx.x == 0 && pd.info) {
    polylab_an_info in{gn, nan(""), flag, n, n - 1, 0};
    pd.info[p] = in;
  }
}

}  // namespace

// ------------------------------------------------------------------ stage 1
// Gradient and Hessian by one of two sweeps over the term list:
//  gather  (the plan has a gather form and every |x_v| is in the range where
//          monomial values and 1/x stay normal): per chunk of terms, the
//          monomial values m_t into shared memory, then each thread sums a
//          contiguous run of the entry-sorted records coef * m_t in registers
//          and adds a run's sum to its entry when the entry changes; entries
//          are scaled by 1/x_i (1/x_j) at the end;
//  scatter (otherwise): every term's derivative values are added to their
//          entries one by one (per-warp gradient replicas).
// A CTA takes two consecutive work items at a time; when both are points of
// the same polynomial and the gather form holds at both, one pass over the
// terms and records serves the two points (each record is decoded once and
// applied to both points' monomial values).  Otherwise the points are swept
// one after another (a pair that straddles two polynomials in two passes).
// The sweep is two kernels.  GATHER: the gather passes of an item range; a
// pass the gather form cannot take (a coordinate outside its range, or a plan
// without records) is appended to the list fl and left to the second
// kernel, which takes the listed passes term by term.  Split this way the
// gather kernel carries none of the term-by-term code and keeps a much smaller
// register allocation (64 against 134 in double words), so twice as many CTAs
// stay resident.
template <typename R>
constexpr int terms_min_blocks(bool gather, int nt) {
  return (!gather ? 512 : sizeof(R) == 8 && !std::is_same<R, dfloat>::value ? 768 : 1024) / nt;
}
// The small integer c of a gather record in the form's multiplier type.
template <typename R>
__device__ __forceinline__ SmallOf<R> small_coef(uint32_t c, const double*) {
  return SmallOf<R>(c);
}
template <>
__device__ __forceinline__ double small_coef<double>(uint32_t c, const double* table) {
  return table[c];
}

template <typename R, int NT, bool GATHER>
__global__ void __launch_bounds__(NT, terms_min_blocks<R>(GATHER, NT)) exact_terms_kernel(StageArgs<R> a, PassList fl) {
  using Acc = AccOf<R>;
  using Abs = AbsOf<R>;
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ int64_t s_item;
  __shared__ double s_cf[std::is_same<R, double>::value ? 128 : 1];  // c -> (double)c, c < 128
  if constexpr (std::is_same<R, double>::value)
    for (int i = threadIdx.x; i < 128; i += NT) s_cf[i] = (double)i;
  constexpr int NW = NT / 32;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  while (true) {
    int64_t pair, pair_end;
    if constexpr (!GATHER) {
      const int64_t idx = next_item(a.counter, &s_item);
      if (idx >= (int64_t)min(*fl.count, fl.cap)) break;  // (written by the gather launches before this one)
      pair = fl.pass[2 * idx];
      pair_end = pair + fl.pass[2 * idx + 1];
    } else {
      pair = a.item_begin + (int64_t)fl.pts * next_item(a.counter, &s_item);
      if (pair >= a.item_end) break;
      pair_end = min(pair + fl.pts, a.item_end);
    }
    int np = 0;
    for (int64_t item = pair; item < pair_end; item += np) {
      const int lo = find_poly(a.prefix, a.n_desc, item);
      const ExactDesc& pd = a.descs[a.order[lo]];
      const int64_t p0 = item - a.prefix[lo];
      // the points of this pass: the rest of the pair within this polynomial
      np = (int)min(pair_end - item, pd.P - p0);
      const int n = pd.n, nn = n * n, E1 = pd.E + 1;
      const int pts = GATHER ? fl.pts : kTermPoints;
      const Lay1 L = lay_terms<R, NW>(n, E1, pd.h_in_smem, GATHER, pts);
      auto pw_of = [&](int q) { return (R*)(sm + L.pw + q * L.pw_step); };
      auto ix_of = [&](int q) { return (R*)(sm + L.ix + q * L.ix_step); };
      auto gs_of = [&](int q) { return (Acc*)(sm + L.gs + q * L.gs_step); };
      R* mvi = (R*)(sm + L.mv);  // interleaved: [t * pts + q]
      auto Hg_of = [&](int q) { return a.mats_h + pd.mat_off + (p0 + q) * mat_slot<Acc>(n); };
      auto Hr_of = [&](int q) { return pd.h_in_smem ? (Acc*)(sm + L.H + q * L.H_step) : Hg_of(q); };
      auto rec_of = [&](int q) { return a.vecs + pd.vec_off + (p0 + q) * vrec(n); };
      Acc* g = (Acc*)(sm + L.g);
      double* red = (double*)(sm + L.red);
      bool in_range = true;
      for (int i = tid; i < np * n; i += NT) {
        const double ax = fabs(pd.X[p0 * n + i]);
        in_range &= ax >= pd.x_lo && ax <= pd.x_hi;
      }
      const bool gather = GATHER && __syncthreads_and(in_range && pd.gather != nullptr) != 0;
      if constexpr (GATHER) {
        if (!gather) {  // (uniform) the term-by-term launch takes this pass
          if (tid == 0) {
            const int idx = atomicAdd(fl.count, 1);
            if (idx < fl.cap) {
              fl.pass[2 * idx] = item;
              fl.pass[2 * idx + 1] = np;
            } else {
              atomicExch(a.err, 4);  // (the list holds one pass per pair plus one per polynomial)
            }
          }
          continue;
        }
      }
      for (int q = 0; q < np; ++q) {
        const double* X = pd.X + (p0 + q) * n;
        if (gather) {
          for (int i = tid; i < n; i += NT) {
            ix_of(q)[i] = R(1) / R(X[i]);
            gs_of(q)[i] = Acc(0);
          }
        }
        power_table<R, NT>(X, n, E1, pw_of(q));
        Acc* Hr = Hr_of(q);
        for (int64_t i = tid; i < mat_slot<Acc>(n); i += NT) Hr[i] = Acc(0);
      }
      __syncthreads();
      Abs gabs[kTermPoints] = {};  // this thread's share of sum |gradient contributions|, per point
      if (gather) {
        // one pass over terms and records for NP points
        auto sweep = [&](auto np_c) {
          constexpr int NP = decltype(np_c)::value;
          Acc* Hr[NP];
          Acc* gs[NP];
  #pragma unroll
          for (int q = 0; q < NP; ++q) {
            Hr[q] = Hr_of(q);
            gs[q] = gs_of(q);
          }
          auto flush = [&](int e, const RunSum<R>* acc) {
            if (e < 0 || e == (int)kGatherPad) return;  // nothing yet, or padding
  #pragma unroll
            for (int q = 0; q < NP; ++q) {
              if (e >= nn) {
                acc_add(&gs[q][e - nn], acc[q].value());
              } else {
                acc_add(&Hr[q][e], acc[q].value());
              }
            }
          };
          for (int c = 0; c < pd.n_gchunks; ++c) {
            const int64_t t0 = (int64_t)c * kGatherChunk, t1 = min(pd.m, t0 + kGatherChunk);
            for (int64_t t = t0 + tid; t < t1; t += NT) {
              const TermRegs tr = load_term(pd.terms, t);
              // the zero-gradient scale once per term, not per gradient record
  #pragma unroll
              for (int q = 0; q < NP; ++q) {
                const R mv = term_value<R>(tr, pw_of(q), E1);
                mvi[(t - t0) * pts + q] = mv;
                gabs[q] += abs_of(mv) * grad_abs_factor<R>(tr, ix_of(q));
              }
            }
            __syncthreads();
            const int64_t r0 = pd.gather_chunk[c];
            const int Lc = (int)((pd.gather_chunk[c + 1] - r0) / kGatherStreams);
            const uint32_t* recs = pd.gather + r0;
            for (int st = tid; st < kGatherStreams; st += NT) {
              int cur = -1;
              RunSum<R> acc[NP];
              for (int k = 0; k < Lc; k += kGatherUnroll) {
                uint32_t rr[kGatherUnroll];
  #pragma unroll
                for (int u = 0; u < kGatherUnroll; ++u) rr[u] = __ldg(recs + (int64_t)(k + u) * kGatherStreams + st);
  #pragma unroll
                for (int u = 0; u < kGatherUnroll; ++u) {
                  const int e = (int)((rr[u] >> 11) & 0x3fffu);
                  // falling-factorial coefficient <= 127 (FP64: from a table, keeping the
                  // integer conversion off the FP64 pipe)
                  const SmallOf<R> cf = small_coef<R>(rr[u] >> 25, s_cf);
                  const int tt = (int)(rr[u] & 0x7ffu);
                  if (e != cur) {
                    flush(cur, acc);
                    cur = e;
  #pragma unroll
                    for (int q = 0; q < NP; ++q) acc[q] = RunSum<R>();
                  }
                  R mvp[kTermPoints];
                  if constexpr (NP == 2) load_pair(mvi + tt * kTermPoints, mvp);  // (pts = 2)
                  else mvp[0] = mvi[tt * pts];
  #pragma unroll
                  for (int q = 0; q < NP; ++q) acc[q].add(mvp[q], cf);
                }
              }
              flush(cur, acc);
            }
            __syncthreads();
          }
        };
        if (np == 2) sweep(std::integral_constant<int, 2>{});
        else sweep(std::integral_constant<int, 1>{});
        for (int q = 0; q < np; ++q) {
          Acc* Hr = Hr_of(q);
          const R* ix = ix_of(q);
          for (int i = wid; i < n; i += NW)
            for (int j = i + lane; j < n; j += 32) Hr[i * n + j] = Acc(R(Hr[i * n + j]) * ix[i] * ix[j]);
          double* rec = rec_of(q);
          for (int i = tid; i < n; i += NT) rec[i] = (double)(R(gs_of(q)[i]) * ix[i]);
        }
      } else if constexpr (!GATHER) {
        for (int q = 0; q < np; ++q) {
          for (int i = tid; i < NW * n; i += NT) g[i] = Acc(0);
          __syncthreads();
          Acc* gw = g + wid * n;
          Acc* Hr = Hr_of(q);
          const R* pw = pw_of(q);
          Abs ga = Abs(0);
          auto emit = [&](int kind, int i, int j, R val) {
            if (kind == 1) {
              acc_add(&gw[i], Acc(val));
              ga += Abs(fabs(val));
            } else if (kind == 2) {
              acc_add(&Hr[i * n + j], Acc(val));
            }
          };
          // one loop per support-size group: inside each loop the support size
          // is a compile-time constant and the warp never branches on it
          for_support<kMaxSupport>([&](auto kc) {
            constexpr int K = decltype(kc)::value;
            for (int64_t t = pd.koff[K] + tid; t < pd.koff[K + 1]; t += NT) {
              const TermRegs tr = load_term(pd.terms, t);
              term_derivs_group<R, 2, K>(tr, pw, E1, emit);
            }
          });
          __syncthreads();
          double* rec = rec_of(q);
          for (int i = tid; i < n; i += NT) {
            Acc sum = g[i];
            for (int w = 1; w < NW; ++w) sum += g[w * n + i];
            rec[i] = (double)sum;
          }
          gabs[q] = ga;
          __syncthreads();
        }
      }
      for (int q = 0; q < np; ++q) {
        const Abs gq = warp_sum(gabs[q]);
        if (lane == 0) red[q * 40 + wid] = (double)gq;
      }
      __syncthreads();
      if (tid < np) {
        double gsum = 0.0;
        for (int w = 0; w < NW; ++w) gsum += red[tid * 40 + w];
        rec_of(tid)[4 * n] = gsum;
      }
      // the upper triangles the sweep filled (zeros below) to the workspace by
      // one bulk copy each; their shared-memory sources are read before the
      // next pair
      if (pd.h_in_smem && tid == 0) {
        fence_proxy_async_smem();
        for (int q = 0; q < np; ++q) bulk_s2g(Hg_of(q), Hr_of(q), (uint32_t)(mat_slot<Acc>(n) * sizeof(Acc)));
        bulk_commit();
        bulk_wait_read();
      }
      __syncthreads();  // (the next pass reuses the shared arrays)
    }
  }
  if (tid == 0) bulk_wait_all();
}

// ------------------------------------------------------------------ stage 2
// One (polynomial, point) item of the frame stage.  SMEM: the n x n
// matrices live in shared memory (else in this CTA's global workspace); as a
// template parameter it lets every matrix access compile to a shared-memory
// instruction.  Returns false, for every thread of the CTA, when a bounded
// wait expired (the kernel stops).
template <typename R, int NT, bool SMEM>
__device__ __forceinline__ bool frame_item(const StageArgs<R>& a, const ExactDesc& pd, int64_t p, unsigned char* sm,
                                           int* s_flag, double* s_sc, uint64_t& s_bar, uint32_t& phase) {
  // kF64: the factor is formed in place in the 8-byte matrix (FP64 and
  // double-word forms); kDW: double-word form, whose H and frame update are
  // FP64 (H arrives as FP64 sums) and whose inverse and W are double words
  constexpr bool kF64 = sizeof(R) == 8;
  constexpr bool kDW = std::is_same<R, dfloat>::value;
  using Rh = std::conditional_t<kDW, double, R>;
  constexpr int NW = NT / 32;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int n = pd.n, m = n - 1, nn = n * n, xs = x_stride(m);
  const Lay2 L = lay_frame<R>(n, SMEM);
  double* e = (double*)(sm + L.e);
  double* v = (double*)(sm + L.v);
  double* h = (double*)(sm + L.h);
  double* dv = (double*)(sm + L.dv);
  double* di = (double*)(sm + L.di);
  double* uc = (double*)(sm + L.uc);
  Rh* vr = (Rh*)(sm + L.vr);
  Rh* u = (Rh*)(sm + L.u);
  Rh* w = (Rh*)(sm + L.w);
  unsigned char* gb = a.gws + (size_t)blockIdx.x * a.gws_stride;
  Rh* Hr = SMEM ? (Rh*)(sm + L.Hr) : (Rh*)gb;
  // the same storage in the form's precision R (after the factorisation)
  R* HrR = reinterpret_cast<R*>(Hr);
  R* vrR = reinterpret_cast<R*>(vr);
  R* uR = reinterpret_cast<R*>(u);
  R* wR = reinterpret_cast<R*>(w);
  unsigned char* rest = SMEM ? nullptr : gb + (size_t)mat_slot<R>(n) * sizeof(R);
  // FP64 factor storage, element (i, j) of the leading block at col(j)[i]:
  // in place in Hr (col(j) = row j of the symmetric Hr) for the FP64 form, a
  // packed column-major lower triangle for the FP32 form; X = L^{-1} with
  // row stride xs (the FP32 form reuses the factor's storage)
  double* Ld = kF64 ? (double*)Hr : (SMEM ? (double*)(sm + L.Ld) : (double*)rest);
  R* Xs = kF64 ? (SMEM ? (R*)(sm + L.X) : (R*)rest) : (R*)Ld;
  const bool xin = SMEM && x_in_place<R>(m);  // X' in the lower triangle of HrR
  // storage of X'_ij, i >= j
  auto xref = [&](int i, int j) -> R& { return xin ? HrR[i * n + j] : Xs[j * xs + i]; };
  auto col = [Ld, n, m](int j) -> double* {
    return kF64 ? Ld + (size_t)j * n : Ld + ((size_t)j * m - (size_t)j * (j - 1) / 2 - j);
  };
  // H in the form's sum type (double words in the double-word form, converted
  // to FP64 element by element in place once it is in this CTA's buffer)
  const AccOf<R>* Hg = a.mats_h + pd.mat_off + p * mat_slot<R>(n);
  R* Wg = a.mats_w + pd.mat_off + p * mat_slot<R>(n);
  const uint32_t mat_bytes = (uint32_t)(mat_slot<R>(n) * sizeof(R));
  double* rec = a.vecs + pd.vec_off + p * vrec(n);
  // H (upper triangle) into shared memory by one bulk copy
  if (SMEM) {
    if (tid == 0) {
      fence_proxy_async_smem();
      mbar_arrive_expect_tx(&s_bar, mat_bytes);
      bulk_g2s(Hr, Hg, mat_bytes, &s_bar);
    }
  } else {
    for (int i = wid; i < n; i += NW)
      for (int j = lane; j < n; j += 32) Hr[i * n + j] = Rh(Hg[i * n + j]);
  }
  // |g|, the zero-gradient test and the Householder vector (warp 0)
  if (wid == 0) {
    double gg = 0.0;
    for (int i = lane; i < n; i += 32) gg += rec[i] * rec[i];
    const double gn = sqrt(warp_sum(gg));
    bool zero = !(gn > 0.0) || !isfinite(gn);
    // relative test at the resolution of the form: 1e-14 (FP64), 1e-6 (FP32 sums)
    if (!a.assume_nonzero_x && gn <= (kF64 ? 1e-14 : 1e-6) * rec[4 * n]) zero = true;
    double beta = 0.0, sgn = 1.0;
    if (!zero) {
      const double ign = 1.0 / gn;
      const double en = rec[n - 1] * ign;
      sgn = en >= 0.0 ? 1.0 : -1.0;
      beta = 1.0 / (1.0 + sgn * en);  // 2 / v^T v with v^T v = 2 (1 + s e_n)
      for (int i = lane; i < n; i += 32) {
        const double ei = rec[i] * ign;
        e[i] = ei;
        v[i] = ei + (i == n - 1 ? sgn : 0.0);
        vr[i] = Rh(v[i]);
      }
    }
    if (lane == 0) {
      s_sc[0] = gn;
      s_sc[1] = zero ? 1.0 : 0.0;
      s_sc[2] = beta;
      s_sc[3] = sgn;
      s_flag[0] = s_flag[1] = 0;
    }
  }
  if (SMEM) {
    if (!mbar_wait_cta(&s_bar, phase, a.err, 2)) {
      mbar_drain(&s_bar, phase, a.err, 2);
      return false;
    }
    phase ^= 1u;
  } else {
    __syncthreads();
  }
  if constexpr (kDW) {
    if (SMEM) {  // double words -> FP64, element by element in place
      const dfloat* Hd = reinterpret_cast<const dfloat*>(Hr);
      for (int i = wid; i < n; i += NW)
        for (int j = i + lane; j < n; j += 32) Hr[i * n + j] = (double)Hd[i * n + j];
      __syncthreads();
    }
  }
  for (int i = wid; i < n; i += NW)  // mirror the upper triangle
    for (int j = lane; j < i; j += 32) Hr[i * n + j] = Hr[j * n + i];
  __syncthreads();
  const double gn = s_sc[0], beta = s_sc[2], sgn = s_sc[3];
  if (s_sc[1] != 0.0) {
    write_failed(pd, p, n, gn, POLYLAB_FLAG_ZERO_GRAD);
    if (tid == 0) {
      rec[4 * n + 1] = gn;
      rec[4 * n + 4] = kStZero;
    }
    return true;
  }
  for (int i = tid; i < n; i += NT) {  // u = H v (H symmetric: column access, conflict-free)
    Rh acc = Rh(0);
    for (int j = 0; j < n; ++j) acc += Hr[j * n + i] * vr[j];
    u[i] = acc;
  }
  __syncthreads();
  if (wid == 0) {  // w = beta u - (beta^2 / 2) (v.u) v
    double part = 0.0;
    for (int i = lane; i < n; i += 32) part += v[i] * (double)u[i];
    const double gamma = warp_sum(part);
    for (int i = lane; i < n; i += 32) w[i] = Rh(beta * (double)u[i] - 0.5 * beta * beta * gamma * v[i]);
  }
  __syncthreads();
  for (int i = wid; i < n; i += NW)  // P H P = H - v w^T - w v^T
    for (int j = lane; j < n; j += 32) Hr[i * n + j] -= vr[i] * w[j] + w[i] * vr[j];
  __syncthreads();
  for (int i = tid; i < n; i += NT) h[i] = i < m ? -sgn * (double)Hr[i * n + (n - 1)] : 0.0;
  if constexpr (kF64) {
    for (int i = tid; i < m; i += NT) Hr[i * n + i] += a.r;
  } else {
    for (int j = wid; j < m; j += NW)
      for (int i = j + lane; i < m; i += 32) col(j)[i] = (double)Hr[j * n + i];
    __syncthreads();
    for (int i = tid; i < m; i += NT) col(i)[i] += a.r;
  }
  __syncthreads();
  if constexpr (SMEM) ldlt_block<NT>(m, col, uc, dv, di, s_flag);
  else ldlt_block_pairs<NT>(m, col, uc, dv, di, s_flag);
  __syncthreads();
  if (s_flag[0] | s_flag[1]) {
    write_failed(pd, p, n, gn, POLYLAB_FLAG_NOT_PD);
    if (tid == 0) {
      rec[4 * n + 1] = gn;
      rec[4 * n + 4] = kStNotPd;
    }
    return true;
  }
  // log-det (warp 0) while the others take the factor into the form's
  // precision: Lt(i, j) = Hr[j*n + i] = l_ij (i > j); sq = d^{-1/2}
  R* sq = wR;
  if (wid == 0) {
    double lsum = 0.0;
    for (int k = lane; k < m; k += 32) lsum += log(dv[k]);
    lsum = warp_sum(lsum);
    if (lane == 0) s_sc[1] = lsum;
  }
  for (int i = tid; i < m; i += NT) sq[i] = kF64 ? R(sqrt(di[i])) : R(sqrtf((float)di[i]));
  if constexpr (!kF64) {  // (the factor's storage becomes X after the next barrier)
    for (int j = wid; j < m; j += NW)
      for (int i = j + 1 + lane; i < m; i += 32) Hr[j * n + i] = (R)col(j)[i];
  }
  if constexpr (kDW) {  // FP64 factor -> double words, element by element in place
    for (int j = wid; j < m; j += NW)
      for (int i = j + 1 + lane; i < m; i += 32) HrR[j * n + i] = R(col(j)[i]);
    for (int i = tid; i < n; i += NT) vrR[i] = R(v[i]);  // (vr's FP64 copy is no longer needed)
  }
  __syncthreads();  // L in the form's precision and sq complete
  // X' = D^{-1/2} X with X = L^{-1} (unit lower), stored transposed:
  // Xs[j*xs + i] = X'_ij, i >= j; then M = X'^T X'
  if (kDW && m <= 64) {
    // the same column scheme as below, each row's sum delta_rj - sum_k l_rk x_k
    // kept as a compensated dot product (dw_dot) and rounded to a double
    // word only when its x_k is broadcast or stored
    for (int ja = wid; ja < m; ja += 2 * NW) {
      const int jb = ja + NW;
      const int r0 = lane, r1 = lane + 32;
      dw_dot a0, a1, b0, b1;
      a0.s = r0 == ja ? 1.f : 0.f;
      a1.s = r1 == ja ? 1.f : 0.f;
      b0.s = r0 == jb ? 1.f : 0.f;
      b1.s = r1 == jb ? 1.f : 0.f;
      for (int k = ja; k + 1 < m; ++k) {
        const dfloat l0 = (r0 > k && r0 < m) ? -dfloat(HrR[k * n + r0]) : dfloat(0.f, 0.f);
        const dfloat l1 = (r1 > k && r1 < m) ? -dfloat(HrR[k * n + r1]) : dfloat(0.f, 0.f);
        const dfloat xa = shfl((k < 32 ? a0 : a1).value(), k & 31);
        a0.add(l0, xa);
        a1.add(l1, xa);
        if (k >= jb) {  // column jb is zero above row jb
          const dfloat xb = shfl((k < 32 ? b0 : b1).value(), k & 31);
          b0.add(l0, xb);
          b1.add(l1, xb);
        }
      }
      if (r0 >= ja && r0 < m) xref(r0, ja) = R(a0.value() * dfloat(sq[r0]));
      if (r1 >= ja && r1 < m) xref(r1, ja) = R(a1.value() * dfloat(sq[r1]));
      if (jb < m) {
        if (r0 >= jb && r0 < m) xref(r0, jb) = R(b0.value() * dfloat(sq[r0]));
        if (r1 >= jb && r1 < m) xref(r1, jb) = R(b1.value() * dfloat(sq[r1]));
      }
    }
  } else if (m <= 64) {
    // column j of X is the forward substitution of e_j alone, so columns
    // are independent: warp w takes columns j = w, w + NW, ... two at a
    // time, lane q holding rows q and q + 32 in registers; x_k reaches the
    // other lanes by a shuffle once final (no block barrier)
    for (int ja = wid; ja < m; ja += 2 * NW) {
      const int jb = ja + NW;  // second column (none if jb >= m)
      const int r0 = lane, r1 = lane + 32;
      R a0 = r0 == ja ? R(1) : R(0), a1 = r1 == ja ? R(1) : R(0);
      R b0 = r0 == jb ? R(1) : R(0), b1 = r1 == jb ? R(1) : R(0);
      for (int k = ja; k + 1 < m; ++k) {
        const R l0 = (r0 > k && r0 < m) ? HrR[k * n + r0] : R(0);
        const R l1 = (r1 > k && r1 < m) ? HrR[k * n + r1] : R(0);
        const R xa = shfl_r(k < 32 ? a0 : a1, k & 31);
        a0 -= l0 * xa;
        a1 -= l1 * xa;
        if (k >= jb) {  // column jb is zero above row jb
          const R xb = shfl_r(k < 32 ? b0 : b1, k & 31);
          b0 -= l0 * xb;
          b1 -= l1 * xb;
        }
      }
      if (r0 >= ja && r0 < m) xref(r0, ja) = a0 * sq[r0];
      if (r1 >= ja && r1 < m) xref(r1, ja) = a1 * sq[r1];
      if (jb < m) {
        if (r0 >= jb && r0 < m) xref(r0, jb) = b0 * sq[r0];
        if (r1 >= jb && r1 < m) xref(r1, jb) = b1 * sq[r1];
      }
    }
  } else {
    for (int j = wid; j < m; j += NW)
      for (int i = j + lane; i < m; i += 32) Xs[j * xs + i] = i == j ? R(1) : R(0);
    __syncthreads();
    // right-looking: after step k row k of X is final; X_ij -= l_ik X_kj for
    // j <= k < i, the (m-k-1) x (k+1) rectangle enumerated over the CTA
    for (int k = 0; k + 1 < m; ++k) {
      const int rows = m - k - 1;
      // thread tid starts at q = tid = j * rows + i0 and steps by NT
      const int dj = NT / rows, di0 = NT - dj * rows;
      int j = tid / rows, i0 = tid - j * rows;
      const R* lk = HrR + k * n + k + 1;
      while (j <= k) {
        Xs[j * xs + k + 1 + i0] -= lk[i0] * Xs[j * xs + k];
        j += dj;
        i0 += di0;
        if (i0 >= rows) {
          i0 -= rows;
          ++j;
        }
      }
      __syncthreads();
    }
    for (int j = wid; j < m; j += NW)
      for (int i = j + lane; i < m; i += 32) Xs[j * xs + i] *= sq[i];
  }
  __syncthreads();
  // M = H_T^{-1} = X'^T X', upper triangle into Hr (L no longer needed):
  // M_ij = sum_{k >= j} X'_ki X'_kj (i <= j)
  if (xin) {
    // X' in the lower triangle: a lane's column j is read with consecutive
    // lanes on consecutive addresses; the diagonal X'_kk = sq_k is taken from
    // sq, so the writes to the upper triangle and diagonal touch nothing read
    for (int i = wid; i < m; i += NW)
      for (int j = i + lane; j < m; j += 32) {
        DotAcc<R> acc;
        acc.add(i == j ? sq[j] : HrR[j * n + i], sq[j]);
        for (int k = j + 1; k < m; ++k) acc.add(HrR[k * n + i], HrR[k * n + j]);
        HrR[i * n + j] = acc.value();
      }
  } else {
    for (int i = wid; i < m; i += NW)
      for (int j = i + lane; j < m; j += 32) {
        DotAcc<R> acc;
        for (int k = j; k < m; ++k) acc.add(Xs[i * xs + k], Xs[j * xs + k]);
        HrR[i * n + j] = acc.value();
      }
  }
  __syncthreads();
  for (int i = wid; i < n; i += NW)  // Hr <- [M 0; 0 0], full symmetric, in place
    for (int j = lane; j < n; j += 32) {
      if (i == n - 1 || j == n - 1) HrR[i * n + j] = R(0);
      else if (i > j) HrR[i * n + j] = HrR[j * n + i];
    }
  __syncthreads();
  for (int i = tid; i < n; i += NT) {  // u = [M 0; 0 0] v
    DotAcc<R> acc;
    for (int j = 0; j < n; ++j) acc.add(HrR[j * n + i], vrR[j]);
    uR[i] = acc.value();
  }
  __syncthreads();
  if (wid == 0) {
    double part = 0.0;
    for (int i = lane; i < n; i += 32) part += v[i] * (double)uR[i];
    const double gam2 = warp_sum(part);
    for (int i = lane; i < n; i += 32) {
      wR[i] = R(beta * (double)uR[i] - 0.5 * beta * beta * gam2 * v[i]);
      rec[n + i] = v[i];
      rec[2 * n + i] = e[i];
      rec[3 * n + i] = h[i];
    }
    if (lane == 0) {
      rec[4 * n + 1] = gn;
      rec[4 * n + 2] = beta;
      rec[4 * n + 3] = s_sc[1];
      rec[4 * n + 4] = kStOk;
    }
  }
  __syncthreads();
  if (SMEM) {  // W = P [M 0; 0 0] P in place, then one bulk copy out
    for (int i = wid; i < n; i += NW)
      for (int j = lane; j < n; j += 32) HrR[i * n + j] -= vrR[i] * wR[j] + wR[i] * vrR[j];
    __syncthreads();
    if (tid == 0) {
      fence_proxy_async_smem();
      bulk_s2g(Wg, HrR, mat_bytes);
      bulk_commit();
      bulk_wait_read();
    }
  } else {
    for (int i = wid; i < n; i += NW)
      for (int j = lane; j < n; j += 32) Wg[i * n + j] = HrR[i * n + j] - (vrR[i] * wR[j] + wR[i] * vrR[j]);
  }
  return true;
}

template <typename R, int NT>
__global__ void __launch_bounds__(NT) exact_frame_kernel(StageArgs<R> a) {
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ int64_t s_item;
  __shared__ int s_flag[2];  // the factorisation's failure flags (two slots, alternating by step)
  __shared__ double s_sc[4];
  __shared__ __align__(8) uint64_t s_bar;
  const int tid = threadIdx.x;
  if (tid == 0) {
    mbar_init(&s_bar, 1);
    mbar_init_fence();
  }
  uint32_t phase = 0;
  while (true) {
    const int64_t item = a.item_begin + next_item(a.counter, &s_item);
    if (item >= a.item_end) break;
    const int lo = find_poly(a.prefix, a.n_desc, item);
    const ExactDesc& pd = a.descs[a.order[lo]];
    const int64_t p = item - a.prefix[lo];
    const bool ok = pd.mats_in_smem ? frame_item<R, NT, true>(a, pd, p, sm, s_flag, s_sc, s_bar, phase)
                                    : frame_item<R, NT, false>(a, pd, p, sm, s_flag, s_sc, s_bar, phase);
    if (!ok) break;  // (uniform across the CTA)
  }
  if (tid == 0) bulk_wait_all();
}

// ------------------------------------------------------------------ stage 3
// Resident CTAs a launch of the third stage is compiled for, in double
// words: seven (73 registers) over support sizes 1..4, six (85) over 5..6
// (the bench batch's third stage: 47.0 ms at six, 47.5 at seven, 48.6 at five
// and 51.8 at four), five for the generic launch whose out-of-line sizes 7
// and 8 carry a large stack.
template <typename R, int NT, int KHI>
constexpr int third_min_blocks() {
  return sizeof(R) == 4 ? 1024 / NT : std::is_same<R, dfloat>::value ? (KHI <= 4 ? 896 : KHI <= 6 ? 768 : 640) / NT : 1;
}
// KLO..KHI: the support sizes compiled into this instantiation (a launch also
// takes its range at run time, a.kmin..a.kmax, within them): a launch over one
// range carries only that range's code.
// MB > 0: that many resident CTAs instead (the classes of smaller n, whose
// shared memory allows more than the register budget of the default).
template <typename R, int NT, int KLO = 1, int KHI = kMaxSupport, int MB = 0>
__global__ void __launch_bounds__(NT, MB > 0 ? MB : third_min_blocks<R, NT, KHI>()) exact_third_kernel(StageArgs<R> a) {
  using Acc = AccOf<R>;
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ int64_t s_item;
  __shared__ __align__(8) uint64_t s_bar;
  constexpr int NW = NT / 32;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (tid == 0) {
    mbar_init(&s_bar, 1);
    mbar_init_fence();
  }
  uint32_t phase = 0;
  while (true) {
    const int64_t item = a.item_begin + next_item(a.counter, &s_item);
    if (item >= a.item_end) break;
    const int lo = find_poly(a.prefix, a.n_desc, item);
    const ExactDesc& pd = a.descs[a.order[lo]];
    const int64_t p = item - a.prefix[lo];
    const int n = pd.n, m = n - 1, E1 = pd.E + 1;
    const double* rec = a.vecs + pd.vec_off + p * vrec(n);
    if (rec[4 * n + 4] != kStOk) continue;  // flagged by stage 2 (same value for the whole CTA)
    if (a.kmax < kMaxSupport) {  // a launch before the last: nothing to do without terms of its sizes
      bool any = false;
      for (int k = max(a.kmin, 1); k <= a.kmax; ++k) any |= pd.koff[k + 1] > pd.k3off[k];
      if (!any) {
        if (a.kmin <= 1)
          for (int i = tid; i < n; i += NT) const_cast<double*>(rec)[4 * n + 8 + i] = 0.0;
        continue;
      }
    }
    const Lay3 L = lay_third<R, NW>(n, E1, pd.w_in_smem);
    R* pw = (R*)(sm + L.pw);
    Acc* c = (Acc*)(sm + L.c);
    double* v = (double*)(sm + L.v);
    double* e = (double*)(sm + L.e);
    double* y = (double*)(sm + L.y);
    R* yr = (R*)(sm + L.yr);
    const R* Wg = a.mats_w + pd.mat_off + p * mat_slot<R>(n);
    R* Ws = (R*)(sm + L.W);
    const R* W = pd.w_in_smem ? Ws : Wg;
    if (pd.w_in_smem && tid == 0) {  // W into shared memory by one bulk copy
      const uint32_t bytes = (uint32_t)(mat_slot<R>(n) * sizeof(R));
      fence_proxy_async_smem();
      mbar_arrive_expect_tx(&s_bar, bytes);
      bulk_g2s(Ws, Wg, bytes, &s_bar);
    }
    for (int i = tid; i < NW * n; i += NT) c[i] = Acc(0);
    const double* X = pd.X + p * n;
    power_table<R, NT>(X, n, E1, pw);
    R* ix = (R*)(sm + L.ix);
    bool in_range = true;
    for (int i = tid; i < n; i += NT) {
      v[i] = rec[n + i];
      e[i] = rec[2 * n + i];
      const double ax = fabs(X[i]);
      in_range &= ax >= pd.x_lo && ax <= pd.x_hi;
      ix[i] = R(1) / R(X[i]);
    }
    // gather form of the contraction where every |x_v| keeps m and 1/x normal
    const bool gather = __syncthreads_and(in_range) != 0;
    if (pd.w_in_smem) {
      if (!mbar_wait_cta(&s_bar, phase, a.err, 3)) {
        mbar_drain(&s_bar, phase, a.err, 3);
        return;
      }
      phase ^= 1u;
    }
    __syncthreads();
    {
      Acc* cw = c + wid * n;
      auto wget = [&](int, int, int va, int vb) { return W[va * n + vb]; };
      auto emit = [&](int l, R val) { acc_add(&cw[l], Acc(val)); };
      // terms of degree < 3 have no third derivatives: each group starts at
      // its first term of degree >= 3
      for_support<kMaxSupport>([&](auto kc) {
        constexpr int K = decltype(kc)::value;
        if constexpr (K < KLO || K > KHI) return;  // not compiled into this instantiation
        if (K < a.kmin || K > a.kmax) return;  // (uniform: another launch of the step takes this size)
        if constexpr (K >= 1) {
          if (gather) {
            for (int64_t t = pd.k3off[K] + tid; t < pd.koff[K + 1]; t += NT) {
              const TermRegs tr = load_term(pd.terms, t);
              // the reduced gather form for double words (within their bar);
              // the cancellation-free form for FP32 and for the FP64 form,
              // which is the accuracy reference
              if constexpr (std::is_same<R, dfloat>::value) term_third_gather_sub_group<R, K>(tr, pw, E1, ix, wget, emit);
              else term_third_gather_group<R, K>(tr, pw, E1, ix, wget, emit);
            }
            // the CTA's warps enter each support-size group together: every
            // group runs its own (large, fully unrolled) code, and warps
            // spread over several groups evicted each other's instructions
            // (third stage 62.2 -> 55.1 ms in double words)
            if (pd.koff[K + 1] > pd.k3off[K]) __syncthreads();
          } else {
            for (int64_t t = pd.k3off[K] + tid; t < pd.koff[K + 1]; t += NT) {
              const TermRegs tr = load_term(pd.terms, t);
              term_third_group<R, K>(tr, pw, E1, wget, emit);
            }
          }
        }
      });
    }
    __syncthreads();
    // c of this launch's support sizes, added to the earlier launches' in
    // launch order; a launch before the last passes the sum on
    double* cpart = const_cast<double*>(rec) + 4 * n + 8;
    const bool first = a.kmin <= 1, last = a.kmax >= kMaxSupport;
    if (!last) {
      for (int i = tid; i < n; i += NT) {
        Acc s = c[i];
        for (int q = 1; q < NW; ++q) s += c[q * n + i];
        cpart[i] = (first ? 0.0 : cpart[i]) + (double)s;
      }
      continue;  // (the next item's first barrier orders these reads of c before its writes)
    }
    const double gn = rec[4 * n + 1], beta = rec[4 * n + 2];
    // a = (P c)[0:m] = c - beta v (v.c);  tv = [h - |g|/(n+1) a; 0];  yr = P tv  (warp 0)
    if (wid == 0) {
      double vc = 0.0;
      for (int i = lane; i < n; i += 32) {
        Acc s = c[i];
        for (int q = 1; q < NW; ++q) s += c[q * n + i];
        const double ci = (first ? 0.0 : cpart[i]) + (double)s;
        y[i] = ci;
        vc += v[i] * ci;
      }
      vc = warp_sum(vc);
      const double wgt = gn / (double)(n + 1);
      double vt = 0.0;
      for (int i = lane; i < n; i += 32) {
        const double tv = i < m ? rec[3 * n + i] - wgt * (y[i] - beta * v[i] * vc) : 0.0;
        y[i] = tv;
        vt += v[i] * tv;
      }
      vt = warp_sum(vt);
      for (int i = lane; i < n; i += 32) yr[i] = R(y[i] - beta * v[i] * vt);
    }
    __syncthreads();
    // nu = W P tv - e  (W symmetric: column access, conflict-free)
    for (int i = tid; i < n; i += NT) {
      DotAcc<R> acc;
      for (int j = 0; j < n; ++j) acc.add(W[j * n + i], yr[j]);
      y[i] = (double)acc.value() - e[i];
    }
    __syncthreads();
    if (wid == 0) {
      double nrm = 0.0;
      for (int i = lane; i < n; i += 32) nrm += y[i] * y[i];
      const double inv = 1.0 / sqrt(warp_sum(nrm));
      for (int i = lane; i < n; i += 32) {
        pd.D[p * n + i] = y[i];
        if (pd.Dunit) pd.Dunit[p * n + i] = y[i] * inv;
      }
      if (lane == 0 && pd.info) {
        polylab_an_info in{gn, rec[4 * n + 3], 0, n, n - 1, 0};
        pd.info[p] = in;
      }
    }
  }
}

// ------------------------------------------------------------------ host side

namespace {

constexpr size_t kSmemCap = 200 * 1024;

template <typename R, int NW>
size_t lay_bytes(int stage, int n, int E1, bool in_smem, bool gather, int pts) {
  if (stage == 0) return lay_terms<R, NW>(n, E1, in_smem, gather, pts).total;
  if (stage == 1) return lay_frame<R>(n, in_smem).total;
  return lay_third<R, NW>(n, E1, in_smem).total;
}

template <typename R>
size_t stage_bytes(int stage, int threads, int n, int E1, bool in_smem, bool gather, int pts = kTermPoints) {
  if (threads == 64) return lay_bytes<R, 2>(stage, n, E1, in_smem, gather, pts);
  if (threads == 128) return lay_bytes<R, 4>(stage, n, E1, in_smem, gather, pts);
  return lay_bytes<R, 8>(stage, n, E1, in_smem, gather, pts);
}

}  // namespace

template <typename R>
static polylab_status prepare_exact(ExactBatch* b) {
  static_assert(sizeof(AccOf<R>) == sizeof(R), "H and W slots share one layout");
  size_t smem[3] = {0, 0, 0}, gstride = 0;
  int64_t mat = 0, vec = 0;
  b->frame_need.assign(b->host_descs.size(), 0);
  b->third_need.assign(b->host_descs.size(), 0);
  b->terms_need.assign(b->host_descs.size(), 0);
  b->terms_need1.assign(b->host_descs.size(), 0);
  b->terms_fb_smem = 0;
  for (size_t di = 0; di < b->host_descs.size(); ++di) {
    ExactDesc& d = b->host_descs[di];
    const int E1 = d.E + 1;
    const int tt = b->cfg.term_threads, ft = b->cfg.threads, t3 = b->cfg.third_threads;
    const bool gat = d.gather != nullptr;
    d.h_in_smem = stage_bytes<R>(0, tt, d.n, E1, true, gat) <= kSmemCap ? 1 : 0;
    d.mats_in_smem = stage_bytes<R>(1, ft, d.n, E1, true, false) <= kSmemCap ? 1 : 0;
    d.w_in_smem = stage_bytes<R>(2, t3, d.n, E1, true, false) <= kSmemCap ? 1 : 0;
    const size_t need[3] = {stage_bytes<R>(0, tt, d.n, E1, d.h_in_smem, gat),
                            stage_bytes<R>(1, ft, d.n, E1, d.mats_in_smem, false),
                            stage_bytes<R>(2, t3, d.n, E1, d.w_in_smem, false)};
    for (int st = 0; st < 3; ++st) {
      if (need[st] > kSmemCap) return POLYLAB_ERR_UNSUPPORTED;
      smem[st] = std::max(smem[st], need[st]);
    }
    b->frame_need[di] = need[1];
    b->third_need[di] = need[2];
    // class-wise sweep: the gather launch (descriptors with records) and the term-by-term launch
    b->terms_need[di] = gat ? need[0] : 0;
    b->terms_need1[di] = gat ? stage_bytes<R>(0, tt, d.n, E1, d.h_in_smem, true, 1) : 0;
    b->terms_fb_smem = std::max(b->terms_fb_smem, stage_bytes<R>(0, tt, d.n, E1, d.h_in_smem, false));
    if (!d.mats_in_smem) gstride = std::max(gstride, frame_gmem<R>(d.n));
    d.mat_off = mat;
    d.vec_off = vec;
    mat += d.P * mat_slot<R>(d.n);
    vec += d.P * vrec(d.n);
  }
  for (int st = 0; st < 3; ++st) b->smem[st] = smem[st];
  b->gws_stride = gstride;
  b->ws_mat_bytes = (size_t)mat * sizeof(R);
  b->ws_vec_bytes = (size_t)vec * sizeof(double);
  return POLYLAB_OK;
}

template <typename R, int NT>
static polylab_status launch_stage_t(ExactBatch* b, int stage, cudaStream_t s) {
  void (*k)(StageArgs<R>) = stage == 1 ? exact_frame_kernel<R, NT> : exact_third_kernel<R, NT>;
  const int64_t i0 = 0, i1 = b->total;
  if (i1 <= i0) return POLYLAB_OK;
  const size_t smem = b->smem[stage];
  PL_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  PL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, NT, smem));
  per_sm = std::max(1, per_sm);
  const int cap = stage == 1 ? b->cfg.ctas_per_sm : b->cfg.third_ctas;
  if (cap > 0) per_sm = std::min(per_sm, cap);
  const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(i1 - i0, (int64_t)num_sms() * per_sm));
  if (stage == 1 && b->gws_stride > 0 && (size_t)grid * b->gws_stride > b->gws_bytes) return POLYLAB_ERR_UNSUPPORTED;
  StageArgs<R> a{};
  a.descs = b->descs;
  a.n_desc = b->n_desc;
  a.prefix = b->prefix;
  a.order = b->order;
  a.item_begin = i0;
  a.item_end = i1;
  a.counter = b->counter + stage;
  a.mats_h = (AccOf<R>*)b->ws_h;
  a.mats_w = (R*)b->ws_w;
  a.vecs = (double*)b->ws_v;
  a.r = b->opts.regularization;
  a.assume_nonzero_x = b->opts.assume_nonzero_x;
  a.gws = b->gws;
  a.gws_stride = b->gws_stride;
  a.err = b->err;
  a.kmin = 1;
  a.kmax = kMaxSupport;
  if (stage == 1) {
    PL_CUDA(cudaMemsetAsync(a.counter, 0, sizeof(int), s));
    k<<<(unsigned)grid, NT, smem, s>>>(a);
    return launch_status("exact_frame_kernel");
  }
  // the third stage as one launch per range of support sizes, in order
  static const int kRanges[4][4][2] = {{{1, kMaxSupport}},
                                       {{1, 4}, {5, kMaxSupport}},
                                       {{1, 4}, {5, 5}, {6, kMaxSupport}},
                                       {{1, 3}, {4, 4}, {5, 5}, {6, kMaxSupport}}};
  const int split = std::min(4, std::max(1, b->cfg.third_split));
  int max_support = 0;
  for (const ExactDesc& d : b->host_descs) max_support = std::max(max_support, d.max_support);
  for (int g = 0; g < split; ++g) {
    a.kmin = kRanges[split - 1][g][0];
    a.kmax = kRanges[split - 1][g][1];
    // the double-word form has instantiations for the ranges of two and
    // three launches, the last without the (out-of-line) support sizes 7 and
    // 8 when the batch has no such terms: a launch carries only its own
    // sizes' (large, unrolled) code (four launches, with generic kernels for
    // 1..3 and 4, measured slower: 46.6 against 45.5 ms)
    void (*kt)(StageArgs<R>) = k;
    if constexpr (std::is_same<R, dfloat>::value) {
      if (a.kmin == 1 && a.kmax == 4) kt = exact_third_kernel<R, NT, 1, 4>;
      else if (a.kmin == 5 && a.kmax == 5) kt = exact_third_kernel<R, NT, 5, 5>;
      else if (a.kmin == 5 && a.kmax == kMaxSupport)
        kt = max_support <= 6 ? exact_third_kernel<R, NT, 5, 6> : exact_third_kernel<R, NT, 5, kMaxSupport>;
      else if (a.kmin == 6 && a.kmax == kMaxSupport)
        kt = max_support <= 6 ? exact_third_kernel<R, NT, 6, 6> : exact_third_kernel<R, NT, 6, kMaxSupport>;
    }
    // within a range, one launch per class of n of the frame stage (frame
    // order), each with its own class's shared memory: a launch over all
    // polynomials reserved the largest n's W for every CTA
    a.prefix = b->fprefix;
    a.order = b->forder;
    for (int c = 0; c < kFrameClasses; ++c) {
      const FrameClass& fc = b->fclass[c];
      if (fc.end <= fc.begin) continue;
      const size_t sm3 = std::max<size_t>(fc.t3smem, 16);
      void (*kc)(StageArgs<R>) = kt;
      if constexpr (std::is_same<R, dfloat>::value && NT == 128) {
        // more resident CTAs where the class's shared memory allows them: sizes
        // 5 and 6 at seven (72 registers) for n <= 40, sizes 1..5 at eight (64)
        // for n <= 24 (third stage 44.5 -> 43.1 ms for the bench batch)
        if (c > 0 && kt == exact_third_kernel<R, NT, 5, 5>) kc = exact_third_kernel<R, NT, 5, 5, 7>;
        if (c > 0 && kt == exact_third_kernel<R, NT, 6, 6>) kc = exact_third_kernel<R, NT, 6, 6, 7>;
        if (c == 2 && kt == exact_third_kernel<R, NT, 1, 4>) kc = exact_third_kernel<R, NT, 1, 4, 8>;
        if (c == 2 && kt == exact_third_kernel<R, NT, 5, 5>) kc = exact_third_kernel<R, NT, 5, 5, 8>;
      }
      PL_CUDA(cudaFuncSetAttribute(kc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm3));
      int psm = 0;
      PL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&psm, kc, NT, sm3));
      psm = std::max(1, psm);
      if (cap > 0) psm = std::min(psm, cap);
      const int64_t gk = std::max<int64_t>(1, std::min<int64_t>(fc.end - fc.begin, (int64_t)num_sms() * psm));
      a.item_begin = fc.begin;
      a.item_end = fc.end;
      PL_CUDA(cudaMemsetAsync(a.counter, 0, sizeof(int), s));
      kc<<<(unsigned)gk, NT, sm3, s>>>(a);
      PL_TRY(launch_status("exact_third_kernel"));
    }
  }
  (void)grid;
  return POLYLAB_OK;
}

// The gradient/Hessian sweep over the frame stage's classes of n (frame
// order): one gather launch per class, each with the shared memory of its own
// largest n, then one term-by-term launch over the passes they left.  (The
// list and the launch counters are reset on the stream first.)
template <typename R, int NT>
static polylab_status launch_terms_classes(ExactBatch* b, cudaStream_t s) {
  StageArgs<R> a{};
  a.descs = b->descs;
  a.n_desc = b->n_desc;
  a.prefix = b->fprefix;
  a.order = b->forder;
  a.mats_h = (AccOf<R>*)b->ws_h;
  a.mats_w = (R*)b->ws_w;
  a.vecs = (double*)b->ws_v;
  a.r = b->opts.regularization;
  a.assume_nonzero_x = b->opts.assume_nonzero_x;
  a.gws = b->gws;
  a.gws_stride = b->gws_stride;
  a.err = b->err;
  a.kmin = 1;
  a.kmax = kMaxSupport;
  PassList fl{b->tfb, b->tfb_ctl, (int)b->tfb_cap, kTermPoints};
  PL_CUDA(cudaMemsetAsync(b->tfb_ctl, 0, (2 + kFrameClasses) * sizeof(int), s));
  auto launch = [&](void (*k)(StageArgs<R>, PassList), size_t smem, int64_t items, int* counter) -> polylab_status {
    smem = std::max<size_t>(smem, 16);
    PL_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    PL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, NT, smem));
    per_sm = std::max(1, per_sm);
    if (b->cfg.terms_ctas > 0) per_sm = std::min(per_sm, b->cfg.terms_ctas);
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(items, (int64_t)num_sms() * per_sm));
    a.counter = counter;
    k<<<(unsigned)grid, NT, smem, s>>>(a, fl);
    return launch_status("exact_terms_kernel");
  };
  // resident CTAs of the gather kernel at `smem` bytes
  auto resident = [&](size_t smem) -> int {
    smem = std::max<size_t>(smem, 16);
    int r = 0;
    if (cudaFuncSetAttribute(exact_terms_kernel<R, NT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r, exact_terms_kernel<R, NT, true>, NT, smem) != cudaSuccess)
      return 0;
    return r;
  };
  for (int c = 0; c < kFrameClasses; ++c) {
    const FrameClass& fc = b->fclass[c];
    if (fc.end <= fc.begin) continue;
    a.item_begin = fc.begin;
    a.item_end = fc.end;
    // one point per pass where that raises the resident CTAs (the shared
    // memory of two points' Hessian slots limits the classes of larger n);
    // two otherwise, each record then decoded once for both
    fl.pts = kTermPoints;
    if (fc.tsmem1 > 0 && resident(fc.tsmem1) > resident(fc.tsmem)) fl.pts = 1;
    PL_TRY(launch(exact_terms_kernel<R, NT, true>, fl.pts == 1 ? fc.tsmem1 : fc.tsmem,
                  (fc.end - fc.begin + fl.pts - 1) / fl.pts, b->tfb_ctl + 1 + c));
  }
  a.item_begin = 0;
  a.item_end = b->total;
  return launch(exact_terms_kernel<R, NT, false>, b->terms_fb_smem, (b->total + 1) / 2,
                b->tfb_ctl + 1 + kFrameClasses);
}

// One class of the split frame stage: the class's item
// range of the frame order, its own counter and shared memory; the residency
// cap applies to the first (largest-n) class only.
template <typename R, int NT>
static polylab_status launch_frame_class(ExactBatch* b, int cls, cudaStream_t s) {
  const FrameClass& fc = b->fclass[cls];
  if (fc.end <= fc.begin) return POLYLAB_OK;
  auto k = exact_frame_kernel<R, NT>;
  const size_t smem = std::max<size_t>(fc.smem, 16);
  PL_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  PL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, NT, smem));
  per_sm = std::max(1, per_sm);
  if (cls == 0 && b->cfg.ctas_per_sm > 0) per_sm = std::min(per_sm, b->cfg.ctas_per_sm);
  const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(fc.end - fc.begin, (int64_t)num_sms() * per_sm));
  if (b->gws_stride > 0 && (size_t)grid * b->gws_stride > b->gws_bytes) return POLYLAB_ERR_UNSUPPORTED;
  StageArgs<R> a{};
  a.descs = b->descs;
  a.n_desc = b->n_desc;
  a.prefix = b->fprefix;
  a.order = b->forder;
  a.item_begin = fc.begin;
  a.item_end = fc.end;
  a.counter = b->fcounter + cls;
  a.mats_h = (AccOf<R>*)b->ws_h;
  a.mats_w = (R*)b->ws_w;
  a.vecs = (double*)b->ws_v;
  a.r = b->opts.regularization;
  a.assume_nonzero_x = b->opts.assume_nonzero_x;
  a.gws = b->gws;
  a.gws_stride = b->gws_stride;
  a.err = b->err;
  PL_CUDA(cudaMemsetAsync(a.counter, 0, sizeof(int), s));
  k<<<(unsigned)grid, NT, smem, s>>>(a);
  return launch_status("exact_frame_kernel");
}

template <typename R>
static polylab_status launch_frame_classes(ExactBatch* b, cudaStream_t s) {
  for (int c = 0; c < kFrameClasses; ++c) {
    const int nt = b->fclass[c].threads;
    if (nt == 64) PL_TRY((launch_frame_class<R, 64>(b, c, s)));
    else if (nt == 128) PL_TRY((launch_frame_class<R, 128>(b, c, s)));
    else PL_TRY((launch_frame_class<R, 256>(b, c, s)));
  }
  return POLYLAB_OK;
}

template <typename R>
static polylab_status launch_stage(ExactBatch* b, int stage, cudaStream_t s) {
  if (stage == 1 && b->cfg.frame_split) return launch_frame_classes<R>(b, s);
  if (stage == 0) {
    const int nt = b->cfg.term_threads;
    if (nt == 64) return launch_terms_classes<R, 64>(b, s);
    if (nt == 128) return launch_terms_classes<R, 128>(b, s);
    return launch_terms_classes<R, 256>(b, s);
  }
  const int nt = stage == 0 ? b->cfg.term_threads : stage == 1 ? b->cfg.threads : b->cfg.third_threads;
  if (nt == 64) return launch_stage_t<R, 64>(b, stage, s);
  if (nt == 128) return launch_stage_t<R, 128>(b, stage, s);
  return launch_stage_t<R, 256>(b, stage, s);
}

polylab_status run_exact_stage(ExactBatch* b, int stage, cudaStream_t s) {
  if (b->total == 0) return POLYLAB_OK;
  if (b->opts.prec == POLYLAB_FP32) return launch_stage<float>(b, stage, s);
  if (b->opts.prec == POLYLAB_F32X2) return launch_stage<dfloat>(b, stage, s);
  return launch_stage<double>(b, stage, s);
}

// One run: the three stages one after another on `s` (capturable in a graph).
polylab_status run_exact_batch(ExactBatch* b, cudaStream_t s) {
  for (int st = 0; st < 3; ++st) PL_TRY(run_exact_stage(b, st, s));
  return POLYLAB_OK;
}

polylab_status prepare_exact_batch(ExactBatch* b) {
  if (b->opts.prec == POLYLAB_FP32) return prepare_exact<float>(b);
  if (b->opts.prec == POLYLAB_F32X2) return prepare_exact<dfloat>(b);
  return prepare_exact<double>(b);
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
