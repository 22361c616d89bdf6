// Internal definitions shared by the CUDA translation units of libpolylab.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <type_traits>
#include <unordered_set>
#include <vector>

#include "polylab.h"

namespace polylab {

// ------------------------------------------------------------------ errors

void set_last_error(const char* where, cudaError_t e);
void set_last_message(const char* msg);

#define PL_CUDA(call)                                   \
  do {                                                  \
    cudaError_t e__ = (call);                           \
    if (e__ != cudaSuccess) {                           \
      ::polylab::set_last_error(#call, e__);            \
      return POLYLAB_ERR_CUDA;                          \
    }                                                   \
  } while (0)

#define PL_TRY(expr)                          \
  do {                                        \
    polylab_status s__ = (expr);              \
    if (s__ != POLYLAB_OK) return s__;        \
  } while (0)

inline polylab_status launch_status(const char* where) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_last_error(where, e);
    return POLYLAB_ERR_CUDA;
  }
  return POLYLAB_OK;
}

// ------------------------------------------------------------ scratch memory
// Stream-ordered scratch buffers: freed in stream order when the guard dies.

// The library's stream-ordered memory pool on the current device: like the
// device's default pool, but it keeps the memory it has mapped across
// synchronisations (release threshold: unlimited), so that a call does not
// map its scratch afresh after the previous call synchronised.  Its memory
// goes back to the system when the process ends.
cudaMemPool_t scratch_pool();

struct Scratch {
  cudaStream_t s;
  std::vector<void*> ptrs;
  explicit Scratch(cudaStream_t st) : s(st) {}
  ~Scratch() {
    for (void* p : ptrs) cudaFreeAsync(p, s);
  }
  template <typename T>
  polylab_status get(T** out, size_t count) {
    *out = nullptr;
    if (count == 0) count = 1;
    void* p = nullptr;
    cudaMemPool_t pool = scratch_pool();
    cudaError_t e = pool ? cudaMallocFromPoolAsync(&p, count * sizeof(T), pool, s)
                         : cudaMallocAsync(&p, count * sizeof(T), s);
    if (e != cudaSuccess) {
      set_last_error("cudaMallocAsync", e);
      cudaGetLastError();
      return POLYLAB_ERR_OOM;
    }
    ptrs.push_back(p);
    *out = static_cast<T*>(p);
    return POLYLAB_OK;
  }
};

// --------------------------------------------------------------- term list
// Terms per chunk of the gather-form sweep (monomial values of one chunk are
// held in shared memory), and the number of record streams per chunk: the
// entry-sorted records of a chunk are cut into kGatherStreams contiguous
// runs of equal length, stored interleaved (record k of stream s at
// k * kGatherStreams + s) so that the threads of a warp, each walking its own
// run, read consecutive addresses.  Runs are padded to a multiple of
// kGatherUnroll records with entry kGatherPad and coefficient 0.
constexpr int kGatherChunk = 2048;
constexpr int kGatherStreams = 256;
constexpr int kGatherUnroll = 8;
constexpr uint32_t kGatherPad = 0x3fff;

// Packed sparse form of one term: at most kMaxSupport active variables, in
// ascending variable order; unused slots have exp == 0.  32 bytes, so a term
// is two aligned 16-byte loads.

constexpr int kMaxSupport = 8;

struct __align__(16) Term {
  double coef;
  uint16_t var[kMaxSupport];
  uint8_t exp[kMaxSupport];
};
static_assert(sizeof(Term) == 32, "Term layout");

// Device-resident preprocessed polynomial (the opaque polylab_plan).
struct GemmOperand;  // defined with the tensor-core contraction

}  // namespace polylab

struct polylab_plan {
  int32_t n = 0;
  int64_t m = 0;
  int32_t max_exp = 0;       // largest single exponent (power-table depth)
  int32_t max_support = 0;   // largest number of active variables in a term
  polylab::Term* terms = nullptr;  // DEVICE, m terms, sorted by (support size, degree)
  // koff[k]: first term with support size k (koff[kMaxSupport + 1] = m);
  // k3off[k]: first term of that group with degree >= 3
  int64_t koff[polylab::kMaxSupport + 2] = {};
  int64_t k3off[polylab::kMaxSupport + 1] = {};
  // gather form of the gradient/Hessian sweep (nullptr when n > 127 or a
  // falling-factorial coefficient exceeds 127): for every chunk of
  // kGatherChunk terms, the (term, entry, coefficient) contributions sorted
  // by entry; entry e < n*n is H(e / n, e % n) (upper triangle), e >= n*n is
  // g(e - n*n); one 32-bit record: term within the chunk (bits 0-10), entry
  // (bits 11-24), coefficient (bits 25-31)
  uint32_t* gather = nullptr;         // DEVICE records
  int64_t* gather_chunk = nullptr;    // DEVICE, n_gchunks + 1 record offsets (multiples of kGatherStreams)
  int32_t n_gchunks = 0;
  int32_t max_degree = 0;
  // sparsity pattern of the Hessian for assembled Hessian-vector products
  // (built on first use by the stochastic path): CSR of every (i, j) that a
  // term's support pairs (both orders) plus the whole diagonal; for term t of
  // support-size group K (t' = t - koff[K]) the CSR positions of its K x K
  // block are hpos[hbase[K] + t' K^2 + a K + b]
  int32_t* hrow = nullptr;  // DEVICE, n + 1
  int32_t* hcol = nullptr;  // DEVICE, hnnz
  int32_t* hpos = nullptr;  // DEVICE
  int64_t hnnz = 0;
  int64_t hbase[polylab::kMaxSupport + 1] = {};
  // derived-coefficient data for the tensor-core forms (nullptr unless built)
  polylab::GemmOperand* gemm = nullptr;
  int64_t closure = -1;
};

namespace polylab {

// A polynomial with FP64 or FP32 coefficients (the two storage precisions of
// the C ABI: polylab_poly / polylab_poly_f32), as the engine and the plan
// builder see it.
template <typename C>
struct PolyIn {
  int32_t n_vars;
  const uint64_t* var_ids;
  int64_t n_terms;
  const uint8_t* exps;
  const C* coef;
};
template <typename C>
struct PolyOut {
  int32_t n_vars;
  uint64_t* var_ids;
  int64_t n_terms;
  uint8_t* exps;
  C* coef;
};
template <typename Pub>
using coef_of = std::remove_cv_t<std::remove_pointer_t<decltype(Pub::coef)>>;
template <typename Pub>
inline PolyIn<coef_of<Pub>> poly_in(const Pub& p) {
  return {p.n_vars, p.var_ids, p.n_terms, p.exps, p.coef};
}
template <typename Pub>
inline PolyOut<coef_of<Pub>> poly_out(const Pub& o) {
  return {o.n_vars, o.var_ids, o.n_terms, o.exps, o.coef};
}
template <typename Pub>
inline void store_out(const PolyOut<coef_of<Pub>>& o, Pub* out) {
  out->n_vars = o.n_vars;
  out->n_terms = o.n_terms;
  out->exps = o.exps;
  out->coef = o.coef;
}

template <typename C>
polylab_status check_poly(const PolyIn<C>* p) {
  if (!p || p->n_vars < 1 || p->n_terms < 0 || !p->var_ids) return POLYLAB_ERR_INVALID_ARG;
  if (p->n_terms > 0 && (!p->exps || !p->coef)) return POLYLAB_ERR_INVALID_ARG;
  std::unordered_set<uint64_t> seen;
  for (int i = 0; i < p->n_vars; ++i)
    if (!seen.insert(p->var_ids[i]).second) return POLYLAB_ERR_DUP_VAR_ID;
  return POLYLAB_OK;
}

// Fill `plan` (terms, m, n, max_exp, max_support); synchronises `s`.  FP32
// coefficients are held in the term list exactly (as doubles).
template <typename C>
polylab_status build_term_plan(const PolyIn<C>* p, cudaStream_t s, polylab_plan* plan);
// Build the Hessian sparsity pattern of `plan` if absent (synchronises `s`).
polylab_status ensure_hessian_pattern(polylab_plan* plan, cudaStream_t s);
polylab_status build_gemm_operand(polylab_plan* plan, cudaStream_t s);
void free_gemm_operand(GemmOperand* g, cudaStream_t s);

// The engine (engine.cu): simplify, product, sum or difference of
// polynomials, coefficient arithmetic and storage in C (double or float).
constexpr int kSimplifyMode = 0, kMulMode = 1, kAddMode = 2, kSubMode = 3;
template <typename C>
polylab_status engine(const PolyIn<C>* pa, const PolyIn<C>* pb, int mode, double zeroprec, PolyOut<C>* out,
                      polylab_alloc_fn alloc, void* ctx, cudaStream_t s);

// Kernel launchers (one per translation unit)
polylab_status eval_direct(const polylab_plan* plan, const double* X, int64_t P, int order, bool fp32,
                           double* F, double* G, double* H, cudaStream_t s);
polylab_status eval_direct_f32(const polylab_plan* plan, const float* X, int64_t P, int order, float* F, float* G,
                               float* H, cudaStream_t s);
polylab_status eval_gemm(const polylab_plan* plan, const double* X, int64_t P, int order, int prec,
                         double* F, double* G, double* H, cudaStream_t s);
polylab_status affine_exact(const polylab_plan* plan, const double* X, int64_t P, const polylab_an_opts* o,
                            double* D, double* Dunit, polylab_an_info* info, cudaStream_t s);
polylab_status affine_ad(const polylab_plan* plan, const double* X, int64_t P, const polylab_an_opts* o, double* D,
                         double* Dunit, polylab_an_info* info, cudaStream_t s);
polylab_status affine_stochastic(const polylab_plan* plan, const double* X, int64_t P,
                                 const polylab_an_opts* o, double* D, double* Dunit, polylab_an_info* info,
                                 cudaStream_t s);

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

int num_sms();

}  // namespace polylab
