// Polynomial algebra on top of the engine: integer powers and symbolic
// partial derivatives (the paper's mpower/prod and diff/jacobian, Sec. 2
// Table "coresemantics" and Sec. 3.3).  Both reduce to the engine's product
// and simplify; results are simplified and in the engine's canonical order.
#include <cstring>
#include <vector>

#include "common.cuh"

namespace polylab {

namespace {

// A polynomial held in library-owned device memory between engine calls.
template <typename C>
struct Owned {
  std::vector<uint64_t> ids;
  int64_t m = 0;
  uint8_t* exps = nullptr;
  C* coef = nullptr;
  PolyIn<C> view() const { return {(int32_t)ids.size(), ids.data(), m, exps, coef}; }
};

// Allocation callback of the engine for intermediates: stream-ordered device
// memory that the Scratch guard frees at the end of the call.
struct ScratchAlloc {
  Scratch* scr;
  bool failed = false;
};
void* scratch_alloc(size_t bytes, void* ctx) {
  auto* a = static_cast<ScratchAlloc*>(ctx);
  unsigned char* p = nullptr;
  if (a->scr->get(&p, bytes) != POLYLAB_OK) {
    a->failed = true;
    return nullptr;
  }
  return p;
}

template <typename C>
polylab_status run_engine(const PolyIn<C>* a, const PolyIn<C>* b, int mode, double zeroprec, Scratch& scr,
                          cudaStream_t s, Owned<C>* res) {
  ScratchAlloc sa{&scr};
  res->ids.assign((size_t)a->n_vars + (b ? b->n_vars : 0), 0);
  PolyOut<C> o{};
  o.var_ids = res->ids.data();
  PL_TRY(engine(a, b, mode, zeroprec, &o, scratch_alloc, &sa, s));
  if (sa.failed) return POLYLAB_ERR_OOM;
  res->ids.resize(o.n_vars);
  res->m = o.n_terms;
  res->exps = o.exps;
  res->coef = o.coef;
  return POLYLAB_OK;
}

template <typename C>
polylab_status copy_out(const Owned<C>& r, PolyOut<C>* out, polylab_alloc_fn alloc, void* ctx, cudaStream_t s) {
  const int n = (int)r.ids.size();
  out->n_vars = n;
  std::memcpy(out->var_ids, r.ids.data(), (size_t)n * sizeof(uint64_t));
  out->n_terms = r.m;
  out->exps = nullptr;
  out->coef = nullptr;
  if (r.m == 0) return POLYLAB_OK;
  out->exps = (uint8_t*)alloc((size_t)r.m * n, ctx);
  out->coef = (C*)alloc((size_t)r.m * sizeof(C), ctx);
  if (!out->exps || !out->coef) return POLYLAB_ERR_OOM;
  PL_CUDA(cudaMemcpyAsync(out->exps, r.exps, (size_t)r.m * n, cudaMemcpyDeviceToDevice, s));
  PL_CUDA(cudaMemcpyAsync(out->coef, r.coef, (size_t)r.m * sizeof(C), cudaMemcpyDeviceToDevice, s));
  return POLYLAB_OK;
}

// d/dx_v of every term: exponent row with a_v - 1 and coefficient a_v c; a
// term without x_v gets coefficient 0 (its row is left as is and the
// simplify that follows drops it, adding exact zeros to nothing else).
template <typename C>
__global__ void diff_terms(const uint8_t* __restrict__ exps, const C* __restrict__ coef, int64_t m, int n, int v,
                           uint8_t* __restrict__ dexps, C* __restrict__ dcoef) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= m) return;
  const uint8_t* row = exps + t * n;
  uint8_t* drow = dexps + t * n;
  for (int c = 0; c < n; ++c) drow[c] = row[c];
  const int a = row[v];
  if (a > 0) {
    drow[v] = (uint8_t)(a - 1);
    dcoef[t] = (C)a * coef[t];
  } else {
    dcoef[t] = C(0);
  }
}

template <typename C>
polylab_status pow_impl(const PolyIn<C>* p, int32_t k, double zeroprec, PolyOut<C>* out, polylab_alloc_fn alloc,
                        void* alloc_ctx, cudaStream_t s) {
  if (!out || !alloc || !out->var_ids || k < 0 || !(zeroprec >= 0.0)) return POLYLAB_ERR_INVALID_ARG;
  PL_TRY(check_poly(p));
  Scratch scr(s);
  if (k == 0) {  // the constant 1 over p's variables
    Owned<C> one;
    one.ids.assign(p->var_ids, p->var_ids + p->n_vars);
    one.m = 1.0 > zeroprec ? 1 : 0;
    if (one.m) {
      PL_TRY(scr.get(&one.exps, (size_t)p->n_vars));
      PL_TRY(scr.get(&one.coef, 1));
      PL_CUDA(cudaMemsetAsync(one.exps, 0, (size_t)p->n_vars, s));
      const C c1 = C(1);
      PL_CUDA(cudaMemcpyAsync(one.coef, &c1, sizeof(C), cudaMemcpyHostToDevice, s));
      PL_CUDA(cudaStreamSynchronize(s));  // c1 lives on this stack frame
    }
    return copy_out(one, out, alloc, alloc_ctx, s);
  }
  // binary exponentiation: base = p^(2^i), acc = product of the bases of k's set bits
  Owned<C> base, acc;
  bool have_acc = false;
  PL_TRY(run_engine<C>(p, nullptr, kSimplifyMode, zeroprec, scr, s, &base));
  for (int32_t e = k;;) {
    if (e & 1) {
      if (!have_acc) {
        acc = base;
        have_acc = true;
      } else {
        const PolyIn<C> av = acc.view(), bv = base.view();
        Owned<C> nxt;
        PL_TRY(run_engine(&av, &bv, kMulMode, zeroprec, scr, s, &nxt));
        acc = nxt;
      }
    }
    e >>= 1;
    if (!e) break;
    const PolyIn<C> bv = base.view();
    Owned<C> sq;
    PL_TRY(run_engine(&bv, &bv, kMulMode, zeroprec, scr, s, &sq));
    base = sq;
  }
  return copy_out(acc, out, alloc, alloc_ctx, s);
}

template <typename C>
polylab_status diff_impl(const PolyIn<C>* p, uint64_t var_id, double zeroprec, PolyOut<C>* out,
                         polylab_alloc_fn alloc, void* alloc_ctx, cudaStream_t s) {
  if (!out || !alloc || !out->var_ids || !(zeroprec >= 0.0)) return POLYLAB_ERR_INVALID_ARG;
  PL_TRY(check_poly(p));
  int v = -1;
  for (int i = 0; i < p->n_vars; ++i)
    if (p->var_ids[i] == var_id) v = i;
  if (v < 0 || p->n_terms == 0) {  // derivative identically zero
    out->n_vars = p->n_vars;
    std::memcpy(out->var_ids, p->var_ids, (size_t)p->n_vars * sizeof(uint64_t));
    out->n_terms = 0;
    out->exps = nullptr;
    out->coef = nullptr;
    return POLYLAB_OK;
  }
  Scratch scr(s);
  uint8_t* dexps;
  C* dcoef;
  PL_TRY(scr.get(&dexps, (size_t)p->n_terms * p->n_vars));
  PL_TRY(scr.get(&dcoef, (size_t)p->n_terms));
  diff_terms<C><<<(unsigned)ceil_div(p->n_terms, 256), 256, 0, s>>>(p->exps, p->coef, p->n_terms, p->n_vars, v,
                                                                    dexps, dcoef);
  PL_TRY(launch_status("diff_terms"));
  PolyIn<C> d = *p;
  d.exps = dexps;
  d.coef = dcoef;
  return engine<C>(&d, nullptr, kSimplifyMode, zeroprec, out, alloc, alloc_ctx, s);
}

// The public structs viewed as PolyIn / PolyOut and back.
template <typename PubIn, typename PubOut, typename F>
polylab_status entry(const PubIn* p, PubOut* out, F&& f) {
  if (!p || !out) return POLYLAB_ERR_INVALID_ARG;
  const auto vp = poly_in(*p);
  auto o = poly_out(*out);
  const polylab_status st = f(&vp, &o);
  store_out(o, out);
  return st;
}

}  // namespace

}  // namespace polylab

using namespace polylab;

extern "C" {

polylab_status polylab_pow(const polylab_poly* p, int32_t k, double zeroprec, polylab_poly_out* out,
                           polylab_alloc_fn alloc, void* alloc_ctx, polylab_stream stream) {
  return entry(p, out, [&](auto* vp, auto* o) {
    return pow_impl(vp, k, zeroprec, o, alloc, alloc_ctx, (cudaStream_t)stream);
  });
}

polylab_status polylab_pow_f32(const polylab_poly_f32* p, int32_t k, double zeroprec, polylab_poly_out_f32* out,
                               polylab_alloc_fn alloc, void* alloc_ctx, polylab_stream stream) {
  return entry(p, out, [&](auto* vp, auto* o) {
    return pow_impl(vp, k, zeroprec, o, alloc, alloc_ctx, (cudaStream_t)stream);
  });
}

polylab_status polylab_diff(const polylab_poly* p, uint64_t var_id, double zeroprec, polylab_poly_out* out,
                            polylab_alloc_fn alloc, void* alloc_ctx, polylab_stream stream) {
  return entry(p, out, [&](auto* vp, auto* o) {
    return diff_impl(vp, var_id, zeroprec, o, alloc, alloc_ctx, (cudaStream_t)stream);
  });
}

polylab_status polylab_diff_f32(const polylab_poly_f32* p, uint64_t var_id, double zeroprec,
                                polylab_poly_out_f32* out, polylab_alloc_fn alloc, void* alloc_ctx,
                                polylab_stream stream) {
  return entry(p, out, [&](auto* vp, auto* o) {
    return diff_impl(vp, var_id, zeroprec, o, alloc, alloc_ctx, (cudaStream_t)stream);
  });
}

}  // extern "C"
