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
struct Owned {
  std::vector<uint64_t> ids;
  int64_t m = 0;
  uint8_t* exps = nullptr;
  double* coef = nullptr;
  polylab_poly view() const {
    polylab_poly p{};
    p.n_vars = (int32_t)ids.size();
    p.var_ids = ids.data();
    p.n_terms = m;
    p.exps = exps;
    p.coef = coef;
    return p;
  }
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

polylab_status run_engine(const polylab_poly* a, const polylab_poly* b, int mode, double zeroprec, Scratch& scr,
                          cudaStream_t s, Owned* res) {
  ScratchAlloc sa{&scr};
  res->ids.assign((size_t)a->n_vars + (b ? b->n_vars : 0), 0);
  polylab_poly_out o{};
  o.var_ids = res->ids.data();
  PL_TRY(engine(a, b, mode, zeroprec, &o, scratch_alloc, &sa, s));
  if (sa.failed) return POLYLAB_ERR_OOM;
  res->ids.resize(o.n_vars);
  res->m = o.n_terms;
  res->exps = o.exps;
  res->coef = o.coef;
  return POLYLAB_OK;
}

polylab_status copy_out(const Owned& r, polylab_poly_out* out, polylab_alloc_fn alloc, void* ctx, cudaStream_t s) {
  const int n = (int)r.ids.size();
  out->n_vars = n;
  std::memcpy(out->var_ids, r.ids.data(), (size_t)n * sizeof(uint64_t));
  out->n_terms = r.m;
  out->exps = nullptr;
  out->coef = nullptr;
  if (r.m == 0) return POLYLAB_OK;
  out->exps = (uint8_t*)alloc((size_t)r.m * n, ctx);
  out->coef = (double*)alloc((size_t)r.m * sizeof(double), ctx);
  if (!out->exps || !out->coef) return POLYLAB_ERR_OOM;
  PL_CUDA(cudaMemcpyAsync(out->exps, r.exps, (size_t)r.m * n, cudaMemcpyDeviceToDevice, s));
  PL_CUDA(cudaMemcpyAsync(out->coef, r.coef, (size_t)r.m * sizeof(double), cudaMemcpyDeviceToDevice, s));
  return POLYLAB_OK;
}

// d/dx_v of every term: exponent row with a_v - 1 and coefficient a_v c; a
// term without x_v gets coefficient 0 (its row is left as is and the
// simplify that follows drops it, adding exact zeros to nothing else).
__global__ void diff_terms(const uint8_t* __restrict__ exps, const double* __restrict__ coef, int64_t m, int n, int v,
                           uint8_t* __restrict__ dexps, double* __restrict__ dcoef) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= m) return;
  const uint8_t* row = exps + t * n;
  uint8_t* drow = dexps + t * n;
  for (int c = 0; c < n; ++c) drow[c] = row[c];
  const int a = row[v];
  if (a > 0) {
    drow[v] = (uint8_t)(a - 1);
    dcoef[t] = (double)a * coef[t];
  } else {
    dcoef[t] = 0.0;
  }
}

}  // namespace

}  // namespace polylab

using namespace polylab;

extern "C" {

polylab_status polylab_pow(const polylab_poly* p, int32_t k, double zeroprec, polylab_poly_out* out,
                           polylab_alloc_fn alloc, void* alloc_ctx, polylab_stream stream) {
  if (!p || !out || !alloc || !out->var_ids || k < 0 || !(zeroprec >= 0.0)) return POLYLAB_ERR_INVALID_ARG;
  PL_TRY(check_poly(p));
  cudaStream_t s = (cudaStream_t)stream;
  Scratch scr(s);
  if (k == 0) {  // the constant 1 over p's variables
    Owned one;
    one.ids.assign(p->var_ids, p->var_ids + p->n_vars);
    one.m = 1.0 > zeroprec ? 1 : 0;
    if (one.m) {
      PL_TRY(scr.get(&one.exps, (size_t)p->n_vars));
      PL_TRY(scr.get(&one.coef, 1));
      PL_CUDA(cudaMemsetAsync(one.exps, 0, (size_t)p->n_vars, s));
      const double c1 = 1.0;
      PL_CUDA(cudaMemcpyAsync(one.coef, &c1, sizeof(double), cudaMemcpyHostToDevice, s));
      PL_CUDA(cudaStreamSynchronize(s));  // c1 lives on this stack frame
    }
    return copy_out(one, out, alloc, alloc_ctx, s);
  }
  // binary exponentiation: base = p^(2^i), acc = product of the bases of k's set bits
  Owned base, acc;
  bool have_acc = false;
  PL_TRY(run_engine(p, nullptr, kSimplifyMode, zeroprec, scr, s, &base));
  for (int32_t e = k;;) {
    if (e & 1) {
      if (!have_acc) {
        acc = base;
        have_acc = true;
      } else {
        const polylab_poly av = acc.view(), bv = base.view();
        Owned nxt;
        PL_TRY(run_engine(&av, &bv, kMulMode, zeroprec, scr, s, &nxt));
        acc = nxt;
      }
    }
    e >>= 1;
    if (!e) break;
    const polylab_poly bv = base.view();
    Owned sq;
    PL_TRY(run_engine(&bv, &bv, kMulMode, zeroprec, scr, s, &sq));
    base = sq;
  }
  return copy_out(acc, out, alloc, alloc_ctx, s);
}

polylab_status polylab_diff(const polylab_poly* p, uint64_t var_id, double zeroprec, polylab_poly_out* out,
                            polylab_alloc_fn alloc, void* alloc_ctx, polylab_stream stream) {
  if (!p || !out || !alloc || !out->var_ids || !(zeroprec >= 0.0)) return POLYLAB_ERR_INVALID_ARG;
  PL_TRY(check_poly(p));
  cudaStream_t s = (cudaStream_t)stream;
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
  double* dcoef;
  PL_TRY(scr.get(&dexps, (size_t)p->n_terms * p->n_vars));
  PL_TRY(scr.get(&dcoef, (size_t)p->n_terms));
  diff_terms<<<(unsigned)ceil_div(p->n_terms, 256), 256, 0, s>>>(p->exps, p->coef, p->n_terms, p->n_vars, v, dexps,
                                                                 dcoef);
  PL_TRY(launch_status("diff_terms"));
  polylab_poly d = *p;
  d.exps = dexps;
  d.coef = dcoef;
  return engine(&d, nullptr, kSimplifyMode, zeroprec, out, alloc, alloc_ctx, s);
}

}  // extern "C"
