// Host side of batched exact affine-normal launches: descriptors, work order,
// configuration and the project's autotuner, plus the public batch API.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>

#include "batch.cuh"

namespace polylab {

polylab_status exact_batch_upload_order(ExactBatch* b, cudaStream_t s) {
  const int n = b->n_desc;
  std::vector<int>& ord = b->host_order;
  ord.resize(n);
  std::iota(ord.begin(), ord.end(), 0);
  if (b->cfg.order == 1) {
    std::vector<double> cost(n);
    for (int i = 0; i < n; ++i) cost[i] = exact_point_cost(b->host_descs[i], b->host_descs[i].max_support);
    std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return cost[x] > cost[y]; });
  }
  b->host_prefix.assign(n + 1, 0);
  for (int i = 0; i < n; ++i) b->host_prefix[i + 1] = b->host_prefix[i] + b->host_descs[ord[i]].P;
  b->total = b->host_prefix[n];
  // the split frame stage's own order: n descending (its cost is set by n)
  std::vector<int>& ford = b->host_forder;
  ford.resize(n);
  std::iota(ford.begin(), ford.end(), 0);
  std::stable_sort(ford.begin(), ford.end(),
                   [&](int x, int y) { return b->host_descs[x].n > b->host_descs[y].n; });
  b->host_fprefix.assign(n + 1, 0);
  for (int i = 0; i < n; ++i) b->host_fprefix[i + 1] = b->host_fprefix[i] + b->host_descs[ford[i]].P;
  exact_frame_classes(b);
  PL_CUDA(cudaMemcpyAsync(b->order, ord.data(), n * sizeof(int), cudaMemcpyHostToDevice, s));
  PL_CUDA(cudaMemcpyAsync(b->prefix, b->host_prefix.data(), (n + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  PL_CUDA(cudaMemcpyAsync(b->forder, ford.data(), n * sizeof(int), cudaMemcpyHostToDevice, s));
  PL_CUDA(cudaMemcpyAsync(b->fprefix, b->host_fprefix.data(), (n + 1) * sizeof(int64_t), cudaMemcpyHostToDevice,
                          s));
  PL_CUDA(cudaStreamSynchronize(s));  // host vectors may change after this returns
  return POLYLAB_OK;
}

// Classes of the split frame stage: n > 40 with the configured CTA size,
// 24 < n <= 40 and n <= 24 with 64 threads (a point's factorisation has
// little parallel work there, and smaller CTAs with smaller shared memory
// keep more points in flight per SM).  Each class is a contiguous range of
// the frame order; its shared memory is the largest need among its members.
void exact_frame_classes(ExactBatch* b) {
  const int bounds[kFrameClasses + 1] = {1 << 30, 40, 24, 0};
  const int n = b->n_desc;
  int i = 0;
  for (int c = 0; c < kFrameClasses; ++c) {
    FrameClass& fc = b->fclass[c];
    fc.n_hi = bounds[c];
    fc.n_lo = bounds[c + 1];
    fc.threads = c == 0 ? b->cfg.threads : 64;
    fc.smem = 0;
    fc.tsmem = 0;
    fc.tsmem1 = 0;
    fc.t3smem = 0;
    fc.begin = b->host_fprefix.empty() ? 0 : b->host_fprefix[i];
    while (i < n && b->host_descs[b->host_forder[i]].n > fc.n_lo) {
      const size_t d = (size_t)b->host_forder[i];
      fc.smem = std::max(fc.smem, d < b->frame_need.size() ? b->frame_need[d] : 0);
      fc.tsmem = std::max(fc.tsmem, d < b->terms_need.size() ? b->terms_need[d] : 0);
      fc.tsmem1 = std::max(fc.tsmem1, d < b->terms_need1.size() ? b->terms_need1[d] : 0);
      fc.t3smem = std::max(fc.t3smem, d < b->third_need.size() ? b->third_need[d] : 0);
      ++i;
    }
    fc.end = b->host_fprefix.empty() ? 0 : b->host_fprefix[i];
  }
}

static int default_threads(const ExactBatch* b) {
  int nmax = 1;
  for (const auto& d : b->host_descs) nmax = std::max(nmax, d.n);
  return nmax <= 16 ? 64 : nmax <= 48 ? 128 : 256;
}

polylab_status exact_batch_init(ExactBatch* b, int n, const polylab_plan* const* plans, const double* const* X,
                                const int64_t* P, const polylab_an_opts* o, double* const* D,
                                double* const* Dunit, polylab_an_info* const* info, cudaStream_t s) {
  b->opts = *o;
  b->n_desc = n;
  b->host_descs.resize(n);
  for (int i = 0; i < n; ++i) {
    const polylab_plan* pl = plans[i];
    if (!pl || P[i] < 0 || (P[i] > 0 && (!X[i] || !D[i]))) return POLYLAB_ERR_INVALID_ARG;
    ExactDesc& d = b->host_descs[i];
    d.terms = pl->terms;
    d.m = pl->m;
    d.n = pl->n;
    d.E = std::max(1, pl->max_exp);
    d.max_support = pl->max_support;
    for (int k = 0; k < kMaxSupport + 2; ++k) d.koff[k] = pl->koff[k];
    for (int k = 0; k < kMaxSupport + 1; ++k) d.k3off[k] = pl->k3off[k];
    d.gather = pl->gather;
    d.gather_chunk = pl->gather_chunk;
    d.n_gchunks = pl->n_gchunks;
    {
      // monomial values c x^a, their partial products and 1/x stay normal:
      // |x|^deg within [1e-30, 1e30] (FP32 sums), [1e-25, 1e25] (double words,
      // whose low word is ~2^-24 of the high one) or [1e-280, 1e280] (FP64)
      const double lim = o->prec == POLYLAB_FP32 ? 30.0 : o->prec == POLYLAB_F32X2 ? 25.0 : 280.0;
      const double deg = std::max(1, pl->max_degree);
      d.x_lo = std::pow(10.0, -lim / deg);
      d.x_hi = std::pow(10.0, lim / deg);
    }
    d.mats_in_smem = 1;
    d.X = X[i];
    d.P = P[i];
    d.D = D[i];
    d.Dunit = Dunit ? Dunit[i] : nullptr;
    d.info = info ? info[i] : nullptr;
  }
  if (b->cfg.threads == 0) b->cfg.threads = default_threads(b);
  if (b->cfg.term_threads == 0) b->cfg.term_threads = 128;
  if (b->cfg.third_threads == 0) b->cfg.third_threads = 128;
  PL_TRY(prepare_exact_batch(b));
  PL_CUDA(cudaMallocAsync(&b->descs, std::max(n, 1) * sizeof(ExactDesc), s));
  PL_CUDA(cudaMallocAsync(&b->order, std::max(n, 1) * sizeof(int), s));
  PL_CUDA(cudaMallocAsync(&b->prefix, (n + 1) * sizeof(int64_t), s));
  PL_CUDA(cudaMallocAsync(&b->counter, 3 * sizeof(int), s));
  PL_CUDA(cudaMallocAsync(&b->forder, std::max(n, 1) * sizeof(int), s));
  PL_CUDA(cudaMallocAsync(&b->fprefix, (n + 1) * sizeof(int64_t), s));
  PL_CUDA(cudaMallocAsync(&b->fcounter, kFrameClasses * sizeof(int), s));
  PL_CUDA(cudaMallocAsync(&b->err, sizeof(int), s));
  PL_CUDA(cudaMemsetAsync(b->err, 0, sizeof(int), s));
  PL_CUDA(cudaMallocAsync(&b->ws_h, std::max<size_t>(b->ws_mat_bytes, 16), s));
  PL_CUDA(cudaMallocAsync(&b->ws_w, std::max<size_t>(b->ws_mat_bytes, 16), s));
  PL_CUDA(cudaMallocAsync(&b->ws_v, std::max<size_t>(b->ws_vec_bytes, 16), s));
  PL_CUDA(cudaMemcpyAsync(b->descs, b->host_descs.data(), n * sizeof(ExactDesc), cudaMemcpyHostToDevice, s));
  PL_TRY(exact_batch_upload_order(b, s));
  if (b->gws_stride > 0) {
    // enough workspace for the largest grid any configuration may launch
    b->gws_bytes = (size_t)num_sms() * 32 * b->gws_stride;
    PL_CUDA(cudaMallocAsync(&b->gws, b->gws_bytes, s));
  }
  {  // passes of the term sweep left to its term-by-term launch: at most one per pair of points (pairs
     // start afresh in each class of n) plus one per polynomial (a pass never spans two)
    int64_t points = 0;
    for (int i = 0; i < n; ++i) points += P[i];
    const int64_t cap = points / 2 + n + 2 + kFrameClasses;
    if (cap > INT32_MAX) return POLYLAB_ERR_UNSUPPORTED;
    b->tfb_cap = cap;
    PL_CUDA(cudaMallocAsync(&b->tfb, (size_t)cap * 2 * sizeof(int64_t), s));
    PL_CUDA(cudaMallocAsync(&b->tfb_ctl, (2 + kFrameClasses) * sizeof(int), s));
  }
  return POLYLAB_OK;
}

// Shared-memory layout depends on the CTA size: recompute it, re-upload the
// descriptors and grow the global workspace when needed.
polylab_status exact_batch_relayout(ExactBatch* b, cudaStream_t s) {
  PL_TRY(prepare_exact_batch(b));
  exact_frame_classes(b);
  PL_CUDA(cudaMemcpyAsync(b->descs, b->host_descs.data(), b->n_desc * sizeof(ExactDesc), cudaMemcpyHostToDevice, s));
  const size_t need = (size_t)num_sms() * 32 * b->gws_stride;
  if (need > b->gws_bytes) {
    if (b->gws) PL_CUDA(cudaFreeAsync(b->gws, s));
    b->gws = nullptr;
    PL_CUDA(cudaMallocAsync(&b->gws, need, s));
    b->gws_bytes = need;
  }
  PL_CUDA(cudaStreamSynchronize(s));
  return POLYLAB_OK;
}

void exact_batch_release(ExactBatch* b, cudaStream_t s) {
  if (b->descs) cudaFreeAsync(b->descs, s);
  if (b->order) cudaFreeAsync(b->order, s);
  if (b->prefix) cudaFreeAsync(b->prefix, s);
  if (b->counter) cudaFreeAsync(b->counter, s);
  if (b->forder) cudaFreeAsync(b->forder, s);
  if (b->fprefix) cudaFreeAsync(b->fprefix, s);
  if (b->fcounter) cudaFreeAsync(b->fcounter, s);
  b->forder = nullptr;
  b->fprefix = nullptr;
  b->fcounter = nullptr;
  if (b->gws) cudaFreeAsync(b->gws, s);
  if (b->err) cudaFreeAsync(b->err, s);
  if (b->tfb) cudaFreeAsync(b->tfb, s);
  if (b->tfb_ctl) cudaFreeAsync(b->tfb_ctl, s);
  b->tfb = nullptr;
  b->tfb_ctl = nullptr;
  b->err = nullptr;
  if (b->ws_h) cudaFreeAsync(b->ws_h, s);
  if (b->ws_w) cudaFreeAsync(b->ws_w, s);
  if (b->ws_v) cudaFreeAsync(b->ws_v, s);
  b->ws_h = b->ws_w = b->ws_v = nullptr;
  for (polylab_plan* p : b->owned_plans) polylab_plan_destroy(p, (polylab_stream)s);
  b->descs = nullptr;
  b->order = nullptr;
  b->prefix = nullptr;
  b->counter = nullptr;
  b->gws = nullptr;
  b->owned_plans.clear();
}

}  // namespace polylab

using namespace polylab;

extern "C" {

polylab_status polylab_batch_create(int32_t n_polys, const polylab_poly* polys, const polylab_plan* const* plans,
                                    const double* const* X, const int64_t* P, const polylab_an_opts* opts,
                                    double* const* D, double* const* Dunit, polylab_an_info* const* info,
                                    polylab_stream stream, polylab_batch** out) {
  if (!out || n_polys < 0 || !opts || (n_polys > 0 && (!X || !P || !D))) return POLYLAB_ERR_INVALID_ARG;
  if (n_polys > 0 && !polys && !plans) return POLYLAB_ERR_INVALID_ARG;
  if (opts->method != POLYLAB_MF_EXACT) return POLYLAB_ERR_UNSUPPORTED;
  if (opts->prec != POLYLAB_FP64 && opts->prec != POLYLAB_FP32 && opts->prec != POLYLAB_F32X2)
    return POLYLAB_ERR_INVALID_ARG;
  if (!(opts->regularization >= 0.0)) return POLYLAB_ERR_INVALID_ARG;
  *out = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  polylab_batch* h = new polylab_batch();
  std::vector<const polylab_plan*> use(n_polys);
  polylab_status st = POLYLAB_OK;
  for (int i = 0; i < n_polys && st == POLYLAB_OK; ++i) {
    use[i] = plans ? plans[i] : nullptr;
    if (!use[i]) {
      polylab_plan* tmp = nullptr;
      st = polylab_plan_create(polys ? &polys[i] : nullptr, POLYLAB_PLAN_TERMS, stream, &tmp);
      if (st == POLYLAB_OK) {
        h->b.owned_plans.push_back(tmp);
        use[i] = tmp;
      }
    } else if (polys && (polys[i].n_vars != use[i]->n || polys[i].n_terms != use[i]->m)) {
      st = POLYLAB_ERR_INVALID_ARG;
    }
  }
  if (st == POLYLAB_OK) st = exact_batch_init(&h->b, n_polys, use.data(), X, P, opts, D, Dunit, info, s);
  if (st != POLYLAB_OK) {
    exact_batch_release(&h->b, s);
    delete h;
    return st;
  }
  *out = h;
  return POLYLAB_OK;
}

polylab_status polylab_batch_run(polylab_batch* b, polylab_stream stream) {
  if (!b) return POLYLAB_ERR_INVALID_ARG;
  return run_exact_batch(&b->b, (cudaStream_t)stream);
}

polylab_status polylab_batch_run_stage(polylab_batch* b, int32_t stage, polylab_stream stream) {
  if (!b || stage < 0 || stage > 2) return POLYLAB_ERR_INVALID_ARG;
  return run_exact_stage(&b->b, stage, (cudaStream_t)stream);
}

polylab_status polylab_batch_check(polylab_batch* b, polylab_stream stream) {
  if (!b) return POLYLAB_ERR_INVALID_ARG;
  int flag = 0;
  PL_CUDA(cudaMemcpyAsync(&flag, b->b.err, sizeof(int), cudaMemcpyDeviceToHost, (cudaStream_t)stream));
  PL_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  if (!flag) return POLYLAB_OK;
  char msg[96];
  if (flag == 4)
    snprintf(msg, sizeof(msg), "the term sweep's list of term-by-term passes overflowed");
  else
    snprintf(msg, sizeof(msg), "a bounded wait of the %s stage expired",
             flag == 2 ? "frame" : flag == 3 ? "third-derivative" : "batch");
  set_last_message(msg);
  PL_CUDA(cudaMemsetAsync(b->b.err, 0, sizeof(int), (cudaStream_t)stream));  // the batch may run again
  PL_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  if (flag == 4) return POLYLAB_ERR_UNSUPPORTED;
  return POLYLAB_ERR_TIMEOUT;
}

polylab_status polylab_batch_get_config(const polylab_batch* b, polylab_batch_config* cfg) {
  if (!b || !cfg) return POLYLAB_ERR_INVALID_ARG;
  cfg->threads = b->b.cfg.threads;
  cfg->ctas_per_sm = b->b.cfg.ctas_per_sm;
  cfg->order = b->b.cfg.order;
  cfg->term_threads = b->b.cfg.term_threads;
  cfg->terms_ctas = b->b.cfg.terms_ctas;
  cfg->third_ctas = b->b.cfg.third_ctas;
  cfg->frame_split = b->b.cfg.frame_split;
  cfg->third_threads = b->b.cfg.third_threads;
  cfg->third_split = b->b.cfg.third_split;
  return POLYLAB_OK;
}

polylab_status polylab_batch_set_config(polylab_batch* b, const polylab_batch_config* cfg, polylab_stream stream) {
  if (!b || !cfg) return POLYLAB_ERR_INVALID_ARG;
  auto ok_threads = [](int t) { return t == 64 || t == 128 || t == 256; };
  if (!ok_threads(cfg->threads) || !ok_threads(cfg->term_threads) || !ok_threads(cfg->third_threads))
    return POLYLAB_ERR_INVALID_ARG;
  auto ok_cap = [](int c) { return c >= 0 && c <= 32; };
  if (!ok_cap(cfg->ctas_per_sm) || !ok_cap(cfg->terms_ctas) || !ok_cap(cfg->third_ctas) ||
      (cfg->order != 0 && cfg->order != 1) ||
      (cfg->frame_split != 0 && cfg->frame_split != 1) || cfg->third_split < 1 || cfg->third_split > 4)
    return POLYLAB_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const bool reorder = cfg->order != b->b.cfg.order;
  b->b.cfg.terms_ctas = cfg->terms_ctas;
  b->b.cfg.third_ctas = cfg->third_ctas;
  b->b.cfg.frame_split = cfg->frame_split;
  b->b.cfg.third_split = cfg->third_split;
  const bool relayout = cfg->threads != b->b.cfg.threads || cfg->term_threads != b->b.cfg.term_threads ||
                        cfg->third_threads != b->b.cfg.third_threads;
  b->b.cfg.third_threads = cfg->third_threads;
  b->b.cfg.threads = cfg->threads;
  b->b.cfg.term_threads = cfg->term_threads;
  b->b.cfg.ctas_per_sm = cfg->ctas_per_sm;
  b->b.cfg.order = cfg->order;
  if (relayout) PL_TRY(exact_batch_relayout(&b->b, s));
  if (reorder) PL_TRY(exact_batch_upload_order(&b->b, s));
  return POLYLAB_OK;
}

polylab_status polylab_batch_autotune(polylab_batch* b, int32_t reps, polylab_stream stream,
                                      polylab_batch_config* chosen, float* best_ms) {
  if (!b || reps < 1) return POLYLAB_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  ExactBatch* eb = &b->b;
  polylab_batch_config cur{eb->cfg.threads,    eb->cfg.ctas_per_sm, eb->cfg.order,
                           eb->cfg.term_threads, eb->cfg.terms_ctas,  eb->cfg.third_ctas,
                           eb->cfg.frame_split,  eb->cfg.third_threads, eb->cfg.third_split};
  cur.terms_ctas = 0;
  cur.third_ctas = 0;
  cudaEvent_t e0, e1;
  PL_CUDA(cudaEventCreate(&e0));
  PL_CUDA(cudaEventCreate(&e1));
  // mean time of `reps` runs of stages [s0, s1] after one warm-up run
  auto time_stages = [&](int s0, int s1, float* ms_out) -> polylab_status {
    for (int r = 0; r <= reps; ++r) {
      if (r == 1) cudaEventRecord(e0, s);
      if (s0 == 0 && s1 == 2) PL_TRY(run_exact_batch(eb, s));
      else
        for (int st = s0; st <= s1; ++st) PL_TRY(run_exact_stage(eb, st, s));
    }
    cudaEventRecord(e1, s);
    PL_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    *ms_out = ms / reps;
    return POLYLAB_OK;
  };
  // try `c` on stages [s0, s1]; configurations a stage cannot run are skipped
  auto trial = [&](const polylab_batch_config& c, int s0, int s1, float* ms) -> polylab_status {
    *ms = 1e30f;
    polylab_status st = polylab_batch_set_config(b, &c, stream);
    if (st == POLYLAB_OK) st = time_stages(s0, s1, ms);
    if (st == POLYLAB_ERR_UNSUPPORTED) {
      *ms = 1e30f;
      return POLYLAB_OK;
    }
    return st;
  };
  polylab_status st = polylab_batch_set_config(b, &cur, stream);
  if (st == POLYLAB_OK) st = run_exact_batch(eb, s);  // every stage's inputs exist from here on
  float best_t = 1e30f, t = 0.f;
  // 1. CTA sizes of the two term sweeps, each timed over its own stage
  for (int sweep = 0; sweep < 2 && st == POLYLAB_OK; ++sweep) {
    polylab_batch_config best = cur;
    best_t = 1e30f;
    for (int tt : {64, 128, 256}) {
      polylab_batch_config c = cur;
      (sweep == 0 ? c.term_threads : c.third_threads) = tt;
      if ((st = trial(c, 2 * sweep, 2 * sweep, &t)) != POLYLAB_OK) break;
      if (t < best_t) {
        best_t = t;
        best = c;
      }
    }
    cur = best;
  }
  // 1b. launches of the third-derivative sweep
  if (st == POLYLAB_OK) {
    polylab_batch_config best = cur;
    best_t = 1e30f;
    for (int sp : {1, 2, 3}) {
      polylab_batch_config c = cur;
      c.third_split = sp;
      if ((st = trial(c, 2, 2, &t)) != POLYLAB_OK) break;
      if (t < best_t) {
        best_t = t;
        best = c;
      }
    }
    cur = best;
  }
  // 2. CTA size and residency cap of the frame stage
  if (st == POLYLAB_OK) {
    polylab_batch_config best = cur;
    best_t = 1e30f;
    for (int split : {1, 0}) {
      for (int threads : {64, 128, 256}) {
        for (int cap : {0, 2, 4}) {
          polylab_batch_config c = cur;
          c.frame_split = split;
          c.threads = threads;
          c.ctas_per_sm = cap;
          if ((st = trial(c, 1, 1, &t)) != POLYLAB_OK) break;
          if (t < best_t) {
            best_t = t;
            best = c;
          }
        }
        if (st != POLYLAB_OK) break;
      }
      if (st != POLYLAB_OK) break;
    }
    cur = best;
  }
  // 3. work order, timed over the whole run
  if (st == POLYLAB_OK) {
    polylab_batch_config best = cur;
    best_t = 1e30f;
    for (int order : {1, 0}) {
      polylab_batch_config c = cur;
      c.order = order;
      if ((st = trial(c, 0, 2, &t)) != POLYLAB_OK) break;
      if (t < best_t) {
        best_t = t;
        best = c;
      }
    }
    cur = best;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  PL_TRY(st);
  if (best_t >= 1e30f) return POLYLAB_ERR_UNSUPPORTED;
  PL_TRY(polylab_batch_set_config(b, &cur, stream));
  if (chosen) *chosen = cur;
  if (best_ms) *best_ms = best_t;
  return POLYLAB_OK;
}

polylab_status polylab_batch_destroy(polylab_batch* b, polylab_stream stream) {
  if (!b) return POLYLAB_OK;
  exact_batch_release(&b->b, (cudaStream_t)stream);
  delete b;
  return launch_status("polylab_batch_destroy");
}

polylab_status polylab_affine_normal_batched(int32_t n_polys, const polylab_poly* polys,
                                             const polylab_plan* const* plans, const double* const* X,
                                             const int64_t* P, const polylab_an_opts* opts, double* const* D,
                                             double* const* Dunit, polylab_an_info* const* info,
                                             polylab_stream stream) {
  polylab_batch* b = nullptr;
  PL_TRY(polylab_batch_create(n_polys, polys, plans, X, P, opts, D, Dunit, info, stream, &b));
  const polylab_status st = polylab_batch_run(b, stream);
  polylab_batch_destroy(b, stream);
  return st;
}

}  // extern "C"
