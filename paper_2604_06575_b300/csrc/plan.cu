// Plans: the device-resident term list of a polynomial, status strings and
// argument checks shared by every entry point.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <unordered_set>
#include <mutex>
#include <vector>

#include "common.cuh"

namespace polylab {

static thread_local char g_last_error[512] = "";

void set_last_error(const char* where, cudaError_t e) {
  snprintf(g_last_error, sizeof(g_last_error), "%s: %s (%s)", where, cudaGetErrorString(e), cudaGetErrorName(e));
}

void set_last_message(const char* msg) { snprintf(g_last_error, sizeof(g_last_error), "%s", msg); }

cudaMemPool_t scratch_pool() {
  static std::mutex mu;
  static std::vector<cudaMemPool_t> pools;  // by device ordinal
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  std::lock_guard<std::mutex> lock(mu);
  if ((int)pools.size() <= dev) pools.resize(dev + 1, nullptr);
  if (!pools[dev]) {
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;  // (the caller falls back to the device's default pool)
    }
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    pools[dev] = pool;
  }
  return pools[dev];
}

int num_sms() {
  static int cached = 0;
  if (!cached) {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    cached = v > 0 ? v : 148;
  }
  return cached;
}

// One warp per term: scan the exponent row, keep the nonzero entries in
// column order.  stats[0] = max exponent, stats[1] = max support.
template <typename C>
__global__ void pack_terms_kernel(const uint8_t* __restrict__ exps, const C* __restrict__ coef, int64_t m,
                                  int n, Term* __restrict__ terms, int* __restrict__ stats) {
  __shared__ Term stage[8];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t t = (int64_t)blockIdx.x * 8 + wib;
  if (t >= m) return;
  Term& st = stage[wib];
  if (lane < kMaxSupport) {
    st.var[lane] = 0;
    st.exp[lane] = 0;
  }
  __syncwarp();
  const uint8_t* row = exps + t * (int64_t)n;
  int count = 0, maxe = 0;
  for (int base = 0; base < n; base += 32) {
    const int j = base + lane;
    const int e = j < n ? row[j] : 0;
    const unsigned mask = __ballot_sync(0xffffffffu, e != 0);
    if (e) {
      const int pos = count + __popc(mask & ((1u << lane) - 1u));
      if (pos < kMaxSupport) {
        st.var[pos] = (uint16_t)j;
        st.exp[pos] = (uint8_t)e;
      }
    }
    count += __popc(mask);
    maxe = max(maxe, e);
  }
  for (int o = 16; o; o >>= 1) maxe = max(maxe, __shfl_xor_sync(0xffffffffu, maxe, o));
  __syncwarp();
  if (lane == 0) {
    st.coef = coef[t];
    terms[t] = st;
    atomicMax(&stats[0], maxe);
    atomicMax(&stats[1], count);
  }
}

// Group boundaries of a term list sorted by (support size, degree).
static void group_offsets(const std::vector<Term>& host, polylab_plan* plan) {
  const int64_t m = (int64_t)host.size();
  std::vector<int> ks(m), ds(m);
  for (int64_t t = 0; t < m; ++t) {
    int k = 0, d = 0;
    for (int q = 0; q < kMaxSupport; ++q) {
      k += host[t].exp[q] != 0;
      d += host[t].exp[q];
    }
    ks[t] = k;
    ds[t] = d;
  }
  int64_t t = 0;
  for (int k = 0; k <= kMaxSupport; ++k) {
    plan->koff[k] = t;
    while (t < m && ks[t] == k && ds[t] < 3) ++t;
    plan->k3off[k] = t;
    while (t < m && ks[t] == k) ++t;
  }
  plan->koff[kMaxSupport + 1] = m;
}

// Gather form of the gradient/Hessian sweep.  With m_t = c_t prod_s x_s^a_s,
//   d_i m_t = a_i m_t / x_i,   d_ij m_t = a_i a_j m_t / (x_i x_j),
//   d_ii m_t = a_i (a_i - 1) m_t / x_i^2,
// so each entry of g and H is (1/x_i)(1/x_j) sum_t coef_t m_t over the terms
// that touch it.  The records of every chunk of kGatherChunk terms are sorted
// by entry, so a sweep sums runs of equal entries in registers.
static polylab_status build_gather(const std::vector<Term>& host, int n, cudaStream_t s, polylab_plan* plan) {
  const int64_t m = (int64_t)host.size();
  int maxdeg = 0;
  for (const Term& t : host) {
    int d = 0;
    for (int q = 0; q < kMaxSupport; ++q) d += t.exp[q];
    maxdeg = std::max(maxdeg, d);
  }
  plan->max_degree = maxdeg;
  if (n > 127 || m == 0) return POLYLAB_OK;
  struct Rec {
    uint64_t key;  // chunk << 48 | entry << 32 | term
    uint32_t coef;
  };
  std::vector<Rec> recs;
  recs.reserve((size_t)m * 8);
  const uint64_t nn = (uint64_t)n * n;
  for (int64_t t = 0; t < m; ++t) {
    const Term& tm = host[t];
    const uint64_t chunk = (uint64_t)(t / kGatherChunk);
    auto add = [&](uint64_t entry, uint32_t coef) {
      recs.push_back({chunk << 48 | entry << 32 | (uint64_t)t, coef});
    };
    for (int a = 0; a < kMaxSupport; ++a) {
      const uint32_t ea = tm.exp[a];
      if (!ea) continue;
      const uint64_t va = tm.var[a];
      add(nn + va, ea);
      if (ea >= 2) add(va * n + va, ea * (ea - 1));
      for (int b = a + 1; b < kMaxSupport; ++b)
        if (tm.exp[b]) add(va * n + tm.var[b], ea * tm.exp[b]);
    }
  }
  for (const Rec& r : recs)
    if (r.coef > 127) return POLYLAB_OK;  // no gather form: coefficients beyond 7 bits
  std::sort(recs.begin(), recs.end(), [](const Rec& x, const Rec& y) { return x.key < y.key; });
  const int nch = (int)((m + kGatherChunk - 1) / kGatherChunk);
  // sorted record range of every chunk
  std::vector<int64_t> sorted_off(nch + 1, (int64_t)recs.size());
  sorted_off[0] = 0;
  for (int c = 0, q = 0; q < (int)recs.size(); ++q) {
    const int ch = (int)(recs[q].key >> 48);
    while (c < ch) sorted_off[++c] = q;
  }
  // interleaved streams: chunk c holds L_c * S records, record k of stream s
  // at k * S + s, stream s = sorted records [s L_c, (s+1) L_c) of the chunk
  constexpr int S = kGatherStreams;
  std::vector<int64_t> off(nch + 1, 0);
  for (int c = 0; c < nch; ++c) {
    const int64_t len = sorted_off[c + 1] - sorted_off[c];
    const int64_t L = (len + S - 1) / S;
    off[c + 1] = off[c] + (L + kGatherUnroll - 1) / kGatherUnroll * kGatherUnroll * S;
  }
  std::vector<uint32_t> dev((size_t)off[nch], kGatherPad << 11);
  for (int c = 0; c < nch; ++c) {
    const int64_t len = sorted_off[c + 1] - sorted_off[c], L = (off[c + 1] - off[c]) / S;
    for (int64_t q = 0; q < len; ++q) {
      const Rec& r = recs[(size_t)(sorted_off[c] + q)];
      const int64_t Ls = (len + S - 1) / S;  // records per stream before padding
      const int64_t s_ = q / Ls, k = q - s_ * Ls;
      const uint32_t t_local = (uint32_t)((r.key & 0xffffffffu) - (uint64_t)c * kGatherChunk);
      const uint32_t entry = (uint32_t)((r.key >> 32) & 0xffffu);
      dev[(size_t)(off[c] + k * S + s_)] = t_local | entry << 11 | r.coef << 25;
    }
  }
  PL_CUDA(cudaMallocAsync(&plan->gather, std::max<size_t>(dev.size(), 1) * sizeof(uint32_t), s));
  PL_CUDA(cudaMallocAsync(&plan->gather_chunk, (nch + 1) * sizeof(int64_t), s));
  PL_CUDA(cudaMemcpyAsync(plan->gather, dev.data(), dev.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, s));
  PL_CUDA(cudaMemcpyAsync(plan->gather_chunk, off.data(), (nch + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  PL_CUDA(cudaStreamSynchronize(s));  // host vectors go out of scope
  plan->n_gchunks = nch;
  return POLYLAB_OK;
}

polylab_status ensure_hessian_pattern(polylab_plan* plan, cudaStream_t s) {
  if (plan->hrow) return POLYLAB_OK;
  const int64_t m = plan->m;
  const int n = plan->n;
  std::vector<Term> host((size_t)m);
  if (m > 0) {
    PL_CUDA(cudaMemcpyAsync(host.data(), plan->terms, m * sizeof(Term), cudaMemcpyDeviceToHost, s));
    PL_CUDA(cudaStreamSynchronize(s));
  }
  std::vector<uint64_t> keys;
  keys.reserve((size_t)n + (size_t)m * 16);
  for (int i = 0; i < n; ++i) keys.push_back((uint64_t)i << 32 | (uint64_t)i);
  for (const Term& t : host)
    for (int a = 0; a < kMaxSupport; ++a)
      for (int b = 0; b < kMaxSupport; ++b)
        if (t.exp[a] && t.exp[b] && a != b) keys.push_back((uint64_t)t.var[a] << 32 | t.var[b]);
  std::sort(keys.begin(), keys.end());
  keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
  if (keys.size() > 0x7fffffffu) return POLYLAB_ERR_UNSUPPORTED;
  std::vector<int32_t> row(n + 1, 0), col(keys.size());
  for (size_t q = 0; q < keys.size(); ++q) {
    row[(keys[q] >> 32) + 1] += 1;
    col[q] = (int32_t)(keys[q] & 0xffffffffu);
  }
  for (int i = 0; i < n; ++i) row[i + 1] += row[i];
  std::vector<int32_t> pos;
  int64_t base = 0;
  for (int K = 0; K <= kMaxSupport; ++K) {
    plan->hbase[K] = base;
    for (int64_t t = plan->koff[K]; t < plan->koff[K + 1]; ++t) {
      int var[kMaxSupport], k = 0;
      for (int q = 0; q < kMaxSupport; ++q)
        if (host[t].exp[q]) var[k++] = host[t].var[q];
      for (int a = 0; a < K; ++a)
        for (int b = 0; b < K; ++b) {
          const uint64_t key = (uint64_t)var[a] << 32 | (uint64_t)var[b];
          pos.push_back((int32_t)(std::lower_bound(keys.begin(), keys.end(), key) - keys.begin()));
        }
    }
    base = (int64_t)pos.size();
  }
  PL_CUDA(cudaMallocAsync(&plan->hrow, (n + 1) * sizeof(int32_t), s));
  PL_CUDA(cudaMallocAsync(&plan->hcol, std::max<size_t>(col.size(), 1) * sizeof(int32_t), s));
  PL_CUDA(cudaMallocAsync(&plan->hpos, std::max<size_t>(pos.size(), 1) * sizeof(int32_t), s));
  PL_CUDA(cudaMemcpyAsync(plan->hrow, row.data(), (n + 1) * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  PL_CUDA(cudaMemcpyAsync(plan->hcol, col.data(), col.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  PL_CUDA(cudaMemcpyAsync(plan->hpos, pos.data(), pos.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  PL_CUDA(cudaStreamSynchronize(s));
  plan->hnnz = (int64_t)col.size();
  return POLYLAB_OK;
}

template <typename C>
polylab_status build_term_plan(const PolyIn<C>* p, cudaStream_t s, polylab_plan* plan) {
  PL_TRY(check_poly(p));
  if (p->n_vars > 65535) return POLYLAB_ERR_UNSUPPORTED;
  plan->n = p->n_vars;
  plan->m = p->n_terms;
  int* stats = nullptr;
  PL_CUDA(cudaMallocAsync(&stats, 2 * sizeof(int), s));
  PL_CUDA(cudaMemsetAsync(stats, 0, 2 * sizeof(int), s));
  PL_CUDA(cudaMallocAsync(&plan->terms, std::max<int64_t>(p->n_terms, 1) * sizeof(Term), s));
  if (p->n_terms > 0) {
    pack_terms_kernel<C><<<(unsigned)ceil_div(p->n_terms, 8), 256, 0, s>>>(p->exps, p->coef, p->n_terms, p->n_vars,
                                                                          plan->terms, stats);
    PL_TRY(launch_status("pack_terms_kernel"));
  }
  int h[2] = {0, 0};
  PL_CUDA(cudaMemcpyAsync(h, stats, sizeof(h), cudaMemcpyDeviceToHost, s));
  PL_CUDA(cudaFreeAsync(stats, s));
  PL_CUDA(cudaStreamSynchronize(s));
  plan->max_exp = h[0];
  plan->max_support = h[1];
  if (h[1] > kMaxSupport) return POLYLAB_ERR_UNSUPPORTED;
  // order the term list by (support size, degree): the per-term kernels branch
  // on the support size, so a warp of consecutive terms then takes one branch
  // and skips low-degree terms together.  Sums are order independent.
  if (p->n_terms > 1) {
    std::vector<Term> host(p->n_terms);
    PL_CUDA(cudaMemcpyAsync(host.data(), plan->terms, p->n_terms * sizeof(Term), cudaMemcpyDeviceToHost, s));
    PL_CUDA(cudaStreamSynchronize(s));
    auto key = [](const Term& t) {
      int k = 0, d = 0;
      for (int q = 0; q < kMaxSupport; ++q) {
        k += t.exp[q] != 0;
        d += t.exp[q];
      }
      return k * 4096 + d;
    };
    std::stable_sort(host.begin(), host.end(), [&](const Term& a, const Term& b) { return key(a) < key(b); });
    PL_CUDA(cudaMemcpyAsync(plan->terms, host.data(), p->n_terms * sizeof(Term), cudaMemcpyHostToDevice, s));
    PL_CUDA(cudaStreamSynchronize(s));
    group_offsets(host, plan);
    PL_TRY(build_gather(host, p->n_vars, s, plan));
  } else {
    std::vector<Term> host(p->n_terms);
    if (p->n_terms > 0) {
      PL_CUDA(cudaMemcpyAsync(host.data(), plan->terms, sizeof(Term), cudaMemcpyDeviceToHost, s));
      PL_CUDA(cudaStreamSynchronize(s));
    }
    group_offsets(host, plan);
    PL_TRY(build_gather(host, p->n_vars, s, plan));
  }
  return POLYLAB_OK;
}

namespace {

template <typename Pub>
polylab_status plan_create(const Pub* p, uint32_t what, polylab_stream stream, polylab_plan** out) {
  if (!out) return POLYLAB_ERR_INVALID_ARG;
  *out = nullptr;
  if (!p || what > POLYLAB_PLAN_GEMM) return POLYLAB_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const auto view = poly_in(*p);
  polylab_plan* plan = new polylab_plan();
  polylab_status st = build_term_plan(&view, s, plan);
  if (st == POLYLAB_OK && (what & POLYLAB_PLAN_GEMM)) st = build_gemm_operand(plan, s);
  if (st != POLYLAB_OK) {
    polylab_plan_destroy(plan, stream);
    return st;
  }
  *out = plan;
  return POLYLAB_OK;
}

}  // namespace

}  // namespace polylab

using namespace polylab;

extern "C" {

const char* polylab_status_string(polylab_status s) {
  switch (s) {
    case POLYLAB_OK: return "POLYLAB_OK";
    case POLYLAB_ERR_INVALID_ARG: return "POLYLAB_ERR_INVALID_ARG";
    case POLYLAB_ERR_EXP_OVERFLOW: return "POLYLAB_ERR_EXP_OVERFLOW";
    case POLYLAB_ERR_DUP_VAR_ID: return "POLYLAB_ERR_DUP_VAR_ID";
    case POLYLAB_ERR_OOM: return "POLYLAB_ERR_OOM";
    case POLYLAB_ERR_CUDA: return "POLYLAB_ERR_CUDA";
    case POLYLAB_ERR_TIMEOUT: return "POLYLAB_ERR_TIMEOUT";
    case POLYLAB_ERR_UNSUPPORTED: return "POLYLAB_ERR_UNSUPPORTED";
  }
  return "POLYLAB_UNKNOWN_STATUS";
}

const char* polylab_last_error(void) { return g_last_error; }

polylab_status polylab_plan_create(const polylab_poly* p, uint32_t what, polylab_stream stream,
                                   polylab_plan** out) {
  return plan_create(p, what, stream, out);
}

polylab_status polylab_plan_create_f32(const polylab_poly_f32* p, uint32_t what, polylab_stream stream,
                                       polylab_plan** out) {
  return plan_create(p, what, stream, out);
}

polylab_status polylab_plan_destroy(polylab_plan* plan, polylab_stream stream) {
  if (!plan) return POLYLAB_OK;
  cudaStream_t s = (cudaStream_t)stream;
  if (plan->terms) cudaFreeAsync(plan->terms, s);
  if (plan->gather) cudaFreeAsync(plan->gather, s);
  if (plan->hrow) cudaFreeAsync(plan->hrow, s);
  if (plan->hcol) cudaFreeAsync(plan->hcol, s);
  if (plan->hpos) cudaFreeAsync(plan->hpos, s);
  if (plan->gather_chunk) cudaFreeAsync(plan->gather_chunk, s);
  if (plan->gemm) free_gemm_operand(plan->gemm, s);
  delete plan;
  return launch_status("polylab_plan_destroy");
}

int64_t polylab_plan_closure_size(const polylab_plan* plan) { return plan ? plan->closure : -1; }

void polylab_an_opts_default(polylab_an_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->method = POLYLAB_MF_EXACT;
  o->regularization = 1e-6;
  o->num_probes = 8;
  o->krylov_tol = 1e-4;
  o->krylov_maxit = 40;
  o->assume_nonzero_x = 0;
  o->seed = 20260321ull;
  o->prec = POLYLAB_FP64;
  o->precond = POLYLAB_PRECOND_JACOBI;
  o->mlp_weights = nullptr;
}

}  // extern "C"
