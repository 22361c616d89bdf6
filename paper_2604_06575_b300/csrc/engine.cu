// simplify and mul (Sec. 2 "simplify"/"mtimes", Sec. 3.2 alignment, Sec. 6.3
// expansion-and-merge workloads) as key generation + LSD radix sort +
// warp-shuffle segmented reduce-by-key + threshold compaction + unpack.
//
// Key = position of the exponent row in Polylab's internal monomial order
// (Sec. 3.1 monolist: graded, then ascending lexicographic order of the
// reversed row).  With S(c, R) = C(R + c, c), the number of monomials of
// degree <= R in c variables, a row alpha of degree d over n variables has
//
//   rank(alpha) = S(n, d-1) + sum_{c = n-1 .. 1} [ S(c, R_c) - S(c, R_c - alpha_c) ],
//   R_c = d - sum_{c' > c} alpha_c'
//
// and only nonzero entries contribute, so a sparse row costs O(support).
// The key therefore needs only ceil(log2 S(n, D)) bits (34 for a product of
// two degree-6 polynomials in 30 variables), and sorting by it emits the
// result in the canonical order directly.  Keys of up to 64 bits sort as
// uint64, up to 128 bits as unsigned __int128.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "common.cuh"
#include "sort.cuh"

namespace polylab {
namespace {

// ------------------------------------------------------- term supports (CSR)
// Supports are stored in DESCENDING merged-column order, the order in which
// the rank formula consumes them.

__global__ void count_support(const uint8_t* __restrict__ exps, int64_t m, int n, uint32_t* __restrict__ cnt,
                              uint32_t* __restrict__ deg, int* __restrict__ maxdeg) {
  const int64_t t = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (t >= m) return;
  const uint8_t* row = exps + t * (int64_t)n;
  uint32_t c = 0, d = 0;
  for (int j = lane; j < n; j += 32) {
    const uint32_t e = row[j];
    c += e != 0;
    d += e;
  }
  for (int o = 16; o; o >>= 1) {
    c += __shfl_xor_sync(0xffffffffu, c, o);
    d += __shfl_xor_sync(0xffffffffu, d, o);
  }
  if (lane == 0) {
    cnt[t] = c;
    deg[t] = d;
    atomicMax(maxdeg, (int)d);
  }
}

// ord[q] = operand column with the q-th smallest merged column; colmap[j] =
// merged column of operand column j.  Entries are emitted for q descending.
__global__ void fill_support(const uint8_t* __restrict__ exps, int64_t m, int n, const int* __restrict__ ord,
                             const int* __restrict__ colmap, const uint32_t* __restrict__ ptr,
                             uint32_t* __restrict__ col, uint8_t* __restrict__ ex) {
  const int64_t t = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (t >= m) return;
  const uint8_t* row = exps + t * (int64_t)n;
  const uint32_t start = ptr[t];
  uint32_t written = 0;
  for (int base = n - 1; base >= 0; base -= 32) {
    const int q = base - lane;
    const int j = q >= 0 ? ord[q] : 0;
    const uint32_t e = q >= 0 ? row[j] : 0u;
    const unsigned mask = __ballot_sync(0xffffffffu, e != 0);
    if (e) {
      const uint32_t pos = written + __popc(mask & ((1u << lane) - 1u));
      col[start + pos] = (uint32_t)colmap[j];
      ex[start + pos] = (uint8_t)e;
    }
    written += __popc(mask);
  }
}

// ------------------------------------------------------------ keys

template <typename K>
__device__ __forceinline__ K tbl(const K* S, int D1, int c, int R) {  // S(c, R), 0 for R < 0
  return R < 0 ? K(0) : S[c * D1 + R];
}

template <typename K>
__global__ void keys_simplify(const uint32_t* __restrict__ ptr, const uint32_t* __restrict__ col,
                              const uint8_t* __restrict__ ex, const uint32_t* __restrict__ deg, int64_t m, int n,
                              const K* __restrict__ S, int D1, K* __restrict__ keys, uint32_t* __restrict__ vals) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= m) return;
  const int d = (int)deg[t];
  K r = tbl(S, D1, n, d - 1);
  int R = d;
  for (uint32_t q = ptr[t]; q < ptr[t + 1]; ++q) {
    const int c = (int)col[q], a = ex[q];
    r += tbl(S, D1, c, R) - tbl(S, D1, c, R - a);
    R -= a;
  }
  keys[t] = r;
  vals[t] = (uint32_t)t;
}

// Item t < ma is term t of A, otherwise term t - ma of B (the sum a + b).
template <typename K>
__global__ void keys_add(const uint32_t* __restrict__ pa, const uint32_t* __restrict__ ca,
                         const uint8_t* __restrict__ ea, const uint32_t* __restrict__ da,
                         const uint32_t* __restrict__ pb, const uint32_t* __restrict__ cb,
                         const uint8_t* __restrict__ eb, const uint32_t* __restrict__ db, int64_t ma, int64_t mb,
                         int n, const K* __restrict__ S, int D1, K* __restrict__ keys, uint32_t* __restrict__ vals) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ma + mb) return;
  const bool fa = t < ma;
  const int64_t i = fa ? t : t - ma;
  const uint32_t* ptr = fa ? pa : pb;
  const uint32_t* col = fa ? ca : cb;
  const uint8_t* ex = fa ? ea : eb;
  const int d = (int)(fa ? da[i] : db[i]);
  K r = tbl(S, D1, n, d - 1);
  int R = d;
  for (uint32_t q = ptr[i]; q < ptr[i + 1]; ++q) {
    const int c = (int)col[q], a = ex[q];
    r += tbl(S, D1, c, R) - tbl(S, D1, c, R - a);
    R -= a;
  }
  keys[t] = r;
  vals[t] = (uint32_t)t;
}

template <typename K>
__global__ void keys_mul(const uint32_t* __restrict__ pa, const uint32_t* __restrict__ ca,
                         const uint8_t* __restrict__ ea, const uint32_t* __restrict__ da,
                         const uint32_t* __restrict__ pb, const uint32_t* __restrict__ cb,
                         const uint8_t* __restrict__ eb, const uint32_t* __restrict__ db, int64_t ma, int64_t mb,
                         int n, const K* __restrict__ S, int D1, K* __restrict__ keys, uint32_t* __restrict__ vals,
                         int* __restrict__ overflow) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= ma * mb) return;
  const int64_t i = k / mb, j = k - i * mb;
  const int d = (int)(da[i] + db[j]);
  K r = tbl(S, D1, n, d - 1);
  int R = d;
  uint32_t qa = pa[i], qa_end = pa[i + 1], qb = pb[j], qb_end = pb[j + 1];
  // merge two descending column lists
  while (qa < qa_end || qb < qb_end) {
    int c, a;
    const int cA = qa < qa_end ? (int)ca[qa] : -1;
    const int cB = qb < qb_end ? (int)cb[qb] : -1;
    if (cA > cB) {
      c = cA;
      a = ea[qa++];
    } else if (cB > cA) {
      c = cB;
      a = eb[qb++];
    } else {
      c = cA;
      a = (int)ea[qa++] + (int)eb[qb++];
      if (a > 255) *overflow = 1;
    }
    r += tbl(S, D1, c, R) - tbl(S, D1, c, R - a);
    R -= a;
  }
  keys[k] = r;
  vals[k] = (uint32_t)k;
}

// ------------------------------------------------- segmented reduce-by-key

template <typename K>
__global__ void mark_heads(const K* __restrict__ keys, int64_t N, uint32_t* __restrict__ head) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < N) head[k] = (k == 0 || keys[k] != keys[k - 1]) ? 1u : 0u;
}

// Coefficient of a sorted item: the input for simplify, one IEEE product for
// mul, the input of either operand for add.
enum Mode { kSimplify = 0, kMul = 1, kAdd = 2, kSub = 3 };  // kSub: a - b, terms as kAdd
static_assert(kSimplify == kSimplifyMode && kMul == kMulMode && kAdd == kAddMode && kSub == kSubMode,
              "engine modes as declared in common.cuh");

// Coefficient of sort item idx, in the coefficient type C of the operands
// (products and negation in C).
template <typename C>
struct CoefOf {
  const C* ca;
  const C* cb;
  int64_t ma, mb;
  int mode;
  __device__ __forceinline__ C operator()(uint32_t idx) const {
    if (mode == kSimplify) return ca[idx];
    if (mode == kAdd) return idx < ma ? ca[idx] : cb[idx - ma];
    if (mode == kSub) return idx < ma ? ca[idx] : -cb[idx - ma];
    const uint32_t i = idx / (uint32_t)mb, j = idx - i * (uint32_t)mb;  // (N < 2^31)
    return ca[i] * cb[j];
  }
};

// Reduce-by-key over the sorted items (runs of equal keys, "segments", start
// at the head items).  A head item's thread sums its segment left to right
// while it is at most kSegShort items long (nearly every segment of a
// product); a longer segment is listed, and one warp per listed segment sums
// it (lane-strided partial sums, then a fixed shuffle tree).  Both orders are
// fixed, so the sums do not depend on scheduling.  Each segment writes its
// sum, a representative item (any item of a segment has the segment's
// exponent row) and its keep flag at its index (slot of its head).
constexpr int kSegShort = 32;

template <typename C>
__device__ __forceinline__ void seg_write(uint32_t sl, C v, uint32_t item, double zeroprec, uint32_t* __restrict__ rep,
                                          C* __restrict__ sums, uint32_t* __restrict__ keep) {
  sums[sl] = v;
  rep[sl] = item;
  keep[sl] = fabs((double)v) > zeroprec ? 1u : 0u;
}

template <typename C>
__global__ void __launch_bounds__(256) seg_short(const uint32_t* __restrict__ vals, const uint32_t* __restrict__ head,
                                                 const uint32_t* __restrict__ slot, int64_t N, CoefOf<C> coef,
                                                 double zeroprec, uint32_t* __restrict__ rep, C* __restrict__ sums,
                                                 uint32_t* __restrict__ keep, uint32_t* __restrict__ long_list,
                                                 uint32_t* __restrict__ long_count) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N || !head[k]) return;
  const uint32_t item = vals[k];
  C v = coef(item);
  for (int64_t j = k + 1; j < N && !head[j]; ++j) {
    if (j - k >= kSegShort) {
      long_list[atomicAdd(long_count, 1u)] = (uint32_t)k;
      return;
    }
    v += coef(vals[j]);
  }
  seg_write(slot[k], v, item, zeroprec, rep, sums, keep);
}

template <typename C>
__global__ void __launch_bounds__(256) seg_long(const uint32_t* __restrict__ vals, const uint32_t* __restrict__ head,
                                                const uint32_t* __restrict__ slot, int64_t N, CoefOf<C> coef,
                                                double zeroprec, uint32_t* __restrict__ rep, C* __restrict__ sums,
                                                uint32_t* __restrict__ keep, const uint32_t* __restrict__ long_list,
                                                const uint32_t* __restrict__ long_count) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t count = *long_count;
  for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < count; w += warps) {
    const int64_t k0 = long_list[w];
    C v = C(0);
    for (int64_t base = k0;; base += 32) {
      const int64_t k = base + lane;
      // the segment ends before the next head (or the end of the items)
      const bool stop = k >= N || (k > k0 && head[k] != 0u);
      const unsigned stops = __ballot_sync(0xffffffffu, stop);
      const int first_stop = stops ? __ffs(stops) - 1 : 32;
      if (lane < first_stop) v += coef(vals[k]);
      if (first_stop < 32) break;
    }
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) seg_write(slot[k0], v, vals[k0], zeroprec, rep, sums, keep);
  }
}

// Exponent rows of the kept merged terms.  Every item of a key's run has the
// same exponent row, so a row is assembled from one representative item: a
// row of the simplify operand, a row of either add operand, or the sum of the
// two factor rows of a product, each from its operand's sparse support (whose
// columns are already merged columns).  A CTA takes 128 consecutive merged
// terms; with `Staged` the rows are built in shared memory and the kept ones
// (contiguous in the output, since kpos is the exclusive scan of keep) leave
// as one coalesced byte range, otherwise (very wide rows) each thread writes
// its row in place.
constexpr int kUnpackThreads = 128;

struct RowSrc {
  const uint32_t* pa;
  const uint32_t* ca;
  const uint8_t* ea;
  const uint32_t* pb;
  const uint32_t* cb;
  const uint8_t* eb;
  int64_t ma, mb;
  int mode;
};

__device__ __forceinline__ void add_support(uint8_t* row, const uint32_t* __restrict__ ptr,
                                            const uint32_t* __restrict__ col, const uint8_t* __restrict__ ex,
                                            int64_t t) {
  for (uint32_t q = ptr[t]; q < ptr[t + 1]; ++q) row[col[q]] += ex[q];
}

__device__ __forceinline__ void build_row(uint8_t* row, uint32_t idx, const RowSrc& r) {
  if (r.mode == kMul) {
    const int64_t i = idx / r.mb, j = idx - i * r.mb;
    add_support(row, r.pa, r.ca, r.ea, i);
    add_support(row, r.pb, r.cb, r.eb, j);
  } else if (r.mode == kSimplify || (int64_t)idx < r.ma) {
    add_support(row, r.pa, r.ca, r.ea, idx);
  } else {
    add_support(row, r.pb, r.cb, r.eb, (int64_t)idx - r.ma);
  }
}

template <typename C, bool Staged>
__global__ void __launch_bounds__(kUnpackThreads) assemble_rows(const uint32_t* __restrict__ rep,
                                                                const C* __restrict__ sums,
                                                                const uint32_t* __restrict__ keep,
                                                                const uint32_t* __restrict__ kpos, int64_t U, int n,
                                                                RowSrc src, uint8_t* __restrict__ out_exps,
                                                                C* __restrict__ out_coef) {
  extern __shared__ __align__(16) unsigned char rows[];
  const int tid = threadIdx.x;
  const int64_t u0 = (int64_t)blockIdx.x * kUnpackThreads, u = u0 + tid;
  const bool kept = u < U && keep[u];
  if constexpr (Staged) {
    uint32_t* rw = reinterpret_cast<uint32_t*>(rows);
    for (int i = tid; i < kUnpackThreads * n / 4 + 1; i += kUnpackThreads) rw[i] = 0;
    __syncthreads();
    const int64_t obase = kpos[u0];  // output row of the first kept term at or after u0
    if (kept) {
      const int64_t o = kpos[u];
      build_row(rows + (o - obase) * n, rep[u], src);
      out_coef[o] = sums[u];
    }
    const int bytes = __syncthreads_count(kept) * n;
    // out: bytes up to the first 4-byte boundary of the destination, then
    // whole words (each packed from four shared-memory bytes), then the rest
    uint8_t* dst = out_exps + obase * n;
    const int head = (int)((4 - ((uintptr_t)dst & 3)) & 3);
    const int lead = head < bytes ? head : bytes;
    const int words = (bytes - lead) >> 2;
    if (tid < lead) dst[tid] = rows[tid];
    uint32_t* dw = reinterpret_cast<uint32_t*>(dst + lead);
    for (int k = tid; k < words; k += kUnpackThreads) {
      const unsigned char* r = rows + lead + 4 * k;
      dw[k] = (uint32_t)r[0] | ((uint32_t)r[1] << 8) | ((uint32_t)r[2] << 16) | ((uint32_t)r[3] << 24);
    }
    const int tail = lead + 4 * words;
    if (tail + tid < bytes) dst[tail + tid] = rows[tail + tid];
  } else {
    if (!kept) return;
    const int64_t o = kpos[u];
    uint8_t* row = out_exps + o * (int64_t)n;
    for (int c = 0; c < n; ++c) row[c] = 0;
    build_row(row, rep[u], src);
    out_coef[o] = sums[u];
  }
}

// ------------------------------------------------------------- host side

struct Operand {
  int64_t m = 0;
  uint32_t* ptr = nullptr;  // m + 1
  uint32_t* col = nullptr;
  uint8_t* ex = nullptr;
  uint32_t* deg = nullptr;
  int maxdeg = 0;
  uint32_t nnz = 0;
};

// Host side of an operand's build: the column maps it uploads (kept until the
// stream is next synchronised, as the copy reads them asynchronously) and the
// support size and top degree the device reports back.
struct OperandHost {
  std::vector<int> ordmap;  // [ord | colmap]
  int maxdeg = 0;
  uint32_t nnz = 0;
};

// First half of an operand's build: per-term support counts and degrees, their
// scan, and the copies of the top degree and the support total to the host.
// Nothing waits here; the caller synchronises once for every operand.
template <class Poly, class Mem>
polylab_status count_operand(const Poly* p, const std::vector<int>& colmap_h, Operand* op, OperandHost* hb,
                             int** ordmap_d, Mem& scr, cudaStream_t s) {
  op->m = p->n_terms;
  const int64_t m = op->m;
  PL_TRY(scr.get(&op->ptr, m + 1));
  PL_TRY(scr.get(&op->deg, m + 1));
  int* dev_max = nullptr;
  PL_TRY(scr.get(&dev_max, 1));
  // operand columns in increasing merged-column order
  std::vector<int>& both = hb->ordmap;
  both.resize(2 * colmap_h.size());
  for (size_t j = 0; j < colmap_h.size(); ++j) both[j] = (int)j;
  std::sort(both.begin(), both.begin() + colmap_h.size(), [&](int x, int y) { return colmap_h[x] < colmap_h[y]; });
  std::copy(colmap_h.begin(), colmap_h.end(), both.begin() + colmap_h.size());
  PL_TRY(scr.get(ordmap_d, both.size()));
  PL_CUDA(cudaMemcpyAsync(*ordmap_d, both.data(), both.size() * sizeof(int), cudaMemcpyHostToDevice, s));
  PL_CUDA(cudaMemsetAsync(dev_max, 0, sizeof(int), s));
  PL_CUDA(cudaMemsetAsync(op->ptr, 0, (m + 1) * sizeof(uint32_t), s));
  if (m > 0) {
    count_support<<<(unsigned)ceil_div(m, 8), 256, 0, s>>>(p->exps, m, p->n_vars, op->ptr, op->deg, dev_max);
    PL_TRY(launch_status("count_support"));
  }
  PL_TRY(exclusive_scan(op->ptr, op->ptr, m + 1, scr, s));
  PL_CUDA(cudaMemcpyAsync(&hb->maxdeg, dev_max, sizeof(int), cudaMemcpyDeviceToHost, s));
  PL_CUDA(cudaMemcpyAsync(&hb->nnz, op->ptr + m, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  return POLYLAB_OK;
}

// Second half, once the host holds the counts: the CSR supports themselves.
template <class Poly, class Mem>
polylab_status fill_operand(const Poly* p, const OperandHost& hb, const int* ordmap_d, Operand* op, Mem& scr,
                            cudaStream_t s) {
  const int64_t m = op->m;
  op->maxdeg = hb.maxdeg;
  op->nnz = hb.nnz;
  PL_TRY(scr.get(&op->col, std::max<uint32_t>(hb.nnz, 1)));
  PL_TRY(scr.get(&op->ex, std::max<uint32_t>(hb.nnz, 1)));
  if (m > 0) {
    fill_support<<<(unsigned)ceil_div(m, 8), 256, 0, s>>>(p->exps, m, p->n_vars, ordmap_d, ordmap_d + p->n_vars,
                                                          op->ptr, op->col, op->ex);
    PL_TRY(launch_status("fill_support"));
  }
  return POLYLAB_OK;
}

// S(c, R) = C(R + c, c) for c = 0..n, R = 0..D, as K; false if S(n, D) >= 2^bits(K).
template <typename K>
bool build_table(int n, int D, std::vector<K>& S) {
  const int D1 = D + 1;
  S.assign((size_t)(n + 1) * D1, K(0));
  for (int R = 0; R <= D; ++R) S[R] = 1;
  for (int c = 1; c <= n; ++c) {
    S[(size_t)c * D1] = 1;
    for (int R = 1; R <= D; ++R) {
      const K a = S[(size_t)(c - 1) * D1 + R], b = S[(size_t)c * D1 + R - 1];
      const K v = a + b;
      if (v < a) return false;  // wrapped
      S[(size_t)c * D1 + R] = v;
    }
  }
  return true;
}

int key_bits_u128(u128 total) {  // bits to represent values 0 .. total-1
  int b = 0;
  u128 t = total - 1;
  while (t) {
    ++b;
    t >>= 1;
  }
  return b;
}

template <typename K, typename C, class Mem>
polylab_status run_pipeline(int n, int D, int64_t N, const std::vector<K>& Sh, int mode, const Operand& A,
                            const Operand& B, const PolyIn<C>* pa, const PolyIn<C>* pb, double zeroprec, int bits,
                            PolyOut<C>* out, polylab_alloc_fn alloc, void* ctx, Mem& scr, cudaStream_t s) {
  const int D1 = D + 1;
  K* S = nullptr;
  PL_TRY(scr.get(&S, Sh.size()));
  PL_CUDA(cudaMemcpyAsync(S, Sh.data(), Sh.size() * sizeof(K), cudaMemcpyHostToDevice, s));
  K *keys, *akeys;
  uint32_t *vals, *avals;
  PL_TRY(scr.get(&keys, N));
  PL_TRY(scr.get(&akeys, N));
  PL_TRY(scr.get(&vals, N));
  PL_TRY(scr.get(&avals, N));
  int* ovf = nullptr;  // [exponent overflow, sort look-back gave up]
  PL_TRY(scr.get(&ovf, 2));
  PL_CUDA(cudaMemsetAsync(ovf, 0, 2 * sizeof(int), s));
  if (mode == kMul) {
    keys_mul<K><<<(unsigned)ceil_div(N, 256), 256, 0, s>>>(A.ptr, A.col, A.ex, A.deg, B.ptr, B.col, B.ex, B.deg, A.m,
                                                           B.m, n, S, D1, keys, vals, ovf);
  } else if (mode == kAdd || mode == kSub) {
    keys_add<K><<<(unsigned)ceil_div(N, 256), 256, 0, s>>>(A.ptr, A.col, A.ex, A.deg, B.ptr, B.col, B.ex, B.deg, A.m,
                                                           B.m, n, S, D1, keys, vals);
  } else {
    keys_simplify<K><<<(unsigned)ceil_div(N, 256), 256, 0, s>>>(A.ptr, A.col, A.ex, A.deg, N, n, S, D1, keys, vals);
  }
  PL_TRY(launch_status("keys"));
  int which = 0;
  PL_TRY((radix_sort<K, Mem>(keys, vals, akeys, avals, N, bits, scr, s, &which, ovf + 1)));
  if (which) {
    std::swap(keys, akeys);
    std::swap(vals, avals);
  }
  // Reduce-by-key into arrays sized for the worst case (every key unique), so
  // that nothing waits for the number U of distinct keys: U is only read on
  // the device, and the keep flags past U stay zero.
  uint32_t *head, *slot, *keep, *kpos, *rep;
  C* sums;
  PL_TRY(scr.get(&head, N));
  PL_TRY(scr.get(&slot, N));
  PL_TRY(scr.get(&rep, N));
  PL_TRY(scr.get(&sums, N));
  PL_TRY(scr.get(&keep, N));
  PL_TRY(scr.get(&kpos, N));
  PL_CUDA(cudaMemsetAsync(keep, 0, (size_t)N * sizeof(uint32_t), s));
  mark_heads<K><<<(unsigned)ceil_div(N, 256), 256, 0, s>>>(keys, N, head);
  PL_TRY(launch_status("mark_heads"));
  PL_TRY(exclusive_scan(head, slot, N, scr, s));
  CoefOf<C> cf{pa->coef, mode != kSimplify ? pb->coef : nullptr, pa->n_terms, mode != kSimplify ? pb->n_terms : 0,
            mode};
  uint32_t* long_list = nullptr;  // heads of the segments longer than kSegShort, then their count
  const int64_t max_long = N / (kSegShort + 1) + 1;
  PL_TRY(scr.get(&long_list, max_long + 1));
  uint32_t* long_count = long_list + max_long;
  PL_CUDA(cudaMemsetAsync(long_count, 0, sizeof(uint32_t), s));
  seg_short<C><<<(unsigned)ceil_div(N, 256), 256, 0, s>>>(vals, head, slot, N, cf, zeroprec, rep, sums, keep,
                                                          long_list, long_count);
  PL_TRY(launch_status("seg_short"));
  const int64_t lblocks = std::min<int64_t>(ceil_div(max_long, 8), (int64_t)num_sms() * 8);
  seg_long<C><<<(unsigned)lblocks, 256, 0, s>>>(vals, head, slot, N, cf, zeroprec, rep, sums, keep, long_list,
                                                long_count);
  PL_TRY(launch_status("seg_long"));
  PL_TRY(exclusive_scan(keep, kpos, N, scr, s));
  // the one wait that sizes the output: kept count, exponent overflow and the
  // sort's look-back word
  uint32_t hM[2] = {0, 0};
  int hflags[2] = {0, 0};
  PL_CUDA(cudaMemcpyAsync(&hM[0], kpos + N - 1, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  PL_CUDA(cudaMemcpyAsync(&hM[1], keep + N - 1, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  PL_CUDA(cudaMemcpyAsync(hflags, ovf, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
  PL_CUDA(cudaStreamSynchronize(s));
  if (hflags[0]) return POLYLAB_ERR_EXP_OVERFLOW;
  if (hflags[1]) {
    set_last_message("radix sort: a look-back wait gave up");
    return POLYLAB_ERR_TIMEOUT;
  }
  const int64_t U = N;  // keep is zero past the distinct keys
  const int64_t M = (int64_t)hM[0] + hM[1];
  out->n_terms = M;
  out->exps = nullptr;
  out->coef = nullptr;
  if (M == 0) return POLYLAB_OK;
  out->exps = (uint8_t*)alloc((size_t)M * n, ctx);
  out->coef = (C*)alloc((size_t)M * sizeof(C), ctx);
  if (!out->exps || !out->coef) return POLYLAB_ERR_OOM;
  const RowSrc rs{A.ptr, A.col, A.ex, B.ptr, B.col, B.ex, A.m, B.m, mode};
  const size_t ush = (size_t)kUnpackThreads * n + 4;
  const unsigned ublocks = (unsigned)ceil_div(U, kUnpackThreads);
  if (ush <= 96 * 1024) {
    if (ush > 48 * 1024)
      PL_CUDA(cudaFuncSetAttribute(assemble_rows<C, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ush));
    assemble_rows<C, true><<<ublocks, kUnpackThreads, ush, s>>>(rep, sums, keep, kpos, U, n, rs, out->exps, out->coef);
  } else {
    assemble_rows<C, false><<<ublocks, kUnpackThreads, 0, s>>>(rep, sums, keep, kpos, U, n, rs, out->exps, out->coef);
  }
  return launch_status("assemble_rows");
}

template <typename C, class Mem>
polylab_status engine_with(Mem& scr, const PolyIn<C>* pa, const PolyIn<C>* pb, int mode, double zeroprec,
                           PolyOut<C>* out, polylab_alloc_fn alloc, void* ctx, cudaStream_t s) {
  if (!out || !alloc || !out->var_ids || !(zeroprec >= 0.0)) return POLYLAB_ERR_INVALID_ARG;
  PL_TRY(check_poly(pa));
  const bool is_mul = mode != kSimplify;  // two operands (mul or add)
  if (is_mul) PL_TRY(check_poly(pb));
  // alignment (Sec. 3.2): merged ids ascending; column maps per operand
  std::vector<uint64_t> ids(pa->var_ids, pa->var_ids + pa->n_vars);
  std::vector<int> mapA(pa->n_vars), mapB;
  int n;
  if (is_mul) {
    ids.insert(ids.end(), pb->var_ids, pb->var_ids + pb->n_vars);
    std::sort(ids.begin(), ids.end());
    ids.erase(std::unique(ids.begin(), ids.end()), ids.end());
    n = (int)ids.size();
    std::unordered_map<uint64_t, int> pos;
    for (int i = 0; i < n; ++i) pos[ids[i]] = i;
    for (int i = 0; i < pa->n_vars; ++i) mapA[i] = pos[pa->var_ids[i]];
    mapB.resize(pb->n_vars);
    for (int i = 0; i < pb->n_vars; ++i) mapB[i] = pos[pb->var_ids[i]];
  } else {
    n = pa->n_vars;
    for (int i = 0; i < n; ++i) mapA[i] = i;
  }
  out->n_vars = n;
  std::memcpy(out->var_ids, ids.data(), ids.size() * sizeof(uint64_t));
  out->n_terms = 0;
  out->exps = nullptr;
  out->coef = nullptr;
  const int64_t N = mode == kMul ? pa->n_terms * pb->n_terms
                   : (mode == kAdd || mode == kSub) ? pa->n_terms + pb->n_terms : pa->n_terms;
  if (N >= ((int64_t)1 << 31)) return POLYLAB_ERR_UNSUPPORTED;
  if (N == 0) return POLYLAB_OK;
  Operand A, B;
  OperandHost ha, hb;
  int *orda = nullptr, *ordb = nullptr;
  PL_TRY(count_operand(pa, mapA, &A, &ha, &orda, scr, s));
  if (is_mul) PL_TRY(count_operand(pb, mapB, &B, &hb, &ordb, scr, s));
  PL_CUDA(cudaStreamSynchronize(s));  // the one wait before the key width is known
  PL_TRY(fill_operand(pa, ha, orda, &A, scr, s));
  if (is_mul) PL_TRY(fill_operand(pb, hb, ordb, &B, scr, s));
  const int D = std::max(1, mode == kMul ? A.maxdeg + B.maxdeg
                            : (mode == kAdd || mode == kSub) ? std::max(A.maxdeg, B.maxdeg) : A.maxdeg);
  std::vector<u128> S128;
  if (!build_table<u128>(n, D, S128)) return POLYLAB_ERR_UNSUPPORTED;
  const u128 total = S128[(size_t)n * (D + 1) + D];
  const int bits = key_bits_u128(total);
  if (bits <= 64) {
    std::vector<uint64_t> S64(S128.size());
    for (size_t i = 0; i < S128.size(); ++i) S64[i] = (uint64_t)S128[i];
    return run_pipeline<uint64_t, C, Mem>(n, D, N, S64, mode, A, B, pa, pb, zeroprec, bits, out, alloc, ctx, scr,
                                          s);
  }
  return run_pipeline<u128, C, Mem>(n, D, N, S128, mode, A, B, pa, pb, zeroprec, bits, out, alloc, ctx, scr, s);
}

}  // namespace

// (declared in common.cuh; the algebra entry points call it too)
template <typename C>
polylab_status engine(const PolyIn<C>* pa, const PolyIn<C>* pb, int mode, double zeroprec, PolyOut<C>* out,
                      polylab_alloc_fn alloc, void* ctx, cudaStream_t s) {
  Scratch scr(s);
  return engine_with<C>(scr, pa, pb, mode, zeroprec, out, alloc, ctx, s);
}
template polylab_status engine<double>(const PolyIn<double>*, const PolyIn<double>*, int, double, PolyOut<double>*,
                                       polylab_alloc_fn, void*, cudaStream_t);
template polylab_status engine<float>(const PolyIn<float>*, const PolyIn<float>*, int, double, PolyOut<float>*,
                                      polylab_alloc_fn, void*, cudaStream_t);

namespace {

// A C entry point: the public structs viewed as PolyIn / PolyOut and back.
template <typename PubIn, typename PubOut>
polylab_status engine_entry(const PubIn* a, const PubIn* b, int mode, double zeroprec, PubOut* out,
                            polylab_alloc_fn alloc, void* ctx, cudaStream_t s) {
  if (!a || !out || (mode != kSimplify && !b)) return POLYLAB_ERR_INVALID_ARG;
  const auto va = poly_in(*a);
  auto vb = va;
  if (b) vb = poly_in(*b);
  auto o = poly_out(*out);
  const polylab_status st = engine(&va, b ? &vb : nullptr, mode, zeroprec, &o, alloc, ctx, s);
  store_out(o, out);
  return st;
}

}  // namespace

namespace {

// ------------------------------------------------ no-allocation simplify
// For callers that may not allocate device memory during a call: all scratch
// of polylab_simplify_noalloc is carved from this file-scope array.  Every
// GPU that loads the library holds it until the process exits.

constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;  // 16 MiB
constexpr int64_t kNoAllocMaxTerms = 65536;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Fixed arena over the static array: 256-byte aligned bump allocation, no frees.
struct Arena {
  unsigned char* base;
  size_t cap;
  size_t used = 0;
  template <typename T>
  polylab_status get(T** out, size_t count) {
    *out = nullptr;
    if (count == 0) count = 1;
    const size_t bytes = (count * sizeof(T) + 255) & ~size_t(255);
    if (bytes > cap - used) {
      char msg[160];
      snprintf(msg, sizeof(msg), "polylab_simplify_noalloc: working set exceeds the %zu-byte static scratch array",
               cap);
      set_last_message(msg);
      return POLYLAB_ERR_UNSUPPORTED;
    }
    *out = reinterpret_cast<T*>(base + used);
    used += bytes;
    return POLYLAB_OK;
  }
};

// Device address of the array on the current device, looked up on every call
// (in host code the symbol itself is only a host-side stand-in; a lookup per
// call stays valid across device resets and new contexts).
polylab_status noalloc_base(unsigned char** out) {
  void* a = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&a, g_noalloc_scratch);
  if (e != cudaSuccess) {
    set_last_error("cudaGetSymbolAddress(g_noalloc_scratch)", e);
    return POLYLAB_ERR_CUDA;
  }
  *out = static_cast<unsigned char*>(a);
  return POLYLAB_OK;
}

// Hands the caller's output buffers to the pipeline instead of allocating.
struct CallerBuffers {
  uint8_t* exps;
  double* coef;
  int64_t capacity;
  int n;
  int calls = 0;
  bool too_small = false;
};

void* caller_buffers(size_t bytes, void* ctx) {
  CallerBuffers* b = static_cast<CallerBuffers*>(ctx);
  const int call = b->calls++;
  const size_t room = call == 0 ? (size_t)b->capacity * (size_t)b->n : (size_t)b->capacity * sizeof(double);
  if (bytes > room) {
    b->too_small = true;
    return nullptr;
  }
  return call == 0 ? static_cast<void*>(b->exps) : static_cast<void*>(b->coef);
}

}  // namespace
}  // namespace polylab

extern "C" {

polylab_status polylab_simplify(const polylab_poly* p, double zeroprec, polylab_poly_out* out,
                                polylab_alloc_fn alloc, void* alloc_ctx, polylab_stream stream) {
  return polylab::engine_entry(p, (const polylab_poly*)nullptr, polylab::kSimplify, zeroprec, out, alloc, alloc_ctx,
                               (cudaStream_t)stream);
}

polylab_status polylab_mul(const polylab_poly* a, const polylab_poly* b, double zeroprec, polylab_poly_out* out,
                           polylab_alloc_fn alloc, void* alloc_ctx, polylab_stream stream) {
  return polylab::engine_entry(a, b, polylab::kMul, zeroprec, out, alloc, alloc_ctx, (cudaStream_t)stream);
}

polylab_status polylab_add(const polylab_poly* a, const polylab_poly* b, double zeroprec, polylab_poly_out* out,
                           polylab_alloc_fn alloc, void* alloc_ctx, polylab_stream stream) {
  return polylab::engine_entry(a, b, polylab::kAdd, zeroprec, out, alloc, alloc_ctx, (cudaStream_t)stream);
}

polylab_status polylab_sub(const polylab_poly* a, const polylab_poly* b, double zeroprec, polylab_poly_out* out,
                           polylab_alloc_fn alloc, void* alloc_ctx, polylab_stream stream) {
  return polylab::engine_entry(a, b, polylab::kSub, zeroprec, out, alloc, alloc_ctx, (cudaStream_t)stream);
}

polylab_status polylab_simplify_f32(const polylab_poly_f32* p, double zeroprec, polylab_poly_out_f32* out,
                                    polylab_alloc_fn alloc, void* alloc_ctx, polylab_stream stream) {
  return polylab::engine_entry(p, (const polylab_poly_f32*)nullptr, polylab::kSimplify, zeroprec, out, alloc,
                               alloc_ctx, (cudaStream_t)stream);
}

polylab_status polylab_mul_f32(const polylab_poly_f32* a, const polylab_poly_f32* b, double zeroprec,
                               polylab_poly_out_f32* out, polylab_alloc_fn alloc, void* alloc_ctx,
                               polylab_stream stream) {
  return polylab::engine_entry(a, b, polylab::kMul, zeroprec, out, alloc, alloc_ctx, (cudaStream_t)stream);
}

polylab_status polylab_add_f32(const polylab_poly_f32* a, const polylab_poly_f32* b, double zeroprec,
                               polylab_poly_out_f32* out, polylab_alloc_fn alloc, void* alloc_ctx,
                               polylab_stream stream) {
  return polylab::engine_entry(a, b, polylab::kAdd, zeroprec, out, alloc, alloc_ctx, (cudaStream_t)stream);
}

polylab_status polylab_sub_f32(const polylab_poly_f32* a, const polylab_poly_f32* b, double zeroprec,
                               polylab_poly_out_f32* out, polylab_alloc_fn alloc, void* alloc_ctx,
                               polylab_stream stream) {
  return polylab::engine_entry(a, b, polylab::kSub, zeroprec, out, alloc, alloc_ctx, (cudaStream_t)stream);
}

polylab_status polylab_simplify_noalloc(const polylab_poly* p, double zeroprec, polylab_poly_out* out,
                                        int64_t capacity, polylab_stream stream) {
  using namespace polylab;
  if (!p || !out || capacity < 0 || (capacity > 0 && (!out->exps || !out->coef))) return POLYLAB_ERR_INVALID_ARG;
  if (p->n_terms > kNoAllocMaxTerms) {
    char msg[160];
    snprintf(msg, sizeof(msg), "polylab_simplify_noalloc: %lld terms exceed the limit of %lld",
             (long long)p->n_terms, (long long)kNoAllocMaxTerms);
    set_last_message(msg);
    return POLYLAB_ERR_UNSUPPORTED;
  }
  unsigned char* base = nullptr;
  PL_TRY(noalloc_base(&base));
  Arena arena{base, kNoAllocScratchBytes};
  CallerBuffers buf{out->exps, out->coef, capacity, p->n_vars};
  const auto vp = poly_in(*p);
  auto o = poly_out(*out);
  const polylab_status st =
      engine_with<double>(arena, &vp, nullptr, kSimplify, zeroprec, &o, caller_buffers, &buf, (cudaStream_t)stream);
  store_out(o, out);
  // the pipeline resets the output pointers; hand the caller's buffers back
  out->exps = buf.exps;
  out->coef = buf.coef;
  // the array is shared by every call: return only once this call's kernels
  // (the last reads the array) are done
  if (st == POLYLAB_OK) PL_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  if (st == POLYLAB_ERR_OOM && buf.too_small) {
    set_last_message("polylab_simplify_noalloc: the result has more terms than `capacity`; n_terms holds the count");
    return POLYLAB_ERR_INVALID_ARG;
  }
  return st;
}

}  // extern "C"
