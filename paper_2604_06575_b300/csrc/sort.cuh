// Device-wide exclusive scan and stable LSD radix sort of (key, uint32) pairs,
// shared by the simplify engine and the derived-coefficient build.  Included
// by several translation units: everything lives in an unnamed namespace.
#pragma once

#include <algorithm>

#include "common.cuh"

namespace polylab {
namespace {

typedef unsigned __int128 u128;

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

// ------------------------------------------------------------------ scan

__global__ void scan_tiles(const uint32_t* __restrict__ in, uint32_t* __restrict__ out, uint32_t* __restrict__ sums,
                           int64_t n) {
  __shared__ uint32_t warp_tot[kScanThreads / 32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  uint32_t v[kScanItems];
  uint32_t run = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    v[i] = base + i < n ? in[base + i] : 0u;
    const uint32_t t = v[i];
    v[i] = run;
    run += t;
  }
  // exclusive scan of thread totals across the block
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t inc = run;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) warp_tot[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    uint32_t t = lane < kScanThreads / 32 ? warp_tot[lane] : 0u;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    if (lane < kScanThreads / 32) warp_tot[lane] = t;
  }
  __syncthreads();
  const uint32_t off = (wid ? warp_tot[wid - 1] : 0u) + inc - run;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i)
    if (base + i < n) out[base + i] = v[i] + off;
  if (threadIdx.x == kScanThreads - 1) sums[blockIdx.x] = warp_tot[kScanThreads / 32 - 1];
}

__global__ void add_tile_offsets(uint32_t* __restrict__ out, const uint32_t* __restrict__ offs, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] += offs[i / kScanTile];
}

// Exclusive scan of n uint32 values (in may alias out).  `Mem` provides the
// scratch buffers (stream-ordered allocations, or a fixed arena).
template <class Mem>
polylab_status exclusive_scan(const uint32_t* in, uint32_t* out, int64_t n, Mem& scr, cudaStream_t s) {
  if (n <= 0) return POLYLAB_OK;
  const int64_t tiles = ceil_div(n, kScanTile);
  uint32_t* sums = nullptr;
  PL_TRY(scr.get(&sums, tiles));
  scan_tiles<<<(unsigned)tiles, kScanThreads, 0, s>>>(in, out, sums, n);
  PL_TRY(launch_status("scan_tiles"));
  if (tiles > 1) {
    PL_TRY(exclusive_scan(sums, sums, tiles, scr, s));
    add_tile_offsets<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(out, sums, n);
    PL_TRY(launch_status("add_tile_offsets"));
  }
  return POLYLAB_OK;
}

// -------------------------------------------------------------- radix sort
// Stable LSD radix sort of (key, uint32) pairs, 8-bit digits, one kernel per
// digit in the manner of Adinets and Merrill, "Onesweep: A Faster Least
// Significant Digit Radix Sort for GPUs" (2022):
//  * a digit pass takes tiles in the order CTAs claim them (an atomic tile
//    counter, so every earlier tile belongs to a CTA that is already running),
//    ranks the tile's items by digit in shared memory (per-warp counts from
//    __match_any_sync, stable), publishes its per-digit counts, and sums the
//    counts of the tiles before it by decoupled look-back over their published
//    words (a word holds a flag -- aggregate of that tile alone, or inclusive
//    prefix -- and the count; each step reads kLookWidth earlier tiles'
//    words at once, since the CTAs of the first wave all start together and
//    find no inclusive word until the first tiles finish); the items are
//    staged in shared memory in digit order meanwhile, and each digit's run
//    of the tile leaves as consecutive addresses;
//  * the global start of each digit comes from that digit position's global
//    histogram: the first is counted by a small kernel, every later one by the
//    pass before it (which holds the keys anyway), and each CTA scans the
//    256 counts itself.
// Look-back waits are bounded: past kLookbackSpins polls the thread sets the
// caller's error word, keeps the counts it has (every count is non-negative,
// so its items' positions can only come out lower, never past the end of the
// output) and publishes, so no CTA waits forever.

constexpr int kSortThreads = 256;  // one thread per digit in the look-back
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortDigits = 256;
static_assert(kSortThreads == kSortDigits, "the look-back maps one thread to one digit");

template <typename K>
struct SortTile {
  static constexpr int ipt = sizeof(K) <= 8 ? 16 : 8;  // items per thread
  static constexpr int items = kSortThreads * ipt;
};

constexpr uint64_t kLookAggregate = 1ull << 62;  // count of this tile alone
constexpr uint64_t kLookInclusive = 2ull << 62;  // count of this and every earlier tile
constexpr uint64_t kLookCount = (1ull << 62) - 1;
constexpr int kLookWidth = 32;
constexpr int kLookbackSpins = 1 << 22;

template <typename K>
__device__ __forceinline__ uint32_t digit_of(K key, int shift) {
  return (uint32_t)(key >> shift) & 0xffu;
}

__device__ __forceinline__ uint64_t look_load(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void look_store(uint64_t* p, uint64_t v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Exclusive scan of one value per thread over a 256-thread block.
__device__ __forceinline__ uint32_t block_excl_scan256(uint32_t v, uint32_t* wsum) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t inc = v;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  __syncthreads();  // wsum may still be read by an earlier call
  if (lane == 31) wsum[wid] = inc;
  __syncthreads();
  uint32_t before = 0;
  for (int w = 0; w < wid; ++w) before += wsum[w];
  return before + inc - v;
}

template <typename K>
size_t sort_pass_smem() {
  constexpr int T = SortTile<K>::items;
  return (size_t)T * sizeof(K) + (size_t)T * 4 + (size_t)kSortWarps * kSortDigits * 4 + (size_t)kSortDigits * 4 +
         (size_t)kSortDigits * 8;
}

// ghist[d] += number of keys whose lowest digit is d.
template <typename K>
__global__ void __launch_bounds__(kSortThreads) sort_count_digit0(const K* __restrict__ keys, int64_t N,
                                                                  uint32_t* __restrict__ ghist) {
  __shared__ uint32_t h[kSortWarps][kSortDigits];
  const int wid = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < kSortWarps * kSortDigits; i += kSortThreads) (&h[0][0])[i] = 0;
  __syncthreads();
  for (int64_t k = (int64_t)blockIdx.x * kSortThreads + threadIdx.x; k < N; k += (int64_t)gridDim.x * kSortThreads)
    atomicAdd(&h[wid][digit_of(keys[k], 0)], 1u);
  __syncthreads();
  uint32_t c = 0;
  for (int w = 0; w < kSortWarps; ++w) c += h[w][threadIdx.x];
  if (c) atomicAdd(&ghist[threadIdx.x], c);
}

template <typename K>
__global__ void __launch_bounds__(kSortThreads) sort_pass(const K* __restrict__ keys, const uint32_t* __restrict__ vals,
                                                          K* __restrict__ okeys, uint32_t* __restrict__ ovals,
                                                          int64_t N, int shift, const uint32_t* __restrict__ hist,
                                                          uint32_t* __restrict__ hist_next,
                                                          uint64_t* __restrict__ look, uint32_t* __restrict__ tile_ctr,
                                                          int* __restrict__ err) {
  constexpr int IPT = SortTile<K>::ipt, TILE = SortTile<K>::items;
  extern __shared__ __align__(16) unsigned char sm[];
  K* sk = reinterpret_cast<K*>(sm);                           // the tile in digit order
  uint32_t* sv = reinterpret_cast<uint32_t*>(sk + TILE);
  uint32_t* wcnt = sv + TILE;                                 // [warp][digit]
  uint32_t* lstart = wcnt + kSortWarps * kSortDigits;         // tile-local start of each digit
  int64_t* gbase = reinterpret_cast<int64_t*>(lstart + kSortDigits);  // global start - local start
  __shared__ uint32_t s_tile;
  __shared__ uint32_t s_wsum[kSortWarps];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  for (int i = tid; i < kSortWarps * kSortDigits; i += kSortThreads) wcnt[i] = 0;
  if (tid == 0) s_tile = atomicAdd(tile_ctr, 1u);
  __syncthreads();
  const uint32_t t = s_tile;
  const int64_t t0 = (int64_t)t * TILE;
  // warp w ranks the contiguous segment [t0 + w * 32 * IPT, + 32 * IPT)
  const int64_t seg = t0 + (int64_t)wid * 32 * IPT;
  K kk[IPT];
  uint32_t vv[IPT], rk[IPT];
  const unsigned lt = (1u << lane) - 1u;
  uint32_t* mycnt = wcnt + wid * kSortDigits;
  // every load of the tile first, all in flight together (the ranking below
  // works on shared memory between warp barriers, which the loads must not
  // wait behind)
#pragma unroll
  for (int it = 0; it < IPT; ++it) {
    const int64_t k = seg + it * 32 + lane;
    kk[it] = k < N ? keys[k] : K(0);
    vv[it] = k < N ? vals[k] : 0u;
  }
#pragma unroll
  for (int it = 0; it < IPT; ++it) {
    const bool ok = seg + it * 32 + lane < N;
    const uint32_t d = ok ? digit_of(kk[it], shift) : uint32_t(kSortDigits);
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const uint32_t before = __popc(peers & lt);
    const uint32_t basec = ok ? mycnt[d] : 0u;
    rk[it] = ok ? basec + before : 0xffffffffu;
    __syncwarp();
    if (ok && before == 0) mycnt[d] = basec + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // thread d: the tile's count of digit d, and each warp's start within it
  const int d = tid;
  uint32_t cnt = 0;
  for (int w = 0; w < kSortWarps; ++w) {
    const uint32_t c = wcnt[w * kSortDigits + d];
    wcnt[w * kSortDigits + d] = cnt;
    cnt += c;
  }
  uint64_t* mine = look + (size_t)t * kSortDigits + d;
  look_store(mine, (t == 0 ? kLookInclusive : kLookAggregate) | cnt);
  // the tile in digit order into shared memory (tile-local starts: a scan of
  // the counts over digits); the look-back below needs none of it
  const uint32_t ls = block_excl_scan256(cnt, s_wsum);
  lstart[d] = ls;
  __syncthreads();
#pragma unroll
  for (int it = 0; it < IPT; ++it) {
    if (rk[it] != 0xffffffffu) {
      const uint32_t dd = digit_of(kk[it], shift);
      const uint32_t lp = lstart[dd] + wcnt[wid * kSortDigits + dd] + rk[it];
      sk[lp] = kk[it];
      sv[lp] = vv[it];
    }
  }
  uint64_t excl = 0;
  if (t > 0) {
    int64_t tp = (int64_t)t - 1;  // nearest tile not yet summed
    int spins = 0;
    while (true) {
      uint64_t w[kLookWidth];
#pragma unroll
      for (int u = 0; u < kLookWidth; ++u)
        w[u] = tp - u >= 0 ? look_load(look + (size_t)(tp - u) * kSortDigits + d) : kLookInclusive;
      bool done = false;
      int used = 0;
#pragma unroll
      for (int u = 0; u < kLookWidth; ++u) {
        if (done || used < u) break;  // stopped at an inclusive word or at one not yet published
        const uint64_t flag = w[u] & ~kLookCount;
        if (flag == 0) break;
        excl += w[u] & kLookCount;
        ++used;
        done = flag == kLookInclusive;
      }
      if (done) break;
      tp -= used;
      if (used < kLookWidth && ++spins > kLookbackSpins) {
        if (err) atomicExch(err, 1);
        break;
      }
    }
    look_store(mine, kLookInclusive | (excl + cnt));
  }
  // the digit's global start: a scan of this position's global histogram
  const uint32_t gs = block_excl_scan256(hist[d], s_wsum);
  gbase[d] = (int64_t)gs + (int64_t)excl - (int64_t)ls;
  __syncthreads();
  // the per-warp counts are free again: they count the next digit
  if (hist_next) {
    for (int i = tid; i < kSortWarps * kSortDigits; i += kSortThreads) wcnt[i] = 0;
    __syncthreads();
  }
  const int n_here = (int)(N - t0 < TILE ? N - t0 : TILE);
  for (int i = tid; i < n_here; i += kSortThreads) {
    const K key = sk[i];
    const int64_t pos = gbase[digit_of(key, shift)] + i;
    okeys[pos] = key;
    ovals[pos] = sv[i];
    if (hist_next) atomicAdd(&mycnt[digit_of(key, shift + 8)], 1u);
  }
  if (hist_next) {
    __syncthreads();
    uint32_t c = 0;
    for (int w = 0; w < kSortWarps; ++w) c += wcnt[w * kSortDigits + d];
    if (c) atomicAdd(&hist_next[d], c);
  }
}

// Sorts (keys, vals) by the low `bits` bits of the key; returns which buffer
// holds the result (0 = the input buffers, 1 = the alternates).  `err` (device
// int, may be null) is set to 1 if a look-back wait gave up: the order is then
// wrong and the caller reports an error when it next reads the word.
template <typename K, class Mem>
polylab_status radix_sort(K* keys, uint32_t* vals, K* akeys, uint32_t* avals, int64_t N, int bits, Mem& scr,
                          cudaStream_t s, int* which, int* err) {
  *which = 0;
  if (N <= 1 || bits <= 0) return POLYLAB_OK;
  constexpr int TILE = SortTile<K>::items;
  const int passes = std::min<int>((bits + 7) / 8, (int)sizeof(K));
  const int64_t tiles = ceil_div(N, TILE);
  uint32_t* ghist = nullptr;  // [passes][256] digit counts, then one tile counter per pass
  uint64_t* look = nullptr;   // [passes][tiles][256] look-back words
  PL_TRY(scr.get(&ghist, (size_t)passes * (kSortDigits + 1)));
  PL_TRY(scr.get(&look, (size_t)passes * tiles * kSortDigits));
  uint32_t* ctr = ghist + (size_t)passes * kSortDigits;
  PL_CUDA(cudaMemsetAsync(ghist, 0, (size_t)passes * (kSortDigits + 1) * 4, s));
  PL_CUDA(cudaMemsetAsync(look, 0, (size_t)passes * tiles * kSortDigits * 8, s));
  const int cgrid = (int)std::min<int64_t>(ceil_div(N, (int64_t)kSortThreads * 16), (int64_t)num_sms() * 4);
  sort_count_digit0<K><<<cgrid, kSortThreads, 0, s>>>(keys, N, ghist);
  PL_TRY(launch_status("sort_count_digit0"));
  const size_t smem = sort_pass_smem<K>();
  PL_CUDA(cudaFuncSetAttribute(sort_pass<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  K* src_k = keys;
  uint32_t* src_v = vals;
  K* dst_k = akeys;
  uint32_t* dst_v = avals;
  for (int p = 0; p < passes; ++p) {
    uint32_t* next = p + 1 < passes ? ghist + (size_t)(p + 1) * kSortDigits : nullptr;
    sort_pass<K><<<(unsigned)tiles, kSortThreads, smem, s>>>(src_k, src_v, dst_k, dst_v, N, 8 * p,
                                                             ghist + (size_t)p * kSortDigits, next,
                                                             look + (size_t)p * tiles * kSortDigits, ctr + p, err);
    PL_TRY(launch_status("sort_pass"));
    std::swap(src_k, dst_k);
    std::swap(src_v, dst_v);
    *which ^= 1;
  }
  return POLYLAB_OK;
}

}  // namespace
}  // namespace polylab
