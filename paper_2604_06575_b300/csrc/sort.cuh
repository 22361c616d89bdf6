// Device-wide exclusive scan and stable LSD radix sort of (key, uint32) pairs,
// shared by the simplify engine and the derived-coefficient build.  Included
// by several translation units: everything lives in an unnamed namespace.
#pragma once

#include <algorithm>

#include "common.cuh"

namespace polylab {
namespace {

typedef unsigned __int128 u128;

// ------------------------------------------------------------------ scan

constexpr int kScanThreads = 256;
constexpr int kScanVecs = 4;                                 // 16-byte vectors per thread
constexpr int kScanTile = kScanThreads * kScanVecs * 4;      // 4096 values

// Exclusive scan of one value per thread over a 256-thread block (wsum: 8
// words of shared memory).
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

// Four consecutive values starting at q (a multiple of 4): one 16-byte load
// when the whole vector lies below n and the array is 16-byte aligned,
// guarded scalar loads otherwise (zeros past n).
__device__ __forceinline__ uint4 scan_load4(const uint32_t* __restrict__ in, int64_t q, int64_t n, bool vec) {
  if (vec && q + 3 < n) return *reinterpret_cast<const uint4*>(in + q);
  uint4 r;
  r.x = q < n ? in[q] : 0u;
  r.y = q + 1 < n ? in[q + 1] : 0u;
  r.z = q + 2 < n ? in[q + 2] : 0u;
  r.w = q + 3 < n ? in[q + 3] : 0u;
  return r;
}

// Scan phase 1: the sum of each 4096-value tile.  Thread t reads vectors
// t, t + 256, ... of the tile (coalesced).
__global__ void __launch_bounds__(kScanThreads) scan_tile_sums(const uint32_t* __restrict__ in, int64_t n, bool vec,
                                                              uint32_t* __restrict__ sums) {
  __shared__ uint32_t wsum[kScanThreads / 32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  uint32_t t = 0;
#pragma unroll
  for (int r = 0; r < kScanVecs; ++r) {
    const uint4 v = scan_load4(in, base + 4 * ((int64_t)r * kScanThreads + threadIdx.x), n, vec);
    t += v.x + v.y + v.z + v.w;
  }
  for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t s = 0;
    for (int w = 0; w < kScanThreads / 32; ++w) s += wsum[w];
    sums[blockIdx.x] = s;
  }
}

// Scan phase 3: each tile scanned from its offset (offs[tile], or 0 with no
// offsets), a block scan per round of vectors; in may alias out.
__global__ void __launch_bounds__(kScanThreads) scan_tiles(const uint32_t* in, uint32_t* out, int64_t n, bool vec,
                                                          const uint32_t* __restrict__ offs) {
  __shared__ uint32_t wsum[kScanThreads / 32];
  __shared__ uint32_t s_total;
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  uint4 v[kScanVecs];
#pragma unroll
  for (int r = 0; r < kScanVecs; ++r)
    v[r] = scan_load4(in, base + 4 * ((int64_t)r * kScanThreads + threadIdx.x), n, vec);
  uint32_t run = offs ? offs[blockIdx.x] : 0u;
#pragma unroll
  for (int r = 0; r < kScanVecs; ++r) {
    const uint32_t g = v[r].x + v[r].y + v[r].z + v[r].w;
    const uint32_t pre = run + block_excl_scan256(g, wsum);
    if (threadIdx.x == kScanThreads - 1) s_total = pre + g;
    uint4 o;
    o.x = pre;
    o.y = o.x + v[r].x;
    o.z = o.y + v[r].y;
    o.w = o.z + v[r].z;
    const int64_t q = base + 4 * ((int64_t)r * kScanThreads + threadIdx.x);
    if (vec && q + 3 < n) {
      *reinterpret_cast<uint4*>(out + q) = o;
    } else {
      if (q < n) out[q] = o.x;
      if (q + 1 < n) out[q + 1] = o.y;
      if (q + 2 < n) out[q + 2] = o.z;
      if (q + 3 < n) out[q + 3] = o.w;
    }
    __syncthreads();
    run = s_total;
  }
}

// Exclusive scan of n uint32 values (in may alias out): tile sums, their own
// exclusive scan (recursively), then every tile from its offset.  `Mem`
// provides the scratch buffers (stream-ordered allocations, or a fixed arena).
template <class Mem>
polylab_status exclusive_scan(const uint32_t* in, uint32_t* out, int64_t n, Mem& scr, cudaStream_t s) {
  if (n <= 0) return POLYLAB_OK;
  const int64_t tiles = ceil_div(n, kScanTile);
  const bool vec = (((uintptr_t)in | (uintptr_t)out) & 15) == 0;
  if (tiles == 1) {
    scan_tiles<<<1, kScanThreads, 0, s>>>(in, out, n, vec, nullptr);
    return launch_status("scan_tiles");
  }
  uint32_t* sums = nullptr;
  PL_TRY(scr.get(&sums, tiles));
  scan_tile_sums<<<(unsigned)tiles, kScanThreads, 0, s>>>(in, n, vec, sums);
  PL_TRY(launch_status("scan_tile_sums"));
  PL_TRY(exclusive_scan(sums, sums, tiles, scr, s));
  scan_tiles<<<(unsigned)tiles, kScanThreads, 0, s>>>(in, out, n, vec, sums);
  return launch_status("scan_tiles");
}

// -------------------------------------------------------------- radix sort
// Stable LSD radix sort of (key, uint32) pairs, 8-bit digits, one kernel per
// digit in the manner of Adinets and Merrill, "Onesweep: A Faster Least
// Significant Digit Radix Sort for GPUs" (2022):
//  * a digit pass takes tiles in the order CTAs claim them (an atomic tile
//    counter, so every earlier tile belongs to a CTA that is already running),
//    ranks the tile's items by digit in shared memory (per-warp counts, the
//    lanes of one digit found by bit ballots; stable), publishes its
//    per-digit counts, and sums the
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

// Lanes of the warp holding the same 8-bit digit d as this lane (lanes whose
// item is past the end, ok = false, form their own class): one ballot per
// digit bit, each lane keeping the lanes that agree with it on that bit.
__device__ __forceinline__ unsigned peers_of_digit(uint32_t d, bool ok) {
  const unsigned v = __ballot_sync(0xffffffffu, ok);
  unsigned peers = ok ? v : ~v;
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    const bool bit = (d >> b) & 1u;
    const unsigned m = __ballot_sync(0xffffffffu, bit);
    peers &= bit ? m : ~m;
  }
  return peers;
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
    const unsigned peers = peers_of_digit(d, ok);
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
    // the previous tile alone first: once the first wave is past, it has
    // usually published its inclusive count already
    const uint64_t w1 = look_load(look + (size_t)tp * kSortDigits + d);
    const bool near = (w1 & ~kLookCount) == kLookInclusive;
    if (near) excl = w1 & kLookCount;
    while (!near) {
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
