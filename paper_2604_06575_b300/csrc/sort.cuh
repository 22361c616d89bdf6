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
// LSD, 8-bit digits.  Tile = 8 warps x 32 lanes x 16 items; within a tile each
// warp owns a contiguous segment and ranks its items stably with
// __match_any_sync; per-digit warp counts are prefix-summed across warps.

constexpr int kSortWarps = 8;
constexpr int kSortIPT = 8;
constexpr int kSortTile = kSortWarps * 32 * kSortIPT;

template <typename K>
__device__ __forceinline__ uint32_t digit_of(K key, int shift) {
  return (uint32_t)(key >> shift) & 0xffu;
}

template <typename K>
__global__ void __launch_bounds__(256) sort_hist(const K* __restrict__ keys, int64_t N, int shift,
                                                 uint32_t* __restrict__ hist, int tiles) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kSortTile;
  for (int i = threadIdx.x; i < kSortTile; i += 256) {
    const int64_t k = base + i;
    if (k < N) atomicAdd(&h[digit_of(keys[k], shift)], 1u);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * tiles + blockIdx.x] = h[threadIdx.x];  // digit-major
}

template <typename K>
__global__ void __launch_bounds__(256) sort_scatter(const K* __restrict__ keys, const uint32_t* __restrict__ vals,
                                                    K* __restrict__ okeys, uint32_t* __restrict__ ovals, int64_t N,
                                                    int shift, const uint32_t* __restrict__ offs, int tiles) {
  __shared__ uint32_t wcnt[kSortWarps][256];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < kSortWarps * 256; i += 256) (&wcnt[0][0])[i] = 0;
  __syncthreads();
  const int64_t seg = (int64_t)blockIdx.x * kSortTile + (int64_t)wid * 32 * kSortIPT;
  K kk[kSortIPT];
  uint32_t vv[kSortIPT], rk[kSortIPT], dg[kSortIPT];
  const unsigned lt = (1u << lane) - 1u;
#pragma unroll
  for (int it = 0; it < kSortIPT; ++it) {
    const int64_t k = seg + it * 32 + lane;
    const bool ok = k < N;
    kk[it] = ok ? keys[k] : K(0);
    vv[it] = ok ? vals[k] : 0u;
    const uint32_t d = ok ? digit_of(kk[it], shift) : 256u;
    dg[it] = d;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const uint32_t before = __popc(peers & lt);
    uint32_t basec = 0;
    if (ok) basec = wcnt[wid][d];
    rk[it] = basec + before;
    __syncwarp();
    if (ok && before == 0) wcnt[wid][d] = basec + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // exclusive prefix over warps for each digit (thread = digit)
  {
    const int d = threadIdx.x;
    uint32_t run = offs[(int64_t)d * tiles + blockIdx.x];
    for (int w = 0; w < kSortWarps; ++w) {
      const uint32_t c = wcnt[w][d];
      wcnt[w][d] = run;
      run += c;
    }
  }
  __syncthreads();
#pragma unroll
  for (int it = 0; it < kSortIPT; ++it) {
    if (dg[it] < 256u) {
      const uint32_t pos = wcnt[wid][dg[it]] + rk[it];
      okeys[pos] = kk[it];
      ovals[pos] = vv[it];
    }
  }
}

// Sorts (keys, vals) by the low `bits` bits of the key; returns which buffer
// holds the result (0 = the input buffers, 1 = the alternates).
template <typename K, class Mem>
polylab_status radix_sort(K* keys, uint32_t* vals, K* akeys, uint32_t* avals, int64_t N, int bits, Mem& scr,
                          cudaStream_t s, int* which) {
  *which = 0;
  if (N <= 1 || bits <= 0) return POLYLAB_OK;
  const int tiles = (int)ceil_div(N, kSortTile);
  uint32_t* hist = nullptr;
  PL_TRY(scr.get(&hist, (size_t)256 * tiles));
  K* src_k = keys;
  uint32_t* src_v = vals;
  K* dst_k = akeys;
  uint32_t* dst_v = avals;
  for (int shift = 0; shift < bits; shift += 8) {
    sort_hist<K><<<tiles, 256, 0, s>>>(src_k, N, shift, hist, tiles);
    PL_TRY(launch_status("sort_hist"));
    PL_TRY(exclusive_scan(hist, hist, (int64_t)256 * tiles, scr, s));
    sort_scatter<K><<<tiles, 256, 0, s>>>(src_k, src_v, dst_k, dst_v, N, shift, hist, tiles);
    PL_TRY(launch_status("sort_scatter"));
    std::swap(src_k, dst_k);
    std::swap(src_v, dst_v);
    *which ^= 1;
  }
  return POLYLAB_OK;
}

}  // namespace
}  // namespace polylab
