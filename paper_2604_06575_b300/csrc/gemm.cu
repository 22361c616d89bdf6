// Derivative evaluation as the dense contraction it is (Sec. 3.3
// differentiation, evaluated at many points):
//
//   Y[p, o] = sum_beta B[p, beta] C[beta, o],   B[p, beta] = prod_v x_{p,v}^{beta_v}
//
// beta runs over the closure set S = {alpha, alpha - e_i, alpha - e_i - e_j}
// of the terms alpha, o over the outputs (f, g_1..g_n, H_ij for i <= j), and
// C[beta, o] collects the falling-factorial coefficients (built once per
// polynomial: "derived-coefficient matrix").
//
// The contraction runs on the 5th-generation tensor cores: one CTA owns 128
// points (the MMA M dimension) and a chunk of output columns (N); per K tile
// it computes the 128 x KT monomial tile B in registers and stores it to
// shared memory in the 128-byte-swizzled K-major layout, while one thread
// bulk-copies the matching pre-swizzled tile of C from HBM (cp.async.bulk
// with mbarrier transaction counts) and issues tcgen05.mma into TMEM
// accumulators (M = 128, N = 256 per instruction).  Two shared-memory stages
// let the producer of tile k+1 overlap the MMAs of tile k.  Tiles of C that
// are all zero are skipped (block sparsity).  The epilogue reads TMEM with
// tcgen05.ld, applies the per-column scale and scatters f, g and the
// symmetric H.
//
// Forms: BF16 operands with per-column coefficient scaling (kind::f16, FP32
// accumulation), and 3xTF32 (kind::tf32: A_hi B_hi + A_hi B_lo + A_lo B_hi,
// FP32 accumulation).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "async.cuh"
#include "common.cuh"
#include "sort.cuh"

namespace polylab {

constexpr int kGemmNPadQuantum = 512;

struct __align__(16) ClosMono {  // support of one closure monomial, ascending variables (32 B)
  uint16_t var[kMaxSupport];
  uint8_t exp[kMaxSupport];
  uint8_t pad[8];
};
static_assert(sizeof(ClosMono) == 32, "ClosMono layout");

struct GemmOperand {
  int n = 0;
  int64_t K = 0, Kpad = 0;  // closure size, padded to 64
  int Npad = 0;             // output columns padded to kGemmNPadQuantum
  ClosMono* mono = nullptr; // Kpad
  // per closure monomial, its factors as rows of the producers' power table
  // (v * Et + e - 1): eight for the BF16 table depth, then eight for the TF32
  // one, 0xffff past the support; built when both tables hold every exponent
  uint16_t* moff = nullptr;  // Kpad x 16
  int* tslots = nullptr;     // Kpad / 64 (BF16 tiles), then Kpad / 32 (TF32 tiles)
  int Et16 = 1, Et32 = 1;
  bool off16 = false, off32 = false;  // the rows are valid for that form's table
  float* scale = nullptr;   // Npad
  uint16_t* tri_i = nullptr;  // Npad: output column -> (kind, i, j) table
  uint16_t* tri_j = nullptr;
  uint8_t* kind = nullptr;
  // BF16: chunks of 512 columns, K tiles of 64, blocks of 512 x 128 B
  unsigned char* b16 = nullptr;
  std::vector<std::vector<int>> live16;  // per chunk: live K tiles
  int* live16_dev = nullptr;             // [chunks][Kt] compacted, -1 padded
  uint8_t* half16_dev = nullptr;         // [chunks][Kt] bit h: half h nonzero
  // TF32 hi/lo: chunks of 256 columns, K tiles of 32, blocks of 256 x 128 B (x2)
  unsigned char* t32 = nullptr;
  std::vector<std::vector<int>> live32;
  int* live32_dev = nullptr;
};

void free_gemm_operand(GemmOperand* g, cudaStream_t s) {
  if (!g) return;
  for (void* p : {(void*)g->mono, (void*)g->moff, (void*)g->tslots, (void*)g->scale, (void*)g->tri_i, (void*)g->tri_j, (void*)g->kind,
                  (void*)g->b16,
                  (void*)g->live16_dev, (void*)g->half16_dev, (void*)g->t32, (void*)g->live32_dev})
    if (p) cudaFreeAsync(p, s);
  delete g;
}

namespace {

constexpr int kCandPerTerm = 1 + kMaxSupport + kMaxSupport * (kMaxSupport + 1) / 2;  // 45

__device__ __forceinline__ uint64_t rank_sparse(const int* var, const int* ex, int k, int n, const uint64_t* S,
                                                int D1) {
  int d = 0;
  for (int s = 0; s < k; ++s) d += ex[s];
  uint64_t r = d > 0 ? S[(size_t)n * D1 + d - 1] : 0;
  int R = d;
  for (int s = k - 1; s >= 0; --s) {  // descending variable order
    const int c = var[s], a = ex[s];
    r += S[(size_t)c * D1 + R] - (R - a >= 0 ? S[(size_t)c * D1 + R - a] : 0);
    R -= a;
  }
  return r;
}

// Candidate closure monomials of each term: alpha, alpha - e_i, alpha - e_i - e_j.
__global__ void closure_candidates(const Term* __restrict__ terms, int64_t m, int n, const uint64_t* __restrict__ S,
                                   int D1, uint64_t* __restrict__ keys, uint32_t* __restrict__ vals) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= m) return;
  const Term tr = terms[t];
  int var[kMaxSupport], ex[kMaxSupport], k = 0;
  for (int s = 0; s < kMaxSupport; ++s)
    if (tr.exp[s]) {
      var[k] = tr.var[s];
      ex[k] = tr.exp[s];
      ++k;
    }
  uint64_t* out = keys + t * kCandPerTerm;
  int slot = 0;
  out[slot++] = rank_sparse(var, ex, k, n, S, D1);
  for (int a = 0; a < k; ++a) {
    ex[a] -= 1;
    out[slot++] = rank_sparse(var, ex, k, n, S, D1);
    for (int b = a; b < k; ++b) {
      if (ex[b] >= 1) {
        ex[b] -= 1;
        out[slot++] = rank_sparse(var, ex, k, n, S, D1);
        ex[b] += 1;
      }
    }
    ex[a] += 1;
  }
  for (; slot < kCandPerTerm; ++slot) out[slot] = ~0ull;
  for (int q = 0; q < kCandPerTerm; ++q) vals[t * kCandPerTerm + q] = 0;
}

__global__ void mark_unique(const uint64_t* __restrict__ keys, int64_t N, uint32_t* __restrict__ head) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < N) head[k] = (keys[k] != ~0ull && (k == 0 || keys[k] != keys[k - 1])) ? 1u : 0u;
}

__global__ void gather_unique(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ head,
                              const uint32_t* __restrict__ pos, int64_t N, uint64_t* __restrict__ out) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < N && head[k]) out[pos[k]] = keys[k];
}

// closure key -> support (inverse of rank_sparse)
__global__ void closure_unrank(const uint64_t* __restrict__ ukeys, int64_t K, int64_t Kpad, int n,
                               const uint64_t* __restrict__ S, int D1, ClosMono* __restrict__ mono) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= Kpad) return;
  ClosMono cm;
  for (int s = 0; s < kMaxSupport; ++s) {
    cm.var[s] = 0;
    cm.exp[s] = 0;
    cm.pad[s] = 0;
  }
  if (q < K) {
    const uint64_t r = ukeys[q];
    const int D = D1 - 1;
    int d = 0;
    while (d < D && S[(size_t)n * D1 + d] <= r) ++d;
    uint64_t w = r - (d > 0 ? S[(size_t)n * D1 + d - 1] : 0);
    int R = d;
    int tv[kMaxSupport], te[kMaxSupport], k = 0;  // collected in descending variable order
    for (int c = n - 1; c >= 1 && R > 0; --c) {
      const uint64_t top = S[(size_t)c * D1 + R];
      int a = 0;
      while (a < R && top - S[(size_t)c * D1 + (R - a - 1)] <= w) ++a;
      if (a) {
        w -= top - S[(size_t)c * D1 + (R - a)];
        R -= a;
        if (k < kMaxSupport) {
          tv[k] = c;
          te[k] = a;
        }
        ++k;
      }
    }
    if (R > 0 && k < kMaxSupport) {
      tv[k] = 0;
      te[k] = R;
      ++k;
    }
    for (int s = 0; s < k && s < kMaxSupport; ++s) {  // ascending
      cm.var[s] = (uint16_t)tv[k - 1 - s];
      cm.exp[s] = (uint8_t)te[k - 1 - s];
    }
    cm.pad[0] = (uint8_t)(k < kMaxSupport ? k : kMaxSupport);  // support size
  }
  mono[q] = cm;
}

// Power-table rows of every closure monomial's factors (see GemmOperand::moff).
// An exponent beyond the table depth Et takes several rows (x^e = (x^Et)^k
// x^r); the host only builds the rows when every monomial fits in eight.
// Unused rows point at the table's row of ones (row n * Et); returns the
// number of rows used.
__device__ __forceinline__ int table_rows(const ClosMono& cm, int n, int Et, uint16_t* out) {
  int k = 0;
  for (int s = 0; s < cm.pad[0] && s < kMaxSupport; ++s) {
    int e = cm.exp[s];
    while (e > 0 && k < 8) {
      const int take = e < Et ? e : Et;
      out[k++] = (uint16_t)(cm.var[s] * Et + take - 1);
      e -= take;
    }
  }
  const int used = k;
  while (k < 8) out[k++] = (uint16_t)(n * Et);
  return used;
}
// Rows of every monomial, and per K tile the most rows any of its monomials
// uses (tslots: BF16 tiles of 64 monomials, then TF32 tiles of 32).
__global__ void closure_offsets(const ClosMono* __restrict__ mono, int64_t Kpad, int n, int Et16, int Et32,
                                uint16_t* __restrict__ moff, int* __restrict__ tslots16,
                                int* __restrict__ tslots32) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= Kpad) return;
  const ClosMono cm = mono[q];
  atomicMax(&tslots16[q / 64], table_rows(cm, n, Et16, moff + q * 16));
  atomicMax(&tslots32[q / 32], table_rows(cm, n, Et32, moff + q * 16 + 8));
}

__device__ __forceinline__ int64_t find_key(const uint64_t* __restrict__ ukeys, int64_t K, uint64_t key) {
  int64_t lo = 0, hi = K;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (ukeys[mid] < key) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ int out_col_upper(int i, int j, int n) {  // i <= j
  return 1 + n + i * (2 * n - i + 1) / 2 + (j - i);
}

// C[beta, o] += coefficient of x^beta in d_o f, from every term.
__global__ void closure_fill(const Term* __restrict__ terms, int64_t m, int n, const uint64_t* __restrict__ S,
                             int D1, const uint64_t* __restrict__ ukeys, int64_t K, int Npad,
                             double* __restrict__ C) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= m) return;
  const Term tr = terms[t];
  int var[kMaxSupport], ex[kMaxSupport], k = 0;
  for (int s = 0; s < kMaxSupport; ++s)
    if (tr.exp[s]) {
      var[k] = tr.var[s];
      ex[k] = tr.exp[s];
      ++k;
    }
  auto add = [&](int o, double v) {
    const int64_t row = find_key(ukeys, K, rank_sparse(var, ex, k, n, S, D1));
    atomicAdd(&C[row * Npad + o], v);
  };
  add(0, tr.coef);
  for (int a = 0; a < k; ++a) {
    const double fa = ex[a];
    ex[a] -= 1;
    add(1 + var[a], tr.coef * fa);
    for (int b = a; b < k; ++b) {
      if (ex[b] >= 1) {
        const double fb = ex[b];  // falling factor: a_b, or a_a - 1 when b == a
        ex[b] -= 1;
        add(out_col_upper(var[a], var[b], n), tr.coef * fa * fb);
        ex[b] += 1;
      }
    }
    ex[a] += 1;
  }
}

// per-column scale: max |C[., o]| (1 when the column is zero)
__global__ void column_scale(const double* __restrict__ C, int64_t Kpad, int Npad, float* __restrict__ scale) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= Npad) return;
  double mx = 0.0;
  for (int64_t k = 0; k < Kpad; ++k) mx = fmax(mx, fabs(C[k * Npad + o]));
  scale[o] = mx > 0.0 ? (float)mx : 1.0f;
}

__host__ __device__ __forceinline__ size_t sw128_offset(int row, int kbyte) {
  return (size_t)(row >> 3) * 1024 + (row & 7) * 128 + ((((kbyte >> 4) ^ (row & 7))) << 4) + (kbyte & 15);
}

__device__ __forceinline__ float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Pack C into the swizzled tile blocks of both forms and flag nonzero tiles.
__global__ void closure_pack(const double* __restrict__ C, const float* __restrict__ scale, int64_t Kpad, int Npad,
                             unsigned char* __restrict__ b16, unsigned char* __restrict__ t32,
                             uint8_t* __restrict__ nz16, uint8_t* __restrict__ nz32) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= Kpad * Npad) return;
  const int64_t k = idx / Npad;
  const int o = (int)(idx - k * Npad);
  const double v = C[idx];
  const float sv = (float)(v / (double)scale[o]);
  const int64_t Kt16 = Kpad / 64, Kt32 = Kpad / 32;
  {  // BF16: chunk of 512 columns, K tile of 64
    const int chunk = o / 512, row = o % 512;
    const int64_t kt = k / 64;
    const int kk = (int)(k % 64);
    const size_t blk = ((size_t)chunk * Kt16 + kt) * (512 * 128);
    const __nv_bfloat16 hb = __float2bfloat16_rn(sv);
    *reinterpret_cast<__nv_bfloat16*>(b16 + blk + sw128_offset(row, kk * 2)) = hb;
    if (v != 0.0) nz16[((size_t)chunk * Kt16 + kt) * 2 + (row >= 256)] = 1;
  }
  {  // TF32 hi/lo: chunk of 256 columns, K tile of 32; hi block then lo block
    const int chunk = o / 256, row = o % 256;
    const int64_t kt = k / 32;
    const int kk = (int)(k % 32);
    const size_t blk = ((size_t)chunk * Kt32 + kt) * (2 * 256 * 128);
    const float hi = tf32_round(sv);
    const float lo = tf32_round(sv - hi);
    *reinterpret_cast<float*>(t32 + blk + sw128_offset(row, kk * 4)) = hi;
    *reinterpret_cast<float*>(t32 + blk + 256 * 128 + sw128_offset(row, kk * 4)) = lo;
    if (v != 0.0) nz32[(size_t)chunk * Kt32 + kt] = 1;
  }
}

// ----------------------------------------------------------- tcgen05 helpers

__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);  // start address (16-byte units)
  d |= (uint64_t)1 << 16;                    // leading byte offset (unused by swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;          // stride byte offset: 8-row groups are 1024 B apart
  d |= (uint64_t)1 << 46;                    // descriptor version for sm_100 family
  d |= (uint64_t)2 << 61;                    // layout: 128-byte swizzle
  return d;
}

// instruction descriptor: D = F32, A/B format (1 = BF16, 2 = TF32), K-major, M = 128, N
__host__ __device__ constexpr uint32_t idesc_of(uint32_t ab_format, uint32_t N) {
  return (1u << 4) | (ab_format << 7) | (ab_format << 10) | ((N >> 3) << 17) | ((128u >> 4) << 24);
}

template <int KIND>  // 0: kind::f16 (BF16), 1: kind::tf32
__device__ __forceinline__ void mma(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  if constexpr (KIND == 0) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            dtmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            dtmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
  }
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// ----------------------------------------------------------- the contraction

struct GemmArgs {
  const double* X;
  int64_t P;
  int n;
  int order;
  int64_t Kt;           // K tiles per chunk
  const ClosMono* mono;
  const float* scale;
  const uint8_t* kind;  // per output column: 0 f, 1 g, 2 H, 3 padding
  const uint16_t* ti;
  const uint16_t* tj;
  const unsigned char* blocks;
  const int* live;      // [chunks][Kt] live K tiles, compacted, -1 padded
  const uint8_t* half;  // BF16: [chunks][Kt] nonzero halves (bit h)
  double* F;
  double* G;
  double* H;
  int* err;
  int Et;   // depth of the per-point power table (x^1..x^Et)
  const uint16_t* moff;  // power-table rows per closure monomial (null: decode var/exp)
  const int* tslots;     // per K tile: rows used by its monomials at most
  int tma;  // 1: the CTA's 128 x n point tile arrives by one tensor-map copy (n even, X 16-byte aligned)
};

template <int KIND>
struct GemmCfg;
template <>
struct GemmCfg<0> {  // BF16
  static constexpr int NC = 512, KT = 64, ESZ = 2, NOPS = 1;
  static constexpr uint32_t BBYTES = NC * 128;  // one block per stage
  static constexpr uint32_t ABYTES = 128 * 128;
};
template <>
struct GemmCfg<1> {  // TF32 hi/lo
  static constexpr int NC = 256, KT = 32, ESZ = 4, NOPS = 2;
  static constexpr uint32_t BBYTES = 2 * NC * 128;
  static constexpr uint32_t ABYTES = 2 * 128 * 128;
};

constexpr int kGemmThreads = 512;  // 4 producer threads per point row; 16 epilogue warps

// 2-D tiled tensor copy global -> shared (TMA), completion on `bar`; the
// innermost coordinate x must be a multiple of 16 bytes / element size
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

template <int KIND>
__global__ void __launch_bounds__(kGemmThreads, 1) gemm_eval_kernel(GemmArgs a, const __grid_constant__ CUtensorMap tmX) {
  using Cf = GemmCfg<KIND>;
  extern __shared__ __align__(1024) unsigned char sm_raw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)sm_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* stA[2] = {sm, sm + Cf::ABYTES};
  unsigned char* stB[2] = {sm + 2 * Cf::ABYTES, sm + 2 * Cf::ABYTES + Cf::BBYTES};
  float* pwt = (float*)(sm + 2 * Cf::ABYTES + 2 * Cf::BBYTES);  // [n][Et][128]: x^(e+1) of row r
  // closure-monomial records of the K tile being produced and of the next one
  // (bulk-copied one tile ahead: they are the same for every CTA and would
  // otherwise be read from L2 by every producer thread)
  ClosMono* recs[2];
  {
    unsigned char* rb = (unsigned char*)(((uintptr_t)(pwt + ((size_t)a.n * a.Et + 1) * 128) + 15) & ~(uintptr_t)15);
    recs[0] = (ClosMono*)rb;
    recs[1] = (ClosMono*)(rb + Cf::KT * sizeof(ClosMono));
  }
  __shared__ __align__(8) uint64_t full[2], done[2], fin, mrec[2], xbar;
  __shared__ uint32_t s_taddr;
  __shared__ int s_started[2];
  __shared__ int s_abort;
  const int tid = threadIdx.x, wid = tid >> 5;
  const int64_t p0 = (int64_t)blockIdx.x * 128;
  const int chunk = blockIdx.y;
  const int n = a.n;

  if (tid == 0) {
    mbar_init(&full[0], 1);
    mbar_init(&full[1], 1);
    mbar_init(&done[0], 1);
    mbar_init(&done[1], 1);
    mbar_init(&fin, 1);
    mbar_init(&mrec[0], 1);
    mbar_init(&mrec[1], 1);
    mbar_init(&xbar, 1);
    s_started[0] = s_started[1] = 0;
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (wid == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_taddr)),
                 "r"((uint32_t)Cf::NC)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  const int Et = a.Et;
  // the CTA's 128 x n points: one tensor-map copy into the (still unused) B
  // stage buffers, rows past P filled with zeros by the copy; or plain loads
  const double* Xt = reinterpret_cast<const double*>(stB[0]);
  if (a.tma) {
    if (tid == 0) {
      mbar_arrive_expect_tx(&xbar, (uint32_t)(128 * n * sizeof(double)));
      tma_load_2d(stB[0], &tmX, 0, (int)p0, &xbar);
    }
    __syncthreads();  // (the barriers' initialisation is visible to every thread from here)
    if (!mbar_wait_cta(&xbar, 0, a.err, 1)) {
      mbar_drain(&xbar, 0, a.err, 1);
      s_abort = 1;
    }
  }
  for (int i = tid; i < n * 128; i += kGemmThreads) {
    const int v = i / 128, rr = i % 128;
    const int64_t p = p0 + rr;
    const float x = a.tma ? (float)Xt[rr * n + v] : (p < a.P ? (float)a.X[p * n + v] : 0.0f);
    float pw = x;
    for (int e = 0; e < Et; ++e) {
      pwt[(v * Et + e) * 128 + rr] = pw;
      pw *= x;
    }
  }
  if (tid < 128) pwt[(size_t)n * Et * 128 + tid] = 1.0f;  // the row of ones (padding rows of a monomial)
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  // the B stage buffers are written by bulk copies from here on: order the
  // generic-proxy reads of the point tile before them
  if (tid == 0) fence_proxy_async_smem();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t taddr = s_taddr;
  const int* live = a.live + (size_t)chunk * a.Kt;
  int nlive = 0;
  while (nlive < a.Kt && live[nlive] >= 0) ++nlive;
  constexpr uint32_t kRecBytes = Cf::KT * sizeof(ClosMono);
  // records: the monomials' power-table rows when the plan built them (same
  // 32-byte stride), else their variables and exponents
  const ClosMono* recsrc = a.moff ? reinterpret_cast<const ClosMono*>(a.moff) : a.mono;
  if (tid == 0 && nlive > 0) {
    mbar_arrive_expect_tx(&mrec[0], kRecBytes);
    bulk_g2s(recs[0], recsrc + (int64_t)live[0] * Cf::KT, kRecBytes, &mrec[0]);
  }
  const unsigned char* gblk = a.blocks + (size_t)chunk * a.Kt * Cf::BBYTES;
  constexpr uint32_t kN = KIND == 0 ? 256 : 256;
  constexpr uint32_t idesc = idesc_of(KIND == 0 ? 1u : 2u, kN);
  const int r = tid & 127;   // this thread's point row
  const int part = tid >> 7;  // which quarter of the row's 16-byte chunks it produces

  for (int it = 0; it < nlive; ++it) {
    const int st = it & 1;
    const int kt = live[it];
    if (it >= 2) {
      if (!mbar_wait(&done[st], ((it - 2) >> 1) & 1, a.err)) s_abort = 1;
    }
    __syncthreads();
    if (s_abort) break;
    if (tid == 0) {
      mbar_arrive_expect_tx(&full[st], Cf::BBYTES);
      bulk_g2s(stB[st], gblk + (size_t)kt * Cf::BBYTES, Cf::BBYTES, &full[st]);
      if (it + 1 < nlive) {  // the other record buffer was last read before the barrier above
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&mrec[st ^ 1], kRecBytes);
        bulk_g2s(recs[st ^ 1], recsrc + (int64_t)live[it + 1] * Cf::KT, kRecBytes, &mrec[st ^ 1]);
      }
    }
    if (!mbar_wait(&mrec[st], (it >> 1) & 1, a.err)) s_abort = 1;
    // monomial tile: row r, KT consecutive closure monomials in 16-byte chunks;
    // thread part q fills chunks 2q and 2q+1
    const ClosMono* mm = recs[st];
    const int ns = a.moff ? a.tslots[kt] : 0;  // rows per monomial in this tile (uniform)
#pragma unroll 1
    for (int c16 = part * 2; c16 < part * 2 + 2; ++c16) {
      constexpr int PER = 16 / Cf::ESZ;
      float val[PER];
      if (a.moff) {
        // the chunk's monomials side by side: one 16-byte load of power-table
        // rows each (the same for the whole warp), then row by row a product
        // per monomial, so the PER products proceed together
        uint32_t ow[PER][4];
#pragma unroll
        for (int q = 0; q < PER; ++q) {
          const uint4 wo = reinterpret_cast<const uint4*>(mm + c16 * PER + q)[KIND == 0 ? 0 : 1];
          ow[q][0] = wo.x;
          ow[q][1] = wo.y;
          ow[q][2] = wo.z;
          ow[q][3] = wo.w;
          val[q] = 1.0f;
        }
#pragma unroll
        for (int s2 = 0; s2 < kMaxSupport; ++s2) {
          if (s2 >= ns) break;
#pragma unroll
          for (int q = 0; q < PER; ++q) {
            const uint32_t o = (ow[q][s2 >> 1] >> ((s2 & 1) * 16)) & 0xffffu;
            val[q] *= pwt[o * 128 + r];
          }
        }
      }
#pragma unroll
      for (int q = 0; q < PER && !a.moff; ++q) {
        const uint4* src = reinterpret_cast<const uint4*>(mm + c16 * PER + q);
        // two 16-byte loads: variables (8 x u16), then exponents (8 x u8)
        const uint4 wv = src[0];
        const uint4 we = src[1];
        const uint32_t vw[4] = {wv.x, wv.y, wv.z, wv.w};
        const uint32_t ew[2] = {we.x, we.y};
        const int kq = we.z & 0xff;  // support size of this monomial (same for the whole warp)
        float prod = 1.0f;
#pragma unroll
        for (int s2 = 0; s2 < kMaxSupport; ++s2) {
          if (s2 >= kq) break;
          const int e = (ew[s2 >> 2] >> ((s2 & 3) * 8)) & 0xff;
          {
            const int v = (vw[s2 >> 1] >> ((s2 & 1) * 16)) & 0xffff;
            if (e <= Et) {
              prod *= pwt[(v * Et + e - 1) * 128 + r];
            } else {
              const float x = pwt[(v * Et) * 128 + r];
              float pw = pwt[(v * Et + Et - 1) * 128 + r];
              for (int u = Et; u < e; ++u) pw *= x;
              prod *= pw;
            }
          }
        }
        val[q] = prod;
      }
      const size_t off = sw128_offset(r, c16 * 16);
      if constexpr (KIND == 0) {
        __nv_bfloat162 h[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) h[q] = __floats2bfloat162_rn(val[2 * q], val[2 * q + 1]);
        *reinterpret_cast<uint4*>(stA[st] + off) = *reinterpret_cast<uint4*>(h);
      } else {
        float hi[4], lo[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          hi[q] = tf32_round(val[q]);
          lo[q] = tf32_round(val[q] - hi[q]);
        }
        *reinterpret_cast<float4*>(stA[st] + off) = make_float4(hi[0], hi[1], hi[2], hi[3]);
        *reinterpret_cast<float4*>(stA[st] + 128 * 128 + off) = make_float4(lo[0], lo[1], lo[2], lo[3]);
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      if (!mbar_wait(&full[st], (it >> 1) & 1, a.err)) {
        s_abort = 1;
      } else {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t aA = smem_u32(stA[st]), aB = smem_u32(stB[st]);
        if constexpr (KIND == 0) {
          const uint8_t hm = a.half[(size_t)chunk * a.Kt + kt];
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            if (!(hm >> h & 1)) continue;
            const uint32_t d = taddr + h * 256;
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) {
              mma<0>(d, desc_sw128(aA + ks * 32), desc_sw128(aB + h * 256 * 128 + ks * 32), idesc,
                     (s_started[h] || ks > 0) ? 1u : 0u);
            }
            s_started[h] = 1;
          }
        } else {
          const uint32_t aAlo = aA + 128 * 128, aBlo = aB + 256 * 128;
#pragma unroll
          for (int ks = 0; ks < 4; ++ks) {
            const uint32_t acc0 = (s_started[0] || ks > 0) ? 1u : 0u;
            mma<1>(taddr, desc_sw128(aA + ks * 32), desc_sw128(aB + ks * 32), idesc, acc0);
            mma<1>(taddr, desc_sw128(aA + ks * 32), desc_sw128(aBlo + ks * 32), idesc, 1u);
            mma<1>(taddr, desc_sw128(aAlo + ks * 32), desc_sw128(aB + ks * 32), idesc, 1u);
          }
          s_started[0] = 1;
        }
        mma_commit(&done[st]);
      }
    }
  }
  // every MMA this CTA issued must be complete before TMEM is read or
  // released, on the abort path too: one more commit covers all of them
  __syncthreads();
  const bool issued = s_started[0] || s_started[1];
  if (issued && tid == 0) mma_commit(&fin);
  if (issued && !mbar_wait(&fin, 0, a.err)) s_abort = 1;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  __syncthreads();
  if (!s_abort && gridDim.y == 1) {
    // every output column is in this CTA: stage 64 points' columns in shared
    // memory (the A/B stage buffers are free now; rows padded to an odd
    // stride) and write each point's f, g and full H in output order, lanes
    // over consecutive addresses
    constexpr int NCS = Cf::NC + 1;
    static_assert(64 * NCS * 4 <= 2 * Cf::ABYTES + 2 * Cf::BBYTES, "staging tile fits the stage buffers");
    float* S = (float*)sm;
    const int nn = n * n, lane = tid & 31;
    constexpr int kCols = Cf::NC / (kGemmThreads / 128);
    for (int hf = 0; hf < 2; ++hf) {
      if (((wid & 3) >> 1) == hf) {  // TMEM quadrants 2hf, 2hf+1 hold rows 64hf..64hf+63
        const int rloc = ((wid & 3) & 1) * 32 + lane;
        for (int c = (wid >> 2) * kCols; c < ((wid >> 2) + 1) * kCols; c += 16) {
          float v[16];
          tmem_ld16(taddr + ((uint32_t)((wid & 3) * 32) << 16) + c, v);  // all lanes of the warp take part
          const bool have = KIND == 0 ? s_started[c / 256] != 0 : s_started[0] != 0;
#pragma unroll
          for (int q = 0; q < 16; ++q) S[rloc * NCS + c + q] = have ? v[q] : 0.0f;
        }
      }
      __syncthreads();
      for (int pr = wid; pr < 64; pr += kGemmThreads / 32) {
        const int64_t p = p0 + 64 * hf + pr;
        if (p >= a.P) continue;
        const float* Sr = S + pr * NCS;
        for (int k = lane; k <= n; k += 32) {  // column 0: f; column 1 + i: g_i
          const double y = (double)Sr[k] * (double)a.scale[k];
          if (k == 0) a.F[p] = y;
          else if (a.order >= 1) a.G[p * n + (k - 1)] = y;
        }
        if (a.order >= 2) {
          int i = lane / n, j = lane - (lane / n) * n;
          for (int k = lane; k < nn; k += 32) {
            const int lo = min(i, j), hi = max(i, j);
            const int col = 1 + n + lo * (2 * n - lo + 1) / 2 + (hi - lo);
            a.H[p * nn + k] = (double)Sr[col] * (double)a.scale[col];
            j += 32;
            while (j >= n) {
              j -= n;
              ++i;
            }
          }
        }
      }
      __syncthreads();
    }
  } else if (s_abort) {
    // a bounded wait gave up: this tile's outputs are NaN (the abort is
    // reported by polylab_eval_check)
    const int nn = n * n;
    for (int idx = tid; idx < 128 * Cf::NC; idx += kGemmThreads) {
      const int64_t p = p0 + idx / Cf::NC;
      const int o = chunk * Cf::NC + idx % Cf::NC;
      const int kd = a.kind[o];
      if (p >= a.P || kd == 3) continue;
      const double y = nan("");
      if (kd == 0) {
        a.F[p] = y;
      } else if (kd == 1) {
        if (a.order >= 1) a.G[p * n + a.ti[o]] = y;
      } else if (a.order >= 2) {
        a.H[p * nn + a.ti[o] * n + a.tj[o]] = y;
        a.H[p * nn + a.tj[o] * n + a.ti[o]] = y;
      }
    }
  } else {
    // several column chunks: warps w, w+4, w+8, w+12 read the same TMEM lane
    // quadrant (rows 32(w%4)..) and split the columns between them
    const int64_t p = p0 + (wid & 3) * 32 + (tid & 31);
    const int nn = n * n;
    constexpr int kCols = Cf::NC / (kGemmThreads / 128);
    for (int c = (wid >> 2) * kCols; c < ((wid >> 2) + 1) * kCols; c += 16) {
      float v[16];
      const int h = c / 256;
      tmem_ld16(taddr + ((uint32_t)((wid & 3) * 32) << 16) + c, v);  // all lanes of the warp take part
      if (p >= a.P) continue;
      const bool have = KIND == 0 ? s_started[h] != 0 : s_started[0] != 0;
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int o = chunk * Cf::NC + c + q;
        const int kd = a.kind[o];
        if (kd == 3) continue;
        const double y = have ? (double)v[q] * (double)a.scale[o] : 0.0;
        if (kd == 0) {
          a.F[p] = y;
        } else if (kd == 1) {
          if (a.order >= 1) a.G[p * n + a.ti[o]] = y;
        } else if (a.order >= 2) {
          const int i = a.ti[o], j = a.tj[o];
          a.H[p * nn + i * n + j] = y;
          a.H[p * nn + j * n + i] = y;
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (wid == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"((uint32_t)Cf::NC)
                 : "memory");
  }
}

template <int KIND>
constexpr size_t gemm_smem(int n, int Et) {
  using Cf = GemmCfg<KIND>;
  return 1024 + 2 * (size_t)Cf::ABYTES + 2 * (size_t)Cf::BBYTES + ((size_t)n * Et + 1) * 128 * 4 + 16 +
         2 * (size_t)Cf::KT * sizeof(ClosMono);
}

// deepest power table that fits next to the stages (at least x itself)
template <int KIND>
int table_depth(int n, int E) {
  int Et = std::max(1, E);
  while (Et > 1 && gemm_smem<KIND>(n, Et) > 225 * 1024) --Et;
  return Et;
}

}  // namespace

// ---------------------------------------------------------------- host side

polylab_status build_gemm_operand(polylab_plan* plan, cudaStream_t s) {
  const int n = plan->n;
  const int64_t m = plan->m;
  if (plan->max_support > kMaxSupport) return POLYLAB_ERR_UNSUPPORTED;
  const int64_t Nout = 1 + n + (int64_t)n * (n + 1) / 2;
  const int Npad = (int)ceil_div(Nout, kGemmNPadQuantum) * kGemmNPadQuantum;
  // degree bound of the closure set and the binomial table S(c, R) = C(R + c, c)
  std::vector<Term> host(std::max<int64_t>(m, 1));
  if (m > 0) {
    PL_CUDA(cudaMemcpyAsync(host.data(), plan->terms, m * sizeof(Term), cudaMemcpyDeviceToHost, s));
    PL_CUDA(cudaStreamSynchronize(s));
  }
  int D = 1;
  for (int64_t t = 0; t < m; ++t) {
    int d = 0;
    for (int q = 0; q < kMaxSupport; ++q) d += host[t].exp[q];
    D = std::max(D, d);
  }
  const int D1 = D + 1;
  std::vector<unsigned __int128> S((size_t)(n + 1) * D1);
  for (int R = 0; R <= D; ++R) S[R] = 1;
  for (int c = 1; c <= n; ++c) {
    S[(size_t)c * D1] = 1;
    for (int R = 1; R <= D; ++R) S[(size_t)c * D1 + R] = S[(size_t)(c - 1) * D1 + R] + S[(size_t)c * D1 + R - 1];
  }
  if (S[(size_t)n * D1 + D] >= ((unsigned __int128)1 << 63)) return POLYLAB_ERR_UNSUPPORTED;
  std::vector<uint64_t> S64(S.size());
  for (size_t i = 0; i < S.size(); ++i) S64[i] = (uint64_t)S[i];

  GemmOperand* g = new GemmOperand();
  plan->gemm = g;
  g->n = n;
  g->Npad = Npad;
  Scratch scr(s);
  uint64_t* dS;
  PL_TRY(scr.get(&dS, S64.size()));
  PL_CUDA(cudaMemcpyAsync(dS, S64.data(), S64.size() * 8, cudaMemcpyHostToDevice, s));
  const int64_t Nc = std::max<int64_t>(m, 1) * kCandPerTerm;
  uint64_t *keys, *akeys;
  uint32_t *vals, *avals;
  PL_TRY(scr.get(&keys, Nc));
  PL_TRY(scr.get(&akeys, Nc));
  PL_TRY(scr.get(&vals, Nc));
  PL_TRY(scr.get(&avals, Nc));
  if (m > 0) {
    closure_candidates<<<(unsigned)ceil_div(m, 128), 128, 0, s>>>(plan->terms, m, n, dS, D1, keys, vals);
    PL_TRY(launch_status("closure_candidates"));
  } else {
    PL_CUDA(cudaMemsetAsync(keys, 0xff, Nc * 8, s));
  }
  int which = 0;
  int* sort_err = nullptr;
  PL_TRY(scr.get(&sort_err, 1));
  PL_CUDA(cudaMemsetAsync(sort_err, 0, sizeof(int), s));
  PL_TRY((radix_sort<uint64_t, Scratch>(keys, vals, akeys, avals, Nc, 64, scr, s, &which, sort_err)));
  if (which) std::swap(keys, akeys);
  uint32_t *head, *pos;
  PL_TRY(scr.get(&head, Nc));
  PL_TRY(scr.get(&pos, Nc));
  mark_unique<<<(unsigned)ceil_div(Nc, 256), 256, 0, s>>>(keys, Nc, head);
  PL_TRY(launch_status("mark_unique"));
  PL_TRY(exclusive_scan(head, pos, Nc, scr, s));
  uint32_t hk[2];
  int herr = 0;
  PL_CUDA(cudaMemcpyAsync(&hk[0], pos + Nc - 1, 4, cudaMemcpyDeviceToHost, s));
  PL_CUDA(cudaMemcpyAsync(&hk[1], head + Nc - 1, 4, cudaMemcpyDeviceToHost, s));
  PL_CUDA(cudaMemcpyAsync(&herr, sort_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  PL_CUDA(cudaStreamSynchronize(s));
  if (herr) {
    set_last_message("radix sort: a look-back wait gave up");
    return POLYLAB_ERR_TIMEOUT;
  }
  const int64_t K = (int64_t)hk[0] + hk[1];
  const int64_t Kpad = std::max<int64_t>(64, ceil_div(K, 64) * 64);
  if ((double)Kpad * Npad > (double)(1ll << 28)) return POLYLAB_ERR_UNSUPPORTED;
  g->K = K;
  g->Kpad = Kpad;
  plan->closure = K;
  uint64_t* ukeys;
  PL_TRY(scr.get(&ukeys, std::max<int64_t>(K, 1)));
  gather_unique<<<(unsigned)ceil_div(Nc, 256), 256, 0, s>>>(keys, head, pos, Nc, ukeys);
  PL_TRY(launch_status("gather_unique"));
  PL_CUDA(cudaMallocAsync(&g->mono, Kpad * sizeof(ClosMono), s));
  closure_unrank<<<(unsigned)ceil_div(Kpad, 128), 128, 0, s>>>(ukeys, K, Kpad, n, dS, D1, g->mono);
  PL_TRY(launch_status("closure_unrank"));
  g->Et16 = table_depth<0>(n, plan->max_exp);
  g->Et32 = table_depth<1>(n, plan->max_exp);
  // rows per monomial at most (support) x ceil(max exponent / depth): valid when that is <= 8
  const int ksup = std::max(1, plan->max_support);
  g->off16 = ksup * ((plan->max_exp + g->Et16 - 1) / g->Et16) <= 8;
  g->off32 = ksup * ((plan->max_exp + g->Et32 - 1) / g->Et32) <= 8;
  if ((g->off16 || g->off32) && (int64_t)n * std::max(g->Et16, g->Et32) < 0xffff) {
    PL_CUDA(cudaMallocAsync(&g->moff, (size_t)Kpad * 16 * sizeof(uint16_t), s));
    PL_CUDA(cudaMallocAsync(&g->tslots, (size_t)(Kpad / 64 + Kpad / 32) * sizeof(int), s));
    PL_CUDA(cudaMemsetAsync(g->tslots, 0, (size_t)(Kpad / 64 + Kpad / 32) * sizeof(int), s));
    closure_offsets<<<(unsigned)ceil_div(Kpad, 128), 128, 0, s>>>(g->mono, Kpad, n, g->Et16, g->Et32, g->moff,
                                                                  g->tslots, g->tslots + Kpad / 64);
    PL_TRY(launch_status("closure_offsets"));
  }
  double* C;
  PL_TRY(scr.get(&C, (size_t)Kpad * Npad));
  PL_CUDA(cudaMemsetAsync(C, 0, (size_t)Kpad * Npad * 8, s));
  if (m > 0) {
    closure_fill<<<(unsigned)ceil_div(m, 128), 128, 0, s>>>(plan->terms, m, n, dS, D1, ukeys, K, Npad, C);
    PL_TRY(launch_status("closure_fill"));
  }
  PL_CUDA(cudaMallocAsync(&g->scale, Npad * sizeof(float), s));
  column_scale<<<(unsigned)ceil_div(Npad, 128), 128, 0, s>>>(C, Kpad, Npad, g->scale);
  PL_TRY(launch_status("column_scale"));
  const int64_t Kt16 = Kpad / 64, Kt32 = Kpad / 32;
  const int ch16 = Npad / 512, ch32 = Npad / 256;
  const size_t b16_bytes = (size_t)ch16 * Kt16 * 512 * 128, t32_bytes = (size_t)ch32 * Kt32 * 2 * 256 * 128;
  PL_CUDA(cudaMallocAsync(&g->b16, b16_bytes, s));
  PL_CUDA(cudaMallocAsync(&g->t32, t32_bytes, s));
  PL_CUDA(cudaMemsetAsync(g->b16, 0, b16_bytes, s));
  PL_CUDA(cudaMemsetAsync(g->t32, 0, t32_bytes, s));
  uint8_t *nz16, *nz32;
  PL_TRY(scr.get(&nz16, (size_t)ch16 * Kt16 * 2));
  PL_TRY(scr.get(&nz32, (size_t)ch32 * Kt32));
  PL_CUDA(cudaMemsetAsync(nz16, 0, (size_t)ch16 * Kt16 * 2, s));
  PL_CUDA(cudaMemsetAsync(nz32, 0, (size_t)ch32 * Kt32, s));
  closure_pack<<<(unsigned)ceil_div(Kpad * Npad, 256), 256, 0, s>>>(C, g->scale, Kpad, Npad, g->b16, g->t32, nz16,
                                                                     nz32);
  PL_TRY(launch_status("closure_pack"));
  std::vector<uint8_t> h16((size_t)ch16 * Kt16 * 2), h32((size_t)ch32 * Kt32);
  PL_CUDA(cudaMemcpyAsync(h16.data(), nz16, h16.size(), cudaMemcpyDeviceToHost, s));
  PL_CUDA(cudaMemcpyAsync(h32.data(), nz32, h32.size(), cudaMemcpyDeviceToHost, s));
  PL_CUDA(cudaStreamSynchronize(s));
  // live-tile lists and the per-tile half masks (BF16)
  std::vector<int> l16((size_t)ch16 * Kt16, -1), l32((size_t)ch32 * Kt32, -1);
  std::vector<uint8_t> half((size_t)ch16 * Kt16, 0);
  g->live16.assign(ch16, {});
  g->live32.assign(ch32, {});
  for (int c = 0; c < ch16; ++c) {
    int q = 0;
    for (int64_t kt = 0; kt < Kt16; ++kt) {
      const uint8_t hm = h16[((size_t)c * Kt16 + kt) * 2] | (h16[((size_t)c * Kt16 + kt) * 2 + 1] << 1);
      half[(size_t)c * Kt16 + kt] = hm;
      if (hm) {
        l16[(size_t)c * Kt16 + q++] = (int)kt;
        g->live16[c].push_back((int)kt);
      }
    }
  }
  for (int c = 0; c < ch32; ++c) {
    int q = 0;
    for (int64_t kt = 0; kt < Kt32; ++kt)
      if (h32[(size_t)c * Kt32 + kt]) {
        l32[(size_t)c * Kt32 + q++] = (int)kt;
        g->live32[c].push_back((int)kt);
      }
  }
  PL_CUDA(cudaMallocAsync(&g->live16_dev, l16.size() * sizeof(int), s));
  PL_CUDA(cudaMallocAsync(&g->live32_dev, l32.size() * sizeof(int), s));
  PL_CUDA(cudaMallocAsync(&g->half16_dev, half.size(), s));
  PL_CUDA(cudaMemcpyAsync(g->live16_dev, l16.data(), l16.size() * sizeof(int), cudaMemcpyHostToDevice, s));
  PL_CUDA(cudaMemcpyAsync(g->live32_dev, l32.data(), l32.size() * sizeof(int), cudaMemcpyHostToDevice, s));
  PL_CUDA(cudaMemcpyAsync(g->half16_dev, half.data(), half.size(), cudaMemcpyHostToDevice, s));
  // output column map
  std::vector<uint8_t> kind(Npad, 3);
  std::vector<uint16_t> ti(Npad, 0), tj(Npad, 0);
  kind[0] = 0;
  for (int i = 0; i < n; ++i) {
    kind[1 + i] = 1;
    ti[1 + i] = (uint16_t)i;
  }
  for (int i = 0; i < n; ++i)
    for (int j = i; j < n; ++j) {
      const int o = 1 + n + i * (2 * n - i + 1) / 2 + (j - i);
      kind[o] = 2;
      ti[o] = (uint16_t)i;
      tj[o] = (uint16_t)j;
    }
  PL_CUDA(cudaMallocAsync(&g->kind, Npad, s));
  PL_CUDA(cudaMallocAsync(&g->tri_i, Npad * 2, s));
  PL_CUDA(cudaMallocAsync(&g->tri_j, Npad * 2, s));
  PL_CUDA(cudaMemcpyAsync(g->kind, kind.data(), Npad, cudaMemcpyHostToDevice, s));
  PL_CUDA(cudaMemcpyAsync(g->tri_i, ti.data(), Npad * 2, cudaMemcpyHostToDevice, s));
  PL_CUDA(cudaMemcpyAsync(g->tri_j, tj.data(), Npad * 2, cudaMemcpyHostToDevice, s));
  PL_CUDA(cudaStreamSynchronize(s));
  return POLYLAB_OK;
}

// Set by a launch of the contraction whose bounded wait gave up; read and
// cleared by polylab_eval_check (one word per device that loads the library).
static __device__ int g_eval_wait_err;

static polylab_status eval_err_word(int** p) {
  PL_CUDA(cudaGetSymbolAddress((void**)p, g_eval_wait_err));
  return POLYLAB_OK;
}

// The tensor map of the points X (P rows of n doubles) with a 128 x n box,
// encoded through the driver entry point the runtime hands out.  False when
// the layout does not allow it (n odd: rows not a multiple of 16 bytes; X not
// 16-byte aligned; n > 128: the box would not fit the staging buffer) or the
// entry point is unavailable -- the kernel then loads the points itself.
static bool encode_points_map(const double* X, int64_t P, int n, CUtensorMap* map) {
  if (n % 2 != 0 || n > 128 || ((uintptr_t)X & 15) != 0 || P >= ((int64_t)1 << 31)) return false;
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
      cudaGetLastError();
      return false;
    }
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  const cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)P};
  const cuuint64_t strides[1] = {(cuuint64_t)n * sizeof(double)};
  const cuuint32_t box[2] = {(cuuint32_t)n, 128u};
  const cuuint32_t estr[2] = {1u, 1u};
  return encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<double*>(X), dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

polylab_status eval_gemm(const polylab_plan* plan, const double* X, int64_t P, int order, int prec, double* F,
                         double* G, double* H, cudaStream_t s) {
  if (P == 0) return POLYLAB_OK;
  const GemmOperand* g = plan->gemm;
  if (!g) return POLYLAB_ERR_INVALID_ARG;
  const int n = plan->n;
  int* err;
  PL_TRY(eval_err_word(&err));
  CUtensorMap tmX{};
  const bool tma = encode_points_map(X, P, n, &tmX);
  GemmArgs a{};
  a.X = X;
  a.P = P;
  a.n = n;
  a.order = order;
  a.mono = g->mono;
  a.scale = g->scale;
  a.kind = g->kind;
  a.ti = g->tri_i;
  a.tj = g->tri_j;
  a.F = F;
  a.G = G;
  a.H = H;
  a.err = err;
  a.tma = tma ? 1 : 0;
  a.moff = (prec == POLYLAB_BF16 ? g->off16 : g->off32) ? g->moff : nullptr;
  a.tslots = g->tslots ? (prec == POLYLAB_BF16 ? g->tslots : g->tslots + g->Kpad / 64) : nullptr;
  const unsigned gx = (unsigned)ceil_div(P, 128);
  if (prec == POLYLAB_BF16) {
    a.Et = table_depth<0>(n, plan->max_exp);
    const size_t smem = gemm_smem<0>(n, a.Et);
    if (smem > 227 * 1024) return POLYLAB_ERR_UNSUPPORTED;
    a.Kt = g->Kpad / 64;
    a.blocks = g->b16;
    a.live = g->live16_dev;
    a.half = g->half16_dev;
    PL_CUDA(cudaFuncSetAttribute(gemm_eval_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    gemm_eval_kernel<0><<<dim3(gx, g->Npad / 512), kGemmThreads, smem, s>>>(a, tmX);
  } else {
    a.Et = table_depth<1>(n, plan->max_exp);
    const size_t smem = gemm_smem<1>(n, a.Et);
    if (smem > 227 * 1024) return POLYLAB_ERR_UNSUPPORTED;
    a.Kt = g->Kpad / 32;
    a.blocks = g->t32;
    a.live = g->live32_dev;
    a.half = nullptr;
    PL_CUDA(cudaFuncSetAttribute(gemm_eval_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    gemm_eval_kernel<1><<<dim3(gx, g->Npad / 256), kGemmThreads, smem, s>>>(a, tmX);
  }
  return launch_status("gemm_eval_kernel");
}

}  // namespace polylab

extern "C" polylab_status polylab_eval_check(polylab_stream stream) {
  using namespace polylab;
  cudaStream_t s = (cudaStream_t)stream;
  int* err;
  PL_TRY(eval_err_word(&err));
  int flag = 0;
  PL_CUDA(cudaMemcpyAsync(&flag, err, sizeof(int), cudaMemcpyDeviceToHost, s));
  PL_CUDA(cudaStreamSynchronize(s));
  if (!flag) return POLYLAB_OK;
  set_last_message("a bounded wait of the tensor-core derivative contraction expired");
  PL_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
  PL_CUDA(cudaStreamSynchronize(s));
  return POLYLAB_ERR_TIMEOUT;
}

extern "C" polylab_status polylab_plan_gemm_info(const polylab_plan* plan, int64_t* K, int32_t* Npad,
                                                 int64_t* bf16_live_halves, int64_t* tf32_live_tiles) {
  if (!plan || !plan->gemm) return POLYLAB_ERR_INVALID_ARG;
  const polylab::GemmOperand* g = plan->gemm;
  if (K) *K = g->K;
  if (Npad) *Npad = g->Npad;
  if (bf16_live_halves) {
    // each live K tile of a 512-column chunk issues one or two 256-column halves
    std::vector<uint8_t> half((size_t)(g->Npad / 512) * (g->Kpad / 64));
    cudaMemcpy(half.data(), g->half16_dev, half.size(), cudaMemcpyDeviceToHost);
    int64_t h = 0;
    for (uint8_t v : half) h += (v & 1) + ((v >> 1) & 1);
    *bf16_live_halves = h;
  }
  if (tf32_live_tiles) {
    int64_t t = 0;
    for (const auto& v : g->live32) t += (int64_t)v.size();
    *tf32_live_tiles = t;
  }
  return POLYLAB_OK;
}
