// Batches of (polynomial, point) work items for the exact affine-normal kernel.
#pragma once

#include <vector>

#include "common.cuh"

namespace polylab {

struct ExactDesc {
  const Term* terms;
  int64_t m;
  int n;
  int E;             // largest exponent (power-table depth)
  int mats_in_smem;  // frame stage: 0 = matrices in the per-CTA global workspace
  int h_in_smem;     // term stage: 0 = H accumulated in the point's workspace slot
  int w_in_smem;     // third stage: 0 = W read from the point's workspace slot
  int64_t mat_off;   // first element of point 0's n x n slot in the matrix workspaces
  int64_t vec_off;   // first element of point 0's record in the vector workspace
  int max_support;
  int64_t koff[kMaxSupport + 2];   // support-size groups of the sorted term list
  int64_t k3off[kMaxSupport + 1];  // first term of degree >= 3 in each group
  const uint32_t* gather;           // gather form of the term sweep (or nullptr)
  const int64_t* gather_chunk;
  int n_gchunks;
  double x_lo, x_hi;  // gather form used when every |x_v| is in [x_lo, x_hi]
  const double* X;   // P x n
  int64_t P;
  double* D;
  double* Dunit;
  polylab_an_info* info;
};

struct ExactConfig {
  int threads = 0;        // frame-stage CTA size: 64, 128 or 256 (0: by largest n)
  int ctas_per_sm = 0;    // cap on resident frame-stage CTAs per SM (0: occupancy limit)
  int order = 1;          // 1: most expensive polynomials first, 0: as given
  int term_threads = 0;   // CTA size of the gradient/Hessian term sweep (0: 128)
  int terms_ctas = 0;     // caps on resident CTAs per SM of the term sweeps (0: occupancy limit)
  int third_ctas = 0;
  int frame_split = 1;    // frame stage in classes of polynomials by n
  int third_threads = 0;  // CTA size of the third-derivative sweep (0: 128)
  int third_split = 2;    // launches of the third-derivative sweep (ranges of support sizes)
};

// A class of the split frame stage: polynomials with n in (n_lo, n_hi], a
// contiguous range of the frame stage's own work order (n descending), run
// as one launch with its own CTA size and shared memory.
constexpr int kFrameClasses = 3;
struct FrameClass {
  int n_lo, n_hi, threads;
  int64_t begin = 0, end = 0;
  size_t smem = 0;
  size_t tsmem = 0;   // the gradient/Hessian sweep's gather launch over the same class (two points per pass)
  size_t tsmem1 = 0;  // the same at one point per pass
  size_t t3smem = 0;  // the third-derivative sweep's launches over the same class
};

struct ExactBatch {
  polylab_an_opts opts{};
  ExactConfig cfg;
  std::vector<ExactDesc> host_descs;
  std::vector<int> host_order;
  std::vector<int64_t> host_prefix;
  ExactDesc* descs = nullptr;  // DEVICE copies
  int* order = nullptr;
  int64_t* prefix = nullptr;
  int* counter = nullptr;  // one work counter per stage
  int* err = nullptr;      // device flag: a bounded wait of a stage expired
  int n_desc = 0;
  int64_t total = 0;
  size_t smem[3] = {0, 0, 0};
  // split frame stage: per-descriptor frame-stage shared memory, the frame
  // work order and prefix (host and DEVICE), the classes, one counter each
  std::vector<size_t> frame_need, third_need;
  std::vector<int> host_forder;
  std::vector<int64_t> host_fprefix;
  int* forder = nullptr;
  int64_t* fprefix = nullptr;
  int* fcounter = nullptr;
  FrameClass fclass[kFrameClasses];
  // the gradient/Hessian sweep by class of n: per-descriptor
  // shared memory of its gather launch, that of the term-by-term launch, the
  // list of passes left to it and [count, one work counter per launch]
  std::vector<size_t> terms_need, terms_need1;  // (two and one points per pass)
  size_t terms_fb_smem = 0;
  int64_t* tfb = nullptr;
  int64_t tfb_cap = 0;
  int* tfb_ctl = nullptr;
  // workspaces: H and W (one n x n slot per point each), small vectors
  void* ws_h = nullptr;
  void* ws_w = nullptr;
  void* ws_v = nullptr;
  size_t ws_mat_bytes = 0, ws_vec_bytes = 0;
  size_t gws_stride = 0;
  unsigned char* gws = nullptr;
  size_t gws_bytes = 0;
  std::vector<polylab_plan*> owned_plans;
};

polylab_status exact_batch_init(ExactBatch* b, int n, const polylab_plan* const* plans, const double* const* X,
                                const int64_t* P, const polylab_an_opts* o, double* const* D,
                                double* const* Dunit, polylab_an_info* const* info, cudaStream_t s);
polylab_status exact_batch_upload_order(ExactBatch* b, cudaStream_t s);
void exact_frame_classes(ExactBatch* b);
polylab_status exact_batch_relayout(ExactBatch* b, cudaStream_t s);
void exact_batch_release(ExactBatch* b, cudaStream_t s);
polylab_status prepare_exact_batch(ExactBatch* b);
polylab_status run_exact_batch(ExactBatch* b, cudaStream_t s);
polylab_status run_exact_stage(ExactBatch* b, int stage, cudaStream_t s);
double exact_point_cost(const ExactDesc& d, int max_support);

}  // namespace polylab

// The opaque public batch handle.
struct polylab_batch {
  polylab::ExactBatch b;
};
