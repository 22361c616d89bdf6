// The learned diagonal-plus-low-rank preconditioner: network shape, feature
// map and forward pass shared by the training kernels and the stochastic
// solver.  Per coordinate i of a point (a_i = |H_ii| + r):
//   f_i = [log(a_i), log(sum_{j != i} sum_t |d_i d_j t(x)| + r), x_i,
//          n e_i^2, log(|g_i| + 1e-30), sum_{j != i} H_ij / a_i,
//          sum_{j != i} H_ij / a_j]
//   h = tanh(W1^T f + b1) (32 units), o = W2^T h + b2 (3 outputs)
//   D_i = exp(clip(o_0, -5, 5)) / a_i,  U_ik = 0.1 o_k / sqrt(a_i)
// and the preconditioner is Pi (D + U U^T) Pi; zero output weights give Jacobi.
// The two signed features carry couplings of one sign shared by many
// coordinates (a collective, soft or stiff, mode of the Hessian), which
// random-sign couplings do not.
// Parameters: one flat vector W1 (7 x 32, row-major), b1, W2 (32 x 3), b2.
#pragma once

#include "common.cuh"

namespace polylab {

constexpr int kMlpF = 7;
constexpr int kMlpH = 32;
constexpr int kMlpO = 3;
constexpr int kMlpParams = kMlpF * kMlpH + kMlpH + kMlpH * kMlpO + kMlpO;  // 355
constexpr int kMlpW1 = 0, kMlpB1 = kMlpF * kMlpH, kMlpW2 = kMlpB1 + kMlpH, kMlpB2 = kMlpW2 + kMlpH * kMlpO;

// rowsum = sum_{j != i} H_ij, rowsum_a = sum_{j != i} H_ij / a_j
__device__ __forceinline__ void mlp_features(float* f, float hdiag, float offsum, float x, float e, float g, int n,
                                             float r, float rowsum, float rowsum_a) {
  const float a = fabsf(hdiag) + r;
  f[0] = logf(a);
  f[1] = logf(offsum + r);
  f[2] = x;
  f[3] = (float)n * e * e;
  f[4] = logf(fabsf(g) + 1e-30f);
  f[5] = rowsum / a;
  f[6] = rowsum_a;
}

// forward pass; h (hidden activations) and o (outputs) returned
__device__ __forceinline__ void mlp_forward(const float* __restrict__ th, const float* f, float* h, float* o) {
#pragma unroll
  for (int j = 0; j < kMlpH; ++j) {
    float a = th[kMlpB1 + j];
#pragma unroll
    for (int q = 0; q < kMlpF; ++q) a += f[q] * th[kMlpW1 + q * kMlpH + j];
    h[j] = tanhf(a);
  }
#pragma unroll
  for (int k = 0; k < kMlpO; ++k) {
    float a = th[kMlpB2 + k];
#pragma unroll
    for (int j = 0; j < kMlpH; ++j) a += h[j] * th[kMlpW2 + j * kMlpO + k];
    o[k] = a;
  }
}

__device__ __forceinline__ void mlp_factors(const float* o, float hdiag, float r, float* D, float* U0, float* U1) {
  const float s = fabsf(hdiag) + r;
  *D = expf(fminf(fmaxf(o[0], -5.0f), 5.0f)) / s;
  const float rs = rsqrtf(s);
  *U0 = 0.1f * o[1] * rs;
  *U1 = 0.1f * o[2] * rs;
}

}  // namespace polylab
