// Training kernels of the learned preconditioner: loss and its gradient by
// hand-written backpropagation, Adam, initialisation and the BF16 packing
// used for inference inside the stochastic solver.
//
// Loss (mean over points and the 4 probes of each point):
//   L = |Pi (D y + U U^T y) - z|^2 / |z|^2,  y = Pi (H + rI) Pi z,
// with (D, U) from the network (see mlp.cuh).  For one point, with
// uy = U^T y, w = D y + U uy, res = w - e (e.w) - z (e.res = 0 since z is in
// e-perp) and gw = 2 res / |z|^2:
//   dL/dD_i = sum_k gw_ik y_ik,
//   dL/dU_ic = sum_k (gw_ik uy_kc + y_ik (U^T gw)_kc),
// then through D_i = exp(clip(o_0))/s_i, U_ic = 0.1 o_c / sqrt(s_i) and the
// tanh layer to the parameters.
#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"
#include "mlp.cuh"

namespace polylab {
namespace {

constexpr int kNZ = 4;      // probes per training point
constexpr int kMlpNT = 256;

template <int N>
__device__ __forceinline__ void block_sum_n(float (&v)[N], float* red) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
  for (int s = 0; s < N; ++s)
    for (int o = 16; o; o >>= 1) v[s] += __shfl_xor_sync(0xffffffffu, v[s], o);
  __syncthreads();
  if (l == 0)
#pragma unroll
    for (int s = 0; s < N; ++s) red[w * N + s] = v[s];
  __syncthreads();
  if (threadIdx.x < N) {
    float acc = 0.f;
    for (int q = 0; q < kMlpNT / 32; ++q) acc += red[q * N + threadIdx.x];
    red[(kMlpNT / 32) * N + threadIdx.x] = acc;
  }
  __syncthreads();
#pragma unroll
  for (int s = 0; s < N; ++s) v[s] = red[(kMlpNT / 32) * N + s];
  __syncthreads();
}

__global__ void __launch_bounds__(kMlpNT) mlp_loss_grad_kernel(const float* __restrict__ theta, int64_t P, int n,
                                                               const float* __restrict__ feats,
                                                               const float* __restrict__ hd,
                                                               const float* __restrict__ E,
                                                               const float* __restrict__ Z,
                                                               const float* __restrict__ Y, float r, float scale,
                                                               float* __restrict__ grad, float* __restrict__ loss) {
  __shared__ float th[kMlpParams];
  __shared__ float gacc[kMlpParams];
  __shared__ float red[(kMlpNT / 32 + 1) * 16];
  __shared__ float s_loss;
  const int tid = threadIdx.x, lane = tid & 31;
  for (int j = tid; j < kMlpParams; j += kMlpNT) {
    th[j] = theta[j];
    gacc[j] = 0.f;
  }
  if (tid == 0) s_loss = 0.f;
  __syncthreads();
  for (int64_t p = blockIdx.x; p < P; p += gridDim.x) {
    const float* fp = feats + p * (int64_t)n * kMlpF;
    const float* hp = hd + p * (int64_t)n;
    const float* ep = E + p * (int64_t)n;
    const float* zp = Z + p * (int64_t)n * kNZ;
    const float* yp = Y + p * (int64_t)n * kNZ;
    auto factors = [&](int i, float* h, float* o, float* D, float* U0, float* U1) {
      float f[kMlpF];
#pragma unroll
      for (int q = 0; q < kMlpF; ++q) f[q] = fp[i * kMlpF + q];
      mlp_forward(th, f, h, o);
      mlp_factors(o, hp[i], r, D, U0, U1);
    };
    // pass A: uy = U^T y and |z|^2 per probe
    float A[3 * kNZ];
#pragma unroll
    for (int s = 0; s < 3 * kNZ; ++s) A[s] = 0.f;
    for (int i = tid; i < n; i += kMlpNT) {
      float h[kMlpH], o[kMlpO], D, U0, U1;
      factors(i, h, o, &D, &U0, &U1);
#pragma unroll
      for (int k = 0; k < kNZ; ++k) {
        const float y = yp[i * kNZ + k], z = zp[i * kNZ + k];
        A[k] += U0 * y;
        A[kNZ + k] += U1 * y;
        A[2 * kNZ + k] += z * z;
      }
    }
    block_sum_n<3 * kNZ>(A, red);
    // pass B: e.w per probe
    float B[kNZ];
#pragma unroll
    for (int k = 0; k < kNZ; ++k) B[k] = 0.f;
    for (int i = tid; i < n; i += kMlpNT) {
      float h[kMlpH], o[kMlpO], D, U0, U1;
      factors(i, h, o, &D, &U0, &U1);
#pragma unroll
      for (int k = 0; k < kNZ; ++k) {
        const float w = D * yp[i * kNZ + k] + U0 * A[k] + U1 * A[kNZ + k];
        B[k] += ep[i] * w;
      }
    }
    block_sum_n<kNZ>(B, red);
    // pass C: loss and U^T gw per probe
    float Cc[2 * kNZ + 1];
#pragma unroll
    for (int s = 0; s < 2 * kNZ + 1; ++s) Cc[s] = 0.f;
    for (int i = tid; i < n; i += kMlpNT) {
      float h[kMlpH], o[kMlpO], D, U0, U1;
      factors(i, h, o, &D, &U0, &U1);
#pragma unroll
      for (int k = 0; k < kNZ; ++k) {
        const float y = yp[i * kNZ + k];
        const float w = D * y + U0 * A[k] + U1 * A[kNZ + k];
        const float res = w - ep[i] * B[k] - zp[i * kNZ + k];
        const float gw = 2.f * res / A[2 * kNZ + k];
        Cc[k] += U0 * gw;
        Cc[kNZ + k] += U1 * gw;
        Cc[2 * kNZ] += res * res / A[2 * kNZ + k];
      }
    }
    block_sum_n<2 * kNZ + 1>(Cc, red);
    if (tid == 0) s_loss += Cc[2 * kNZ];
    // pass D: backpropagation, warp-reduced parameter gradients
    for (int base = (tid & ~31); base < n; base += kMlpNT) {
      const int i = base + lane;
      float f[kMlpF], h[kMlpH], o[kMlpO], go[kMlpO];
#pragma unroll
      for (int q = 0; q < kMlpF; ++q) f[q] = 0.f;
#pragma unroll
      for (int k = 0; k < kMlpO; ++k) go[k] = 0.f;
      if (i < n) {
#pragma unroll
        for (int q = 0; q < kMlpF; ++q) f[q] = fp[i * kMlpF + q];
        mlp_forward(th, f, h, o);
        float D, U0, U1;
        mlp_factors(o, hp[i], r, &D, &U0, &U1);
        float gD = 0.f, gU0 = 0.f, gU1 = 0.f;
#pragma unroll
        for (int k = 0; k < kNZ; ++k) {
          const float y = yp[i * kNZ + k];
          const float w = D * y + U0 * A[k] + U1 * A[kNZ + k];
          const float res = w - ep[i] * B[k] - zp[i * kNZ + k];
          const float gw = 2.f * res / A[2 * kNZ + k];
          gD += gw * y;
          gU0 += gw * A[k] + y * Cc[k];
          gU1 += gw * A[kNZ + k] + y * Cc[kNZ + k];
        }
        const float s = fabsf(hp[i]) + r;
        go[0] = (o[0] > -5.f && o[0] < 5.f) ? gD * D : 0.f;
        go[1] = gU0 * 0.1f * rsqrtf(s);
        go[2] = gU1 * 0.1f * rsqrtf(s);
      } else {
#pragma unroll
        for (int j = 0; j < kMlpH; ++j) h[j] = 0.f;
      }
      // output layer
#pragma unroll
      for (int j = 0; j < kMlpH; ++j) {
        float gh = 0.f;
#pragma unroll
        for (int k = 0; k < kMlpO; ++k) {
          float v = h[j] * go[k];
          for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
          if (lane == 0) atomicAdd(&gacc[kMlpW2 + j * kMlpO + k], v);
          gh += go[k] * th[kMlpW2 + j * kMlpO + k];
        }
        const float ga = gh * (1.f - h[j] * h[j]);
        float vb = ga;
        for (int off = 16; off; off >>= 1) vb += __shfl_xor_sync(0xffffffffu, vb, off);
        if (lane == 0) atomicAdd(&gacc[kMlpB1 + j], vb);
#pragma unroll
        for (int q = 0; q < kMlpF; ++q) {
          float v = f[q] * ga;
          for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
          if (lane == 0) atomicAdd(&gacc[kMlpW1 + q * kMlpH + j], v);
        }
      }
#pragma unroll
      for (int k = 0; k < kMlpO; ++k) {
        float v = go[k];
        for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if (lane == 0) atomicAdd(&gacc[kMlpB2 + k], v);
      }
    }
    __syncthreads();
  }
  __syncthreads();
  for (int j = tid; j < kMlpParams; j += kMlpNT) atomicAdd(&grad[j], gacc[j] * scale);
  if (tid == 0) atomicAdd(loss, s_loss * scale);
}

__global__ void mlp_adam_kernel(float* __restrict__ th, const float* __restrict__ g, float* __restrict__ m,
                                float* __restrict__ v, int step, float lr) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= kMlpParams) return;
  const float b1 = 0.9f, b2 = 0.999f;
  m[j] = b1 * m[j] + (1.f - b1) * g[j];
  v[j] = b2 * v[j] + (1.f - b2) * g[j] * g[j];
  const float mh = m[j] / (1.f - powf(b1, (float)step));
  const float vh = v[j] / (1.f - powf(b2, (float)step));
  th[j] -= lr * mh / (sqrtf(vh) + 1e-8f);
}

__device__ __forceinline__ uint64_t mix64(uint64_t seed, uint64_t k) {
  uint64_t z = seed + (k + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// W1 ~ U(-1, 1) / sqrt(F); the low-rank outputs' weights (columns 1, 2 of
// W2) ~ U(-1, 1) * 0.05; everything else 0.  The diagonal output starts at
// Jacobi; the low-rank head must not start at zero weights, where U = 0 and
// the gradient of U U^T with respect to U vanishes (training would never
// leave it).
__global__ void mlp_init_kernel(float* __restrict__ th, uint64_t seed) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= kMlpParams) return;
  const double u = (double)(mix64(seed, j) >> 11) * (1.0 / 9007199254740992.0);
  float v = 0.f;
  if (j < kMlpB1) v = (float)((2.0 * u - 1.0) / sqrt((double)kMlpF));
  else if (j >= kMlpW2 && j < kMlpB2 && (j - kMlpW2) % kMlpO != 0) v = (float)((2.0 * u - 1.0) * 0.05);
  th[j] = v;
}

__global__ void mlp_pack_kernel(const float* __restrict__ th, __nv_bfloat16* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < kMlpParams) out[j] = __float2bfloat16_rn(th[j]);
}

}  // namespace
}  // namespace polylab

using namespace polylab;

extern "C" {

int32_t polylab_mlp_param_count(void) { return kMlpParams; }

polylab_status polylab_mlp_init(float* params, uint64_t seed, polylab_stream stream) {
  if (!params) return POLYLAB_ERR_INVALID_ARG;
  mlp_init_kernel<<<2, 256, 0, (cudaStream_t)stream>>>(params, seed);
  return launch_status("mlp_init_kernel");
}

polylab_status polylab_mlp_loss_grad(const float* params, int64_t P, int32_t n, const float* feats, const float* hdiag,
                                     const float* e, const float* Z, const float* Y, double regularization,
                                     float* grad, float* loss, polylab_stream stream) {
  if (!params || !grad || !loss || P < 1 || n < 1 || !feats || !hdiag || !e || !Z || !Y)
    return POLYLAB_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  PL_CUDA(cudaMemsetAsync(grad, 0, kMlpParams * sizeof(float), s));
  PL_CUDA(cudaMemsetAsync(loss, 0, sizeof(float), s));
  const int grid = (int)std::min<int64_t>(P, (int64_t)num_sms() * 4);
  mlp_loss_grad_kernel<<<grid, kMlpNT, 0, s>>>(params, P, n, feats, hdiag, e, Z, Y, (float)regularization,
                                               1.0f / (float)(P * kNZ), grad, loss);
  return launch_status("mlp_loss_grad_kernel");
}

polylab_status polylab_mlp_adam(float* params, const float* grad, float* m, float* v, int32_t step, float lr,
                                polylab_stream stream) {
  if (!params || !grad || !m || !v || step < 1) return POLYLAB_ERR_INVALID_ARG;
  mlp_adam_kernel<<<2, 256, 0, (cudaStream_t)stream>>>(params, grad, m, v, step, lr);
  return launch_status("mlp_adam_kernel");
}

polylab_status polylab_mlp_pack(const float* params, void* packed, polylab_stream stream) {
  if (!params || !packed) return POLYLAB_ERR_INVALID_ARG;
  mlp_pack_kernel<<<2, 256, 0, (cudaStream_t)stream>>>(params, (__nv_bfloat16*)packed);
  return launch_status("mlp_pack_kernel");
}

}  // extern "C"
