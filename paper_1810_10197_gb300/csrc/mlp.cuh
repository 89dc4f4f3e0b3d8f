// Learned step-size proposal: a 16-64-64-1 perceptron with bfloat16 weights and FP32
// arithmetic.  Parameter vector layout (float): W1[64][16], b1[64], W2[64][64], b2[64],
// w3[64], b3.  y = w3 . relu(W2 relu(W1 x + b1) + b2) + b3 proposes log(h_next / h).
#pragma once

#include <cuda_bf16.h>

namespace dns {

constexpr int kMlpIn = 16, kMlpH = 64;
constexpr int kMlpOffW1 = 0;
constexpr int kMlpOffB1 = kMlpOffW1 + kMlpH * kMlpIn;
constexpr int kMlpOffW2 = kMlpOffB1 + kMlpH;
constexpr int kMlpOffB2 = kMlpOffW2 + kMlpH * kMlpH;
constexpr int kMlpOffW3 = kMlpOffB2 + kMlpH;
constexpr int kMlpOffB3 = kMlpOffW3 + kMlpH;
constexpr int kMlpParams = kMlpOffB3 + 1;   // 5313

// weights as deployed: rounded to bfloat16 (nearest even), computed in FP32
__device__ __forceinline__ float bf16r(float w) { return __bfloat162float(__float2bfloat16_rn(w)); }

// Block-parallel forward of one feature vector (threads 0..63 active), all threads of the
// block must call it.  feat: 16 floats in shared memory; work: 128 floats of shared memory.
// Returns y in thread 0.
__device__ __forceinline__ float mlp_forward_block(const float* __restrict__ P, const float* feat,
                                                   float* work) {
  const int t = threadIdx.x;
  if (t < kMlpH) {
    float z = bf16r(P[kMlpOffB1 + t]);
#pragma unroll
    for (int i = 0; i < kMlpIn; ++i) z = fmaf(bf16r(P[kMlpOffW1 + t * kMlpIn + i]), feat[i], z);
    work[t] = fmaxf(z, 0.f);
  }
  __syncthreads();
  if (t < kMlpH) {
    float z = bf16r(P[kMlpOffB2 + t]);
    for (int j = 0; j < kMlpH; ++j) z = fmaf(bf16r(P[kMlpOffW2 + t * kMlpH + j]), work[j], z);
    work[kMlpH + t] = fmaxf(z, 0.f) * bf16r(P[kMlpOffW3 + t]);
  }
  __syncthreads();
  float y = 0.f;
  if (t == 0) {
    y = bf16r(P[kMlpOffB3]);
    for (int k = 0; k < kMlpH; ++k) y += work[kMlpH + k];
  }
  __syncthreads();
  return y;
}

// Host launchers (mlp.cu).
cudaError_t launch_mlp_forward(const float* P, const float* X, int n, float* Y, cudaStream_t s);
cudaError_t launch_mlp_train(float* P, const float* X, const float* T, int n, int steps, int batch,
                             float lr, unsigned seed, float* loss_hist, float* grad_out, cudaStream_t s);

}  // namespace dns
