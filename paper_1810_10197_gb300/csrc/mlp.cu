// Training and inference kernels of the learned step-size proposal (mlp.cuh), and their C ABI.
// The network is tiny (5313 parameters): one CTA trains it with Adam, all state in shared
// memory; the forward pass uses bfloat16-rounded weights and FP32 arithmetic.
#include <cmath>

#include "../../include/dns.h"
#include "mlp.cuh"

namespace dns {

namespace {

constexpr int kMaxBatch = 128;
constexpr int kTrainThreads = 512;

__device__ __forceinline__ unsigned mix32(unsigned x) {
  x ^= x >> 16; x *= 0x7feb352dU; x ^= x >> 15; x *= 0x846ca68bU; x ^= x >> 16;
  return x;
}

// One CTA.  grad_out != null: loss and gradient over samples 0..n-1 (n <= kMaxBatch), no update.
// Otherwise `steps` Adam steps (beta1 0.9, beta2 0.999, eps 1e-8) on random mini-batches of
// `batch` samples; P is updated in place and loss_hist[step] records each batch loss.
__global__ void __launch_bounds__(kTrainThreads)
k_mlp_train(float* Pg, const float* __restrict__ X, const float* __restrict__ T, int n, int steps,
            int batch, float lr, unsigned seed, float* loss_hist, float* grad_out) {
  extern __shared__ float sm[];
  float* P = sm;
  float* Pb = P + kMlpParams;
  float* G = Pb + kMlpParams;
  float* Mo = G + kMlpParams;
  float* Vo = Mo + kMlpParams;
  float* A1 = Vo + kMlpParams;
  float* A2 = A1 + kMaxBatch * kMlpH;
  float* DY = A2 + kMaxBatch * kMlpH;
  int* IDX = reinterpret_cast<int*>(DY + kMaxBatch);
  float* red = reinterpret_cast<float*>(IDX + kMaxBatch);
  const int tid = threadIdx.x, nth = blockDim.x;
  for (int i = tid; i < kMlpParams; i += nth) { P[i] = Pg[i]; Mo[i] = 0.f; Vo[i] = 0.f; }
  const bool grad_only = grad_out != nullptr;
  const int nsteps = grad_only ? 1 : steps;
  const int B = grad_only ? n : batch;
  float b1p = 1.f, b2p = 1.f;
  for (int step = 0; step < nsteps; ++step) {
    for (int b = tid; b < B; b += nth)
      IDX[b] = grad_only ? b : (int)(mix32(seed ^ mix32(0x9E3779B1U * (unsigned)(step + 1) + (unsigned)b)) % (unsigned)n);
    for (int i = tid; i < kMlpParams; i += nth) { Pb[i] = bf16r(P[i]); G[i] = 0.f; }
    if (tid < 32) red[tid] = 0.f;
    __syncthreads();
    for (int e = tid; e < B * kMlpH; e += nth) {
      const int b = e / kMlpH, j = e % kMlpH;
      const float* x = X + (size_t)IDX[b] * kMlpIn;
      float z = Pb[kMlpOffB1 + j];
#pragma unroll
      for (int i = 0; i < kMlpIn; ++i) z = fmaf(Pb[kMlpOffW1 + j * kMlpIn + i], x[i], z);
      A1[e] = fmaxf(z, 0.f);
    }
    __syncthreads();
    for (int e = tid; e < B * kMlpH; e += nth) {
      const int b = e / kMlpH, k = e % kMlpH;
      float z = Pb[kMlpOffB2 + k];
      for (int j = 0; j < kMlpH; ++j) z = fmaf(Pb[kMlpOffW2 + k * kMlpH + j], A1[b * kMlpH + j], z);
      A2[e] = fmaxf(z, 0.f);
    }
    __syncthreads();
    float lsum = 0.f;
    for (int b = tid; b < B; b += nth) {
      float y = Pb[kMlpOffB3];
      for (int k = 0; k < kMlpH; ++k) y = fmaf(Pb[kMlpOffW3 + k], A2[b * kMlpH + k], y);
      const float r = y - T[IDX[b]];
      DY[b] = 2.f * r / (float)B;
      lsum += r * r;
    }
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if ((tid & 31) == 0) red[tid >> 5] = lsum;
    __syncthreads();
    for (int k = tid; k <= kMlpH; k += nth) {
      float s = 0.f;
      if (k < kMlpH) {
        for (int b = 0; b < B; ++b) s = fmaf(DY[b], A2[b * kMlpH + k], s);
        G[kMlpOffW3 + k] = s;
      } else {
        for (int b = 0; b < B; ++b) s += DY[b];
        G[kMlpOffB3] = s;
      }
    }
    __syncthreads();
    for (int e = tid; e < B * kMlpH; e += nth) {
      const int b = e / kMlpH, k = e % kMlpH;
      A2[e] = A2[e] > 0.f ? DY[b] * Pb[kMlpOffW3 + k] : 0.f;
    }
    __syncthreads();
    for (int e = tid; e < kMlpH * kMlpH + kMlpH; e += nth) {
      float s = 0.f;
      if (e < kMlpH * kMlpH) {
        const int k = e / kMlpH, j = e % kMlpH;
        for (int b = 0; b < B; ++b) s = fmaf(A2[b * kMlpH + k], A1[b * kMlpH + j], s);
        G[kMlpOffW2 + e] = s;
      } else {
        const int k = e - kMlpH * kMlpH;
        for (int b = 0; b < B; ++b) s += A2[b * kMlpH + k];
        G[kMlpOffB2 + k] = s;
      }
    }
    __syncthreads();
    for (int e = tid; e < B * kMlpH; e += nth) {
      const int b = e / kMlpH, j = e % kMlpH;
      float s = 0.f;
      if (A1[e] > 0.f)
        for (int k = 0; k < kMlpH; ++k) s = fmaf(A2[b * kMlpH + k], Pb[kMlpOffW2 + k * kMlpH + j], s);
      A1[e] = s;
    }
    __syncthreads();
    for (int e = tid; e < kMlpH * kMlpIn + kMlpH; e += nth) {
      float s = 0.f;
      if (e < kMlpH * kMlpIn) {
        const int j = e / kMlpIn, i = e % kMlpIn;
        for (int b = 0; b < B; ++b) s = fmaf(A1[b * kMlpH + j], X[(size_t)IDX[b] * kMlpIn + i], s);
        G[kMlpOffW1 + e] = s;
      } else {
        const int j = e - kMlpH * kMlpIn;
        for (int b = 0; b < B; ++b) s += A1[b * kMlpH + j];
        G[kMlpOffB1 + j] = s;
      }
    }
    __syncthreads();
    float loss = 0.f;
    if (tid == 0) {
      for (int w = 0; w < (nth + 31) / 32; ++w) loss += red[w];
      loss /= (float)B;
      if (loss_hist) loss_hist[step] = loss;
    }
    if (grad_only) {
      for (int i = tid; i < kMlpParams; i += nth) grad_out[i] = G[i];
      return;
    }
    b1p *= 0.9f;
    b2p *= 0.999f;
    for (int i = tid; i < kMlpParams; i += nth) {
      const float g = G[i];
      Mo[i] = 0.9f * Mo[i] + 0.1f * g;
      Vo[i] = 0.999f * Vo[i] + 0.001f * g * g;
      const float mh = Mo[i] / (1.f - b1p), vh = Vo[i] / (1.f - b2p);
      P[i] -= lr * mh / (sqrtf(vh) + 1e-8f);
    }
    __syncthreads();
  }
  for (int i = tid; i < kMlpParams; i += nth) Pg[i] = P[i];
}

__global__ void k_mlp_forward(const float* __restrict__ P, const float* __restrict__ X, int n, float* Y) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n) return;
  const float* x = X + (size_t)b * kMlpIn;
  float a1[kMlpH];
  for (int j = 0; j < kMlpH; ++j) {
    float z = bf16r(P[kMlpOffB1 + j]);
    for (int i = 0; i < kMlpIn; ++i) z = fmaf(bf16r(P[kMlpOffW1 + j * kMlpIn + i]), x[i], z);
    a1[j] = fmaxf(z, 0.f);
  }
  float y = bf16r(P[kMlpOffB3]);
  for (int k = 0; k < kMlpH; ++k) {
    float z = bf16r(P[kMlpOffB2 + k]);
    for (int j = 0; j < kMlpH; ++j) z = fmaf(bf16r(P[kMlpOffW2 + k * kMlpH + j]), a1[j], z);
    y = fmaf(bf16r(P[kMlpOffW3 + k]), fmaxf(z, 0.f), y);
  }
  Y[b] = y;
}

size_t train_smem() {
  return (size_t)5 * kMlpParams * sizeof(float) + (size_t)2 * kMaxBatch * kMlpH * sizeof(float) +
         (size_t)kMaxBatch * (sizeof(float) + sizeof(int)) + 32 * sizeof(float);
}

}  // namespace

cudaError_t launch_mlp_forward(const float* P, const float* X, int n, float* Y, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_mlp_forward<<<(n + 127) / 128, 128, 0, s>>>(P, X, n, Y);
  return cudaGetLastError();
}

cudaError_t launch_mlp_train(float* P, const float* X, const float* T, int n, int steps, int batch,
                             float lr, unsigned seed, float* loss_hist, float* grad_out, cudaStream_t s) {
  const size_t smem = train_smem();
  cudaError_t e = cudaFuncSetAttribute(k_mlp_train, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_mlp_train<<<1, kTrainThreads, smem, s>>>(P, X, T, n, steps, batch, lr, seed, loss_hist, grad_out);
  return cudaGetLastError();
}

}  // namespace dns

extern "C" {

dns_status dns_mlp_forward(const float* params, const float* x, int n, float* y, void* stream) {
  if (!params || !x || !y || n < 0) return DNS_ERR_ARG;
  return dns::launch_mlp_forward(params, x, n, y, reinterpret_cast<cudaStream_t>(stream)) == cudaSuccess
             ? DNS_OK : DNS_ERR_CUDA;
}

dns_status dns_mlp_loss_grad(const float* params, const float* x, const float* t, int n, float* grad,
                             float* loss, void* stream) {
  if (!params || !x || !t || !grad || !loss || n < 1 || n > dns::kMaxBatch) return DNS_ERR_ARG;
  return dns::launch_mlp_train(const_cast<float*>(params), x, t, n, 0, n, 0.f, 0u, loss, grad,
                               reinterpret_cast<cudaStream_t>(stream)) == cudaSuccess ? DNS_OK : DNS_ERR_CUDA;
}

dns_status dns_mlp_train(float* params, const float* x, const float* t, int n, int steps, int batch,
                         float lr, unsigned seed, float* loss_hist, void* stream) {
  if (!params || !x || !t || n < 1 || steps < 0 || batch < 1 || batch > dns::kMaxBatch || !(lr > 0.f))
    return DNS_ERR_ARG;
  return dns::launch_mlp_train(params, x, t, n, steps, batch, lr, seed, loss_hist, nullptr,
                               reinterpret_cast<cudaStream_t>(stream)) == cudaSuccess ? DNS_OK : DNS_ERR_CUDA;
}

}  // extern "C"
