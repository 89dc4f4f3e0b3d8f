// dns_measure_fp64_rate: the issue rate of this GPU's FP64 pipe, measured.  The FP64 form of
// the passes is bound by that pipe (an FP64 right-hand side at 256^3 has about 2 flops per
// byte of traffic, far above the FP64 ridge), so its roofline is stated against this
// measured rate rather than a datasheet figure.
#include <cmath>

#include "../../include/dns.h"

namespace {

constexpr int kChains = 8;        // independent dependency chains per thread
constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 8;

// kChains chains of x <- x a + b (DFMA) or x <- x + b (DADD), `iters` times each.  The
// results are folded and written only if they reach an impossible value, so the loop stays.
template <bool FMA>
__global__ void __launch_bounds__(kThreads) k_probe_fp64(double* sink, int iters, double a, double b) {
  double x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = 1.0 + 1e-3 * (threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = FMA ? fma(x[c], a, b) : x[c] + b;
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == -1.0) sink[0] = s;
}

template <bool FMA>
cudaError_t time_probe(cudaStream_t st, int blocks, int iters, double* sink, float* ms) {
  cudaEvent_t e0, e1;
  cudaError_t e;
  if ((e = cudaEventCreate(&e0)) != cudaSuccess) return e;
  if ((e = cudaEventCreate(&e1)) != cudaSuccess) { cudaEventDestroy(e0); return e; }
  const double a = 0.9999999, b = 1e-7;
  k_probe_fp64<FMA><<<blocks, kThreads, 0, st>>>(sink, iters / 8, a, b);   // warm-up
  cudaEventRecord(e0, st);
  k_probe_fp64<FMA><<<blocks, kThreads, 0, st>>>(sink, iters, a, b);
  cudaEventRecord(e1, st);
  e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return e;
}

}  // namespace

extern "C" dns_status dns_measure_fp64_rate(void* stream, double* dfma_per_s, double* dadd_per_s) {
  if (!dfma_per_s || !dadd_per_s) return DNS_ERR_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return DNS_ERR_CUDA;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  double* sink = nullptr;
  // a one-double scratch for the impossible-value store (freed below)
  if (cudaMalloc(&sink, sizeof(double)) != cudaSuccess) return DNS_ERR_OOM;
  const int blocks = sms * kBlocksPerSm;
  const int iters = 16384;
  float ms_fma = 0.f, ms_add = 0.f;
  cudaError_t e = time_probe<true>(st, blocks, iters, sink, &ms_fma);
  if (e == cudaSuccess) e = time_probe<false>(st, blocks, iters, sink, &ms_add);
  cudaFree(sink);
  if (e != cudaSuccess || !(ms_fma > 0.f) || !(ms_add > 0.f)) return DNS_ERR_CUDA;
  const double instr = (double)blocks * kThreads * (double)iters * kChains;
  *dfma_per_s = instr / (ms_fma * 1e-3);
  *dadd_per_s = instr / (ms_add * 1e-3);
  return DNS_OK;
}
