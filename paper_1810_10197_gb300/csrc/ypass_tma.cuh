// The y passes (P2 inverse, P4 forward) in FP32 for ny = 256 with tensor-map tile copies and
// register-resident line transforms: the same results as k_py, by a different schedule.
//
// A CTA of 128 threads takes 8 consecutive kz columns of one (field, x) plane.  The TMA
// engine copies the tile -- 8 complex columns (64 bytes) of every row of the plane -- in one
// tensor-map box load into shared memory, with the 64-byte swizzle (the 16-byte chunks of
// a row permuted by bits 7-8 of its address) so that the 16 rows a half-warp reads in one
// column fall on 8 distinct bank groups; the copy completes on an mbarrier.  A group of 16
// threads owns one column: thread t takes the points y = t + 16 r (r = 0..15) into registers
// (the band between the retained ky of an inverse transform is zero), runs the 16 x 16
// transform of the register-resident z pass (one exchange through a padded per-column
// buffer; in the forward pass it shares the box's shared memory), writes the points it then
// holds (t + 16 m) into the box, and one tensor-map box store copies the tile to the output
// plane.  Columns past Mz are zero-filled by the load
// and skipped by the store.  Global loads and stores leave the LSU path: the element-wise
// copies and the shared-memory Stockham stages of k_py keep the L1TEX unit about 80% busy at
// 256^3.
//
// A wait for the load is bounded as in the z pass; one that runs out marks the step
// controller DNS_ERR_TIMEOUT and the CTA returns after a second bounded wait.
#pragma once

#include <cuda.h>

#include "zpass_rr.cuh"

namespace dns {

// shared memory: 1024-byte alignment slack | the box (256 rows x 64 B) | the exchange buffers
// of the 8 columns (8 x LSTR complex) | stage-1 twiddles | mbarrier.  In the forward pass the
// exchange buffers share the box's memory (the box is idle during the transform), which
// leaves room for more CTAs per SM; the inverse pass measured faster with separate buffers
// (0.091 against 0.094 ms at 256^3; forward 0.045 against 0.049 ms shared).
constexpr size_t kYtmaBox = (size_t)256 * 64;
constexpr size_t kYtmaXbuf = (size_t)8 * ZrrPlan<256>::LSTR * sizeof(float2);
static_assert(kYtmaXbuf >= kYtmaBox, "the exchange buffers cover a whole box");
template <bool INVERSE> __host__ __device__ constexpr size_t ytma_smem() {
  return 1024 + (INVERSE ? kYtmaBox + kYtmaXbuf : kYtmaXbuf) + 256 * sizeof(float2) + 16;
}

// stage-1 twiddles of the 256-point transform from a y pass's stage table (16 x 16 plan:
// entry (j, r) of stage 1 sits at j 15 + (r - 1) and holds W256^{j r}); tw1[r 16 + j] = W256^{j r}
__device__ __forceinline__ void rr256_twiddles(float2* tw1, const void* tab) {
  const float2* __restrict__ tws = reinterpret_cast<const float2*>(tab);
  for (int i = threadIdx.x; i < 256; i += blockDim.x) {
    const int r = i / 16, j = i % 16;
    tw1[i] = r == 0 ? make_float2(1.f, 0.f) : tws[j * 15 + (r - 1)];
  }
}

// byte offset of complex column c (0..7) of row r in a 64-byte-swizzled box of 64-byte rows
__device__ __forceinline__ int swz64(int r, int c) { return r * 64 + ((c * 8) ^ (((r >> 1) & 3) << 4)); }

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* tm, int x, int y, int z,
                                            unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
      ::"r"(smem_u32(dst)), "l"(reinterpret_cast<unsigned long long>(tm)), "r"(x), "r"(y), "r"(z),
        "r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void tma_store_3d(const CUtensorMap* tm, int x, int y, int z, const void* src) {
  asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];"
               ::"l"(reinterpret_cast<unsigned long long>(tm)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(src))
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// wait until the shared-memory sources of this thread's bulk stores have been read
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }

// tm_in / tm_out: FP32 views [planes][rows][2 Mz] of the pass input and output (rows My or
// ny), box {16, rows, 1}, 64-byte swizzle.  grid (ceil(Mz / 8), nx, fields).
template <bool INVERSE>
__global__ void __launch_bounds__(128) k_py_tma(const PassArgs a, const __grid_constant__ CUtensorMap tm_in,
                                                const __grid_constant__ CUtensorMap tm_out) {
  constexpr int N = 256, G = 16, TZ = 8;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (gated_off(a.ctrl, a.gate_k1)) return;
  const Geom& g = a.g;
  const unsigned base = smem_u32(smem_raw);
  unsigned char* box = smem_raw + (((base + 1023u) & ~1023u) - base);      // 1024-byte aligned
  float2* xbuf = reinterpret_cast<float2*>(INVERSE ? box + kYtmaBox : box);  // [8][LSTR]
  float2* tw1 = xbuf + TZ * ZrrPlan<N>::LSTR;                                 // [16][16]
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(tw1 + 256);
  const int tid = threadIdx.x, gi = tid / G, t = tid % G;
  const int plane = blockIdx.z * g.nx + blockIdx.y, kz0 = blockIdx.x * TZ;
  const int My = g.My, Ky = g.Ky;
  const int rows_in = INVERSE ? My : N;
  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_expect_tx(bar, (unsigned)rows_in * 64u);
    tma_load_3d(box, &tm_in, 2 * kz0, 0, plane, bar);
  }
  rr256_twiddles(tw1, a.tw);
  __syncthreads();
  const bool arrived = mbar_wait_bounded(bar, 0);
  if (!__syncthreads_and(arrived)) {
    if (tid == 0) {
      if (a.ctrl) {
        DnsCtrl* cw = const_cast<DnsCtrl*>(a.ctrl);
        cw->status = ST_TIMEOUT;
        cw->done = 1;
      }
      mbar_wait_bounded(bar, 0);   // let the copy still in flight land (bounded)
    }
    return;
  }
  // the column's points y = t + 16 r
  float2 v[16];
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    const int y = t + G * r;
    int row = y;
    if (INVERSE) row = y <= Ky ? y : (y >= N - Ky ? y - (N - My) : -1);
    v[r] = row >= 0 ? *reinterpret_cast<const float2*>(box + swz64(row, gi)) : make_float2(0.f, 0.f);
  }
  __syncthreads();                                    // the box is read: it takes the output
  float2* xb = xbuf + gi * ZrrPlan<N>::LSTR;
  zrr_fft<N, INVERSE ? +1 : -1, float2>(v, xb, tw1, t);
  if (!INVERSE) __syncthreads();                      // shared region: every exchange is done
#pragma unroll
  for (int m = 0; m < 16; ++m) {
    const int k = t + G * m;
    int row = k;
    if (!INVERSE) row = k <= Ky ? k : (k >= N - Ky ? k - (N - My) : -1);
    if (row >= 0) *reinterpret_cast<float2*>(box + swz64(row, gi)) = v[m];
  }
  fence_proxy_async_smem();                           // the box store reads what was written
  __syncthreads();
  if (tid == 0) {
    tma_store_3d(&tm_out, 2 * kz0, 0, plane, box);
    bulk_commit();
    bulk_wait_read();
  }
}

}  // namespace dns
