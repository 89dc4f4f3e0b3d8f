// The y passes (P2 inverse, P4 forward) in FP32 for ny = 128 and 256 with tensor-map tile
// copies and register-resident line transforms: the same results as k_py, by a different
// schedule.
//
// A CTA of 128 threads takes TZ consecutive kz columns of one (field, x) plane (8 at ny = 256,
// 16 at 128).  The TMA engine copies the tile -- TZ complex columns (64 or 128 bytes) of every
// row of the plane -- in one tensor-map box load into shared memory, with the swizzle of the
// row width (the 16-byte chunks of a row permuted by bits 7-8 or 7-9 of its address) so that
// the rows a half-warp reads in one column fall on distinct bank groups; the copy completes
// on an mbarrier.  A group of G = ny / 16 threads owns one column: thread t takes the points
// y = t + G r (r = 0..15) into registers (the band between the retained ky of an inverse
// transform is zero), runs the 16 x G transform of the register-resident z pass (one
// exchange through a padded per-column buffer; in the forward pass it shares the box's
// shared memory), writes the points it then holds (t + G m) into the box, and one tensor-map
// box store copies the tile to the output plane.  Columns past Mz are zero-filled by the load
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

// Tile geometry for line length N (16 x G plan, G = N / 16 threads per column): 128 / G
// columns per CTA (8 at 256, 16 at 128), rows of 8 bytes per column (64 or 128 bytes, with
// the 64- or 128-byte swizzle).
template <int N> struct YtmaTile {
  static constexpr int G = N / 16, TZ = 128 / G, ROWB = TZ * 8;
  static constexpr size_t BOX = (size_t)N * ROWB;
  static constexpr size_t XBUF = (size_t)TZ * ZrrPlan<N>::LSTR * sizeof(float2);
  static_assert(N == 128 || N == 256, "tensor-map y passes: 128 or 256 points");
  static_assert(XBUF >= BOX, "the exchange buffers cover a whole box");
};
// shared memory: 1024-byte alignment slack | the box (N rows) | the exchange buffers of the
// columns | stage-1 twiddles | mbarrier.  In the forward pass the exchange buffers share the
// box's memory (the box is idle during the transform), which leaves room for more CTAs per
// SM; the inverse pass measured faster with separate buffers (0.091 against 0.094 ms at
// 256^3; forward 0.045 against 0.049 ms shared).
template <int N, bool INVERSE> __host__ __device__ constexpr size_t ytma_smem() {
  using P = YtmaTile<N>;
  return 1024 + (INVERSE ? P::BOX + P::XBUF : P::XBUF) + 16 * P::G * sizeof(float2) + 16;
}

// stage-1 twiddles of the N-point transform (16 x G plan) from an x or y pass's stage table:
// entry (j, r) of stage 1 sits at j (G - 1) + (r - 1) and holds W_N^{j r}; tw1[r 16 + j] = W_N^{j r}
template <int N>
__device__ __forceinline__ void rr_twiddles(float2* tw1, const void* tab) {
  constexpr int G = N / 16;
  const float2* __restrict__ tws = reinterpret_cast<const float2*>(tab);
  for (int i = threadIdx.x; i < 16 * G; i += blockDim.x) {
    const int r = i / 16, j = i % 16;
    tw1[i] = r == 0 ? make_float2(1.f, 0.f) : tws[j * (G - 1) + (r - 1)];
  }
}
__device__ __forceinline__ void rr256_twiddles(float2* tw1, const void* tab) { rr_twiddles<256>(tw1, tab); }

// byte offset of byte b of row r in a swizzled box of ROWB-byte rows (64-byte swizzle: the
// 16-byte chunk index XOR address bits 7-8; 128-byte swizzle: XOR bits 7-9)
template <int ROWB> __device__ __forceinline__ int swz(int r, int b) {
  static_assert(ROWB == 64 || ROWB == 128, "64- or 128-byte rows");
  return ROWB == 64 ? r * 64 + (b ^ (((r >> 1) & 3) << 4)) : r * 128 + (b ^ ((r & 7) << 4));
}
// complex column c (0..7) of row r in a 64-byte-swizzled box of 64-byte rows
__device__ __forceinline__ int swz64(int r, int c) { return swz<64>(r, c * 8); }

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
// ny), box {2 TZ, rows, 1}, swizzle of the row width.  grid (ceil(Mz / TZ), nx, fields).
template <int N, bool INVERSE>
__global__ void __launch_bounds__(128) k_py_tma(const PassArgs a, const __grid_constant__ CUtensorMap tm_in,
                                                const __grid_constant__ CUtensorMap tm_out) {
  using P = YtmaTile<N>;
  constexpr int G = P::G, TZ = P::TZ, ROWB = P::ROWB;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (gated_off(a.ctrl, a.gate_k1)) return;
  const Geom& g = a.g;
  const unsigned base = smem_u32(smem_raw);
  unsigned char* box = smem_raw + (((base + 1023u) & ~1023u) - base);        // 1024-byte aligned
  float2* xbuf = reinterpret_cast<float2*>(INVERSE ? box + P::BOX : box);      // [TZ][LSTR]
  float2* tw1 = xbuf + TZ * ZrrPlan<N>::LSTR;                                  // [G][16]
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(tw1 + 16 * G);
  const int tid = threadIdx.x, gi = tid / G, t = tid % G;
  const int plane = blockIdx.z * g.nx + blockIdx.y, kz0 = blockIdx.x * TZ;
  const int My = g.My, Ky = g.Ky;
  const int rows_in = INVERSE ? My : N;
  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_expect_tx(bar, (unsigned)rows_in * ROWB);
    tma_load_3d(box, &tm_in, 2 * kz0, 0, plane, bar);
  }
  rr_twiddles<N>(tw1, a.tw);
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
  // the column's points y = t + G r
  float2 v[16];
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    const int y = t + G * r;
    int row = y;
    if (INVERSE) row = y <= Ky ? y : (y >= N - Ky ? y - (N - My) : -1);
    v[r] = row >= 0 ? *reinterpret_cast<const float2*>(box + swz<ROWB>(row, gi * 8)) : make_float2(0.f, 0.f);
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
    if (row >= 0) *reinterpret_cast<float2*>(box + swz<ROWB>(row, gi * 8)) = v[m];
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
