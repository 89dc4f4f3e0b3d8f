// The x-inverse pass (P1) in FP32 for nx = 256, velocity form, with tensor-map tile copies and
// register-resident line transforms: the same result as k_p1, by a different schedule.
//
// A CTA of 128 threads takes 8 consecutive (ky, kz) columns.  The TMA engine copies the
// tile's stage input -- 8 complex values of every retained kx row of each of the 3 fields --
// in three tensor-map box loads on one mbarrier: FP64 rows of 128 bytes with the 128-byte
// swizzle (the 16-byte chunks of a row permuted by bits 7-9 of its address), or, for the
// FP32 stage-input scratch of the DNS_FP32 form, rows of 64 bytes with the 64-byte swizzle.
// A group of 16 threads owns one column: thread t reads Y_c (c = 0..2) at the modes whose
// transform position is t + 16 r (positions 0..Kx and nx-Kx..nx-1 hold the retained kx, the
// rest are zero), converts them to FP32, scales by 1/(nx ny nz) and keeps the 48 values in
// registers.  The input's shared memory then holds the exchange buffers and two output boxes:
// the six lines u0, u1, u2, omega0, omega1, omega2 (omega = i kappa x u formed from the
// registers) are transformed one after another (the z pass's 16 x 16 plan, one exchange),
// written into an output box (256 x rows of 8 FP32 complex, 64-byte swizzle) and copied to
// the pass output by a tensor-map box store, the two boxes alternating so that a store
// overlaps the next line's transform.
//
// The stage input is named by a controller slot that the kernel resolves; the launcher
// passes tensor maps for the buffers the slot can name (two at most) and the kernel takes the
// one at the resolved address.  The wait for the loads is bounded as in the z pass; a wait
// that runs out, or a stage input at no mapped address, marks the step controller
// DNS_ERR_TIMEOUT and the CTA returns.
#pragma once

#include <cuda.h>

#include "ypass_tma.cuh"

namespace dns {

// shared memory of k_p1_tma: 1024-byte alignment slack | the input region (three field boxes,
// each rounded up to 1024 bytes; later the exchange buffers and two output boxes) | stage-1
// twiddles | mbarrier
__host__ __device__ constexpr size_t xtma_in_box(int Mx, bool y32) {
  return ((size_t)Mx * (y32 ? 64 : 128) + 1023) / 1024 * 1024;
}
constexpr size_t kXtmaXbuf = (size_t)8 * ZrrPlan<256>::LSTR * sizeof(float2);   // 17408 = 17 x 1024
constexpr size_t kXtmaOutBox = (size_t)256 * 64;
__host__ __device__ constexpr size_t xtma_region(int Mx, bool y32) {
  return 3 * xtma_in_box(Mx, y32) > kXtmaXbuf + 2 * kXtmaOutBox ? 3 * xtma_in_box(Mx, y32)
                                                                  : kXtmaXbuf + 2 * kXtmaOutBox;
}
__host__ __device__ constexpr size_t xtma_p1_smem(int Mx, bool y32) {
  return 1024 + xtma_region(Mx, y32) + 256 * sizeof(float2) + 16;
}

// byte offset of complex column c (0..7) of row r in a 128-byte-swizzled box of 128-byte rows
__device__ __forceinline__ int swz128(int r, int c) { return r * 128 + ((c ^ (r & 7)) << 4); }

__device__ __forceinline__ void bulk_wait_read_1() { asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); }

// tm_y0 / tm_y1: views [3][Mx][2 MyMz] of the buffers a.ycand[0] / a.ycand[1] (FP64, or FP32
// when Y32), box {16, Mx, 1}; tm_out: FP32 view [6][nx][2 MyMz] of the pass output, box
// {16, nx, 1}.  grid ceil(MyMz / 8).
template <int N, bool Y32>
__global__ void __launch_bounds__(128, 3) k_p1_tma(const PassArgs a, const __grid_constant__ CUtensorMap tm_y0,
                                                   const __grid_constant__ CUtensorMap tm_y1,
                                                   const __grid_constant__ CUtensorMap tm_out) {
  static_assert(N == 256, "tensor-map x-inverse pass: nx = 256");
  constexpr int G = 16, TC = 8;
  constexpr int ROWB = Y32 ? 64 : 128;                 // bytes per input box row
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (gated_off(a.ctrl, a.gate_k1)) return;
  const Geom& g = a.g;
  const int Kx = g.Kx, Mx = g.Mx;
  const size_t inbox = xtma_in_box(Mx, Y32);
  const unsigned base = smem_u32(smem_raw);
  unsigned char* region = smem_raw + (((base + 1023u) & ~1023u) - base);   // 1024-byte aligned
  float2* xbuf = reinterpret_cast<float2*>(region);                          // after the input is read
  unsigned char* obox = region + kXtmaXbuf;                                  // 2 output boxes
  float2* tw1 = reinterpret_cast<float2*>(region + xtma_region(Mx, Y32));
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(tw1 + 256);
  const int tid = threadIdx.x, gi = tid / G, t = tid % G;
  const int col0 = blockIdx.x * TC;
  const double2* Y = resolve_in(a.y, a.ctrl, a.yslot);
  const CUtensorMap* tmy = (const void*)Y == a.ycand[0] ? &tm_y0 : ((const void*)Y == a.ycand[1] ? &tm_y1 : nullptr);
  if (!tmy) {   // uniform over the grid, before any barrier
    if (tid == 0 && a.ctrl) {
      DnsCtrl* cw = const_cast<DnsCtrl*>(a.ctrl);
      cw->status = ST_TIMEOUT;
      cw->done = 1;
    }
    return;
  }
  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_expect_tx(bar, 3u * (unsigned)Mx * ROWB);
    for (int f = 0; f < 3; ++f) tma_load_3d(region + f * inbox, tmy, 2 * col0, 0, f, bar);
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
      mbar_wait_bounded(bar, 0);   // let the copies still in flight land (bounded)
    }
    return;
  }
  const int MyMz = g.MyMz;
  const int col = min(col0 + gi, MyMz - 1);
  const int jy = col / g.Mz, kz = col - jy * g.Mz;
  const float s = (float)g.inv_n3, sx = (float)g.sx;
  const float ky = (float)g.sy * (float)signed_mode(jy, g.Ky, g.My), kzz = (float)g.sz * (float)kz;
  // stage input at this thread's 16 transform positions p = t + 16 r, scaled
  float2 y0[16], y1[16], y2[16];
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    const int p = t + G * r;
    const int ix = p <= Kx ? p : (p >= N - Kx ? p - (N - Mx) : -1);
    float2 a0 = make_float2(0.f, 0.f), a1 = a0, a2 = a0;
    if (ix >= 0) {
      if constexpr (Y32) {
        const int o = swz64(ix, gi);
        a0 = *reinterpret_cast<const float2*>(region + o);
        a1 = *reinterpret_cast<const float2*>(region + inbox + o);
        a2 = *reinterpret_cast<const float2*>(region + 2 * inbox + o);
      } else {
        const int o = swz128(ix, gi);
        const double2 d0 = *reinterpret_cast<const double2*>(region + o);
        const double2 d1 = *reinterpret_cast<const double2*>(region + inbox + o);
        const double2 d2 = *reinterpret_cast<const double2*>(region + 2 * inbox + o);
        a0 = make_float2(d2f_bits(d0.x), d2f_bits(d0.y));
        a1 = make_float2(d2f_bits(d1.x), d2f_bits(d1.y));
        a2 = make_float2(d2f_bits(d2.x), d2f_bits(d2.y));
      }
    }
    y0[r] = cscale(a0, s); y1[r] = cscale(a1, s); y2[r] = cscale(a2, s);
  }
  __syncthreads();                       // the input is read: the region takes the exchanges and outputs
  float2* xb = xbuf + gi * ZrrPlan<N>::LSTR;
#pragma unroll
  for (int f = 0; f < 6; ++f) {
    float2 v[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const int p = t + G * r;
      const float kx = sx * (float)(p <= N / 2 ? p : p - N);
      float2 c;
      if (f == 0) c = y0[r];
      else if (f == 1) c = y1[r];
      else if (f == 2) c = y2[r];
      else if (f == 3) c = make_float2(ky * y2[r].x - kzz * y1[r].x, ky * y2[r].y - kzz * y1[r].y);
      else if (f == 4) c = make_float2(kzz * y0[r].x - kx * y2[r].x, kzz * y0[r].y - kx * y2[r].y);
      else c = make_float2(kx * y1[r].x - ky * y0[r].x, kx * y1[r].y - ky * y0[r].y);
      v[r] = f < 3 ? c : make_float2(-c.y, c.x);     // omega = i (kappa x u)
    }
    zrr_fft<N, +1, float2>(v, xb, tw1, t);
    unsigned char* ob = obox + (f & 1) * kXtmaOutBox;
    if (f >= 2) {                        // the store of line f - 2 has read this box
      if (tid == 0) bulk_wait_read_1();
      __syncthreads();
    }
#pragma unroll
    for (int m = 0; m < 16; ++m) *reinterpret_cast<float2*>(ob + swz64(t + G * m, gi)) = v[m];
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      tma_store_3d(&tm_out, 2 * col0, 0, f, ob);
      bulk_commit();
    }
  }
  if (tid == 0) bulk_wait_read();
}

}  // namespace dns
