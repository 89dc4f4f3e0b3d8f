// The five passes of one pseudo-spectral right-hand-side evaluation, Eq. (ufdef):
//
//   P1  x-inverse : retained Y -> (u, omega = i kappa x Y) / (nx ny nz), inverse DFT along x
//   P2  y-inverse : inverse DFT along y of the 6 fields (retained kz planes only)
//   P3  z + cross : inverse real DFT along z (6 fields), u x omega in physical space, forward
//                   real DFT along z keeping kz <= Kz (3 fields)
//   P4  y-forward : forward DFT along y keeping |ky| <= Ky
//   P5  x-forward : forward DFT along x keeping |kx| <= Kx, then Leray projection, viscous
//                   term and forcing: k = P(kappa) N - nu |kappa|^2 Y + F   (FP64 epilogue)
//
// Intermediate layouts (T = double or float complex, kz innermost):
//   after P1: A[6][nx][My][Mz]   after P2: B[6][nx][ny][Mz]   after P3: A[3][nx][ny][Mz]
//   after P4: B[3][nx][My][Mz]   (A and B are two scratch buffers reused across passes)
// Only retained (ky, kz) columns are transformed along x and only retained kz planes along y,
// so the work and traffic skip the modes the 2/3 rule zeroes.
#pragma once

#include <type_traits>

#include "common.cuh"
#include "fft.cuh"

namespace dns {

struct PassArgs {
  Geom g;
  const DnsCtrl* ctrl;   // may be null (plain right-hand side)
  int gate_k1;           // skip unless ctrl->need_k1
  int yslot;             // slot of the stage input (P1, P5), -1 = use y
  int kslot;             // slot of the output (P5), -1 = use kout
  const double2* y;      // stage input, compact [3][Mx][My][Mz]
  double2* kout;         // output, compact
  const void* in;        // pass input (T complex)
  void* out;             // pass output (T complex)
  const void* tw;        // twiddle tables (T complex) of this pass's axis, see twiddle_count
  double nu;
  double kf2;            // forcing band |kappa|^2 <= kf2 (0: no forcing)
  double kappa_d;        // density diffusivity (Boussinesq)
  double ri;             // Richardson number (Boussinesq)
  int var_py;            // y passes: 0 full tile, 1 half width, 2 tensor-map tiles (FP32, ny = 128, 256), autotuned
  int var_p3;            // tile variant of the z pass (0: full, 1: half the lines), autotuned
  int p3_bulk;           // z pass: stage input rows with bulk copies (rows a multiple of 16 B)
  int p3_stall;          // debug: block 0's bulk-copy barrier expects this many extra bytes
  int epi32;             // P5 epilogue (viscous term, forcing) in FP32 (DNS_FP32 form)
  int p3_rr;             // z pass: the register-resident FP32 kernel where it applies (autotuned)
  int x_tma;             // x-inverse pass: the tensor-map FP32 kernel where it applies (autotuned)
  const void* ycand[2];  // the buffers the stage-input slot can name (null: unknown), for P1's tensor maps
  int ycand_f32;         // those buffers hold the FP32 stage-input scratch (DNS_FP32 form)
};

// The register-resident FP32 z pass (zpass_rr.cuh) handles nz = 64, 128, 256 in the velocity
// form.  It takes a launch when selected and when a tile's rows can be bulk-copied: TL Mz
// complex values per field starting on a 16-byte boundary, a multiple of 16 bytes long
// (Mz even, or nx ny even).
__host__ __device__ constexpr bool zrr_supported(int nz) { return nz == 64 || nz == 128 || nz == 256; }
inline bool p3_rr_applies(const PassArgs& a) {
  return a.p3_rr && !a.g.bouss && zrr_supported(a.g.nz) &&
         (a.g.Mz % 2 == 0 || ((long long)a.g.nx * a.g.ny) % 2 == 0);
}

// The FP32 y passes with tensor-map tile copies (ypass_tma.cuh, y-pass variant 2) handle
// ny = 128 and 256 with an even number of retained kz planes (rows of 16-byte multiples).
__host__ __device__ constexpr bool ytma_supported(int ny, int Mz) { return (ny == 256 || ny == 128) && Mz % 2 == 0; }
// The FP32 x-inverse pass with tensor-map tile copies (xpass_tma.cuh) handles nx = 256 in the
// velocity form with an even number of retained (ky, kz) columns, when the buffers the
// stage-input slot can name are known.
inline bool x_tma_applies(const PassArgs& a) {
  return a.x_tma && !a.g.bouss && a.g.nx == 256 && a.g.MyMz % 2 == 0 && a.ycand[0] != nullptr;
}

// ---- bulk copies (TMA engine) completing on a CTA-local mbarrier ---------------------------
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// global -> shared, `bytes` a multiple of 16, both addresses 16-byte aligned
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}
// count `bytes` of the barrier's expected transaction bytes as arrived (no data moves)
__device__ __forceinline__ void mbar_complete_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.complete_tx.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
               : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
  return ok != 0;
}
// Bounded wait: gives up after about half a second (1e9 clock cycles) or 2^24 polls.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity) {
  const long long t0 = clock64();
  for (int it = 0; it < (1 << 24); ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if (clock64() - t0 > 1000000000LL) return false;
  }
  return false;
}

// Column tiles: kz-contiguous columns handled per CTA in the x and y passes (128-byte rows),
// and z lines per CTA in the z pass.
template <typename T, int N> __host__ __device__ constexpr int p1_cols() {
  // double-word: half the FP64 tile, so that two or three CTAs share an SM (its kernels are
  // issue-bound and need the extra warps; the FP64 ones are bound by the FP64 pipe)
  return is_dw<T>() ? (N >= 512 ? 2 : 4) : sizeof(T) == 4 ? (N >= 512 ? 8 : 16) : (N >= 512 ? 4 : 8);
}
template <typename T, int VAR = 0> __host__ __device__ constexpr int py_cols() {
  return (sizeof(T) == 4 ? 16 : 8) >> VAR;
}
template <typename T, int MZ, bool BOUSS = false, int VAR = 0> __host__ __device__ constexpr int p3_lines() {
  return (BOUSS ? (MZ >= 256 ? 2 : 4) : (MZ >= 256 ? 4 : 8)) >> VAR;
}
// z-pass line stride: lines whose threads share a half-warp (FP32) or quarter-warp (FP64)
// start at bank offsets that the first Stockham stage's writes do not overlap.
template <typename V, int MZ> __host__ __device__ constexpr int p3_ld() {
  constexpr int unit = sizeof(V) == 8 ? 16 : 8;               // elements per 128 bytes
  constexpr int base = (MZ + 1) + ((MZ + 1) >> pad_shift<V>());
  constexpr int G = plan_threads(MZ), R0 = plan_radix(MZ, 0);
  constexpr int res = G >= unit ? 0 : (R0 == 8 && 2 * G == unit ? unit / 4 : G);
  return base + ((res - base % unit) % unit + unit) % unit;
}
// twiddle entries of a pass: x and y passes hold the stage tables of their line length n; the
// z pass holds exp(-2 pi i k / nz) for k <= nz/2, then the stage tables of nz/2.
__host__ __device__ constexpr int twiddle_count_xy(int n) { return plan_tw_size(n); }
__host__ __device__ constexpr int twiddle_count_z(int nz) { return nz / 2 + 1 + plan_tw_size(nz / 2); }

// Entry i of a pass's twiddle table as a fraction num/den of a full turn: the value is
// exp(-2 pi i num/den).  Stage tables of line length L: stage s >= 1 stores (jm, r) at
// offset + jm (R-1) + (r-1) with angle jm r / (NS R).
__host__ __device__ inline void stage_twiddle_turns(int L, int idx, int* num, int* den) {
  int off = 0;
  for (int s = 1; s < plan_stages(L); ++s) {
    const int R = plan_radix(L, s), NS = plan_ns(L, s), sz = NS * (R - 1);
    if (idx < off + sz) {
      const int q = idx - off;
      *num = (q / (R - 1)) * (q % (R - 1) + 1);
      *den = NS * R;
      return;
    }
    off += sz;
  }
  *num = 0;
  *den = 1;
}
__host__ __device__ inline int axis_twiddle_count(int n, bool zaxis) {
  return zaxis ? twiddle_count_z(n) : twiddle_count_xy(n);
}
__host__ __device__ inline void axis_twiddle_turns(int n, bool zaxis, int i, int* num, int* den) {
  if (!zaxis) { stage_twiddle_turns(n, i, num, den); return; }
  if (i <= n / 2) { *num = i; *den = n; return; }
  stage_twiddle_turns(n / 2, i - (n / 2 + 1), num, den);
}

template <typename V> __device__ __forceinline__ V zero2() { return mk<V>(0, 0); }

// Asynchronous global->shared copy of one complex element (8 or 16 bytes); `valid` false
// writes zeros (src-size 0: nothing is read from `src`, which must still be a valid address).
// Every thread issues all its copies, then cp_async_wait() and a barrier: many loads stay in
// flight per thread instead of one.
template <typename V>
__device__ __forceinline__ void cp_async_elem(V* dst, const V* src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  if constexpr (sizeof(V) == 16) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 16 : 0) : "memory");
  } else {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 8 : 0) : "memory");
  }
}
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Visit (row, q) for row < rows, q < len: one warp per row, lanes along q (coalesced, no
// division) when the CTA is whole warps; otherwise a flat loop.
template <int NTH, typename F>
__device__ __forceinline__ void for_rows(int rows, int len, F&& fn) {
  const int tid = threadIdx.x;
  if constexpr (NTH % 32 == 0) {
    const int lane = tid & 31, wid = tid >> 5;
    for (int row = wid; row < rows; row += NTH / 32)
      for (int q = lane; q < len; q += 32) fn(row, q);
  } else {
    for (int i = tid; i < rows * len; i += NTH) fn(i / len, i % len);
  }
}

template <typename V>
__device__ __forceinline__ void copy_tw(V* dst, const V* __restrict__ src, int n) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
}

// ------------------------------------------------------------------------------------------
// P1: x-inverse with the curl fused in.  grid (ceil(MyMz/(TC/2)), 1 or 2): y = 0 -> the six
// lines u, omega of TC/2 columns (the state is read and converted once per mode), y = 1 ->
// density (Boussinesq: one field over 3 TC columns, output field 6).
// ------------------------------------------------------------------------------------------
// FP32 lines up to 256 points: registers bounded for two CTAs per SM (768-thread blocks)
template <typename T, int NX> __host__ __device__ constexpr int p1_min_blocks() {
  return std::is_same<T, float>::value && NX <= 256 ? 2 : 0;
}
template <typename T, int NX, bool BOUSS>
__global__ void __launch_bounds__(FftPlan<NX>::G * 3 * p1_cols<T, NX>(), p1_min_blocks<T, NX>())
k_p1(const PassArgs a) {
  using V = v2_t<T>;
  constexpr int TC = p1_cols<T, NX>();
  constexpr int TC2 = TC / 2;                  // columns of the u, omega blocks (6 lines each)
  constexpr int G = FftPlan<NX>::G;
  constexpr int LD = line_ld<V, NX>();
  constexpr int NTW = twiddle_count_xy(NX);
  static_assert(TC % 2 == 0, "x-inverse tiles hold an even number of columns");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* tw = reinterpret_cast<V*>(smem_raw);
  V* lines = tw + NTW;
  if (gated_off(a.ctrl, a.gate_k1)) return;
  const Geom& g = a.g;
  const double2* __restrict__ Y = resolve_in(a.y, a.ctrl, a.yslot);
  // FP32 stage-input scratch (fp32 form; compile-time false for the other element types)
  const bool y32 = std::is_same<T, float>::value && in_is_f32(a.ctrl, a.yslot);
  V* __restrict__ out = reinterpret_cast<V*>(a.out);
  const int tid = threadIdx.x, nth = blockDim.x;
  constexpr int NTH = G * 3 * TC;
  T* colk = reinterpret_cast<T*>(lines + 6 * TC2 * LD);   // ky, kz of each column
  copy_tw(tw, reinterpret_cast<const V*>(a.tw), NTW);
  const T s = (T)g.inv_n3;
  const T sx = (T)g.sx, sy = (T)g.sy, sz = (T)g.sz;
  if constexpr (BOUSS) {
    if (blockIdx.y == 1) {   // density: lines are 3 TC columns of one field
      constexpr int TC3 = 3 * TC;
      const int c0 = blockIdx.x * TC3;
      if (c0 >= g.MyMz) return;   // uniform over the CTA, before any barrier
      for_rows<NTH>(TC3, NX - g.Mx, [&](int l, int q) { lines[l * LD + pidx<V>(g.Kx + 1 + q)] = zero2<V>(); });
      __syncthreads();
      for (int i = tid; i < g.Mx * TC3; i += nth) {
        const int ix = i / TC3, c = i - ix * TC3, col = c0 + c;
        V f = zero2<V>();
        if (col < g.MyMz) {
          const size_t yi = 3 * g.M + (size_t)ix * g.MyMz + col;
          if constexpr (std::is_same<T, float>::value) {
            f = cscale(y_as_f32(Y, yi, y32), s);
          } else {
            const double2 d = Y[yi];
            f = cscale(mk<V>(from_f64<T>(d.x), from_f64<T>(d.y)), s);
          }
        }
        lines[c * LD + pidx<V>(ix <= g.Kx ? ix : NX - g.Mx + ix)] = f;
      }
      __syncthreads();
      line_fft<V, NX, +1>(lines + (tid / G) * LD, tid % G, tw);
      for (int i = tid; i < NX * TC3; i += nth) {
        const int x = i / TC3, c = i - x * TC3, col = c0 + c;
        if (col < g.MyMz) out[((size_t)6 * NX + x) * g.MyMz + col] = lines[c * LD + pidx<V>(x)];
      }
      return;
    }
  }
  const int col0 = blockIdx.x * TC2;
  for_rows<NTH>(6 * TC2, NX - g.Mx, [&](int l, int q) { lines[l * LD + pidx<V>(g.Kx + 1 + q)] = zero2<V>(); });
  if (tid < TC2) {
    const int col = min(col0 + tid, g.MyMz - 1);
    const int jy = col / g.Mz, kz = col - jy * g.Mz;
    colk[2 * tid] = sy * (T)signed_mode(jy, g.Ky, g.My);
    colk[2 * tid + 1] = sz * (T)kz;
  }
  __syncthreads();
  // thread tid owns column c = tid mod TC2 and modes r0 + k RS: constant strides, no division
  constexpr int RS = NTH / TC2;
  const int c = tid % TC2, r0 = tid / TC2, col = col0 + c;
  const bool ok = col < g.MyMz;
  const T ky = colk[2 * c], kzz = colk[2 * c + 1];
  for (int ix = r0; ix < g.Mx; ix += RS) {
    V u0 = zero2<V>(), u1 = u0, u2 = u0, w0 = u0, w1 = u0, w2 = u0;
    if (ok) {
      const size_t off = (size_t)ix * g.MyMz + col;
      V y0, y1, y2;
      if constexpr (std::is_same<T, float>::value) {
        y0 = y_as_f32(Y, off, y32); y1 = y_as_f32(Y, off + g.M, y32); y2 = y_as_f32(Y, off + 2 * g.M, y32);
      } else {
        const double2 d0 = Y[off], d1 = Y[off + g.M], d2 = Y[off + 2 * g.M];
        y0 = mk<V>(from_f64<T>(d0.x), from_f64<T>(d0.y));
        y1 = mk<V>(from_f64<T>(d1.x), from_f64<T>(d1.y));
        y2 = mk<V>(from_f64<T>(d2.x), from_f64<T>(d2.y));
      }
      u0 = cscale(y0, s); u1 = cscale(y1, s); u2 = cscale(y2, s);
      const T kx = sx * (T)signed_mode(ix, g.Kx, g.Mx);
      // omega = i kappa x Y, scaled by 1/(nx ny nz): i (kappa x u) with u already scaled
      const V cx = mk<V>(ky * u2.x - kzz * u1.x, ky * u2.y - kzz * u1.y);
      const V cy = mk<V>(kzz * u0.x - kx * u2.x, kzz * u0.y - kx * u2.y);
      const V cz = mk<V>(kx * u1.x - ky * u0.x, kx * u1.y - ky * u0.y);
      w0 = mk<V>(-cx.y, cx.x);
      w1 = mk<V>(-cy.y, cy.x);
      w2 = mk<V>(-cz.y, cz.x);
    }
    const int pos = pidx<V>(ix <= g.Kx ? ix : NX - g.Mx + ix);
    lines[(0 * TC2 + c) * LD + pos] = u0;
    lines[(1 * TC2 + c) * LD + pos] = u1;
    lines[(2 * TC2 + c) * LD + pos] = u2;
    lines[(3 * TC2 + c) * LD + pos] = w0;
    lines[(4 * TC2 + c) * LD + pos] = w1;
    lines[(5 * TC2 + c) * LD + pos] = w2;
  }
  __syncthreads();
  line_fft<V, NX, +1>(lines + (tid / G) * LD, tid % G, tw);
  if constexpr (G % (1 << pad_shift<V>()) == 0 && NTH % (6 * TC2) == 0 && (NTH / (6 * TC2)) == G) {
    // thread: column cc, field f, rows x = xq + G k -- the padded line index and the output
    // address advance by constants (G + G / 2^pad per step in shared memory)
    const int cc = tid % TC2, rest = tid / TC2, f = rest % 6, xq = rest / 6, cl = col0 + cc;
    if (cl < g.MyMz) {
      V* op = out + ((size_t)f * NX + xq) * g.MyMz + cl;
      const V* lp = lines + (f * TC2 + cc) * LD + pidx<V>(xq);
      constexpr int LSTEP = G + (G >> pad_shift<V>());
      const size_t ostep = (size_t)G * g.MyMz;
#pragma unroll 4
      for (int k = 0; k < NX / G; ++k, op += ostep, lp += LSTEP) *op = *lp;
    }
  } else {
    for (int i = tid; i < 6 * NX * TC2; i += nth) {
      const int f = i / (NX * TC2), r = i - f * (NX * TC2), x = r / TC2, cc = r - x * TC2, cl = col0 + cc;
      if (cl < g.MyMz) out[((size_t)f * NX + x) * g.MyMz + cl] = lines[(f * TC2 + cc) * LD + pidx<V>(x)];
    }
  }
}

// ------------------------------------------------------------------------------------------
// P2 / P4: DFT along y for one (field, x) and TZ kz columns.  grid (ceil(Mz/TZ), nx, nf).
// INVERSE: retained ky -> all y.  Forward: all y -> retained ky.
// ------------------------------------------------------------------------------------------
template <typename T, int NY, bool INVERSE, int VAR>
__global__ void __launch_bounds__(FftPlan<NY>::G * py_cols<T, VAR>())
k_py(const PassArgs a) {
  using V = v2_t<T>;
  constexpr int TZ = py_cols<T, VAR>();
  constexpr int G = FftPlan<NY>::G;
  constexpr int LD = line_ld<V, NY>();
  constexpr int NTW = twiddle_count_xy(NY);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* tw = reinterpret_cast<V*>(smem_raw);
  V* lines = tw + NTW;
  if (gated_off(a.ctrl, a.gate_k1)) return;
  const Geom& g = a.g;
  const V* __restrict__ in = reinterpret_cast<const V*>(a.in);
  V* __restrict__ out = reinterpret_cast<V*>(a.out);
  const int f = blockIdx.z, x = blockIdx.y, kz0 = blockIdx.x * TZ;
  const int tid = threadIdx.x;
  const int Mz = g.Mz;
  copy_tw(tw, reinterpret_cast<const V*>(a.tw), NTW);
  // The CTA has G TZ threads: thread tid owns column c = tid mod TZ and rows y0 + k G, so the
  // element loops advance by constant strides (no per-element division).
  const int c = tid % TZ, y0 = tid / TZ, kz = kz0 + c;
  const bool ok = kz < Mz;
  V* const line = lines + c * LD;
  if (INVERSE) {
    // rows |ky| <= Ky from the retained box, the band between zero-filled
    const V* src = in + ((size_t)f * g.nx + x) * g.My * Mz + (ok ? kz : 0);
    const int Ky = g.Ky, shift = NY - g.My;
    for (int y = y0; y < NY; y += G) {
      const bool load = ok && (y <= Ky || y > Ky + shift);
      const int jy = y <= Ky ? y : y - shift;
      cp_async_elem(&line[pidx<V>(y)], load ? src + (size_t)jy * Mz : src, load);
    }
  } else {
    const V* src = in + ((size_t)f * g.nx + x) * NY * Mz + (ok ? kz : 0);
    const size_t step = (size_t)G * Mz;
    const V* sp = src + (size_t)y0 * Mz;
    for (int y = y0; y < NY; y += G, sp += step) cp_async_elem(&line[pidx<V>(y)], ok ? sp : src, ok);
  }
  cp_async_wait();
  __syncthreads();
  line_fft<V, NY, INVERSE ? +1 : -1>(lines + (tid / G) * LD, tid % G, tw);
  if (!ok) return;
  if (INVERSE) {
    V* dp = out + ((size_t)f * g.nx + x) * NY * Mz + kz + (size_t)y0 * Mz;
    const size_t step = (size_t)G * Mz;
    for (int y = y0; y < NY; y += G, dp += step) *dp = line[pidx<V>(y)];
  } else {
    V* dst = out + ((size_t)f * g.nx + x) * g.My * Mz + kz;
    const int Ky = g.Ky, shift = NY - g.My;
    for (int jy = y0; jy < g.My; jy += G) dst[(size_t)jy * Mz] = line[pidx<V>(jy <= Ky ? jy : jy + shift)];
  }
}

// ------------------------------------------------------------------------------------------
// P3: z lines.  Inverse real DFT of 6 fields through an MZ = nz/2 point complex DFT of the
// packed sequence z_n = x_2n + i x_2n+1, u x omega on both packed halves, forward real DFT
// of the 3 products the same way.  grid ceil(nx ny / TL).
//   C2R pre-step : Z_k = (X_k + conj X_{M-k}) + i e^{+2 pi i k/nz} (X_k - conj X_{M-k})
//   R2C post-step: X_k = (Z_k + conj Z_{M-k})/2 - (i/2) e^{-2 pi i k/nz} (Z_k - conj Z_{M-k})
// ------------------------------------------------------------------------------------------
// byte offset of the z pass's staging rows: after `elems` elements of V, rounded up to 16
template <typename V> __host__ __device__ constexpr size_t p3_stage_offset(size_t elems) {
  return (elems * sizeof(V) + 15) / 16 * 16;
}

template <typename T, int MZ, bool BOUSS, int VAR>
__global__ void __launch_bounds__(FftPlan<MZ>::G * (BOUSS ? 7 : 6) * p3_lines<T, MZ, BOUSS, VAR>())
k_p3(const PassArgs a) {
  using V = v2_t<T>;
  constexpr int TL = p3_lines<T, MZ, BOUSS, VAR>();
  constexpr int NIN = BOUSS ? 7 : 6;    // u, omega (, rho)
  constexpr int NOUT = BOUSS ? 6 : 3;   // u x omega (, rho u)
  constexpr int G = FftPlan<MZ>::G;
  constexpr int LD = p3_ld<V, MZ>();
  constexpr int NTW = twiddle_count_z(2 * MZ);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* tw = reinterpret_cast<V*>(smem_raw);      // [0, MZ]: exp(-2 pi i k / nz); then stages
  V* tws = tw + MZ + 1;
  V* lines = tw + NTW;                         // NIN*TL lines of LD
  if (gated_off(a.ctrl, a.gate_k1)) return;
  const Geom& g = a.g;
  const V* __restrict__ in = reinterpret_cast<const V*>(a.in);
  V* __restrict__ out = reinterpret_cast<V*>(a.out);
  const long long nxy = (long long)g.nx * g.ny;
  const long long xy0 = (long long)blockIdx.x * TL;
  const int Mz = g.Mz;
  const int tid = threadIdx.x, nth = blockDim.x;
  constexpr int NTH = G * NIN * TL;
  // bulk path: unpadded staging rows [NIN TL][Mz] after the lines (16-byte aligned), then the
  // mbarrier; the C2R pre-step reads the staging rows
  V* stage = reinterpret_cast<V*>(smem_raw + p3_stage_offset<V>(NTW + NIN * TL * LD));
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(stage + (size_t)NIN * TL * Mz);
  const bool bulk = a.p3_bulk != 0;
  if (bulk && tid == 0) mbar_init(bar, 1);
  copy_tw(tw, reinterpret_cast<const V*>(a.tw), NTW);
  if (bulk) {
    __syncthreads();
    const unsigned extra = blockIdx.x == 0 ? (unsigned)a.p3_stall : 0u;
    if (tid == 0) {
      const unsigned row_bytes = (unsigned)(Mz * sizeof(V));
      const long long rows_here = (nxy - xy0) < TL ? (nxy - xy0) : TL;
      mbar_expect_tx(bar, (unsigned)(NIN * rows_here) * row_bytes + extra);
      for (int f = 0; f < NIN; ++f)
        for (int l = 0; l < rows_here; ++l)
          bulk_g2s(stage + (size_t)(f * TL + l) * Mz, in + ((size_t)f * nxy + xy0 + l) * Mz, row_bytes, bar);
    }
    // every thread polls (bounded); the block agrees on the outcome
    const bool arrived = mbar_wait_bounded(bar, 0);
    if (!__syncthreads_and(arrived)) {
      if (tid == 0) {
        if (a.ctrl) {
          DnsCtrl* cw = const_cast<DnsCtrl*>(a.ctrl);
          cw->status = ST_TIMEOUT;
          cw->done = 1;
        }
        // let copies still in flight land before the block exits: the bytes of the debug
        // stall never arrive, so count them as arrived; the phase then completes exactly
        // when every real copy has landed (the wait stays bounded for any other cause)
        if (extra) mbar_complete_tx(bar, extra);
        mbar_wait_bounded(bar, 0);
      }
      return;
    }
  } else {
    // rows (field, line): kz < Mz from memory, Mz..MZ zero
    for_rows<NTH>(NIN * TL, MZ + 1, [&](int row, int kz) {
      const int f = row / TL, l = row - f * TL;
      const long long xy = xy0 + l;
      const bool ok = kz < Mz && xy < nxy;
      cp_async_elem(&lines[row * LD + pidx<V>(kz)], ok ? &in[((size_t)f * nxy + xy) * Mz + kz] : in, ok);
    });
    cp_async_wait();
    __syncthreads();
  }
  // C2R pre-step on pairs (k, MZ-k), k = 0..MZ/2, of the NIN input lines; each line by the G
  // threads that transform it
  auto prestep = [&]() {
    V* L = lines + (tid / G) * LD;
    const V* S = stage + (size_t)(tid / G) * Mz;
    for (int k = tid % G; k <= MZ / 2; k += G) {
      const int m = MZ - k;
      const V xk = bulk ? (k < Mz ? S[k] : zero2<V>()) : L[pidx<V>(k)];
      const V xm = bulk ? (m < Mz ? S[m] : zero2<V>()) : L[pidx<V>(m)];
      // s = X_k + conj X_m, t = e^{+2 pi i k/nz} (X_k - conj X_m); Z_k = s + i t.  The partner
      // k' = m has s' = conj s and t' = conj t (e^{+2 pi i m/nz} = -e^{-2 pi i k/nz}), so
      // Z_m = conj(s) + i conj(t) costs two more additions.
      const V s = cadd(xk, cconj(xm));
      const V t = cmul(cconj(tw[k]), csub(xk, cconj(xm)));
      if (k != 0 && k != m) L[pidx<V>(m)] = mk<V>(badd(s.x, t.y), bsub(t.x, s.y));
      L[pidx<V>(k)] = mk<V>(bsub(s.x, t.y), badd(s.y, t.x));
    }
  };
  // u x omega (and rho u) on both packed halves (real part: even z, imaginary part: odd z);
  // conjugated when CJ (see below)
  auto cross = [&](auto cj) {
    constexpr bool CJ = decltype(cj)::value;
    for (int i = tid; i < TL * MZ; i += nth) {
      const int l = i / MZ, n = pidx<V>(i - l * MZ);
      const V u0 = lines[(0 * TL + l) * LD + n], u1 = lines[(1 * TL + l) * LD + n], u2 = lines[(2 * TL + l) * LD + n];
      const V w0 = lines[(3 * TL + l) * LD + n], w1 = lines[(4 * TL + l) * LD + n], w2 = lines[(5 * TL + l) * LD + n];
      V p0 = mk<V>(bdot2(u1.x, w2.x, -u2.x, w1.x), bdot2(u1.y, w2.y, -u2.y, w1.y));
      V p1 = mk<V>(bdot2(u2.x, w0.x, -u0.x, w2.x), bdot2(u2.y, w0.y, -u0.y, w2.y));
      V p2 = mk<V>(bdot2(u0.x, w1.x, -u1.x, w0.x), bdot2(u0.y, w1.y, -u1.y, w0.y));
      if constexpr (CJ) { p0 = cconj(p0); p1 = cconj(p1); p2 = cconj(p2); }
      lines[(0 * TL + l) * LD + n] = p0;
      lines[(1 * TL + l) * LD + n] = p1;
      lines[(2 * TL + l) * LD + n] = p2;
      if constexpr (BOUSS) {
        const V r = lines[(6 * TL + l) * LD + n];
        V q0 = mk<V>(r.x * u0.x, r.y * u0.y), q1 = mk<V>(r.x * u1.x, r.y * u1.y), q2 = mk<V>(r.x * u2.x, r.y * u2.y);
        if constexpr (CJ) { q0 = cconj(q0); q1 = cconj(q1); q2 = cconj(q2); }
        lines[(3 * TL + l) * LD + n] = q0;
        lines[(4 * TL + l) * LD + n] = q1;
        lines[(5 * TL + l) * LD + n] = q2;
      }
    }
  };
  const int line = tid / G;
  // Double-word: the two phases share one copy of the line transform (its butterflies are
  // long; two inlined copies overflow the instruction cache).  The products are stored
  // conjugated, transformed by the same inverse DFT -- conj(DFT^+(conj z)) is the forward DFT
  // of z -- and the post-step conjugates on reading.  FP32/FP64: two unrolled transforms.
  // Threads on lines past the active count idle in the second transform but take part in
  // the barriers.
  constexpr bool SHARE = is_dw<T>();
  if constexpr (SHARE) {
#pragma unroll 1
    for (int ph = 0; ph < 2; ++ph) {
      if (ph == 0) {
        prestep();
        line_sync<MZ>();
      } else {
        cross(std::true_type{});
        __syncthreads();
      }
      const int nact = ph == 0 ? NIN * TL : NOUT * TL;
      line_fft<V, MZ, +1>(lines + (line < nact ? line : 0) * LD, tid % G, tws, line < nact);
    }
  } else {
    prestep();
    line_sync<MZ>();
    line_fft<V, MZ, +1>(lines + line * LD, tid % G, tws);
    cross(std::false_type{});
    __syncthreads();
    line_fft<V, MZ, -1>(lines + (line < NOUT * TL ? line : 0) * LD, tid % G, tws, line < NOUT * TL);
  }
  // R2C post-step, keep kz <= Kz
  for_rows<NTH>(NOUT * TL, Mz, [&](int row, int k) {
    const int c = row / TL, l = row - c * TL;
    const long long xy = xy0 + l;
    if (xy >= nxy) return;
    const V* L = lines + row * LD;
    V zk = L[pidx<V>(k)], zm = L[pidx<V>((MZ - k) % MZ)];
    if constexpr (SHARE) { zk = cconj(zk); zm = cconj(zm); }
    const V s = cadd(zk, cconj(zm)), d = csub(zk, cconj(zm));
    const V od = cmul(tw[k], d);                   // e^{-2 pi i k / nz} (Z_k - conj Z_{M-k})
    // X = s/2 - (i/2) od
    out[((size_t)c * nxy + xy) * Mz + k] = mk<V>(bhalf(badd(s.x, od.y)), bhalf(bsub(s.y, od.x)));
  });
}

// ------------------------------------------------------------------------------------------
// P5: x-forward + epilogue.  grid ceil(MyMz/TC).  The Leray projection runs in the
// transform precision T; the viscous term and forcing are FP64 (FP64 and double-word forms)
// or FP32 (fp32 form, DNS_FP32, whose k carries FP32 accuracy: the epilogue then has no FP64
// instruction).  k is stored FP64, except into the FP32 k slots of an fp32 context
// (stored FP32 and read as FP32 by its stage sums and error norm).
// Boussinesq (Section 3.2): fields 0..2 hold (u x omega)^, 3..5 (rho u)^; the buoyancy
// -Ri rho e_z (kappa != 0) enters before the projection, and the density equation is
// -i kappa . (rho u)^ - kappa_d |kappa|^2 rho.
// ------------------------------------------------------------------------------------------
template <typename T, int NX> __host__ __device__ constexpr int p5_cols(bool bouss) {
  return bouss ? p1_cols<T, NX>() / 2 : p1_cols<T, NX>();
}
// FP32 lines up to 256 points: two CTAs per SM (the register budget of two 768-thread
// blocks, which these fit without spilling; the shared-memory tile fits twice), so that one
// CTA's loads overlap the other's transform and epilogue.  Longer lines would spill.
// Other element types: 0, no bound (an explicit minimum of one CTA lets the allocator take
// more registers than it does without a minimum: 225 instead of 160 for the 256-point
// double-word kernel, one CTA per SM instead of two).
template <typename T, int NX> __host__ __device__ constexpr int p5_min_blocks() {
  return std::is_same<T, float>::value && NX <= 256 ? 2 : 0;
}
template <typename T, int NX, bool BOUSS>
__global__ void __launch_bounds__(FftPlan<NX>::G * 3 * p1_cols<T, NX>(), p5_min_blocks<T, NX>())
k_p5(const PassArgs a) {
  using V = v2_t<T>;
  constexpr int TC = p5_cols<T, NX>(BOUSS);
  constexpr int NF = BOUSS ? 6 : 3;
  constexpr int G = FftPlan<NX>::G;
  constexpr int LD = line_ld<V, NX>();
  constexpr int NTW = twiddle_count_xy(NX);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* tw = reinterpret_cast<V*>(smem_raw);
  V* lines = tw + NTW;
  if (gated_off(a.ctrl, a.gate_k1)) return;
  const Geom& g = a.g;
  const double2* __restrict__ Y = resolve_in(a.y, a.ctrl, a.yslot);
  double2* __restrict__ K = resolve_out(a.kout, a.ctrl, a.kslot);
  // FP32 k slots and stage-input scratch (fp32 form; compile-time false for the other types)
  const bool k32 = std::is_same<T, float>::value && out_is_f32(a.ctrl, a.kslot);
  const bool y32 = std::is_same<T, float>::value && in_is_f32(a.ctrl, a.yslot);
  const V* __restrict__ in = reinterpret_cast<const V*>(a.in);
  const int col0 = blockIdx.x * TC;
  const int tid = threadIdx.x, nth = blockDim.x;
  copy_tw(tw, reinterpret_cast<const V*>(a.tw), NTW);
  // thread tid owns column c = tid mod TC and rows r0 + k RS: constant strides, no division
  constexpr int RS = G * NF;
  const int cc = tid % TC, r0 = tid / TC, ccol = col0 + cc;
  const bool cok = ccol < g.MyMz;
  if constexpr (G % (1 << pad_shift<V>()) == 0) {
    // thread: column cc, field f = r0 mod NF, rows x = xq + G k -- constant strides in both
    // memories (G + G / 2^pad per step in the padded line)
    const int f = r0 % NF, xq = r0 / NF;
    const V* ip = in + ((size_t)f * NX + xq) * g.MyMz + (cok ? ccol : 0);
    const size_t istep = (size_t)G * g.MyMz;
    V* lp = &lines[(f * TC + cc) * LD + pidx<V>(xq)];
    constexpr int LSTEP = G + (G >> pad_shift<V>());
#pragma unroll 4
    for (int k = 0; k < NX / G; ++k, ip += istep, lp += LSTEP) cp_async_elem(lp, cok ? ip : in, cok);
  } else {
    const V* ip = in + (size_t)r0 * g.MyMz + (cok ? ccol : 0);
    const size_t istep = (size_t)RS * g.MyMz;
    for (int row = r0; row < NF * NX; row += RS, ip += istep) {
      const int f = row / NX, x = row - f * NX;
      cp_async_elem(&lines[(f * TC + cc) * LD + pidx<V>(x)], cok ? ip : in, cok);
    }
  }
  cp_async_wait();
  __syncthreads();
  line_fft<V, NX, -1>(lines + (tid / G) * LD, tid % G, tw);
  const double fc = (a.ctrl && a.kf2 > 0) ? a.ctrl->forcing_coef : 0.0;
  // |kappa|^2 split per axis (FP64): x part per retained kx, y+z part per column
  double* k2x = reinterpret_cast<double*>(lines + NF * TC * LD);
  double* k2yz = k2x + g.Mx;
  for (int i = tid; i < g.Mx; i += nth) {
    const double kx = g.sx * signed_mode(i, g.Kx, g.Mx);
    k2x[i] = kx * kx;
  }
  const T sx = (T)g.sx, sy = (T)g.sy, sz = (T)g.sz;
  T* colk = reinterpret_cast<T*>(k2yz + TC);
  for (int c = tid; c < TC; c += nth) {
    const int col = min(col0 + c, g.MyMz - 1);
    const int jy = col / g.Mz, kz = col - jy * g.Mz;
    const double ky = g.sy * signed_mode(jy, g.Ky, g.My), kzz = g.sz * kz;
    k2yz[c] = ky * ky + kzz * kzz;
    colk[2 * c] = sy * (T)signed_mode(jy, g.Ky, g.My);
    colk[2 * c + 1] = sz * (T)kz;
  }
  __syncthreads();
  const T kf2 = (T)a.kf2;
  const T fsc = (T)g.fwd_scale;
  const int c = cc, col = ccol;
  if (!cok) return;
  for (int ix = r0; ix < g.Mx; ix += RS) {
    const int pos = pidx<V>(ix <= g.Kx ? ix : NX - g.Mx + ix);
    V n0 = lines[(0 * TC + c) * LD + pos], n1 = lines[(1 * TC + c) * LD + pos], n2 = lines[(2 * TC + c) * LD + pos];
    if (fsc != (T)1) { n0 = cscale(n0, fsc); n1 = cscale(n1, fsc); n2 = cscale(n2, fsc); }
    const T kx = sx * (T)signed_mode(ix, g.Kx, g.Mx);
    const T ky = colk[2 * c], kzz = colk[2 * c + 1];
    const T k2 = kx * kx + ky * ky + kzz * kzz;
    const size_t off = (size_t)ix * g.MyMz + col;
    double2 rho = make_double2(0.0, 0.0);
    float2 rho32 = make_float2(0.f, 0.f);
    if constexpr (BOUSS) {
      if constexpr (std::is_same<T, float>::value) {
        rho32 = y_as_f32(Y, off + 3 * g.M, y32);
        if (!y32) rho = Y[off + 3 * g.M];   // an FP64 stage input keeps its FP64 value
        if (k2 > (T)0) n2 = mk<V>(n2.x - (T)a.ri * rho32.x, n2.y - (T)a.ri * rho32.y);
      } else {
        rho = Y[off + 3 * g.M];
        if (k2 > (T)0) {
          const T ri = (T)a.ri;
          n2 = mk<V>(n2.x - ri * from_f64<T>(rho.x), n2.y - ri * from_f64<T>(rho.y));
        }
      }
    }
    if (k2 > (T)0) {
      const T ik2 = (T)1 / k2;
      const T dr = (kx * n0.x + ky * n1.x + kzz * n2.x) * ik2;
      const T di = (kx * n0.y + ky * n1.y + kzz * n2.y) * ik2;
      n0 = mk<V>(n0.x - kx * dr, n0.y - kx * di);
      n1 = mk<V>(n1.x - ky * dr, n1.y - ky * di);
      n2 = mk<V>(n2.x - kzz * dr, n2.y - kzz * di);
    }
    double k2d = 0.0;
    bool fp32_epi = false;
    // FP64 epilogue: k = N + (-nu |kappa|^2 + forcing) Y in FP64
    const auto epi64 = [&]() {
      const double2 y0 = Y[off], y1 = Y[off + g.M], y2 = Y[off + 2 * g.M];
      k2d = k2x[ix] + k2yz[c];
      double vis = -a.nu * k2d;
      if (fc != 0.0 && k2 > (T)0 && k2 <= kf2) vis += fc;
      K[off] = make_double2(fma(vis, y0.x, to_f64(n0.x)), fma(vis, y0.y, to_f64(n0.y)));
      K[off + g.M] = make_double2(fma(vis, y1.x, to_f64(n1.x)), fma(vis, y1.y, to_f64(n1.y)));
      K[off + 2 * g.M] = make_double2(fma(vis, y2.x, to_f64(n2.x)), fma(vis, y2.y, to_f64(n2.y)));
    };
    if constexpr (std::is_same<T, float>::value) {
      fp32_epi = a.epi32 != 0;
      if (fp32_epi) {
        T vis = -(T)a.nu * k2;
        if (fc != 0.0 && k2 > (T)0 && k2 <= kf2) vis += (T)fc;
        const float2 y0 = y_as_f32(Y, off, y32), y1 = y_as_f32(Y, off + g.M, y32), y2 = y_as_f32(Y, off + 2 * g.M, y32);
        const float2 r0 = make_float2(fmaf(vis, y0.x, n0.x), fmaf(vis, y0.y, n0.y));
        const float2 r1 = make_float2(fmaf(vis, y1.x, n1.x), fmaf(vis, y1.y, n1.y));
        const float2 r2 = make_float2(fmaf(vis, y2.x, n2.x), fmaf(vis, y2.y, n2.y));
        if (k32) {
          float2* K32 = reinterpret_cast<float2*>(K);
          K32[off] = r0; K32[off + g.M] = r1; K32[off + 2 * g.M] = r2;
        } else {
          K[off] = make_double2(to_f64(r0.x), to_f64(r0.y));
          K[off + g.M] = make_double2(to_f64(r1.x), to_f64(r1.y));
          K[off + 2 * g.M] = make_double2(to_f64(r2.x), to_f64(r2.y));
        }
      } else {
        epi64();
      }
    } else {
      epi64();
    }
    if (off == 0 && a.ctrl && a.kslot >= SLOT_K1 && a.ctrl->inject_rhs >= 0) {
      // debug fault injection (dns_debug_inject): this evaluation's running index is the count
      // before the attempt plus its position in the attempt (k_1 first when it is evaluated)
      DnsCtrl* cw = const_cast<DnsCtrl*>(a.ctrl);
      const long long idx = cw->n_rhs + (a.kslot - SLOT_K1) - (cw->need_k1 ? 0 : 1);
      if (idx == cw->inject_rhs) {
        if (k32) reinterpret_cast<float2*>(K)[0] = make_float2(__uint_as_float(0x7fc00000u), 0.f);
        else K[0] = make_double2(__longlong_as_double(0x7ff8000000000000ULL), 0.0);
        cw->inject_rhs = -1;
      }
    }
    if constexpr (BOUSS) {
      const V f0 = lines[(3 * TC + c) * LD + pos], f1 = lines[(4 * TC + c) * LD + pos], f2 = lines[(5 * TC + c) * LD + pos];
      V kd = mk<V>(kx * f0.x + ky * f1.x + kzz * f2.x, kx * f0.y + ky * f1.y + kzz * f2.y);
      if (fsc != (T)1) kd = cscale(kd, fsc);
      // -i (kappa . F) = (Im, -Re)
      bool dens_done = false;
      if constexpr (std::is_same<T, float>::value) {
        if (fp32_epi) {
          const float visr = -(float)a.kappa_d * k2;
          const float2 rr = make_float2(fmaf(visr, rho32.x, kd.y), fmaf(visr, rho32.y, -kd.x));
          if (k32) reinterpret_cast<float2*>(K)[off + 3 * g.M] = rr;
          else K[off + 3 * g.M] = make_double2(to_f64(rr.x), to_f64(rr.y));
          dens_done = true;
        }
      }
      if (!dens_done) {
        const double visr = -a.kappa_d * k2d;
        K[off + 3 * g.M] = make_double2(fma(visr, rho.x, to_f64(kd.y)), fma(visr, rho.y, -to_f64(kd.x)));
      }
    }
  }
}

// ------------------------------------------------------------------------------------------
// Host side: launch pass `which` (1..5) for element type T (instantiated in passes_f64.cu and
// passes_f32.cu).  Returns cudaErrorInvalidValue for an unsupported line length.
// ------------------------------------------------------------------------------------------
template <typename T> cudaError_t launch_pass(int which, const PassArgs& a, cudaStream_t s);

}  // namespace dns
