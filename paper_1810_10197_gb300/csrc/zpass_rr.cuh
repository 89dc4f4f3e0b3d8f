// The z pass (P3) in FP32 with line transforms held in registers (velocity form, nz = 64,
// 128, 256): inverse real DFT of u and omega along z, u x omega, forward real DFT keeping
// kz <= Kz -- the same result as k_p3, by a different schedule.
//
// Two real fields per complex transform of the full length N = nz.  For fields a, b with
// half spectra A_k, B_k (k <= Kz, zero above by the 2/3 rule) the complex sequence
//   Z_k = A_k + i B_k,  Z_{N-k} = conj(A_k) + i conj(B_k)  (0 < k <= Kz),  Z_0 = Re A_0 + i Re B_0
// has the inverse DFT z(n) = a(n) + i b(n): three transforms give (u0, u1), (u2, w0),
// (w1, w2).  Forward: P = DFT(p0 + i p1) gives X0_k = (P_k + conj P_{N-k}) / 2 and
// X1_k = (P_k - conj P_{N-k}) / (2i); p2 takes a transform of its own (imaginary part 0).
// The real-input steps of the packed half-length transform (pre- and post-twiddles and the
// pairs k, M-k) are gone; each transform is longer.
//
// Each length N = 16 G is two radix stages, 16 x G, done by G threads of one warp with 16
// values each: stage 0 is one 16-point DFT per thread on the values at positions t + G r,
// one exchange through shared memory (padded rows, conflict-free), stage 1 is 16/G G-point
// DFTs per thread after the twiddles.  A thread ends holding the points n = t + G m
// (m = 0..15) of all three transforms, which are exactly the positions its forward stage 0
// reads: u x omega is formed in registers and no exchange separates the two transforms.
//
// Input: persistent CTAs walk tiles of TL consecutive (x, y) lines; the six input rows of a
// tile (TL Mz contiguous complex values per field) arrive by six bulk copies (TMA engine)
// into one shared-memory stage, completing on an mbarrier.  The CTA reads a whole tile into
// registers first, then issues the next tile's copies into the same stage and transforms
// while they run: one stage of shared memory, so more CTAs share an SM.  Every wait is
// bounded as in k_p3.
#pragma once

#include <type_traits>

#include "passes.cuh"

namespace dns {

template <int N, int NT = 128> struct ZrrPlan {
  static constexpr int G = N / 16;           // threads per line = stage-0 butterflies = stage-1 radix
  static constexpr int NB1 = 16 / G;         // stage-1 butterflies per thread
  static constexpr int TL = NT / G;          // lines per tile: NT threads per CTA (even)
  static constexpr int S = G + 1;            // row stride of the exchange (odd: conflict-free columns)
  // line stride of the exchange buffers: lines sharing a half-warp start on disjoint banks
  static constexpr int LSTR = G == 16 ? 16 * 17 : (G == 8 ? 16 * 9 + 8 : 16 * 5 + 4);
  static_assert(N == 64 || N == 128 || N == 256, "register-resident z pass: nz = 64, 128, 256");
  static_assert(LSTR >= N, "exchange buffer holds a line in natural order");

  static_assert(TL % 2 == 0, "tiles of an even number of lines (16-byte bulk copies)");
};

// Dynamic shared memory of k_p3_rr for Mz retained kz planes: one input stage of six fields,
// the exchange buffers, the stage-1 twiddles and the mbarrier.
template <int N> __host__ __device__ constexpr size_t zrr_smem(int Mz) {
  using P = ZrrPlan<N, 128>;
  return ((size_t)6 * P::TL * Mz + (size_t)P::TL * P::LSTR + 16 * P::G) * sizeof(float2) + 8;
}

// Register values of the transforms: float2 (every complex operation as paired FADD2 / FMUL2
// / FFMA2 instructions) or hf2, the same two floats with paired complex sums but scalar
// complex products and multiplications by +-i.  A paired product needs its operands as
// broadcast, swapped and negated register pairs, which costs register moves; the scalar
// product is four instructions with none.  The tile variant selects the form.
struct __align__(8) hf2 { float x, y; };
template <typename RV> __device__ __forceinline__ RV to_rv(float2 a) { RV r; r.x = a.x; r.y = a.y; return r; }
__device__ __forceinline__ float2 f2_of(hf2 a) { return make_float2(a.x, a.y); }
__device__ __forceinline__ hf2 hf2_of(float2 a) { hf2 r; r.x = a.x; r.y = a.y; return r; }
template <> __device__ __forceinline__ hf2 cadd<hf2>(hf2 a, hf2 b) { return hf2_of(__fadd2_rn(f2_of(a), f2_of(b))); }
// a - b = b (-1) + a, one rounding: the exact FP32 difference
template <> __device__ __forceinline__ hf2 csub<hf2>(hf2 a, hf2 b) {
  return hf2_of(__ffma2_rn(f2_of(b), make_float2(-1.f, -1.f), f2_of(a)));
}
// 4-point DFT with the +-i rotation of the odd difference written into the scalar sums
template <int SIGN> struct Dft<4, SIGN, hf2> {
  static __device__ __forceinline__ void run(hf2* v) {
    const hf2 s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
    const hf2 s13 = cadd(v[1], v[3]), e = csub(v[1], v[3]);
    v[0] = cadd(s02, s13);
    v[2] = csub(s02, s13);
    // X1 = d02 + SIGN i e, X3 = d02 - SIGN i e
    v[1] = mk<hf2>(SIGN > 0 ? d02.x - e.y : d02.x + e.y, SIGN > 0 ? d02.y + e.x : d02.y - e.x);
    v[3] = mk<hf2>(SIGN > 0 ? d02.x + e.y : d02.x - e.y, SIGN > 0 ? d02.y - e.x : d02.y + e.x);
  }
};

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// One transform's stage 1 after the stage-0 values of every thread of the line are in the
// exchange buffer xb (Y_t[s] at s S + t): butterfly j = t + G b reads Y_r[j] (r = 0..G-1),
// applies W_N^{j r} (tw1[r 16 + j] = exp(-2 pi i j r / N), lanes on consecutive entries;
// conjugated for the inverse) and leaves the G outputs at positions j + 16 s, i.e.
// n = t + G m with m = b + NB1 s.
template <int N, int SIGN, typename RV>
__device__ __forceinline__ void zrr_stage1(const float2* xb, const float2* tw1, int t, RV (&o)[16]) {
  using P = ZrrPlan<N>;
  constexpr int G = P::G, NB1 = P::NB1, S = P::S;
#pragma unroll
  for (int b = 0; b < NB1; ++b) {
    const int j = t + G * b;
    RV w[G];
#pragma unroll
    for (int r = 0; r < G; ++r) w[r] = to_rv<RV>(xb[j * S + r]);
#pragma unroll
    for (int r = 1; r < G; ++r) {
      const RV tw = to_rv<RV>(tw1[r * 16 + j]);
      w[r] = SIGN < 0 ? cmul(w[r], tw) : cmulc(w[r], tw);
    }
    Dft<G, SIGN, RV>::run(w);
#pragma unroll
    for (int s = 0; s < G; ++s) o[b + NB1 * s] = w[s];
  }
}

// The whole transform of the 16 values v[r] at positions t + G r; the result replaces v
// (position t + G m at v[m]).  Ends with the exchange buffer free again.
template <int N, int SIGN, typename RV>
__device__ __forceinline__ void zrr_fft(RV (&v)[16], float2* xb, const float2* tw1, int t) {
  using P = ZrrPlan<N>;
  Dft<16, SIGN, RV>::run(v);
#pragma unroll
  for (int s = 0; s < 16; ++s) xb[s * P::S + t] = make_float2(v[s].x, v[s].y);
  __syncwarp();
  zrr_stage1<N, SIGN>(xb, tw1, t, v);
  __syncwarp();
}

template <int N, bool PAIRED>
__global__ void __launch_bounds__(128, 3) k_p3_rr(const PassArgs a) {
  using P = ZrrPlan<N, 128>;
  using RV = typename std::conditional<PAIRED, float2, hf2>::type;
  constexpr int G = P::G, TL = P::TL;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (gated_off(a.ctrl, a.gate_k1)) return;
  const Geom& g = a.g;
  const int Mz = g.Mz, Kz = g.Kz;
  const long long nxy = (long long)g.nx * g.ny;
  const long long ntiles = (nxy + TL - 1) / TL;
  const int tile_elems = TL * Mz;                       // per field; TL even: 16-byte multiple
  float2* stage = reinterpret_cast<float2*>(smem_raw);  // [6][TL Mz]
  float2* xbuf = stage + 6 * tile_elems;                // [TL][LSTR]
  float2* tw1 = xbuf + TL * P::LSTR;                    // [G][16]
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(tw1 + 16 * G);
  const int tid = threadIdx.x, l = tid / G, t = tid % G;
  const float2* __restrict__ in = reinterpret_cast<const float2*>(a.in);
  float2* __restrict__ out = reinterpret_cast<float2*>(a.out);
  const float2* __restrict__ twg = reinterpret_cast<const float2*>(a.tw);   // exp(-2 pi i k / N), k <= N/2
  for (int i = tid; i < 16 * G; i += blockDim.x) {
    const int m = ((i / 16) * (i % 16)) % N;      // r = i / 16, j = i % 16
    const float2 w = m <= N / 2 ? twg[m] : twg[N - m];
    tw1[i] = m <= N / 2 ? w : make_float2(w.x, -w.y);
  }
  if (tid == 0) mbar_init(bar, 1);
  __syncthreads();
  const unsigned extra0 = blockIdx.x == 0 ? (unsigned)a.p3_stall : 0u;
  // tile -> the stage: six bulk copies of rows * Mz complex values (one per field)
  auto issue = [&](long long tile, unsigned extra) {
    const long long xy0 = tile * TL;
    const long long rows = (nxy - xy0) < TL ? (nxy - xy0) : TL;
    const unsigned bytes = (unsigned)(rows * Mz * (long long)sizeof(float2));
    mbar_expect_tx(bar, 6 * bytes + extra);
    for (int f = 0; f < 6; ++f)
      bulk_g2s(stage + (size_t)f * tile_elems, in + ((size_t)f * nxy + xy0) * Mz, bytes, bar);
  };
  if (tid == 0 && (long long)blockIdx.x < ntiles) issue(blockIdx.x, extra0);
  float2* xb = xbuf + l * P::LSTR;
  int it = 0;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
    const unsigned par = (unsigned)it & 1u;
    const bool arrived = mbar_wait_bounded(bar, par);
    if (!__syncthreads_and(arrived)) {
      if (tid == 0) {
        if (a.ctrl) {
          DnsCtrl* cw = const_cast<DnsCtrl*>(a.ctrl);
          cw->status = ST_TIMEOUT;
          cw->done = 1;
        }
        // let copies still in flight land before the block exits (the debug stall's bytes
        // never arrive: count them as arrived first; the wait stays bounded for any cause)
        if (it == 0 && extra0) mbar_complete_tx(bar, extra0);
        mbar_wait_bounded(bar, par);
      }
      return;
    }
    const long long xy = tile * TL + l;
    const bool live = xy < nxy;
    const float2* Sl = stage + l * Mz;
    // ---- the tile's inputs into registers: Z for (u0, u1), (u2, w0), (w1, w2) --------------
    RV zr[3][16];
#pragma unroll
    for (int p = 0; p < 3; ++p) {
      const float2* Sa = Sl + (2 * p) * tile_elems;
      const float2* Sb = Sa + tile_elems;
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        // Z_k from A_k, B_k (k <= Kz) or from their conjugates at N - k (k >= N - Kz)
        const int k = t + G * r;
        RV z = mk<RV>(0.f, 0.f);
        if (k <= Kz) {
          const float2 A = Sa[k], B = Sb[k];
          z = k == 0 ? mk<RV>(A.x, B.x) : mk<RV>(A.x - B.y, A.y + B.x);
        } else if (k >= N - Kz) {
          const float2 A = Sa[N - k], B = Sb[N - k];
          z = mk<RV>(A.x + B.y, B.x - A.y);
        }
        zr[p][r] = z;
      }
    }
    // the stage is read: the next tile's copies run while this one is transformed
    __syncthreads();
    if (tid == 0 && tile + (long long)gridDim.x < ntiles) {
      fence_proxy_async_smem();
      issue(tile + (long long)gridDim.x, 0);
    }
    // ---- three inverse transforms ----------------------------------------------------------
#pragma unroll
    for (int p = 0; p < 3; ++p) zrr_fft<N, +1, RV>(zr[p], xb, tw1, t);
    // ---- u x omega at the thread's 16 points ------------------------------------------------
    RV q[16], rr[16];
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      const float u0 = zr[0][m].x, u1 = zr[0][m].y, u2 = zr[1][m].x;
      const float w0 = zr[1][m].y, w1 = zr[2][m].x, w2 = zr[2][m].y;
      q[m] = mk<RV>(fmaf(u1, w2, -u2 * w1), fmaf(u2, w0, -u0 * w2));
      rr[m] = mk<RV>(fmaf(u0, w1, -u1 * w0), 0.f);
    }
    // ---- forward: p0 + i p1, split by conjugate symmetry through the exchange buffer -------
    zrr_fft<N, -1, RV>(q, xb, tw1, t);
#pragma unroll
    for (int m = 0; m < 16; ++m) xb[t + G * m] = make_float2(q[m].x, q[m].y);
    __syncwarp();
    if (live) {
      float2* o0 = out + (size_t)xy * Mz;
      float2* o1 = out + ((size_t)nxy + xy) * Mz;
      for (int k = t; k < Mz; k += G) {
        const float2 pk = xb[k], pm = xb[(N - k) & (N - 1)];
        o0[k] = make_float2(0.5f * (pk.x + pm.x), 0.5f * (pk.y - pm.y));
        o1[k] = make_float2(0.5f * (pk.y + pm.y), 0.5f * (pm.x - pk.x));
      }
    }
    __syncwarp();
    // ---- forward: p2 (real) --------------------------------------------------------------
    zrr_fft<N, -1, RV>(rr, xb, tw1, t);
    if (live) {
      float2* o2 = out + ((size_t)2 * nxy + xy) * Mz;
#pragma unroll
      for (int m = 0; m < 16; ++m) {
        const int k = t + G * m;
        if (k < Mz) o2[k] = make_float2(rr[m].x, rr[m].y);
      }
    }
  }
}

}  // namespace dns
