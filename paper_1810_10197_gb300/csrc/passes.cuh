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
  const void* tw;        // twiddle table (T complex) for this pass's axis
  double nu;
  double kf2;            // forcing band |kappa|^2 <= kf2 (0: no forcing)
};

template <int N> __host__ __device__ constexpr int p1_cols() { return N >= 512 ? 4 : 8; }
template <int N> __host__ __device__ constexpr int p3_lines() { return N >= 256 ? 4 : 8; }
constexpr int kTZ = 8;   // kz columns per CTA in the y passes

template <typename V> __device__ __forceinline__ V zero2() { return mk<V>(0, 0); }

// ------------------------------------------------------------------------------------------
// P1: x-inverse with the curl fused in.  grid (ceil(MyMz/TC), 2): y = 0 -> u, 1 -> omega.
// ------------------------------------------------------------------------------------------
template <typename T, int NX>
__global__ void __launch_bounds__(FftPlan<NX>::G * 3 * p1_cols<NX>())
k_p1(const PassArgs a) {
  using V = v2_t<T>;
  constexpr int TC = p1_cols<NX>();
  constexpr int G = FftPlan<NX>::G;
  constexpr int LD = NX + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* tw = reinterpret_cast<V*>(smem_raw);
  V* lines = tw + NX;
  if (gated_off(a.ctrl, a.gate_k1)) return;
  const Geom& g = a.g;
  const double2* __restrict__ Y = resolve_in(a.y, a.ctrl, a.yslot);
  V* __restrict__ out = reinterpret_cast<V*>(a.out);
  const V* __restrict__ twg = reinterpret_cast<const V*>(a.tw);
  const int half = blockIdx.y;
  const int col0 = blockIdx.x * TC;
  const int tid = threadIdx.x, nth = blockDim.x;
  for (int i = tid; i < NX; i += nth) tw[i] = twg[i];
  const int nzero = NX - g.Mx;
  for (int i = tid; i < 3 * TC * nzero; i += nth) {
    const int l = i / nzero, q = i - l * nzero;
    lines[l * LD + g.Kx + 1 + q] = zero2<V>();
  }
  for (int i = tid; i < g.Mx * TC; i += nth) {
    const int ix = i / TC, c = i - ix * TC, col = col0 + c;
    double2 f0 = make_double2(0, 0), f1 = f0, f2 = f0;
    if (col < g.MyMz) {
      const size_t off = (size_t)ix * g.MyMz + col;
      const double2 y0 = Y[off], y1 = Y[off + g.M], y2 = Y[off + 2 * g.M];
      const double s = g.inv_n3;
      if (half == 0) {
        f0 = make_double2(y0.x * s, y0.y * s);
        f1 = make_double2(y1.x * s, y1.y * s);
        f2 = make_double2(y2.x * s, y2.y * s);
      } else {
        const int jy = col / g.Mz, kz = col - jy * g.Mz;
        const double kx = g.sx * signed_mode(ix, g.Kx, g.Mx);
        const double ky = g.sy * signed_mode(jy, g.Ky, g.My);
        const double kzz = g.sz * kz;
        // omega = i kappa x Y
        const double cx_r = ky * y2.x - kzz * y1.x, cx_i = ky * y2.y - kzz * y1.y;
        const double cy_r = kzz * y0.x - kx * y2.x, cy_i = kzz * y0.y - kx * y2.y;
        const double cz_r = kx * y1.x - ky * y0.x, cz_i = kx * y1.y - ky * y0.y;
        f0 = make_double2(-cx_i * s, cx_r * s);
        f1 = make_double2(-cy_i * s, cy_r * s);
        f2 = make_double2(-cz_i * s, cz_r * s);
      }
    }
    const int pos = ix <= g.Kx ? ix : NX - g.Mx + ix;
    lines[(0 * TC + c) * LD + pos] = mk<V>((T)f0.x, (T)f0.y);
    lines[(1 * TC + c) * LD + pos] = mk<V>((T)f1.x, (T)f1.y);
    lines[(2 * TC + c) * LD + pos] = mk<V>((T)f2.x, (T)f2.y);
  }
  __syncthreads();
  line_fft<V, NX, +1, 1>(lines + (tid / G) * LD, tid % G, tw);
  for (int i = tid; i < 3 * NX * TC; i += nth) {
    const int f = i / (NX * TC), r = i - f * (NX * TC), x = r / TC, c = r - x * TC, col = col0 + c;
    if (col < g.MyMz) out[((size_t)(half * 3 + f) * NX + x) * g.MyMz + col] = lines[(f * TC + c) * LD + x];
  }
}

// ------------------------------------------------------------------------------------------
// P2 / P4: DFT along y for one (field, x) and kTZ kz columns.  grid (ceil(Mz/kTZ), nx, nf).
// INVERSE: retained ky -> all y.  Forward: all y -> retained ky.
// ------------------------------------------------------------------------------------------
template <typename T, int NY, bool INVERSE>
__global__ void __launch_bounds__(FftPlan<NY>::G * kTZ)
k_py(const PassArgs a) {
  using V = v2_t<T>;
  constexpr int G = FftPlan<NY>::G;
  constexpr int LD = NY + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* tw = reinterpret_cast<V*>(smem_raw);
  V* lines = tw + NY;
  if (gated_off(a.ctrl, a.gate_k1)) return;
  const Geom& g = a.g;
  const V* __restrict__ in = reinterpret_cast<const V*>(a.in);
  V* __restrict__ out = reinterpret_cast<V*>(a.out);
  const V* __restrict__ twg = reinterpret_cast<const V*>(a.tw);
  const int f = blockIdx.z, x = blockIdx.y, kz0 = blockIdx.x * kTZ;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int Mz = g.Mz;
  for (int i = tid; i < NY; i += nth) tw[i] = twg[i];
  if (INVERSE) {
    const int nzero = NY - g.My;
    for (int i = tid; i < kTZ * nzero; i += nth) {
      const int l = i / nzero, q = i - l * nzero;
      lines[l * LD + g.Ky + 1 + q] = zero2<V>();
    }
    const V* src = in + ((size_t)f * g.nx + x) * g.My * Mz;
    for (int i = tid; i < g.My * kTZ; i += nth) {
      const int jy = i / kTZ, c = i - jy * kTZ, kz = kz0 + c;
      const V v = kz < Mz ? src[(size_t)jy * Mz + kz] : zero2<V>();
      const int pos = jy <= g.Ky ? jy : NY - g.My + jy;
      lines[c * LD + pos] = v;
    }
  } else {
    const V* src = in + ((size_t)f * g.nx + x) * NY * Mz;
    for (int i = tid; i < NY * kTZ; i += nth) {
      const int y = i / kTZ, c = i - y * kTZ, kz = kz0 + c;
      lines[c * LD + y] = kz < Mz ? src[(size_t)y * Mz + kz] : zero2<V>();
    }
  }
  __syncthreads();
  line_fft<V, NY, INVERSE ? +1 : -1, 1>(lines + (tid / G) * LD, tid % G, tw);
  if (INVERSE) {
    V* dst = out + ((size_t)f * g.nx + x) * NY * Mz;
    for (int i = tid; i < NY * kTZ; i += nth) {
      const int y = i / kTZ, c = i - y * kTZ, kz = kz0 + c;
      if (kz < Mz) dst[(size_t)y * Mz + kz] = lines[c * LD + y];
    }
  } else {
    V* dst = out + ((size_t)f * g.nx + x) * g.My * Mz;
    for (int i = tid; i < g.My * kTZ; i += nth) {
      const int jy = i / kTZ, c = i - jy * kTZ, kz = kz0 + c;
      const int pos = jy <= g.Ky ? jy : NY - g.My + jy;
      if (kz < Mz) dst[(size_t)jy * Mz + kz] = lines[c * LD + pos];
    }
  }
}

// ------------------------------------------------------------------------------------------
// P3: z lines.  Inverse real DFT of 6 fields through an MZ = nz/2 point complex DFT of the
// packed sequence z_n = x_2n + i x_2n+1, u x omega on both packed halves, forward real DFT
// of the 3 products the same way.  grid ceil(nx ny / TL).
//   C2R pre-step : Z_k = (X_k + conj X_{M-k}) + i e^{+2 pi i k/nz} (X_k - conj X_{M-k})
//   R2C post-step: X_k = (Z_k + conj Z_{M-k})/2 - (i/2) e^{-2 pi i k/nz} (Z_k - conj Z_{M-k})
// ------------------------------------------------------------------------------------------
template <typename T, int MZ>
__global__ void __launch_bounds__(FftPlan<MZ>::G * 6 * p3_lines<MZ>())
k_p3(const PassArgs a) {
  using V = v2_t<T>;
  constexpr int TL = p3_lines<MZ>();
  constexpr int G = FftPlan<MZ>::G;
  constexpr int LD = MZ + 1;
  constexpr int NZ = 2 * MZ;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* tw = reinterpret_cast<V*>(smem_raw);      // NZ entries: exp(-2 pi i m / NZ)
  V* lines = tw + NZ;                          // 6*TL lines of LD
  if (gated_off(a.ctrl, a.gate_k1)) return;
  const Geom& g = a.g;
  const V* __restrict__ in = reinterpret_cast<const V*>(a.in);
  V* __restrict__ out = reinterpret_cast<V*>(a.out);
  const V* __restrict__ twg = reinterpret_cast<const V*>(a.tw);
  const long long nxy = (long long)g.nx * g.ny;
  const long long xy0 = (long long)blockIdx.x * TL;
  const int Mz = g.Mz;
  const int tid = threadIdx.x, nth = blockDim.x;
  for (int i = tid; i < NZ; i += nth) tw[i] = twg[i];
  {
    const int nzero = MZ + 1 - Mz;   // positions Mz..MZ
    for (int i = tid; i < 6 * TL * nzero; i += nth) {
      const int l = i / nzero, q = i - l * nzero;
      lines[l * LD + Mz + q] = zero2<V>();
    }
  }
  for (int i = tid; i < 6 * TL * Mz; i += nth) {
    const int f = i / (TL * Mz), r = i - f * (TL * Mz);
    const int l = r / Mz, kz = r - l * Mz;
    const long long xy = xy0 + l;
    lines[(f * TL + l) * LD + kz] = xy < nxy ? in[((size_t)f * nxy + xy) * Mz + kz] : zero2<V>();
  }
  __syncthreads();
  // C2R pre-step on pairs (k, MZ-k), k = 0..MZ/2
  {
    constexpr int NP = MZ / 2 + 1;
    for (int i = tid; i < 6 * TL * NP; i += nth) {
      const int l = i / NP, k = i - l * NP;
      V* L = lines + l * LD;
      const int m = MZ - k;
      const V xk = L[k], xm = L[m];
      // Z_k
      {
        const V s = cadd(xk, cconj(xm)), d = csub(xk, cconj(xm));
        const V w = cconj(tw[k]);                         // e^{+2 pi i k / NZ}
        const V zk = cadd(s, mul_si<+1>(cmul(w, d)));
        if (k != 0 && k != m) {
          const V s2 = cadd(xm, cconj(xk)), d2 = csub(xm, cconj(xk));
          const V w2 = cconj(tw[m]);
          L[m] = cadd(s2, mul_si<+1>(cmul(w2, d2)));
        }
        L[k] = zk;
      }
    }
  }
  __syncthreads();
  line_fft<V, MZ, +1, 2>(lines + (tid / G) * LD, tid % G, tw);
  // u x omega on both packed halves (real part: even z, imaginary part: odd z)
  for (int i = tid; i < TL * MZ; i += nth) {
    const int l = i / MZ, n = i - l * MZ;
    const V u0 = lines[(0 * TL + l) * LD + n], u1 = lines[(1 * TL + l) * LD + n], u2 = lines[(2 * TL + l) * LD + n];
    const V w0 = lines[(3 * TL + l) * LD + n], w1 = lines[(4 * TL + l) * LD + n], w2 = lines[(5 * TL + l) * LD + n];
    lines[(0 * TL + l) * LD + n] = mk<V>(u1.x * w2.x - u2.x * w1.x, u1.y * w2.y - u2.y * w1.y);
    lines[(1 * TL + l) * LD + n] = mk<V>(u2.x * w0.x - u0.x * w2.x, u2.y * w0.y - u0.y * w2.y);
    lines[(2 * TL + l) * LD + n] = mk<V>(u0.x * w1.x - u1.x * w0.x, u0.y * w1.y - u1.y * w0.y);
  }
  __syncthreads();
  // forward complex DFT of the 3 packed product lines; threads on lines >= 3 TL idle but
  // still take part in the barriers
  {
    const int line = tid / G;
    line_fft<V, MZ, -1, 2>(lines + (line < 3 * TL ? line : 0) * LD, tid % G, tw, line < 3 * TL);
  }
  // R2C post-step, keep kz <= Kz
  for (int i = tid; i < 3 * TL * Mz; i += nth) {
    const int c = i / (TL * Mz), r = i - c * (TL * Mz);
    const int l = r / Mz, k = r - l * Mz;
    const long long xy = xy0 + l;
    if (xy >= nxy) continue;
    const V* L = lines + (c * TL + l) * LD;
    const V zk = L[k], zm = L[(MZ - k) % MZ];
    const V s = cadd(zk, cconj(zm)), d = csub(zk, cconj(zm));
    const V od = cmul(tw[k], d);                   // e^{-2 pi i k / NZ} (Z_k - conj Z_{M-k})
    const T hf = (T)0.5;
    // X = s/2 - (i/2) od
    out[((size_t)c * nxy + xy) * Mz + k] = mk<V>(hf * (s.x + od.y), hf * (s.y - od.x));
  }
}

// ------------------------------------------------------------------------------------------
// P5: x-forward + FP64 epilogue.  grid ceil(MyMz/TC).
// ------------------------------------------------------------------------------------------
template <typename T, int NX>
__global__ void __launch_bounds__(FftPlan<NX>::G * 3 * p1_cols<NX>())
k_p5(const PassArgs a) {
  using V = v2_t<T>;
  constexpr int TC = p1_cols<NX>();
  constexpr int G = FftPlan<NX>::G;
  constexpr int LD = NX + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* tw = reinterpret_cast<V*>(smem_raw);
  V* lines = tw + NX;
  if (gated_off(a.ctrl, a.gate_k1)) return;
  const Geom& g = a.g;
  const double2* __restrict__ Y = resolve_in(a.y, a.ctrl, a.yslot);
  double2* __restrict__ K = resolve_out(a.kout, a.ctrl, a.kslot);
  const V* __restrict__ in = reinterpret_cast<const V*>(a.in);
  const V* __restrict__ twg = reinterpret_cast<const V*>(a.tw);
  const int col0 = blockIdx.x * TC;
  const int tid = threadIdx.x, nth = blockDim.x;
  for (int i = tid; i < NX; i += nth) tw[i] = twg[i];
  for (int i = tid; i < 3 * NX * TC; i += nth) {
    const int f = i / (NX * TC), r = i - f * (NX * TC), x = r / TC, c = r - x * TC, col = col0 + c;
    lines[(f * TC + c) * LD + x] = col < g.MyMz ? in[((size_t)f * NX + x) * g.MyMz + col] : zero2<V>();
  }
  __syncthreads();
  line_fft<V, NX, -1, 1>(lines + (tid / G) * LD, tid % G, tw);
  const double fc = (a.ctrl && a.kf2 > 0) ? a.ctrl->forcing_coef : 0.0;
  for (int i = tid; i < g.Mx * TC; i += nth) {
    const int ix = i / TC, c = i - ix * TC, col = col0 + c;
    if (col >= g.MyMz) continue;
    const int pos = ix <= g.Kx ? ix : NX - g.Mx + ix;
    const V n0 = lines[(0 * TC + c) * LD + pos], n1 = lines[(1 * TC + c) * LD + pos], n2 = lines[(2 * TC + c) * LD + pos];
    const int jy = col / g.Mz, kz = col - jy * g.Mz;
    const double kx = g.sx * signed_mode(ix, g.Kx, g.Mx);
    const double ky = g.sy * signed_mode(jy, g.Ky, g.My);
    const double kzz = g.sz * kz;
    const double k2 = kx * kx + ky * ky + kzz * kzz;
    double nr0 = n0.x, ni0 = n0.y, nr1 = n1.x, ni1 = n1.y, nr2 = n2.x, ni2 = n2.y;
    if (k2 > 0) {
      const double ik2 = 1.0 / k2;
      const double dr = (kx * nr0 + ky * nr1 + kzz * nr2) * ik2;
      const double di = (kx * ni0 + ky * ni1 + kzz * ni2) * ik2;
      nr0 -= kx * dr; ni0 -= kx * di;
      nr1 -= ky * dr; ni1 -= ky * di;
      nr2 -= kzz * dr; ni2 -= kzz * di;
    }
    const size_t off = (size_t)ix * g.MyMz + col;
    const double2 y0 = Y[off], y1 = Y[off + g.M], y2 = Y[off + 2 * g.M];
    double vis = -a.nu * k2;
    if (fc != 0.0 && k2 > 0 && k2 <= a.kf2) vis += fc;
    K[off] = make_double2(nr0 + vis * y0.x, ni0 + vis * y0.y);
    K[off + g.M] = make_double2(nr1 + vis * y1.x, ni1 + vis * y1.y);
    K[off + 2 * g.M] = make_double2(nr2 + vis * y2.x, ni2 + vis * y2.y);
  }
}

// ------------------------------------------------------------------------------------------
// Host side: launch pass `which` (1..5) for element type T (instantiated in passes_f64.cu and
// passes_f32.cu).  Returns cudaErrorInvalidValue for an unsupported line length.
// ------------------------------------------------------------------------------------------
template <typename T> cudaError_t launch_pass(int which, const PassArgs& a, cudaStream_t s);

}  // namespace dns
