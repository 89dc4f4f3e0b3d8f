// Batched line FFTs in shared memory: mixed-radix (2,3,4,8,16) Stockham auto-sort stages,
// each thread doing whole radix-R butterflies in registers.
//
// A CTA holds several lines of length N in shared memory; G threads cooperate on one line.
// Stage s (radix R, NS = product of the earlier radices) reads R elements of butterfly j at
// stride N/R, applies twiddles W_{NS R}^{(j mod NS) r}, does an R-point DFT in registers
// and writes them to (j - j mod NS) R + j mod NS + r NS.  All reads of a stage finish
// (barrier) before any write, so one buffer suffices.  SIGN = -1 forward, +1 inverse
// (unnormalised both ways).
#pragma once

#include "common.cuh"

namespace dns {

// Radix plans: stage radices (1 = unused) and G, the threads that share one line.  One
// constexpr source for device templates and host-side twiddle-table construction.
__host__ __device__ constexpr int plan_radix(int n, int s) {
  switch (n) {
    case 4: return s == 0 ? 4 : 1;
    case 6: return s == 0 ? 2 : (s == 1 ? 3 : 1);
    case 8: return s == 0 ? 8 : 1;
    case 12: return s == 0 ? 4 : (s == 1 ? 3 : 1);
    case 16: return s < 2 ? 4 : 1;
    case 24: return s == 0 ? 8 : (s == 1 ? 3 : 1);
    case 32: return s == 0 ? 8 : (s == 1 ? 4 : 1);
    case 48: return s < 2 ? 4 : 3;
    case 64: return s < 2 ? 8 : 1;
    case 96: return s == 0 ? 8 : (s == 1 ? 4 : 3);
    case 128: return s == 0 ? 16 : (s == 1 ? 8 : 1);
    case 192: return s == 0 ? 16 : (s == 1 ? 4 : 3);
    case 256: return s < 2 ? 16 : 1;
    case 384: return s == 0 ? 16 : (s == 1 ? 8 : 3);
    case 512: return 8;
    case 768: return s < 2 ? 16 : 3;
  }
  return 0;
}
__host__ __device__ constexpr int plan_threads(int n) {
  switch (n) {
    case 4: case 8: return 1;
    case 6: return 3;
    case 12: case 16: return 4;
    case 24: case 32: case 64: case 128: return 8;
    case 48: case 96: case 192: case 256: return 16;
    case 384: case 512: return 32;
    case 768: return 64;
  }
  return 0;
}
__host__ __device__ constexpr int plan_stages(int n) {
  return plan_radix(n, 2) > 1 ? 3 : (plan_radix(n, 1) > 1 ? 2 : 1);
}
// product of the radices before stage s
__host__ __device__ constexpr int plan_ns(int n, int s) {
  return s == 0 ? 1 : (s == 1 ? plan_radix(n, 0) : plan_radix(n, 0) * plan_radix(n, 1));
}
// offset of stage s's twiddle table (stages >= 1 only; NS (R-1) entries each)
__host__ __device__ constexpr int plan_tw_offset(int n, int s) {
  return s <= 1 ? 0 : plan_ns(n, 1) * (plan_radix(n, 1) - 1);
}
__host__ __device__ constexpr int plan_tw_size(int n) {
  int t = 0;
  for (int s = 1; s < plan_stages(n); ++s) t += plan_ns(n, s) * (plan_radix(n, s) - 1);
  return t;
}

template <int N> struct FftPlan {
  static constexpr int S = plan_stages(N), R0 = plan_radix(N, 0), R1 = plan_radix(N, 1),
                       R2 = plan_radix(N, 2), G = plan_threads(N);
  static_assert(R0 * R1 * R2 == N, "unsupported line length");
};

template <int N, int s> struct StageInfo {
  static constexpr int R = plan_radix(N, s);
  static constexpr int NS = plan_ns(N, s);
  static constexpr int TWOFF = plan_tw_offset(N, s);
};

// Shared-memory layout of a line: element p sits at p + p / (128 B / element size), so
// stride-R butterfly writes spread over all banks; LD is the (odd) line stride.
template <typename V> __host__ __device__ constexpr int pad_shift() { return sizeof(V) == 8 ? 4 : 3; }
template <typename V> __host__ __device__ __forceinline__ constexpr int pidx(int p) { return p + (p >> pad_shift<V>()); }
template <typename V, int N> __host__ __device__ constexpr int line_ld() {
  return (N + (N >> pad_shift<V>())) | 1;
}

// ---- R-point DFTs in registers: X_k = sum_r v_r exp(SIGN 2 pi i r k / R) -------------------

template <int R, int SIGN, typename V> struct Dft;

template <int SIGN, typename V> struct Dft<2, SIGN, V> {
  static __device__ __forceinline__ void run(V* v) {
    V a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  }
};

template <int SIGN, typename V> struct Dft<3, SIGN, V> {
  static __device__ __forceinline__ void run(V* v) {
    using T = decltype(V::x);
    const T h3 = (T)0.86602540378443864676;   // sqrt(3)/2
    V a = v[0], t = cadd(v[1], v[2]), d = csub(v[1], v[2]);
    V s = mk<V>(fma((T)-0.5, t.x, a.x), fma((T)-0.5, t.y, a.y));
    V q = mul_si<SIGN>(cscale(d, h3));
    v[0] = cadd(a, t);
    v[1] = cadd(s, q);
    v[2] = csub(s, q);
  }
};

template <int SIGN, typename V> struct Dft<4, SIGN, V> {
  static __device__ __forceinline__ void run(V* v) {
    V s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
    V s13 = cadd(v[1], v[3]), d13 = mul_si<SIGN>(csub(v[1], v[3]));
    v[0] = cadd(s02, s13);
    v[2] = csub(s02, s13);
    v[1] = cadd(d02, d13);
    v[3] = csub(d02, d13);
  }
};

// multiply by W8^1 = (1 + SIGN i)/sqrt2 and W8^3 = (-1 + SIGN i)/sqrt2
template <int SIGN, typename V> __device__ __forceinline__ V w8_1(V a) {
  using T = decltype(V::x);
  const T r = (T)0.70710678118654752440;
  return SIGN < 0 ? mk<V>(bmul(badd(a.x, a.y), r), bmul(bsub(a.y, a.x), r))
                  : mk<V>(bmul(bsub(a.x, a.y), r), bmul(badd(a.y, a.x), r));
}
template <int SIGN, typename V> __device__ __forceinline__ V w8_3(V a) {
  using T = decltype(V::x);
  const T r = (T)0.70710678118654752440;
  return SIGN < 0 ? mk<V>(bmul(bsub(a.y, a.x), r), -bmul(badd(a.x, a.y), r))
                  : mk<V>(-bmul(badd(a.x, a.y), r), bmul(bsub(a.x, a.y), r));
}

template <int SIGN, typename V> struct Dft<8, SIGN, V> {
  // 8 = 4 x 2: n = 2 n1 + n2, k = k1 + 4 k2
  static __device__ __forceinline__ void run(V* v) {
    V e[4] = {v[0], v[2], v[4], v[6]};
    V o[4] = {v[1], v[3], v[5], v[7]};
    Dft<4, SIGN, V>::run(e);
    Dft<4, SIGN, V>::run(o);
    o[1] = w8_1<SIGN>(o[1]);
    o[2] = mul_si<SIGN>(o[2]);
    o[3] = w8_3<SIGN>(o[3]);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      v[k] = cadd(e[k], o[k]);
      v[k + 4] = csub(e[k], o[k]);
    }
  }
};

template <int SIGN, typename V> struct Dft<16, SIGN, V> {
  // 16 = 4 x 4: n = 4 n1 + n2, k = k1 + 4 k2; inner twiddle W16^{n2 k1}
  static __device__ __forceinline__ void run(V* v) {
    using T = decltype(V::x);
    const T c1 = (T)0.92387953251128675613, s1 = (T)0.38268343236508977173;
    V y[4][4];
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) {
      y[n2][0] = v[n2]; y[n2][1] = v[4 + n2]; y[n2][2] = v[8 + n2]; y[n2][3] = v[12 + n2];
      Dft<4, SIGN, V>::run(y[n2]);
    }
    const T ps1 = SIGN > 0 ? s1 : -s1, pc1 = SIGN > 0 ? c1 : -c1;   // SIGN s1, SIGN c1
    // n2 = 1: W^0, W^1, W^2, W^3
    y[1][1] = cmul(y[1][1], mk<V>(c1, ps1));
    y[1][2] = w8_1<SIGN>(y[1][2]);
    y[1][3] = cmul(y[1][3], mk<V>(s1, pc1));
    // n2 = 2: W^0, W^2, W^4, W^6
    y[2][1] = w8_1<SIGN>(y[2][1]);
    y[2][2] = mul_si<SIGN>(y[2][2]);
    y[2][3] = w8_3<SIGN>(y[2][3]);
    // n2 = 3: W^0, W^3, W^6, W^9
    y[3][1] = cmul(y[3][1], mk<V>(s1, pc1));
    y[3][2] = w8_3<SIGN>(y[3][2]);
    y[3][3] = cmul(y[3][3], mk<V>(-c1, -ps1));
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
      V z[4] = {y[0][k1], y[1][k1], y[2][k1], y[3][k1]};
      Dft<4, SIGN, V>::run(z);
#pragma unroll
      for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = z[k2];
    }
  }
};

// FP64 16- and 8-point DFTs with the twiddles of the second radix-4 layer factored for
// fused multiply-adds (the FP64 forms are bound by the FP64 pipe's issue rate, so every
// instruction counts): with W = exp(SIGN i pi / 8) = c (1 + SIGN i t), t = tan(pi / 8),
//   W^3 = SIGN i c (1 - SIGN i t),  W^9 = -c (1 + SIGN i t),  W^2 = r (1 + SIGN i),
//   W^6 = r (-1 + SIGN i),  r = 1 / sqrt(2),
// the common scale (c or r) of a column's twiddled terms is applied once, inside the fused
// multiply-adds of its output butterflies: 144 instead of 160 FP64 instructions per 16-point
// DFT, 52 instead of 56 per 8-point DFT.  Same values as the generic forms up to rounding.
namespace fma_dft {
__device__ __forceinline__ double2 rot(double2 a, int S) { return make_double2(-S * a.y, S * a.x); }   // S i a
// (X, Y) outputs of a radix-4 column whose odd terms share the scale k: s02 + k S, s02 - k S,
// d02 + k S i D, d02 - k S i D with S = p + q, D = p - q
template <int SIGN>
__device__ __forceinline__ void out4(double2 s02, double2 d02, double2 p, double2 q, double k, double2* X0,
                                     double2* X1, double2* X2, double2* X3) {
  const double2 S = make_double2(p.x + q.x, p.y + q.y), D = make_double2(p.x - q.x, p.y - q.y);
  *X0 = make_double2(fma(k, S.x, s02.x), fma(k, S.y, s02.y));
  *X2 = make_double2(fma(-k, S.x, s02.x), fma(-k, S.y, s02.y));
  // S i D = (-SIGN D.y, SIGN D.x)
  *X1 = make_double2(fma(-SIGN * k, D.y, d02.x), fma(SIGN * k, D.x, d02.y));
  *X3 = make_double2(fma(SIGN * k, D.y, d02.x), fma(-SIGN * k, D.x, d02.y));
}
}  // namespace fma_dft

template <int SIGN> struct Dft<16, SIGN, double2> {
  static __device__ __forceinline__ void run(double2* v) {
    using namespace fma_dft;
    constexpr double c = 0.92387953251128675613, t = 0.41421356237309504880, r = 0.70710678118654752440;
    constexpr double St = SIGN * t;
    double2 y[4][4];
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) {
      y[n2][0] = v[n2]; y[n2][1] = v[4 + n2]; y[n2][2] = v[8 + n2]; y[n2][3] = v[12 + n2];
      Dft<4, SIGN, double2>::run(y[n2]);
    }
    double2 z[4];
    // k1 = 0: no twiddles
    z[0] = y[0][0]; z[1] = y[1][0]; z[2] = y[2][0]; z[3] = y[3][0];
    Dft<4, SIGN, double2>::run(z);
    v[0] = z[0]; v[4] = z[1]; v[8] = z[2]; v[12] = z[3];
    {  // k1 = 1: W^1 = c (1 + S i t), W^2 = r (1 + S i), W^3 = S i c (1 - S i t)
      const double2 a1 = y[1][1], a2 = y[2][1], a3 = y[3][1], z0 = y[0][1];
      const double2 p = make_double2(fma(-St, a1.y, a1.x), fma(St, a1.x, a1.y));
      const double2 q = rot(make_double2(fma(St, a3.y, a3.x), fma(-St, a3.x, a3.y)), SIGN);
      const double2 A = make_double2(a2.x - SIGN * a2.y, a2.y + SIGN * a2.x);
      const double2 s02 = make_double2(fma(r, A.x, z0.x), fma(r, A.y, z0.y));
      const double2 d02 = make_double2(fma(-r, A.x, z0.x), fma(-r, A.y, z0.y));
      out4<SIGN>(s02, d02, p, q, c, &v[1], &v[5], &v[9], &v[13]);
    }
    {  // k1 = 2: W^2 = r (1 + S i), W^4 = S i, W^6 = r (-1 + S i)
      const double2 a1 = y[1][2], a2 = y[2][2], a3 = y[3][2], z0 = y[0][2];
      const double2 p = make_double2(a1.x - SIGN * a1.y, a1.y + SIGN * a1.x);
      const double2 q = make_double2(-a3.x - SIGN * a3.y, SIGN * a3.x - a3.y);
      const double2 z2 = rot(a2, SIGN);
      const double2 s02 = make_double2(z0.x + z2.x, z0.y + z2.y), d02 = make_double2(z0.x - z2.x, z0.y - z2.y);
      out4<SIGN>(s02, d02, p, q, r, &v[2], &v[6], &v[10], &v[14]);
    }
    {  // k1 = 3: W^3 = S i c (1 - S i t), W^6 = r (-1 + S i), W^9 = -c (1 + S i t)
      const double2 a1 = y[1][3], a2 = y[2][3], a3 = y[3][3], z0 = y[0][3];
      const double2 p = rot(make_double2(fma(St, a1.y, a1.x), fma(-St, a1.x, a1.y)), SIGN);
      const double2 q = make_double2(fma(St, a3.y, -a3.x), fma(-St, a3.x, -a3.y));
      const double2 A = make_double2(-a2.x - SIGN * a2.y, SIGN * a2.x - a2.y);
      const double2 s02 = make_double2(fma(r, A.x, z0.x), fma(r, A.y, z0.y));
      const double2 d02 = make_double2(fma(-r, A.x, z0.x), fma(-r, A.y, z0.y));
      out4<SIGN>(s02, d02, p, q, c, &v[3], &v[7], &v[11], &v[15]);
    }
  }
};

template <int SIGN> struct Dft<8, SIGN, double2> {
  // 8 = 4 x 2 (n = 2 n1 + n2, k = k1 + 4 k2): W8^1 = r (1 + S i), W8^3 = r (-1 + S i)
  static __device__ __forceinline__ void run(double2* v) {
    using namespace fma_dft;
    constexpr double r = 0.70710678118654752440;
    double2 e[4] = {v[0], v[2], v[4], v[6]};
    double2 o[4] = {v[1], v[3], v[5], v[7]};
    Dft<4, SIGN, double2>::run(e);
    Dft<4, SIGN, double2>::run(o);
    const double2 A1 = make_double2(o[1].x - SIGN * o[1].y, o[1].y + SIGN * o[1].x);
    const double2 A3 = make_double2(-o[3].x - SIGN * o[3].y, SIGN * o[3].x - o[3].y);
    const double2 o2 = rot(o[2], SIGN);
    v[0] = make_double2(e[0].x + o[0].x, e[0].y + o[0].y);
    v[4] = make_double2(e[0].x - o[0].x, e[0].y - o[0].y);
    v[1] = make_double2(fma(r, A1.x, e[1].x), fma(r, A1.y, e[1].y));
    v[5] = make_double2(fma(-r, A1.x, e[1].x), fma(-r, A1.y, e[1].y));
    v[2] = make_double2(e[2].x + o2.x, e[2].y + o2.y);
    v[6] = make_double2(e[2].x - o2.x, e[2].y - o2.y);
    v[3] = make_double2(fma(r, A3.x, e[3].x), fma(r, A3.y, e[3].y));
    v[7] = make_double2(fma(-r, A3.x, e[3].x), fma(-r, A3.y, e[3].y));
  }
};

// The same factoring for FP32 values as paired instructions (FFMA2 / FADD2): the register-
// resident transforms are bound by instruction issue.
namespace fma_dft {
__device__ __forceinline__ float2 swp(float2 a) { return make_float2(a.y, a.x); }
template <int SIGN>
__device__ __forceinline__ void out4(float2 s02, float2 d02, float2 p, float2 q, float k, float2* X0, float2* X1,
                                     float2* X2, float2* X3) {
  const float2 S = __fadd2_rn(p, q), D = __fadd2_rn(p, make_float2(-q.x, -q.y));
  *X0 = __ffma2_rn(make_float2(k, k), S, s02);
  *X2 = __ffma2_rn(make_float2(-k, -k), S, s02);
  const float2 Ds = swp(D);   // S i D = (-SIGN D.y, SIGN D.x)
  *X1 = __ffma2_rn(make_float2(-SIGN * k, SIGN * k), Ds, d02);
  *X3 = __ffma2_rn(make_float2(SIGN * k, -SIGN * k), Ds, d02);
}
}  // namespace fma_dft

template <int SIGN> struct Dft<16, SIGN, float2> {
  static __device__ __forceinline__ void run(float2* v) {
    using namespace fma_dft;
    constexpr float c = 0.92387953251128675613f, t = 0.41421356237309504880f, r = 0.70710678118654752440f;
    constexpr float St = SIGN * t;
    float2 y[4][4];
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) {
      y[n2][0] = v[n2]; y[n2][1] = v[4 + n2]; y[n2][2] = v[8 + n2]; y[n2][3] = v[12 + n2];
      Dft<4, SIGN, float2>::run(y[n2]);
    }
    float2 z[4] = {y[0][0], y[1][0], y[2][0], y[3][0]};
    Dft<4, SIGN, float2>::run(z);
    v[0] = z[0]; v[4] = z[1]; v[8] = z[2]; v[12] = z[3];
    {  // k1 = 1: W^1 = c (1 + S i t), W^2 = r (1 + S i), W^3 = S i c (1 - S i t)
      const float2 a1 = y[1][1], a2 = y[2][1], a3 = y[3][1], z0 = y[0][1];
      const float2 p = __ffma2_rn(make_float2(-St, St), swp(a1), a1);
      const float2 R = __ffma2_rn(make_float2(St, -St), swp(a3), a3);
      const float2 q = make_float2(-SIGN * R.y, SIGN * R.x);
      const float2 A = __ffma2_rn(make_float2(-(float)SIGN, (float)SIGN), swp(a2), a2);
      out4<SIGN>(__ffma2_rn(make_float2(r, r), A, z0), __ffma2_rn(make_float2(-r, -r), A, z0), p, q, c,
                 &v[1], &v[5], &v[9], &v[13]);
    }
    {  // k1 = 2: W^2 = r (1 + S i), W^4 = S i, W^6 = r (-1 + S i)
      const float2 a1 = y[1][2], a2 = y[2][2], a3 = y[3][2], z0 = y[0][2];
      const float2 p = __ffma2_rn(make_float2(-(float)SIGN, (float)SIGN), swp(a1), a1);
      const float2 q = __ffma2_rn(make_float2(-(float)SIGN, (float)SIGN), swp(a3), make_float2(-a3.x, -a3.y));
      const float2 z2 = make_float2(-SIGN * a2.y, SIGN * a2.x);
      out4<SIGN>(__fadd2_rn(z0, z2), __fadd2_rn(z0, make_float2(-z2.x, -z2.y)), p, q, r, &v[2], &v[6], &v[10],
                 &v[14]);
    }
    {  // k1 = 3: W^3 = S i c (1 - S i t), W^6 = r (-1 + S i), W^9 = -c (1 + S i t)
      const float2 a1 = y[1][3], a2 = y[2][3], a3 = y[3][3], z0 = y[0][3];
      const float2 R = __ffma2_rn(make_float2(St, -St), swp(a1), a1);
      const float2 p = make_float2(-SIGN * R.y, SIGN * R.x);
      const float2 q = __ffma2_rn(make_float2(St, -St), swp(a3), make_float2(-a3.x, -a3.y));
      const float2 A = __ffma2_rn(make_float2(-(float)SIGN, (float)SIGN), swp(a2), make_float2(-a2.x, -a2.y));
      out4<SIGN>(__ffma2_rn(make_float2(r, r), A, z0), __ffma2_rn(make_float2(-r, -r), A, z0), p, q, c,
                 &v[3], &v[7], &v[11], &v[15]);
    }
  }
};

// ---- one Stockham stage and the whole line transform ------------------------------------

// Linear padded indexing.  A stage reads j + r B (j < B) and writes q + r NS with
// q = (j - j mod NS) R + j mod NS.  When pidx(j + r B) = pidx(j) + pidx(r B) for every j, r
// (and likewise for the writes), each element's padded index is one run-time base per
// butterfly plus a compile-time offset: no per-element index arithmetic.  Power-of-two
// strides satisfy this; stages next to a radix-3 stage may not, and keep the general form.
// Checked exhaustively at compile time.
template <typename V, int N, int s> __host__ __device__ constexpr bool stage_loads_linear() {
  constexpr int R = StageInfo<N, s>::R, B = N / R;
  for (int j = 0; j < B; ++j)
    for (int r = 0; r < R; ++r)
      if (pidx<V>(j + r * B) != pidx<V>(j) + pidx<V>(r * B)) return false;
  return true;
}
template <typename V, int N, int s> __host__ __device__ constexpr bool stage_stores_linear() {
  constexpr int R = StageInfo<N, s>::R, B = N / R, NS = StageInfo<N, s>::NS;
  for (int j = 0; j < B; ++j) {
    const int q = (j - j % NS) * R + j % NS;
    for (int r = 0; r < R; ++r)
      if (pidx<V>(q + r * NS) != pidx<V>(q) + pidx<V>(r * NS)) return false;
  }
  return true;
}

// The G threads of a line are consecutive (line = tid / G) and, when G divides 32, lie in one
// warp: the stages of a line then need only warp-level ordering, and line_fft ends
// with one block barrier for what the caller does next.
template <int N> __host__ __device__ constexpr bool warp_local() { return 32 % plan_threads(N) == 0; }
template <int N> __device__ __forceinline__ void stage_sync() {
  if constexpr (warp_local<N>()) __syncwarp();
  else __syncthreads();
}
// ordering for work a line's own G threads did on it before line_fft
template <int N> __device__ __forceinline__ void line_sync() { stage_sync<N>(); }

// tws: the stage twiddle tables of this line length; stage s >= 1 holds, at
// TWOFF + jm (R-1) + (r-1), exp(SIGN' 2 pi i jm r / (NS R)) with SIGN' = -1 (conjugated for
// inverse transforms).
template <typename V, int N, int SIGN, int s>
__device__ __forceinline__ void fft_stage(V* x, int g, const V* tws, bool active) {
  constexpr int R = StageInfo<N, s>::R;
  constexpr int NS = StageInfo<N, s>::NS;
  constexpr int B = N / R;
  constexpr int G = FftPlan<N>::G;
  constexpr int PER = (B + G - 1) / G;
  V v[PER][R];
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    const int j = g + p * G;
    if (active && ((B % G == 0) || j < B)) {
      if constexpr (stage_loads_linear<V, N, s>()) {
        const V* xj = x + pidx<V>(j);
#pragma unroll
        for (int r = 0; r < R; ++r) v[p][r] = xj[pidx<V>(r * B)];
      } else {
#pragma unroll
        for (int r = 0; r < R; ++r) v[p][r] = x[pidx<V>(j + r * B)];
      }
      if (NS > 1) {
        const int jm = j % NS;
        const V* t = tws + StageInfo<N, s>::TWOFF + jm * (R - 1) - 1;
#pragma unroll
        for (int r = 1; r < R; ++r) {
          const V w = t[r];
          v[p][r] = SIGN < 0 ? cmul(v[p][r], w) : cmulc(v[p][r], w);
        }
      }
      Dft<R, SIGN, V>::run(v[p]);
    }
  }
  stage_sync<N>();
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    const int j = g + p * G;
    if (active && ((B % G == 0) || j < B)) {
      const int jm = j % NS;
      const int base = (j - jm) * R + jm;
      if constexpr (stage_stores_linear<V, N, s>()) {
        V* xq = x + pidx<V>(base);
#pragma unroll
        for (int r = 0; r < R; ++r) xq[pidx<V>(r * NS)] = cnorm(v[p][r]);
      } else {
#pragma unroll
        for (int r = 0; r < R; ++r) x[pidx<V>(base + r * NS)] = cnorm(v[p][r]);
      }
    }
  }
  stage_sync<N>();
}

// The same stage with NS and the twiddle offset known at run time only (NS a power of two):
// consecutive stages of equal radix share one copy of this code (see line_fft).
template <typename V, int N, int SIGN, int R>
__device__ __forceinline__ void fft_stage_rt(V* x, int g, const V* tws, bool active, int ns, int twoff) {
  constexpr int B = N / R;
  constexpr int G = FftPlan<N>::G;
  constexpr int PER = (B + G - 1) / G;
  V v[PER][R];
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    const int j = g + p * G;
    if (active && ((B % G == 0) || j < B)) {
#pragma unroll
      for (int r = 0; r < R; ++r) v[p][r] = x[pidx<V>(j + r * B)];
      if (ns > 1) {
        const V* t = tws + twoff + (j & (ns - 1)) * (R - 1) - 1;
#pragma unroll
        for (int r = 1; r < R; ++r) {
          const V w = t[r];
          v[p][r] = SIGN < 0 ? cmul(v[p][r], w) : cmulc(v[p][r], w);
        }
      }
      Dft<R, SIGN, V>::run(v[p]);
    }
  }
  stage_sync<N>();
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    const int j = g + p * G;
    if (active && ((B % G == 0) || j < B)) {
      const int jm = j & (ns - 1);
      const int base = (j - jm) * R + jm;
#pragma unroll
      for (int r = 0; r < R; ++r) x[pidx<V>(base + r * ns)] = cnorm(v[p][r]);
    }
  }
  stage_sync<N>();
}

// Transform the line at x (length N, padded layout) with G = FftPlan<N>::G threads
// (g = 0..G-1).  Every thread of the CTA must call this (it contains barriers); the caller
// syncs before, and the CTA is synchronised on return.  Threads with active = false only take part in the barriers.  In double-word
// arithmetic (dw2 elements) leading stages of equal radix run as a loop over one copy of the
// stage code: those butterflies are long, and unrolled copies of them overflow the
// instruction cache.  The FP32 and FP64 forms keep every stage unrolled (their code is short,
// and compile-time strides schedule better).
template <typename V, int N, int SIGN>
__device__ __forceinline__ void line_fft(V* x, int g, const V* tws, bool active = true) {
  constexpr int S = FftPlan<N>::S, R0 = FftPlan<N>::R0, R1 = FftPlan<N>::R1, R2 = FftPlan<N>::R2;
  constexpr bool share = is_dw<decltype(V::x)>();
  constexpr int RUN = (share && S >= 2 && R1 == R0) ? ((S == 3 && R2 == R0) ? 3 : 2) : 1;
  if constexpr (RUN > 1) {
#pragma unroll 1
    for (int st = 0; st < RUN; ++st) {
      const int ns = st == 0 ? 1 : (st == 1 ? R0 : R0 * R0);
      const int twoff = st <= 1 ? 0 : R0 * (R0 - 1);
      fft_stage_rt<V, N, SIGN, R0>(x, g, tws, active, ns, twoff);
    }
  } else {
    fft_stage<V, N, SIGN, 0>(x, g, tws, active);
  }
  if constexpr (S > 1 && RUN < 2) fft_stage<V, N, SIGN, 1>(x, g, tws, active);
  if constexpr (S > 2 && RUN < 3) fft_stage<V, N, SIGN, 2>(x, g, tws, active);
  if constexpr (warp_local<N>()) __syncthreads();
}

}  // namespace dns
