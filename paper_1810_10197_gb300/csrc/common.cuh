// Shared device-side definitions: complex helpers, grid geometry, the controller record.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace dns {

// the FP64/FP32 fma overloads stay visible next to the double-word one declared below
using ::fma;

// ---- double-word numbers ("float-float"): x = hi + lo, two FP32 values -------------------
// On this part FP32 instructions issue at 64 times the FP64 rate.  A number held as an
// unevaluated sum of two FP32 values has about 48 significant bits, and its arithmetic costs
// a handful of FP32 instructions per operation, so transforms in this form run several times
// faster than in FP64 at a rounding error near 2^-47 per operation (FP64: 2^-53).
// Building blocks, written from their published definitions:
//   TwoSum (Knuth, TAOCP vol. 2): s + e = a + b exactly, no condition on a, b;
//   Fast2Sum (Dekker 1971): the same in 3 operations when |a| >= |b| (or a = 0);
//   TwoProd with FMA: p + e = a b exactly (e = fma(a, b, -p)).
// The sum adds the high parts exactly and the low parts once (normwise error <= 2u^2 (|x|+|y|),
// u = 2^-24); the product keeps the three leading partial products (relative error <= 4u^2)
// -- the double-word algorithms analysed by Joldes, Muller and Popescu (ACM TOMS 44, 2017).
// Every step uses the _rn intrinsics, which the compiler neither contracts into FMAs nor
// reorders.  The exponent range is FP32's: values below about 1e-30 keep fewer bits, which is
// harmless here because errors are measured against the norm of each field.
struct __align__(8) dw {
  float hi, lo;
  dw() = default;
  __host__ __device__ constexpr dw(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ constexpr dw(int i) : hi((float)i), lo(0.0f) {}
  // exact split of an FP64 value to 48 bits (compile-time constants fold; a run-time value
  // costs one FP64 subtraction -- the hot conversions use from_f64<dw>)
  __host__ __device__ constexpr dw(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
};
struct __align__(16) dw2 { dw x, y; };

__device__ __forceinline__ dw two_sum(float a, float b) {
  const float s = __fadd_rn(a, b), bb = __fsub_rn(s, a);
  return dw(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb)));
}
__device__ __forceinline__ dw fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return dw(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ dw operator+(dw x, dw y) {
  const dw s = two_sum(x.hi, y.hi);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}
__device__ __forceinline__ dw operator-(dw x) { return dw(-x.hi, -x.lo); }
__device__ __forceinline__ dw operator-(dw x, dw y) { return x + (-y); }
__device__ __forceinline__ dw operator*(dw x, dw y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  return fast_two_sum(p, e);
}
// x y + z with one normalisation
__device__ __forceinline__ dw fma(dw x, dw y, dw z) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  const dw s = two_sum(p, z.hi);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(e, z.lo)));
}
// a b + c d (the parts of a complex product) with one normalisation
__device__ __forceinline__ dw dot2(dw a, dw b, dw c, dw d) {
  const float p = __fmul_rn(a.hi, b.hi), q = __fmul_rn(c.hi, d.hi);
  float ep = __fmaf_rn(a.hi, b.hi, -p);
  ep = __fmaf_rn(a.hi, b.lo, ep);
  ep = __fmaf_rn(a.lo, b.hi, ep);
  float eq = __fmaf_rn(c.hi, d.hi, -q);
  eq = __fmaf_rn(c.hi, d.lo, eq);
  eq = __fmaf_rn(c.lo, d.hi, eq);
  const dw s = two_sum(p, q);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(ep, eq)));
}
// 1 / y: the FP32 reciprocal refined by one Newton step in double-word arithmetic
__device__ __forceinline__ dw recip(dw y) {
  const float r = __frcp_rn(y.hi);
  float e = __fmaf_rn(-y.hi, r, 1.0f);
  e = __fmaf_rn(-y.lo, r, e);
  return fast_two_sum(r, __fmul_rn(r, e));
}
__device__ __forceinline__ dw operator/(dw x, dw y) { return x * recip(y); }
__device__ __forceinline__ bool operator==(dw x, dw y) { return x.hi == y.hi && x.lo == y.lo; }
__device__ __forceinline__ bool operator!=(dw x, dw y) { return !(x == y); }
__device__ __forceinline__ bool operator>(dw x, dw y) { return x.hi > y.hi || (x.hi == y.hi && x.lo > y.lo); }
__device__ __forceinline__ bool operator<=(dw x, dw y) { return !(x > y); }

template <typename T> __host__ __device__ constexpr bool is_dw() { return false; }
template <> __host__ __device__ constexpr bool is_dw<dw>() { return true; }

template <typename T> struct V2;
template <> struct V2<double> { using type = double2; };
template <> struct V2<float> { using type = float2; };
template <> struct V2<dw> { using type = dw2; };
template <typename T> using v2_t = typename V2<T>::type;

template <typename V> __device__ __forceinline__ V mk(decltype(V::x) a, decltype(V::x) b) {
  V r; r.x = a; r.y = b; return r;
}
template <typename V> __device__ __forceinline__ V cadd(V a, V b) { return mk<V>(a.x + b.x, a.y + b.y); }
template <typename V> __device__ __forceinline__ V csub(V a, V b) { return mk<V>(a.x - b.x, a.y - b.y); }
// a * b
template <typename V> __device__ __forceinline__ V cmul(V a, V b) {
  return mk<V>(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// a * conj(b)
template <typename V> __device__ __forceinline__ V cmulc(V a, V b) {
  return mk<V>(fma(a.x, b.x, a.y * b.y), fma(a.y, b.x, -a.x * b.y));
}
// s * i * a for s = +1 / -1
template <int S, typename V> __device__ __forceinline__ V mul_si(V a) {
  return S > 0 ? mk<V>(-a.y, a.x) : mk<V>(a.y, -a.x);
}
template <typename V> __device__ __forceinline__ V cscale(V a, decltype(V::x) s) { return mk<V>(a.x * s, a.y * s); }
template <typename V> __device__ __forceinline__ V cconj(V a) { return mk<V>(a.x, -a.y); }
// FP32 complex arithmetic as paired instructions (FADD2 / FMUL2 / FFMA2, sm_100 and later):
// one instruction for both components, each rounded exactly like its scalar _rn counterpart.
template <> __device__ __forceinline__ float2 cadd<float2>(float2 a, float2 b) { return __fadd2_rn(a, b); }
template <> __device__ __forceinline__ float2 csub<float2>(float2 a, float2 b) {
  return __fadd2_rn(a, make_float2(-b.x, -b.y));
}
template <> __device__ __forceinline__ float2 cmul<float2>(float2 a, float2 b) {
  const float2 t = __fmul2_rn(make_float2(a.y, a.y), make_float2(b.y, b.x));   // (ay by, ay bx)
  return __ffma2_rn(make_float2(a.x, a.x), b, make_float2(-t.x, t.y));
}
template <> __device__ __forceinline__ float2 cmulc<float2>(float2 a, float2 b) {
  const float2 t = __fmul2_rn(make_float2(a.y, a.y), make_float2(b.y, b.x));   // (ay by, ay bx)
  return __ffma2_rn(make_float2(a.x, a.x), make_float2(b.x, -b.y), make_float2(t.x, t.y));
}

// Complex sums of double-word values inside the transforms: the exact TwoSum of the high parts
// and one rounded sum of the low parts, without renormalising (8 FP32 instructions instead of
// 11).  A butterfly chains a few of these, so |lo| may grow to a few ulp of hi; the normwise
// error stays O(u^2), products take un-normalised operands as they are, and cnorm
// renormalises (Fast2Sum) when a stage stores its results.
__device__ __forceinline__ dw add_u(dw x, dw y) {
  const dw s = two_sum(x.hi, y.hi);
  return dw(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}
// product without the final renormalisation (4 FP32 instructions instead of 7)
__device__ __forceinline__ dw mul_u(dw x, dw y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, e);
  return dw(p, __fmaf_rn(x.lo, y.hi, e));
}
// a b + c d without the final renormalisation
__device__ __forceinline__ dw dot2_u(dw a, dw b, dw c, dw d) {
  const float p = __fmul_rn(a.hi, b.hi), q = __fmul_rn(c.hi, d.hi);
  float ep = __fmaf_rn(a.hi, b.hi, -p);
  ep = __fmaf_rn(a.hi, b.lo, ep);
  ep = __fmaf_rn(a.lo, b.hi, ep);
  float eq = __fmaf_rn(c.hi, d.hi, -q);
  eq = __fmaf_rn(c.hi, d.lo, eq);
  eq = __fmaf_rn(c.lo, d.hi, eq);
  const dw s = two_sum(p, q);
  return dw(s.hi, __fadd_rn(s.lo, __fadd_rn(ep, eq)));
}
// Butterfly-internal arithmetic: plain for FP32/FP64, un-normalised for double-word.
template <typename T> __device__ __forceinline__ T badd(T a, T b) { return a + b; }
template <typename T> __device__ __forceinline__ T bsub(T a, T b) { return a - b; }
template <typename T> __device__ __forceinline__ T bmul(T a, T b) { return a * b; }
// a b + c d, and x / 2 (exact in every form)
template <typename T> __device__ __forceinline__ T bdot2(T a, T b, T c, T d) { return fma(a, b, c * d); }
template <typename T> __device__ __forceinline__ T bhalf(T x) { return x * (T)0.5; }
template <> __device__ __forceinline__ dw bdot2<dw>(dw a, dw b, dw c, dw d) { return dot2_u(a, b, c, d); }
template <> __device__ __forceinline__ dw bhalf<dw>(dw x) { return dw(__fmul_rn(x.hi, 0.5f), __fmul_rn(x.lo, 0.5f)); }
template <> __device__ __forceinline__ dw badd<dw>(dw a, dw b) { return add_u(a, b); }
template <> __device__ __forceinline__ dw bsub<dw>(dw a, dw b) { return add_u(a, -b); }
template <> __device__ __forceinline__ dw bmul<dw>(dw a, dw b) { return mul_u(a, b); }
template <> __device__ __forceinline__ dw2 cadd<dw2>(dw2 a, dw2 b) { return mk<dw2>(add_u(a.x, b.x), add_u(a.y, b.y)); }
template <> __device__ __forceinline__ dw2 csub<dw2>(dw2 a, dw2 b) { return mk<dw2>(add_u(a.x, -b.x), add_u(a.y, -b.y)); }
// (Paired FADD2 forms of these sums cut the instruction count by a fifth but not the time: the
// pairs cost register moves, and one paired chain has half the independent work of two
// scalar chains, which these kernels need to hide latency.)
template <typename V> __device__ __forceinline__ V cnorm(V a) { return a; }
template <> __device__ __forceinline__ dw2 cnorm<dw2>(dw2 a) {
  return mk<dw2>(fast_two_sum(a.x.hi, a.x.lo), fast_two_sum(a.y.hi, a.y.lo));
}
// double-word complex products: each part is one a b + c d, left un-normalised (what follows
// is a butterfly sum or an explicit renormalisation)
template <> __device__ __forceinline__ dw2 cmul<dw2>(dw2 a, dw2 b) {
  return mk<dw2>(dot2_u(a.x, b.x, -a.y, b.y), dot2_u(a.x, b.y, a.y, b.x));
}
template <> __device__ __forceinline__ dw2 cmulc<dw2>(dw2 a, dw2 b) {
  return mk<dw2>(dot2_u(a.x, b.x, a.y, b.y), dot2_u(a.y, b.x, -a.x, b.y));
}

// Conversions between FP64 and FP32 with integer bit arithmetic.  On this part FP64<->FP32
// conversion instructions issue on the FP64 pipe (1/64 of the FP32 rate); the mixed-precision
// passes convert every mode, so they use these instead.
//   d2f_bits: significand rounded to 24 bits (nearest, ties away from zero), exponent
//             rebiased from 1023 to 127; magnitudes that round below 2^-126 give a signed
//             zero, above the largest float an infinity; NaN stays NaN.  Branch-free.
//   f2d_bits: exact; FP32 subnormals flush to signed zero; inf/NaN preserved.
__device__ __forceinline__ float d2f_bits(double x) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const unsigned s = (unsigned)(bits >> 32) & 0x80000000u;
  const unsigned long long mag = bits & 0x7FFFFFFFFFFFFFFFull;
  const unsigned long long r = mag + (1ull << 28);                  // + half a float ulp
  const unsigned rhi = (unsigned)(r >> 32), rlo = (unsigned)r;
  const unsigned e = rhi >> 20;                                      // exponent after rounding
  // bits 31..23 of (r >> 29) hold e mod 512; subtracting 896 << 23 modulo 2^32 leaves e - 896
  // in the float's exponent field for 897 <= e <= 1150, the normal float range
  unsigned b = __funnelshift_r(rlo, rhi, 29) - (896u << 23);
  b = e < 897u ? 0u : b;
  b = e > 1150u ? 0x7F800000u : b;
  b = mag > 0x7FF0000000000000ull ? 0x7FC00000u : b;
  return __uint_as_float(s | b);
}
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned s = b & 0x80000000u, e = (b >> 23) & 0xffu, m = b & 0x7fffffu;
  if (e == 0u) return __hiloint2double((int)s, 0);
  const unsigned eh = (e == 0xffu) ? 0x7ffu : e + 896u;
  return __hiloint2double((int)(s | (eh << 20) | (m >> 3)), (int)(m << 29));
}
template <typename T> __device__ __forceinline__ T from_f64(double x);
template <> __device__ __forceinline__ double from_f64<double>(double x) { return x; }
template <> __device__ __forceinline__ float from_f64<float>(double x) { return d2f_bits(x); }
// x = hi + lo: hi rounded to FP32, lo the rounded remainder (x - hi is exact in FP64)
template <> __device__ __forceinline__ dw from_f64<dw>(double x) {
  const float h = d2f_bits(x);
  return dw(h, d2f_bits(x - f2d_bits(h)));
}
__device__ __forceinline__ double to_f64(double x) { return x; }
__device__ __forceinline__ double to_f64(float x) { return f2d_bits(x); }
__device__ __forceinline__ double to_f64(dw x) { return f2d_bits(x.hi) + f2d_bits(x.lo); }

// Grid geometry shared by every kernel.  Retained ("compact") spectral arrays are
// [3][Mx][My][Mz] with Mx = 2Kx+1 (kx = i for i <= Kx, i - Mx above), Mz = Kz+1.
struct Geom {
  int nx, ny, nz, nzh;
  int Kx, Ky, Kz;
  int Mx, My, Mz;
  int MyMz;
  long long M;          // Mx*My*Mz
  double sx, sy, sz;    // 2 pi / L per axis
  double inv_n3;        // 1 / (snx sny snz), the state grid's inverse-DFT normalisation
  double nmodes_half;   // snx sny (snz/2+1), divisor of the error norm
  int nc;               // state components: 3 (velocity) or 4 (velocity, density)
  int bouss;            // Boussinesq form (Section 3.2)
  // state grid (the caller's half-spectrum layout).  Equal to the transform grid nx, ny, nz
  // for the 2/3 rule; N with a transform grid of 3N/2 for the 3/2 padding rule.
  int snx, sny, snz, snzh;
  double fwd_scale;     // (snx sny snz) / (nx ny nz): forward transforms on the padded grid
};

__host__ __device__ __forceinline__ int signed_mode(int i, int K, int Mc) { return i <= K ? i : i - Mc; }

// Buffer slots resolved at the start of each attempt (ping-pong for first-same-as-last).
enum Slot : int {
  SLOT_U = 0,        // u_n
  SLOT_K1 = 1,       // k_1 .. k_8 at SLOT_K1 + (i-1)
  SLOT_Y = 9,        // scratch stage input
  SLOT_UNEW = 10,    // u_{n+1} (last stage input of an FSAL pair)
  SLOT_COUNT = 16
};

// Device-resident step controller state.  One writer (the controller kernel, one thread).
struct DnsCtrl {
  double2* slot[SLOT_COUNT];
  double2* uu[2];
  double2* kk[2];
  double2* kfix[9];     // fixed stage buffers k_2..k_7 (index = stage number)
  double t, t_end, h, h_try, err, rtol, atol;
  double errc[4];
  double forcing_coef;  // power / (2 E_f) of the current stage input
  int method;
  int parity;
  int skip;             // this attempt does nothing (finished or failed)
  int need_k1;          // k_1 must be evaluated in this attempt
  int k1_valid;
  int done;
  int status;
  int clipped;
  int after_reject;
  int accepted;
  int max_rejects;
  int f32_slots;        // k_1..k_8 and the stage-input scratch hold FP32 complex values
                        // (fp32 form, DNS_FP32); u_n and u_{n+1} are FP64 in every form
  long long n_rhs, n_acc, n_rej, n_attempts, rejects_in_row;
  // controller variant: 0 = Section 2.2.1, 1 = PI, 2 = learned proposal (MLP)
  int ctrl_kind;
  int hist_n;           // accepted steps in the history (<= 5), newest first
  int rej_since;        // rejections since the last accepted step
  int trace_diag;       // trace E, Omega, eps after every attempt
  double err_prev;      // err of the last accepted step (PI)
  double hist_err[5], hist_h[5];
  int hist_rej[5];
  int pad2_;
  const float* mlp;     // network parameters of the learned proposal
  double* trace;        // [trace_cap][kTraceCols] attempt records
  long long trace_cap, trace_n;
  long long inject_rhs;   // debug: the right-hand side with this running index returns NaN (-1: none)
};

// attempt record: t at the start, h used, err, accepted, n_rhs so far, E, Omega, eps
constexpr int kTraceCols = 8;

__device__ __forceinline__ const double2* resolve_in(const double2* p, const DnsCtrl* c, int slot) {
  return (c && slot >= 0) ? c->slot[slot] : p;
}
__device__ __forceinline__ double2* resolve_out(double2* p, const DnsCtrl* c, int slot) {
  return (c && slot >= 0) ? c->slot[slot] : p;
}
// whether a pass output (a k slot) resolved through a controller slot is stored as FP32 complex
__device__ __forceinline__ bool out_is_f32(const DnsCtrl* c, int slot) {
  return c && slot >= 0 && c->f32_slots != 0;
}
// whether a pass input resolved through a controller slot is the FP32 stage-input scratch
__device__ __forceinline__ bool in_is_f32(const DnsCtrl* c, int slot) {
  return c && slot == SLOT_Y && c->f32_slots != 0;
}
// a stage-input value as FP32: read from the FP32 scratch, or rounded from FP64 (d2f_bits)
__device__ __forceinline__ float2 y_as_f32(const double2* Y, size_t i, bool y32) {
  if (y32) return reinterpret_cast<const float2*>(Y)[i];
  const double2 d = Y[i];
  return make_float2(d2f_bits(d.x), d2f_bits(d.y));
}
// gate: skip flags a launch may check (the k_1 evaluation runs only when needed)
__device__ __forceinline__ bool gated_off(const DnsCtrl* c, int only_if_need_k1) {
  if (!c) return false;
  if (c->skip) return true;
  return only_if_need_k1 && !c->need_k1;
}

enum DnsStatusDev : int { ST_OK = 0, ST_NONFINITE = 4, ST_UNDERFLOW = 5, ST_MAX_REJECTS = 6, ST_TIMEOUT = 7 };

}  // namespace dns
