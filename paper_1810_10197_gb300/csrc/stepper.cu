// Runge-Kutta stage sums, embedded error norm and the device step controller (Section 2.2 of
// arXiv:1810.10197), plus the copies between the half-spectrum layout and the retained box.
#include "stepper.cuh"
#include "mlp.cuh"

namespace dns {

namespace {

inline int grid_for(long long n, int threads, int cap) {
  long long b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  return (int)(b < cap ? b : cap);
}

// Y = u + h * sum_j coef_j k_j, terms added in ascending j (fused multiply-adds: on this part
// the FP64 pipe, not HBM, bounds the FP64 version, so the instruction count matters).
// F32 (the fp32 form, DNS_FP32, whose k_j carry FP32 accuracy and are stored as FP32 complex
// values): the increment sum_j (h coef_j) k_j is formed in FP32 and added to u in FP64; its
// rounding (~6e-8 of the increment) lies below the error the k_j already carry, and the
// kernel is HBM-bound (the FP64 pipe issues at 1/64 of the FP32 rate).
template <int NT, bool F32>
__global__ void k_stage_sum(const StageArgs a) {
  const DnsCtrl* c = a.ctrl;
  if (gated_off(c, a.gate_k1)) return;
  const double h = c->h_try;
  const double2* __restrict__ u = c->slot[a.uslot];
  double2* __restrict__ y = c->slot[a.yslot];
  const double2* k[NT];
#pragma unroll
  for (int j = 0; j < NT; ++j) k[j] = c->slot[a.kslot[j]];
  const long long stride = (long long)gridDim.x * blockDim.x;
  if constexpr (F32) {
    // an intermediate stage input goes to the FP32 scratch (the x passes read it as FP32);
    // u_{n+1} stays FP64
    const bool y32 = a.yslot == SLOT_Y && c->f32_slots;
    const float2* k32[NT];
#pragma unroll
    for (int j = 0; j < NT; ++j) k32[j] = reinterpret_cast<const float2*>(k[j]);
    float hc[NT];
#pragma unroll
    for (int j = 0; j < NT; ++j) hc[j] = (float)(h * a.coef[j]);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < a.n2; i += stride) {
      float2 kv = k32[0][i];
      float ar = hc[0] * kv.x, ai = hc[0] * kv.y;
#pragma unroll
      for (int j = 1; j < NT; ++j) {
        kv = k32[j][i];
        ar = fmaf(hc[j], kv.x, ar);
        ai = fmaf(hc[j], kv.y, ai);
      }
      const double2 uv = u[i];
      if (y32) reinterpret_cast<float2*>(y)[i] = make_float2(d2f_bits(uv.x) + ar, d2f_bits(uv.y) + ai);
      else y[i] = make_double2(uv.x + (double)ar, uv.y + (double)ai);
    }
  } else {
    // the terms (h a_ij) k_j accumulate onto u by fused multiply-adds: NT FP64 instructions a
    // real value (the FP64 pipe bounds this kernel); rounding at most NT/2 units in the last
    // place of u
    double hc[NT];
#pragma unroll
    for (int j = 0; j < NT; ++j) hc[j] = h * a.coef[j];
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < a.n2; i += stride) {
      const double2 uv = u[i];
      double ar = uv.x, ai = uv.y;
#pragma unroll
      for (int j = 0; j < NT; ++j) {
        const double2 kv = k[j][i];
        ar = fma(hc[j], kv.x, ar);
        ai = fma(hc[j], kv.y, ai);
      }
      y[i] = make_double2(ar, ai);
    }
  }
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Deterministic block sum of NV values (fixed tree), result valid in thread 0.
template <int NV>
__device__ __forceinline__ void block_sum(double v[NV], double* sh /* NV*32 */) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int q = 0; q < NV; ++q) v[q] = warp_sum(v[q]);
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) sh[q * 32 + w] = v[q];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      double s = 0.0;
      for (int i = 0; i < nw; ++i) s += sh[q * 32 + i];
      v[q] = s;
    }
  }
}
__device__ __forceinline__ void block_sum3(double v[3], double* sh) { block_sum<3>(v, sh); }

// FP64 square root and reciprocal for the error norm: an FP32 seed (the approximate
// reciprocal square root / reciprocal instructions) refined by one Newton-Raphson step in
// FP64, y <- y (3 - x y^2) / 2 and r <- r + r (1 - x r), which squares the seed's relative
// error (~2^-22 -> ~1e-13).  The norm needs FP64 accuracy, not correct rounding, and the
// FP64 pipe issues at 1/64 of the FP32 rate.  Arguments outside [2^-120, 2^120] (and zero)
// take the library operations.
__device__ __forceinline__ bool in_seed_range(double x) {
  const unsigned e = ((unsigned)__double2hiint(x) >> 20) & 0x7FFu;   // x >= 0 here
  return e > 903u && e < 1143u;
}
__device__ __forceinline__ float rsqrt_seed(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcp_seed(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ double sqrt_nr(double x) {
  if (!in_seed_range(x)) return sqrt(x);
  const double y0 = f2d_bits(rsqrt_seed(d2f_bits(x)));
  const double y1 = y0 * fma(-0.5 * x, y0 * y0, 1.5);
  return x * y1;
}
__device__ __forceinline__ double rcp_nr(double x) {
  if (!in_seed_range(x)) return 1.0 / x;
  const double r0 = f2d_bits(rcp_seed(d2f_bits(x)));
  return fma(r0, fma(-x, r0, 1.0), r0);
}

// Per-block partial sums of (|e| / sc)^2 per component, e = h sum_j (b_j - bhat_j) k_j,
// sc = atol + rtol max(|u_n|, |u_{n+1}|)  (Section 2.2.1).
// F32 (the fp32 form, DNS_FP32, k_j stored as FP32 complex values): e, sc, the ratio and each
// thread's sum of squares in FP32 (u_n, u_{n+1} converted by d2f_bits, integer
// instructions), the block and grid sums in FP64; the k_j carry FP32 accuracy, so err keeps
// all the accuracy they hold.  Nonzero
// tolerances outside [1e-30, 1e30] take FP64 arithmetic (the FP32 k_j widened exactly).
template <int NT, bool F32>
__global__ void __launch_bounds__(kRedThreads) k_err_partials(const ErrArgs a) {
  __shared__ double sh[4 * 32];
  const DnsCtrl* c = a.ctrl;
  if (c->skip) return;
  const double h = c->h_try, rtol = c->rtol, atol = c->atol;
  const double2* __restrict__ u0 = c->slot[SLOT_U];
  const double2* __restrict__ u1 = c->slot[SLOT_UNEW];
  const double2* k[NT];
#pragma unroll
  for (int j = 0; j < NT; ++j) k[j] = c->slot[a.kslot[j]];
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  const long long stride = (long long)gridDim.x * blockDim.x;
  const bool rt_ok = rtol == 0.0 || (rtol >= 1e-30 && rtol <= 1e30);
  const bool at_ok = atol == 0.0 || (atol >= 1e-30 && atol <= 1e30);
  if (F32 && rt_ok && at_ok) {
    const float2* k32[NT];
#pragma unroll
    for (int j = 0; j < NT; ++j) k32[j] = reinterpret_cast<const float2*>(k[j]);
    float hc[NT];
#pragma unroll
    for (int j = 0; j < NT; ++j) hc[j] = (float)(h * a.coef[j]);
    const float rt = (float)rtol, at = (float)atol;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (q >= a.nc) break;
      // a thread's terms (M / (blocks x threads), about 8 at 256^3) are summed in FP32 and
      // added to the FP64 partial once: no FP64 instruction per mode
      float accf = 0.f;
      for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < a.M; i += stride) {
        const long long idx = q * a.M + i;
        float2 kv = k32[0][idx];
        float er = hc[0] * kv.x, ei = hc[0] * kv.y;
#pragma unroll
        for (int j = 1; j < NT; ++j) {
          kv = k32[j][idx];
          er = fmaf(hc[j], kv.x, er);
          ei = fmaf(hc[j], kv.y, ei);
        }
        const double2 a0 = u0[idx], a1 = u1[idx];
        const float x0 = d2f_bits(a0.x), y0 = d2f_bits(a0.y);
        const float x1 = d2f_bits(a1.x), y1 = d2f_bits(a1.y);
        const float m2 = fmaxf(fmaf(x0, x0, y0 * y0), fmaf(x1, x1, y1 * y1));
        const float inv = 1.0f / fmaf(rt, sqrtf(m2), at);
        const float tr = er * inv, ti = ei * inv;
        // a zero error adds nothing, also where sc = 0 (atol = 0 on a mode that is zero in
        // both solutions: 0 * inf would be NaN)
        if (er != 0.f || ei != 0.f) accf = fmaf(tr, tr, fmaf(ti, ti, accf));
      }
      acc[q] = f2d_bits(accf);
    }
  } else {
  double hc[NT];                        // h (b_j - bhat_j)
#pragma unroll
  for (int j = 0; j < NT; ++j) hc[j] = h * a.coef[j];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if (q >= a.nc) break;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < a.M; i += stride) {
      const long long idx = q * a.M + i;
      // F32 here: FP32 k slots, widened exactly (tolerances outside the FP32 range)
      const auto kval = [&](int j) {
        if (F32) {
          const float2 v = reinterpret_cast<const float2*>(k[j])[idx];
          return make_double2(f2d_bits(v.x), f2d_bits(v.y));
        }
        return k[j][idx];
      };
      double2 kv = kval(0);
      double er = hc[0] * kv.x, ei = hc[0] * kv.y;
#pragma unroll
      for (int j = 1; j < NT; ++j) {
        kv = kval(j);
        er = fma(hc[j], kv.x, er);
        ei = fma(hc[j], kv.y, ei);
      }
      const double2 a0 = u0[idx], a1 = u1[idx];
      const double m2 = fmax(fma(a0.x, a0.x, a0.y * a0.y), fma(a1.x, a1.x, a1.y * a1.y));
      const double sc = fma(rtol, sqrt_nr(m2), atol);
      const double e2 = fma(er, er, ei * ei);
      // a zero error adds nothing, also where sc = 0 (see the FP32 arm above)
      if (e2 != 0.0) acc[q] = fma(e2, rcp_nr(sc * sc), acc[q]);
    }
  }
  }
  block_sum<4>(acc, sh);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < 4; ++q) a.partials[blockIdx.x * kRedStride + q] = acc[q];
  }
}

__device__ __forceinline__ bool adaptive_method(int m) { return m == 2 || m == 4; }
__device__ __forceinline__ int method_stages(int m) { return m == 0 ? 4 : (m >= 3 ? 7 : 8); }

__global__ void k_begin_attempt(DnsCtrl* c, int method) {
  if (c->done || c->status != 0) { c->skip = 1; return; }
  const double rem = c->t_end - c->t;
  if (!(rem > 0.0)) { c->done = 1; c->skip = 1; return; }
  const double h = c->h;
  // the last step lands exactly on t_end, also when h falls short of it by rounding only
  c->clipped = h >= rem * (1.0 - 1e-10);
  c->h_try = c->clipped ? rem : h;
  if (!(c->h_try >= 1e-12 * fmax(1.0, fabs(c->t)))) {
    c->status = ST_UNDERFLOW; c->done = 1; c->skip = 1; return;
  }
  c->skip = 0;
  const int p = c->parity;
  c->slot[SLOT_U] = c->uu[p];
  c->slot[SLOT_UNEW] = c->uu[1 - p];
  c->slot[SLOT_K1] = c->kk[p];
  for (int i = 2; i <= 7; ++i) c->slot[SLOT_K1 + i - 1] = c->kfix[i];
  if (method != 0) c->slot[SLOT_K1 + method_stages(method) - 1] = c->kk[1 - p];   // last k of an FSAL pair
  c->need_k1 = (method == 0) ? 1 : !c->k1_valid;
}

// Section 2.2.1: err = max_j sqrt(S_j / (nx ny (nz/2+1))); accept iff err <= 1;
// h_new = h min(dmax, max(dmin, 0.8 err^(-1/5))), dmax = 1 right after a rejection.
// Variants after an accepted step: PI (0.8 err^(-0.7/5) err_prev^(0.4/5)) or the learned
// correction of it, PI exp(clamp(mlp(features), +-log 1.5)), once 4 accepted steps are
// known (before that, and when the network's output is not finite, the PI factor); a
// rejected attempt takes the Section 2.2.1 factor.
__global__ void __launch_bounds__(kRedThreads) k_controller(DnsCtrl* c, const double* partials,
                                                            int method, int nstages, int nblk,
                                                            double nmodes, int nc) {
  __shared__ double sh[4][kRedThreads];
  __shared__ float feat[kMlpIn];
  __shared__ float work[2 * kMlpH];
  __shared__ int use_mlp;
  __shared__ double s_err, s_fac;
  __shared__ int s_accept;
  if (c->skip) return;
  const int tid = threadIdx.x;
  double s[4] = {0.0, 0.0, 0.0, 0.0};
  if (method != 0) {
    for (int b = tid; b < nblk; b += blockDim.x) {
#pragma unroll
      for (int q = 0; q < 4; ++q) s[q] += partials[b * kRedStride + q];
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) sh[q][tid] = s[q];
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (tid < w) {
#pragma unroll
      for (int q = 0; q < 4; ++q) sh[q][tid] += sh[q][tid + w];
    }
    __syncthreads();
  }
  if (tid == 0) {
    c->n_attempts += 1;
    c->n_rhs += (nstages - 1) + c->need_k1;
    double err = 0.0;
    bool nan = false;
    if (method != 0) {
      for (int q = 0; q < nc; ++q) {
        const double e = sqrt(sh[q][0] / nmodes);
        c->errc[q] = e;
        if (e != e) nan = true;
        err = e > err ? e : err;
      }
      if (nan) err = __longlong_as_double(0x7ff8000000000000ULL);
      c->k1_valid = 1;
    }
    bool accept = true;
    double fac = 1.0;
    int mlp_now = 0;
    if (adaptive_method(method)) {
      const bool fin = isfinite(err);
      accept = fin && err <= 1.0;
      const double dmax = c->after_reject ? 1.0 : 2.0;
      if (!fin) fac = 0.01;
      else if (err == 0.0) fac = dmax;
      else fac = fmin(dmax, fmax(0.01, 0.8 * pow(err, -1.0 / 5.0)));
      if (accept && (c->ctrl_kind == 1 || (c->ctrl_kind == 2 && c->mlp)) && err > 0.0)
        fac = fmin(dmax, fmax(0.01, 0.8 * pow(err, -(0.7 / 5.0)) * pow(c->err_prev, 0.4 / 5.0)));
      if (accept && c->ctrl_kind == 2 && c->mlp) {
        for (int i = 4; i > 0; --i) {
          c->hist_err[i] = c->hist_err[i - 1]; c->hist_h[i] = c->hist_h[i - 1]; c->hist_rej[i] = c->hist_rej[i - 1];
        }
        c->hist_err[0] = err; c->hist_h[0] = c->h_try; c->hist_rej[0] = c->rej_since;
        c->hist_n = min(c->hist_n + 1, 5);
        if (c->hist_n >= 4) {
          const double h0 = c->hist_h[0];
          for (int i = 0; i < 4; ++i) {
            const double hp = (i + 1 < c->hist_n) ? c->hist_h[i + 1] : c->hist_h[i];
            feat[4 * i + 0] = (float)log10(fmax(c->hist_err[i], 1e-300));
            feat[4 * i + 1] = (float)log(c->hist_h[i] / h0);
            feat[4 * i + 2] = (float)c->hist_rej[i];
            feat[4 * i + 3] = (float)log(c->hist_h[i] / hp);
          }
          mlp_now = 1;
        }
      }
    }
    s_err = err;
    s_fac = fac;
    s_accept = accept ? 1 : 0;
    use_mlp = mlp_now;
  }
  __syncthreads();
  float y = 0.f;
  if (use_mlp) y = mlp_forward_block(c->mlp, feat, work);
  if (tid != 0) return;
  const double err = s_err;
  const bool accept = s_accept != 0;
  double fac = s_fac;
  if (use_mlp && isfinite(y) && err > 0.0) {
    // learned correction of the PI factor, bounded by 1.5x either way
    const double corr = fmin(log(1.5), fmax(-log(1.5), (double)y));
    const double lpi = log(0.8) - (0.7 / 5.0) * log(err) + (0.4 / 5.0) * log(c->err_prev);
    const double lf = fmin(log(2.0), fmax(log(0.01), lpi + corr));
    fac = exp(lf);
    if (c->after_reject) fac = fmin(1.0, fac);
  }
  const double t_before = c->t;
  c->err = err;
  double h_new = c->h;
  if (adaptive_method(method)) h_new = c->h_try * fac;
  if (accept) {
    c->t = c->clipped ? c->t_end : c->t + c->h_try;
    c->parity ^= 1;
    c->after_reject = 0;
    c->rejects_in_row = 0;
    c->rej_since = 0;
    if (err > 0.0) c->err_prev = err;
    c->n_acc += 1;
    if (method == 0) c->k1_valid = 0;
  } else {
    c->after_reject = 1;
    c->rejects_in_row += 1;
    c->rej_since += 1;
    c->n_rej += 1;
    if (c->rejects_in_row > c->max_rejects) {
      c->status = isfinite(err) ? ST_MAX_REJECTS : ST_NONFINITE;
      c->done = 1;
    }
  }
  c->accepted = accept ? 1 : 0;
  c->h = h_new;
  if (c->t >= c->t_end) c->done = 1;
  if (c->trace && c->trace_n < c->trace_cap) {
    double* r = c->trace + c->trace_n * kTraceCols;
    const double qnan = __longlong_as_double(0x7ff8000000000000ULL);
    r[0] = t_before; r[1] = c->h_try; r[2] = err; r[3] = accept ? 1.0 : 0.0; r[4] = (double)c->n_rhs;
    r[5] = qnan; r[6] = qnan; r[7] = qnan;
    c->trace_n += 1;
  }
}

// E, Omega and eps of the current state for the last trace record (eps from the carried-over
// derivative k_1 = f(u_n) of a first-same-as-last pair).
__global__ void __launch_bounds__(kRedThreads) k_trace_partials(const Geom g, const DnsCtrl* c,
                                                                double* partials) {
  __shared__ double sh[3 * 32];
  if (c->skip || !c->trace_diag || !c->trace) return;
  const double2* __restrict__ u = c->uu[c->parity];
  const double2* __restrict__ f = c->kk[c->parity];
  const float2* __restrict__ f32 = reinterpret_cast<const float2*>(f);   // FP32 k slots
  double v[3] = {0.0, 0.0, 0.0};
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < g.M; r += stride) {
    const int ix = (int)(r / g.MyMz), rem = (int)(r - (long long)ix * g.MyMz);
    const int jy = rem / g.Mz, kz = rem - jy * g.Mz;
    const double kx = g.sx * signed_mode(ix, g.Kx, g.Mx), ky = g.sy * signed_mode(jy, g.Ky, g.My);
    const double kzz = g.sz * kz;
    const double k2 = kx * kx + ky * ky + kzz * kzz;
    const double w = kz == 0 ? 1.0 : 2.0;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const double2 a = u[q * g.M + r];
      double2 b;
      if (c->f32_slots) {
        const float2 b32 = f32[q * g.M + r];
        b = make_double2(f2d_bits(b32.x), f2d_bits(b32.y));
      } else {
        b = f[q * g.M + r];
      }
      const double m2 = a.x * a.x + a.y * a.y;
      v[0] += w * m2;
      v[1] += w * k2 * m2;
      v[2] += w * (a.x * b.x + a.y * b.y);
    }
  }
  block_sum3(v, sh);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < 3; ++q) partials[blockIdx.x * kRedStride + q] = v[q];
  }
}

__global__ void __launch_bounds__(kRedThreads) k_trace_finish(const Geom g, DnsCtrl* c, const double* partials,
                                                              int nblk, int method) {
  __shared__ double sh[3][kRedThreads];
  if (c->skip || !c->trace_diag || !c->trace || c->trace_n == 0) return;
  const int tid = threadIdx.x;
  double s[3] = {0.0, 0.0, 0.0};
  for (int b = tid; b < nblk; b += blockDim.x) {
#pragma unroll
    for (int q = 0; q < 3; ++q) s[q] += partials[b * kRedStride + q];
  }
#pragma unroll
  for (int q = 0; q < 3; ++q) sh[q][tid] = s[q];
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (tid < w) {
#pragma unroll
      for (int q = 0; q < 3; ++q) sh[q][tid] += sh[q][tid + w];
    }
    __syncthreads();
  }
  if (tid == 0) {
    double* r = c->trace + (c->trace_n - 1) * kTraceCols;
    const double n6 = g.inv_n3 * g.inv_n3;
    r[5] = 0.5 * sh[0][0] * n6;
    r[6] = 0.5 * sh[1][0] * n6;
    r[7] = (method != 0 && c->k1_valid) ? -sh[2][0] * n6 : __longlong_as_double(0x7ff8000000000000ULL);
  }
}

__global__ void k_ctrl_set(DnsCtrl* c, int what, int kind, const float* mlp, double* trace,
                           long long cap, int diag) {
  if (what == 0) { c->ctrl_kind = kind; c->mlp = mlp; c->hist_n = 0; }
  else if (what == 1) { c->trace = trace; c->trace_cap = cap; c->trace_n = 0; c->trace_diag = diag; }
  else { c->inject_rhs = cap; }
}

__global__ void k_ctrl_reset(DnsCtrl* c, double t) {
  c->hist_n = 0; c->rej_since = 0; c->err_prev = 1.0; c->trace_n = 0;
  c->t = t; c->t_end = t; c->h = 0.0; c->h_try = 0.0; c->err = 0.0;
  c->errc[0] = c->errc[1] = c->errc[2] = c->errc[3] = 0.0;
  c->parity = 0; c->skip = 0; c->need_k1 = 1; c->k1_valid = 0; c->done = 1; c->status = 0;
  c->clipped = 0; c->after_reject = 0; c->accepted = 0;
  c->n_rhs = c->n_acc = c->n_rej = c->n_attempts = c->rejects_in_row = 0;
}

__global__ void k_ctrl_config(DnsCtrl* c, double t_end, int method, double rtol, double atol,
                              double h0, int max_rejects) {
  c->method = method;
  c->t_end = t_end; c->rtol = rtol; c->atol = atol;
  if (h0 > 0.0) { c->h = h0; c->after_reject = 0; }
  c->max_rejects = max_rejects;
  c->rejects_in_row = 0;
  c->done = (c->status != 0) || !(c->t < t_end);
}

__global__ void k_gather(const Geom g, const double2* __restrict__ full, double2* __restrict__ cmp) {
  const long long n = (long long)g.nc * g.M;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const long long q = i / g.M, r = i - q * g.M;
    const int ix = (int)(r / g.MyMz), rem = (int)(r - (long long)ix * g.MyMz);
    const int jy = rem / g.Mz, kz = rem - jy * g.Mz;
    const int fx = ix <= g.Kx ? ix : g.snx - g.Mx + ix;
    const int fy = jy <= g.Ky ? jy : g.sny - g.My + jy;
    cmp[i] = full[((q * g.snx + fx) * g.sny + fy) * (long long)g.snzh + kz];
  }
}

__global__ void k_scatter(const Geom g, const double2* __restrict__ cmp, double2* __restrict__ full) {
  const long long n = (long long)g.nc * g.M;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const long long q = i / g.M, r = i - q * g.M;
    const int ix = (int)(r / g.MyMz), rem = (int)(r - (long long)ix * g.MyMz);
    const int jy = rem / g.Mz, kz = rem - jy * g.Mz;
    const int fx = ix <= g.Kx ? ix : g.snx - g.Mx + ix;
    const int fy = jy <= g.Ky ? jy : g.sny - g.My + jy;
    full[((q * g.snx + fx) * g.sny + fy) * (long long)g.snzh + kz] = cmp[i];
  }
}

__global__ void k_copy_slot(const DnsCtrl* c, int slot, double2* __restrict__ dst, long long n) {
  const double2* __restrict__ src = c->slot[slot];
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) dst[i] = src[i];
}

// Constant-power forcing coefficient power / (2 E_f), E_f = sum_{0<|kappa|<=kf} w |Y|^2 / (2 N^6).
__global__ void __launch_bounds__(kRedThreads) k_forcing_coef(const Geom g, DnsCtrl* c, int yslot,
                                                              double kf, double power, int gate_k1) {
  __shared__ double sh[3 * 32];
  if (gated_off(c, gate_k1)) return;
  const double2* __restrict__ Y = c->slot[yslot];
  const bool y32 = in_is_f32(c, yslot);   // FP32 stage-input scratch (fp32 form)
  const int bx = min(g.Kx, (int)floor(kf / g.sx)), by = min(g.Ky, (int)floor(kf / g.sy));
  const int bz = min(g.Kz, (int)floor(kf / g.sz));
  const int nxb = 2 * bx + 1, nyb = 2 * by + 1, nzb = bz + 1;
  double v[3] = {0.0, 0.0, 0.0};
  const double kf2 = kf * kf;
  for (int i = threadIdx.x; i < nxb * nyb * nzb; i += blockDim.x) {
    const int mx = i / (nyb * nzb) - bx, r = i % (nyb * nzb), my = r / nzb - by, mz = r % nzb;
    const double kx = g.sx * mx, ky = g.sy * my, kz = g.sz * mz;
    const double k2 = kx * kx + ky * ky + kz * kz;
    if (!(k2 > 0.0 && k2 <= kf2)) continue;
    const int ix = mx >= 0 ? mx : mx + g.Mx, jy = my >= 0 ? my : my + g.My;
    const long long off = ((long long)ix * g.My + jy) * g.Mz + mz;
    const double w = mz == 0 ? 1.0 : 2.0;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      double2 y;
      if (y32) {
        const float2 y2 = reinterpret_cast<const float2*>(Y)[q * g.M + off];
        y = make_double2(f2d_bits(y2.x), f2d_bits(y2.y));
      } else {
        y = Y[q * g.M + off];
      }
      v[q] += w * (y.x * y.x + y.y * y.y);
    }
  }
  block_sum3(v, sh);
  if (threadIdx.x == 0) {
    const double ef = (v[0] + v[1] + v[2]) * g.inv_n3 * g.inv_n3 * 0.5;
    c->forcing_coef = ef > 0.0 ? power / (2.0 * ef) : 0.0;
  }
}

// Band rescale forcing (Section 3.3.1), first half: per-block sums of w |u_n|^2 and
// w |u_{n+1}|^2 over all retained modes, after an accepted step only.  w = 1 at kz = 0, else 2
// (kz is the fastest index of the retained box; the Nyquist plane is never retained).
__global__ void __launch_bounds__(kRedThreads) k_rescale_partials(const Geom g, const DnsCtrl* c,
                                                                  double* partials) {
  __shared__ double sh[2 * 32];
  if (c->skip || !c->accepted) return;
  const double2* __restrict__ u0 = c->uu[c->parity ^ 1];
  const double2* __restrict__ u1 = c->uu[c->parity];
  const long long n = (long long)g.nc * g.M;
  double v[2] = {0.0, 0.0};
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const double w = (i % g.Mz) == 0 ? 1.0 : 2.0;
    const double2 a = u0[i], b = u1[i];
    v[0] += w * fma(a.x, a.x, a.y * a.y);
    v[1] += w * fma(b.x, b.x, b.y * b.y);
  }
  block_sum<2>(v, sh);
  if (threadIdx.x == 0) {
    partials[blockIdx.x * kRedStride + 0] = v[0];
    partials[blockIdx.x * kRedStride + 1] = v[1];
  }
}

// Second half (one block): E_f = band energy of u_{n+1} on 0 < |kappa| <= kf; the band is
// multiplied by alpha = sqrt(1 + (E_n - E_{n+1}) / E_f), which returns the total energy to E_n.
// Without band energy, or with alpha^2 <= 0, the state is left as it is.  A rescaled state
// invalidates the carried-over derivative k_1 of a first-same-as-last pair.
__global__ void __launch_bounds__(kRedThreads) k_rescale_apply(const Geom g, DnsCtrl* c, const double* partials,
                                                               int nblk, double kf) {
  __shared__ double sh[2][kRedThreads];
  __shared__ double sb[3 * 32];
  __shared__ double s_alpha;
  if (c->skip || !c->accepted) return;
  const int tid = threadIdx.x;
  double s0 = 0.0, s1 = 0.0;
  for (int b = tid; b < nblk; b += blockDim.x) {
    s0 += partials[b * kRedStride + 0];
    s1 += partials[b * kRedStride + 1];
  }
  sh[0][tid] = s0;
  sh[1][tid] = s1;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (tid < w) { sh[0][tid] += sh[0][tid + w]; sh[1][tid] += sh[1][tid + w]; }
    __syncthreads();
  }
  double2* __restrict__ u = c->uu[c->parity];
  const int bx = min(g.Kx, (int)floor(kf / g.sx)), by = min(g.Ky, (int)floor(kf / g.sy));
  const int bz = min(g.Kz, (int)floor(kf / g.sz));
  const int nyb = 2 * by + 1, nzb = bz + 1, nbox = (2 * bx + 1) * nyb * nzb;
  const double kf2 = kf * kf;
  double v[3] = {0.0, 0.0, 0.0};
  for (int i = tid; i < nbox; i += blockDim.x) {
    const int mx = i / (nyb * nzb) - bx, r = i % (nyb * nzb), my = r / nzb - by, mz = r % nzb;
    const double kx = g.sx * mx, ky = g.sy * my, kz = g.sz * mz;
    const double k2 = kx * kx + ky * ky + kz * kz;
    if (!(k2 > 0.0 && k2 <= kf2)) continue;
    const int ix = mx >= 0 ? mx : mx + g.Mx, jy = my >= 0 ? my : my + g.My;
    const long long off = ((long long)ix * g.My + jy) * g.Mz + mz;
    const double w = mz == 0 ? 1.0 : 2.0;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const double2 y = u[q * g.M + off];
      v[q] += w * (y.x * y.x + y.y * y.y);
    }
  }
  block_sum3(v, sb);
  if (tid == 0) {
    const double ef = v[0] + v[1] + v[2];
    const double a2 = ef > 0.0 ? 1.0 + (sh[0][0] - sh[1][0]) / ef : 0.0;
    s_alpha = a2 > 0.0 ? sqrt(a2) : 1.0;
    if (a2 > 0.0) c->k1_valid = 0;
  }
  __syncthreads();
  const double alpha = s_alpha;
  if (alpha == 1.0) return;
  for (int i = tid; i < nbox; i += blockDim.x) {
    const int mx = i / (nyb * nzb) - bx, r = i % (nyb * nzb), my = r / nzb - by, mz = r % nzb;
    const double kx = g.sx * mx, ky = g.sy * my, kz = g.sz * mz;
    const double k2 = kx * kx + ky * ky + kz * kz;
    if (!(k2 > 0.0 && k2 <= kf2)) continue;
    const int ix = mx >= 0 ? mx : mx + g.Mx, jy = my >= 0 ? my : my + g.My;
    const long long off = ((long long)ix * g.My + jy) * g.Mz + mz;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      double2& y = u[q * g.M + off];
      y = make_double2(alpha * y.x, alpha * y.y);
    }
  }
}

// Partial sums for E, Omega, eps: sum w |u|^2, sum w |kappa|^2 |u|^2, sum w Re(conj(u).f).
__global__ void __launch_bounds__(kRedThreads) k_diag_partials(const Geom g, const double2* __restrict__ u,
                                                               const double2* __restrict__ f,
                                                               double* partials) {
  __shared__ double sh[3 * 32];
  double v[3] = {0.0, 0.0, 0.0};
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < g.M; r += stride) {
    const int ix = (int)(r / g.MyMz), rem = (int)(r - (long long)ix * g.MyMz);
    const int jy = rem / g.Mz, kz = rem - jy * g.Mz;
    const double kx = g.sx * signed_mode(ix, g.Kx, g.Mx), ky = g.sy * signed_mode(jy, g.Ky, g.My);
    const double kzz = g.sz * kz;
    const double k2 = kx * kx + ky * ky + kzz * kzz;
    const double w = kz == 0 ? 1.0 : 2.0;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const double2 a = u[q * g.M + r], b = f[q * g.M + r];
      const double m2 = a.x * a.x + a.y * a.y;
      v[0] += w * m2;
      v[1] += w * k2 * m2;
      v[2] += w * (a.x * b.x + a.y * b.y);
    }
  }
  block_sum3(v, sh);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < 3; ++q) partials[blockIdx.x * kRedStride + q] = v[q];
  }
}

// Energy spectrum: per-block shell histograms of w |u|^2 (velocity), then a fixed-order sum.
__global__ void __launch_bounds__(kRedThreads) k_spectrum_partials(const Geom g, const double2* __restrict__ u,
                                                                   double* partials, int nshell) {
  extern __shared__ double hist[];
  for (int i = threadIdx.x; i < nshell; i += blockDim.x) hist[i] = 0.0;
  __syncthreads();
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < g.M; r += stride) {
    const int ix = (int)(r / g.MyMz), rem = (int)(r - (long long)ix * g.MyMz);
    const int jy = rem / g.Mz, kz = rem - jy * g.Mz;
    const double kx = g.sx * signed_mode(ix, g.Kx, g.Mx), ky = g.sy * signed_mode(jy, g.Ky, g.My);
    const double kzz = g.sz * kz;
    const int sh = (int)rint(sqrt(kx * kx + ky * ky + kzz * kzz));
    const double w = kz == 0 ? 1.0 : 2.0;
    double m2 = 0.0;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const double2 a = u[q * g.M + r];
      m2 += a.x * a.x + a.y * a.y;
    }
    if (sh < nshell) atomicAdd(&hist[sh], w * m2);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nshell; i += blockDim.x) partials[(size_t)blockIdx.x * nshell + i] = hist[i];
}

__global__ void k_spectrum_finish(const double* partials, int nblk, int nshell, double scale, double* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nshell) return;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += partials[(size_t)b * nshell + i];
  out[i] = s * scale;
}

}  // namespace

constexpr int kSpecBlocks = 152;
cudaError_t launch_spectrum(const Geom& g, const double2* u, double* partials, int nshell, double* out,
                            cudaStream_t s) {
  const size_t smem = (size_t)nshell * sizeof(double);
  k_spectrum_partials<<<kSpecBlocks, kRedThreads, smem, s>>>(g, u, partials, nshell);
  k_spectrum_finish<<<(nshell + 127) / 128, 128, 0, s>>>(partials, kSpecBlocks, nshell,
                                                          0.5 * g.inv_n3 * g.inv_n3, out);
  return cudaGetLastError();
}

__global__ void f32_slots_from_f64(const double* __restrict__ x, float* __restrict__ y, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = d2f_bits(x[i]);
}

template <bool F32>
cudaError_t stage_sum_nt(const StageArgs& a, int blocks, cudaStream_t s) {
  switch (a.nterms) {
    case 1: k_stage_sum<1, F32><<<blocks, 256, 0, s>>>(a); break;
    case 2: k_stage_sum<2, F32><<<blocks, 256, 0, s>>>(a); break;
    case 3: k_stage_sum<3, F32><<<blocks, 256, 0, s>>>(a); break;
    case 4: k_stage_sum<4, F32><<<blocks, 256, 0, s>>>(a); break;
    case 5: k_stage_sum<5, F32><<<blocks, 256, 0, s>>>(a); break;
    case 6: k_stage_sum<6, F32><<<blocks, 256, 0, s>>>(a); break;
    case 7: k_stage_sum<7, F32><<<blocks, 256, 0, s>>>(a); break;
    case 8: k_stage_sum<8, F32><<<blocks, 256, 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <bool F32>
cudaError_t err_partials_nt(const ErrArgs& a, cudaStream_t s) {
  switch (a.nterms) {
    case 6: k_err_partials<6, F32><<<kRedBlocks, kRedThreads, 0, s>>>(a); break;
    case 7: k_err_partials<7, F32><<<kRedBlocks, kRedThreads, 0, s>>>(a); break;
    case 5: k_err_partials<5, F32><<<kRedBlocks, kRedThreads, 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_stage_sum(const StageArgs& a, cudaStream_t s) {
  const int blocks = grid_for(a.n2, 256, 152 * 16);
  return a.f32 ? stage_sum_nt<true>(a, blocks, s) : stage_sum_nt<false>(a, blocks, s);
}

cudaError_t launch_f32_from_f64(const double* x, float* y, long long n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  f32_slots_from_f64<<<grid_for(n, 256, 152 * 8), 256, 0, s>>>(x, y, n);
  return cudaGetLastError();
}

cudaError_t launch_err_partials(const ErrArgs& a, cudaStream_t s) {
  return a.f32 ? err_partials_nt<true>(a, s) : err_partials_nt<false>(a, s);
}

cudaError_t launch_begin_attempt(DnsCtrl* c, int method, cudaStream_t s) {
  k_begin_attempt<<<1, 1, 0, s>>>(c, method);
  return cudaGetLastError();
}

cudaError_t launch_controller(DnsCtrl* c, const double* partials, int method, int nstages,
                              double nmodes, int nc, cudaStream_t s) {
  k_controller<<<1, kRedThreads, 0, s>>>(c, partials, method, nstages, kRedBlocks, nmodes, nc);
  return cudaGetLastError();
}

cudaError_t launch_trace_diag(const Geom& g, DnsCtrl* c, double* partials, int method, cudaStream_t s) {
  k_trace_partials<<<kRedBlocks, kRedThreads, 0, s>>>(g, c, partials);
  k_trace_finish<<<1, kRedThreads, 0, s>>>(g, c, partials, kRedBlocks, method);
  return cudaGetLastError();
}

cudaError_t launch_ctrl_set_controller(DnsCtrl* c, int kind, const float* mlp, cudaStream_t s) {
  k_ctrl_set<<<1, 1, 0, s>>>(c, 0, kind, mlp, nullptr, 0, 0);
  return cudaGetLastError();
}

cudaError_t launch_ctrl_set_trace(DnsCtrl* c, double* trace, long long cap, int diag, cudaStream_t s) {
  k_ctrl_set<<<1, 1, 0, s>>>(c, 1, 0, nullptr, trace, cap, diag);
  return cudaGetLastError();
}

cudaError_t launch_ctrl_inject(DnsCtrl* c, long long rhs_index, cudaStream_t s) {
  k_ctrl_set<<<1, 1, 0, s>>>(c, 2, 0, nullptr, nullptr, rhs_index, 0);
  return cudaGetLastError();
}

cudaError_t launch_ctrl_reset(DnsCtrl* c, double t, cudaStream_t s) {
  k_ctrl_reset<<<1, 1, 0, s>>>(c, t);
  return cudaGetLastError();
}

cudaError_t launch_ctrl_config(DnsCtrl* c, double t_end, int method, double rtol, double atol,
                               double h0, int max_rejects, cudaStream_t s) {
  k_ctrl_config<<<1, 1, 0, s>>>(c, t_end, method, rtol, atol, h0, max_rejects);
  return cudaGetLastError();
}

cudaError_t launch_gather(const Geom& g, const double2* full, double2* compact, cudaStream_t s) {
  k_gather<<<grid_for((long long)g.nc * g.M, 256, 152 * 16), 256, 0, s>>>(g, full, compact);
  return cudaGetLastError();
}

cudaError_t launch_scatter(const Geom& g, const double2* compact, double2* full, cudaStream_t s) {
  k_scatter<<<grid_for((long long)g.nc * g.M, 256, 152 * 16), 256, 0, s>>>(g, compact, full);
  return cudaGetLastError();
}

cudaError_t launch_copy_slot(DnsCtrl* c, int slot, double2* dst, long long n2, cudaStream_t s) {
  k_copy_slot<<<grid_for(n2, 256, 152 * 16), 256, 0, s>>>(c, slot, dst, n2);
  return cudaGetLastError();
}

cudaError_t launch_forcing_coef(const Geom& g, DnsCtrl* c, int yslot, double kf, double power,
                                int gate_k1, cudaStream_t s) {
  k_forcing_coef<<<1, kRedThreads, 0, s>>>(g, c, yslot, kf, power, gate_k1);
  return cudaGetLastError();
}

cudaError_t launch_rescale(const Geom& g, DnsCtrl* c, double* partials, double kf, cudaStream_t s) {
  k_rescale_partials<<<kRedBlocks, kRedThreads, 0, s>>>(g, c, partials);
  k_rescale_apply<<<1, kRedThreads, 0, s>>>(g, c, partials, kRedBlocks, kf);
  return cudaGetLastError();
}

cudaError_t launch_diag_partials(const Geom& g, const double2* u, const double2* f,
                                 double* partials, cudaStream_t s) {
  k_diag_partials<<<kRedBlocks, kRedThreads, 0, s>>>(g, u, f, partials);
  return cudaGetLastError();
}

}  // namespace dns
