/*
 * dns.h -- C ABI of libdns: a GB300 (sm_103a) implementation of the Fourier pseudo-spectral
 * incompressible Navier-Stokes right-hand side in rotational form, integrated with the
 * Bogacki-Shampine 5(4) pair under embedded local-error step control, or with classical RK4.
 *
 * Method: Ketcheson, Mortensen, Parsani & Schilling, "More efficient time integration for
 * Fourier pseudo-spectral DNS of incompressible turbulence", arXiv:1810.10197.
 *
 * Conventions used by every call
 *   - Grid nx x ny x nz (each even, from the supported set below) on [0,lx) x [0,ly) x [0,lz);
 *     wavenumber kappa_a = 2 pi m / l_a for integer mode number m.
 *   - A spectral field is the half spectrum of a real 3D DFT taken along z:
 *     complex128 (interleaved re, im doubles), layout [3][nx][ny][nz/2+1], component-major,
 *     kz contiguous; kx, ky in FFT order (0..n/2-1, -n/2..-1).
 *   - Forward DFT unnormalised: uhat_k = sum_x u(x) exp(-i kappa.x); the inverse carries
 *     1/(nx ny nz) (the convention behind E = ||uhat||^2 / (2 N^6), Section 3.1).
 *   - 2/3-rule dealiasing: a mode is kept iff |m_a| <= K_a = floor((n_a - 1)/3) on every axis.
 *     Fields passed in are truncated to that box; fields returned are zero outside it.
 *
 * Ownership and errors
 *   - Every pointer argument stays owned by the caller; the library copies in and out and
 *     never frees or retains caller memory past the call.  Device pointers must come from
 *     cudaMalloc (e.g. a torch CUDA tensor's data_ptr()) on the context's device; host
 *     pointers may be pageable or pinned (pinned is faster).
 *   - Calls return a dns_status; no exception or longjmp crosses the ABI.  DNS_ERR_ARG leaves
 *     the context usable.  A CUDA error or a device-side failure makes the context "failed":
 *     every later call except dns_last_error/dns_destroy returns DNS_ERR_STATE.
 *   - The context owns all its device work buffers (allocated in dns_create).
 *   - Work is enqueued on the context's stream (dns_set_stream; default: the legacy default
 *     stream).  Calls documented as "synchronous" wait for that stream before returning.
 *   - A context is not thread-safe: use one context per host thread.
 *
 * Supported transform sizes (2/3 rule: nx, ny, nz; 3/2 rule: 3nx/2, 3ny/2, 3nz/2):
 *   {8,12,16,24,32,48,64,96,128,192,256,384,512,768}.
 */
#ifndef DNS_H
#define DNS_H

#include <stddef.h>

/* Exported entry points (the library hides every other symbol). */
#if defined(__GNUC__)
#define DNS_API __attribute__((visibility("default")))
#else
#define DNS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dns_ctx dns_ctx;

typedef enum {
    DNS_OK = 0,
    DNS_ERR_ARG = 1,             /* invalid argument; context unchanged                     */
    DNS_ERR_CUDA = 2,            /* a CUDA call failed; context is failed                    */
    DNS_ERR_OOM = 3,             /* device allocation failed in dns_create                   */
    DNS_ERR_NONFINITE = 4,       /* the error estimate stayed non-finite through max rejects */
    DNS_ERR_STEP_UNDERFLOW = 5,  /* step size fell below 1e-12 max(1,|t|)                   */
    DNS_ERR_MAX_REJECTS = 6,     /* more than max_rejects rejections in a row               */
    DNS_ERR_TIMEOUT = 7,         /* a bounded device wait ran out (see dns_debug_stall)      */
    DNS_ERR_STATE = 8,           /* context failed earlier, or no state was set             */
    DNS_ERR_UNSUPPORTED = 9      /* grid size outside the supported set                     */
} dns_status;

/* Time integrators of Section 2.2.  BS5 is the Bogacki-Shampine 5(4) pair of Appendix A with
 * the b-hat error estimator; DP5 the Dormand-Prince 5(4) pair of Appendix A.  *_FIXED take
 * fixed steps and still evaluate the error norm; *_ADAPTIVE use the controller. */
typedef enum { DNS_RK4 = 0, DNS_BS5_FIXED = 1, DNS_BS5_ADAPTIVE = 2, DNS_DP5_FIXED = 3,
               DNS_DP5_ADAPTIVE = 4 } dns_method;

/* DNS_FP64: every step in double precision.  DNS_FP32_MIXED: the transforms and the
 * nonlinear term in single precision; state, stage sums, viscous term, error norm and step
 * control in double precision (the projection in single precision, on the transformed
 * product).  DNS_FP32: as DNS_FP32_MIXED, and further the derivatives k_i, the intermediate
 * stage inputs, the stage increments, the projection epilogue (viscous term, forcing) and
 * the embedded error combination in single precision: the k_i carry single-precision
 * accuracy in both forms, so this form keeps the same error floor and moves about half the
 * bytes outside the transforms; the state u_n, the update u_{n+1} = u_n + increment, the
 * error norm's sums and step control stay double.  DNS_FP32X2: the transforms, the nonlinear term
 * and the projection in double-word arithmetic -- each number an unevaluated sum of two FP32
 * values, about 48 significant bits (rounding near 2^-47 per operation instead of FP64's
 * 2^-53) at the FP32 instruction rate; state, stage sums, viscous term, error norm and step
 * control in double precision.  DNS_FP32X2 needs transform lengths of 32 or more on every
 * axis (else DNS_ERR_UNSUPPORTED).  The paper fixes no precision; its runs were FP64. */
typedef enum { DNS_FP64 = 0, DNS_FP32_MIXED = 1, DNS_FP32X2 = 2, DNS_FP32 = 3 } dns_precision;

/* Forcing (Section 3.3.1 injects energy into 0 < |kappa| <= kf).  kind 0: none.  kind 1:
 * constant power as a right-hand-side term F_k = power/(2 E_f) uhat_k on 0 < |kappa| <= kf,
 * E_f the band energy, so that dE/dt gains exactly `power`.  kind 2: the paper's own scheme,
 * a rescale after every accepted step: the band 0 < |kappa| <= kf of the new state is
 * multiplied by alpha = sqrt(1 + (E_n - E_{n+1}) / E_f), E_f the band energy of the new
 * state, so that the total energy returns to its value before the step (`power` is unused;
 * the right-hand side has no forcing term; a first-same-as-last pair re-evaluates k_1 after
 * each rescale).  kf > 0 for kinds 1 and 2. */
typedef struct {
    int kind;
    double kf;
    double power;
} dns_forcing;

typedef struct {
    int nx, ny, nz;
    double lx, ly, lz;           /* domain lengths; 0 means 2 pi                             */
    double nu;                   /* kinematic viscosity, 1/Re                                 */
    int precision;               /* dns_precision                                             */
    dns_forcing forcing;
    int dealias;                 /* 0: 2/3 truncation rule (default); 1: 3/2 padding rule of
                                    Section 2.1.1 -- the state holds N frequencies per axis
                                    (nx ny nz = N, each a multiple of 4, 3N/2 supported),
                                    products are formed on the (3N/2)^3 grid, the result keeps
                                    |m| <= N/2 - 1 and the Nyquist modes are zero. */
} dns_config;

/* Outcome of the last attempt and running counters since the last dns_set_state. */
typedef struct {
    int accepted;                /* last attempt accepted                                     */
    int status;                  /* device status word (a dns_status value)                   */
    double err;                  /* last embedded error norm (0 for RK4)                      */
    double h_used;               /* step size of the last attempt (after clipping to t_end)   */
    double h_next;               /* controller's proposal for the next attempt                */
    double t;                    /* current time of the state                                 */
    long long n_rhs;             /* right-hand-side evaluations                               */
    long long n_acc, n_rej;      /* accepted / rejected attempts                              */
} dns_step_info;

/* Create a context for an nx x ny x nz grid on the current CUDA device (Eq. ufdef with
 * viscosity nu, optional forcing, precision a dns_precision).  Domain [0, 2 pi)^3. */
DNS_API dns_status dns_create(int nx, int ny, int nz, double nu, const dns_forcing* forcing,
                      int precision, dns_ctx** out);
/* As dns_create, with domain lengths from cfg. */
DNS_API dns_status dns_create_ex(const dns_config* cfg, dns_ctx** out);
/* Boussinesq form, Eqs. (ufdefboussinesq) and (rhofdefboussinesq) of Section 3.2:
 *   d(uhat)/dt   = P(kappa)[(u x omega)^ - Ri rhohat e_z] - nu |kappa|^2 uhat
 *   d(rhohat)/dt = -i kappa . (rho u)^ - kappa |kappa|^2 rhohat
 * (the buoyancy's kappa = 0 mode is dropped: a mean body force is balanced by the mean
 * pressure gradient).  The state has 4 components [4][nx][ny][nz/2+1]: velocity then the
 * density deviation rho; every state/RHS call of this context uses that layout, and the
 * error norm takes the maximum over the 4 components.  cfg->forcing must be kind 0;
 * kappa is the density diffusivity 1/(Re Pr), ri the Richardson number. */
DNS_API dns_status dns_create_boussinesq(const dns_config* cfg, double kappa, double ri, dns_ctx** out);
DNS_API void dns_destroy(dns_ctx* ctx);
/* Message for the last non-OK status of this context ("" if none).  Valid until next call. */
DNS_API const char* dns_last_error(const dns_ctx* ctx);

/* Stream for all later work (a cudaStream_t as void*; NULL = legacy default stream). */
DNS_API dns_status dns_set_stream(dns_ctx* ctx, void* stream);

/* Load the state uhat (layout above) at time t; where = 0: device pointer, 1: host pointer.
 * Truncates to the 2/3 box, resets the step counters and the controller (next h comes from
 * dns_integrate's h0).  Asynchronous for device input, synchronous for host input.  A host
 * input has only its retained modes copied (about 0.3 of the array at the 2/3 rule; pinned
 * memory transfers by DMA at full speed, pageable memory through the driver's staging). */
DNS_API dns_status dns_set_state(dns_ctx* ctx, const void* uhat, int where, double t);
/* Write the current state (zero outside the 2/3 box); where as above.  Synchronous. */
DNS_API dns_status dns_get_state(dns_ctx* ctx, void* uhat, int where);

/* Eq. (ufdef), once: f = P(kappa) [u x omega]^ - nu |kappa|^2 uhat (+ forcing), evaluated
 * pseudo-spectrally with 2/3 dealiasing (Section 2.1).  uhat and f are device pointers in the
 * layout above (may not alias).  Asynchronous on the context's stream. */
DNS_API dns_status dns_rhs(dns_ctx* ctx, const void* uhat_dev, void* f_dev);

/* One attempted step from the current state with step size h (clipped to t_end if t_end >
 * t), embedded error norm with (rtol, atol) and the controller of Section 2.2.1 (adaptive
 * methods accept iff err <= 1 and propose h_new).  Synchronous; fills info if non-NULL.
 * Tolerances: rtol, atol >= 0, not both 0; the adaptive methods need atol > 0 (else
 * DNS_ERR_ARG): modes that are zero up to rounding make a purely relative norm arbitrary.
 * A mode with e = 0 adds nothing to the norm, also where its scale is 0. */
DNS_API dns_status dns_step(dns_ctx* ctx, int method, double h, double rtol, double atol,
                    double t_end, dns_step_info* info);

/* Integrate from the current time to t_end.  h0 > 0 sets the step (fixed methods) or the
 * first proposal (adaptive); h0 <= 0 keeps the controller's current proposal.  The last step
 * is clipped to land on t_end.  max_rejects consecutive rejections (default 30 when <= 0)
 * end the run with DNS_ERR_MAX_REJECTS (DNS_ERR_NONFINITE if err was not finite).
 * The attempts run as one CUDA graph launch (a device-side loop; at most 1e8 attempts, else
 * DNS_ERR_STATE), built once per method and context and rebuilt after dns_set_tiles,
 * dns_autotune or dns_set_trace; with dns_profile_enable on, attempts are enqueued from the
 * host instead.  Synchronous; fills info if non-NULL. */
DNS_API dns_status dns_integrate(dns_ctx* ctx, double t_end, int method, double rtol, double atol,
                         double h0, int max_rejects, dns_step_info* info);

/* Enqueue exactly n step attempts toward t_end without waiting (for timing loops); attempts
 * after t_end is reached do nothing on the device.  Read the outcome with dns_get_info. */
DNS_API dns_status dns_enqueue_attempts(dns_ctx* ctx, int n, int method, double rtol, double atol,
                                double t_end, double h0);
/* Synchronous read of the controller state and counters. */
DNS_API dns_status dns_get_info(dns_ctx* ctx, dns_step_info* info);

/* Kinetic energy E, enstrophy Omega and dissipation rate eps = -dE/dt of the current state
 * (Section 3.1, half-spectrum weights).  eps uses one right-hand-side evaluation.
 * Synchronous. */
DNS_API dns_status dns_diagnostics(dns_ctx* ctx, double* E, double* Omega, double* eps);

/* Energy spectrum of the current state (Section 3.3): E(k) = sum over shell k of
 * w |uhat|^2 / (2 (nx ny nz)^2), shell k = nearest integer to |kappa| (velocity components;
 * half-spectrum weights as dns_diagnostics).  *nshells receives the number of shells
 * (0..K|kappa|max); out[0..min(cap, nshells)-1] receives E(k).  cap <= 0 or out NULL only
 * queries the count.  Synchronous. */
DNS_API dns_status dns_spectrum(dns_ctx* ctx, double* out, int cap, int* nshells);

/* Per-kernel timing with CUDA events on the context's stream.  enable != 0 starts recording
 * (and clears earlier records).  dns_profile_get returns, for kernel index i < count, its
 * name, number of launches and summed duration in ms (synchronous). */
DNS_API dns_status dns_profile_enable(dns_ctx* ctx, int enable);
DNS_API int dns_profile_count(dns_ctx* ctx);
DNS_API dns_status dns_profile_get(dns_ctx* ctx, int i, const char** name, long long* launches,
                           double* total_ms);

/* Attempt trace.  dns_set_trace allocates room for `capacity` records in the context (0
 * frees it) and clears it; each later attempt appends one record of DNS_TRACE_COLS doubles:
 *   t at the start, h used, err, accepted (1/0), RHS evaluations so far, E, Omega, eps
 * The last three (Section 3.1, of the state after the attempt) are filled only when
 * `diagnostics` != 0 (NaN otherwise; eps also NaN for RK4).  Records beyond the capacity
 * are dropped.  dns_trace copies min(n, cap) records to the host array `out` (row-major)
 * and returns the number recorded in *n.  Synchronous. */
#define DNS_TRACE_COLS 8
DNS_API dns_status dns_set_trace(dns_ctx* ctx, long long capacity, int diagnostics);
DNS_API dns_status dns_trace(dns_ctx* ctx, double* out, long long cap, long long* n);

/* Step-size controller of the adaptive method.  DNS_CTRL_I: Section 2.2.1 (default).
 * DNS_CTRL_PI: after an accepted step h_new = h min(2, max(0.01, 0.8 err^-0.14 err_prev^0.08))
 * (the PI controller the paper names as future work, Section 4, with exponents 0.7/(q+1),
 * 0.4/(q+1)).  DNS_CTRL_MLP: after an accepted step, once 4 accepted steps are known, a
 * learned correction of the PI factor, h_new = h min(2, max(0.01,
 * 0.8 err^-0.14 err_prev^0.08 exp(clamp(y, -log 1.5, log 1.5)))) with y from the network
 * below (capped at 1 right after a rejection); before that, and when y is not finite, the PI
 * factor.  In every variant the embedded error norm still accepts or rejects each step, and
 * a rejected attempt takes the Section 2.2.1 factor.
 * mlp_params_dev: DNS_MLP_PARAMS floats on the device (copied in), for DNS_CTRL_MLP only. */
typedef enum { DNS_CTRL_I = 0, DNS_CTRL_PI = 1, DNS_CTRL_MLP = 2 } dns_controller;
DNS_API dns_status dns_set_controller(dns_ctx* ctx, int kind, const float* mlp_params_dev);

/* The learned proposal's network (not in the paper): inputs 16 features of the 4 newest
 * accepted steps (newest first, each [log10 err, log(h_i/h_0), rejections before it,
 * log(h_i/h_{i+1})]), output y, the log of the correction to the Section 2.2.1 factor.  Parameters (float): W1[64][16], b1[64],
 * W2[64][64], b2[64], w3[64], b3; y = w3.relu(W2 relu(W1 x + b1) + b2) + b3, evaluated with the
 * weights rounded to bfloat16 and FP32 arithmetic.  All pointers are device pointers;
 * asynchronous on `stream`.
 *   dns_mlp_forward:   y[b] for x[n][16].
 *   dns_mlp_loss_grad: mean squared error against t[n] and its gradient (n <= 128).
 *   dns_mlp_train:     `steps` Adam steps (lr, beta 0.9/0.999) on random mini-batches of
 *                      `batch` (<= 128) samples drawn with a counter hash of `seed`; params
 *                      updated in place; loss_hist[steps] (may be NULL) receives batch losses. */
#define DNS_MLP_PARAMS 5313
DNS_API dns_status dns_mlp_forward(const float* params, const float* x, int n, float* y, void* stream);
DNS_API dns_status dns_mlp_loss_grad(const float* params, const float* x, const float* t, int n, float* grad,
                             float* loss, void* stream);
DNS_API dns_status dns_mlp_train(float* params, const float* x, const float* t, int n, int steps, int batch,
                         float lr, unsigned seed, float* loss_hist, void* stream);

/* Ensembles of independent simulations (uneven sizes allowed), advanced together.
 * dns_create_batch makes one context per config (each owns its buffers; all on the current
 * device).  Load each instance's state through dns_batch_context + dns_set_state (or read it
 * with dns_get_state); the contexts belong to the batch: do not destroy them yourself.
 * dns_integrate_batch integrates every instance i from its current time to t_end[i] with its
 * own tolerances and first step h0[i] (<= 0 keeps the current proposal), by ONE launch of a
 * CUDA graph: one conditional loop per instance, side by side, each running that instance's
 * attempts until it is done or fails (at most 10^7 attempts each).  The loops do not wait
 * for one another.
 * The graph is built on the first call for a method and reused.  Synchronous; info[i]
 * receives each instance's outcome; returns the first non-OK instance status (or DNS_OK). */
typedef struct dns_batch dns_batch;
DNS_API dns_status dns_create_batch(int count, const dns_config* cfgs, dns_batch** out);
DNS_API void dns_destroy_batch(dns_batch* batch);
DNS_API const char* dns_batch_last_error(const dns_batch* batch);
DNS_API dns_status dns_batch_context(dns_batch* batch, int i, dns_ctx** out);
DNS_API dns_status dns_integrate_batch(dns_batch* batch, int method, const double* t_end, const double* rtol,
                               const double* atol, const double* h0, dns_step_info* info);

/* Autotuner of the FFT tile shapes and kernels.
 * y argument (var_py): bits 0-1 the y passes' kernel -- 0 full column tile, 1 half tile, 2
 * (single-precision forms, ny = 256, an even number of retained kz planes; elsewhere it runs
 * 0) one tensor-map box load and one box store per tile of 8 kz columns of a (field, x) plane
 * (the TMA engine, a swizzled shared-memory box, line transforms held in registers); bit 2
 * the x-inverse pass's kernel, set: tensor-map box loads of the stage input and a box store
 * per output line (single-precision forms, velocity equations, nx = 256, an even number of
 * retained (ky, kz) columns; elsewhere the shared-memory kernel).  Values 0, 1, 2, 4, 5, 6.
 * z argument (var_p3): bit 0 the tile variant (lines per CTA, full or half), bit 1 set =
 * input rows copied element by element instead of by bulk copies (the TMA engine, completing
 * on a shared-memory barrier; used where a row is a multiple of 16 bytes and the staging fits
 * in shared memory, else element copies anyway); codes 4 and 5 are the register-resident
 * FP32 kernel (two real fields per complex line transform held in registers, u x omega
 * between the transforms without a shared-memory round trip, persistent CTAs fed by bulk
 * copies that overlap the previous tile's transforms) with fully paired FP32 arithmetic
 * (FADD2/FMUL2/FFMA2) or paired sums and scalar products; they apply to the single-precision
 * forms of the velocity equations with nz = 64, 128 or 256 and elsewhere run codes 0 and 1.
 * dns_autotune times `reps` launches of each choice on this context's buffers with CUDA
 * events on its stream, keeps the fastest, and caches the choice per (grid, precision, form)
 * for the process and, if the environment variable DNS_TUNE_CACHE names a file, in that file
 * (read on first use, appended to).  variants (may be NULL) receives {y argument, z argument}.
 * dns_create_batch tunes every instance.  dns_set_tiles sets them by hand (DNS_ERR_ARG for
 * other values); the default is 6 and 4.  Synchronous.
 * A bulk or tensor copy's completion is awaited with a bound (about half a second); a wait
 * that runs out marks the step controller DNS_ERR_TIMEOUT instead of hanging. */
DNS_API dns_status dns_autotune(dns_ctx* ctx, int reps, int* variants);
DNS_API dns_status dns_set_tiles(dns_ctx* ctx, int var_py, int var_p3);

/* Checkpoint and resume (the paper restarts its turbulence runs from a spun-up state,
 * Section 3.3.2).  dns_save writes the current state, the carried-over derivative k_1 of a
 * first-same-as-last pair (when valid) and the controller's state (t, h, step history,
 * counters, controller kind) to `path`; dns_load reads them into a context with the same
 * state grid, dealiasing rule and component count.  The physical parameters (nu, forcing,
 * precision, kappa, Ri) are the loading context's own, so a forced spin-up can be resumed
 * as an unforced run.  A checkpoint taken with the learned controller needs
 * dns_set_controller(ctx, DNS_CTRL_MLP, params) before dns_load (the network parameters are
 * not stored).  Continuing a loaded context with h0 = 0 reproduces the uninterrupted run bit
 * for bit.
 *
 * File layout, little-endian: "DNSCKPT1", u32 version (1), i32 nx ny nz dealias ncomp
 * precision, f64 2pi/lx 2pi/ly 2pi/lz nu kappa Ri, i32 forcing kind, f64 kf power, f64 t h
 * h_try err err_prev rtol atol errc[4], i32 method k1_valid after_reject accepted clipped
 * controller hist_n rej_since hist_rej[5], f64 hist_err[5] hist_h[5], i64 n_rhs n_acc n_rej
 * n_attempts rejects_in_row, i64 M (retained modes per component), complex128 state[ncomp][M]
 * (retained box, kz fastest), complex128 k1[ncomp][M] when k1_valid, u32 CRC-32 of all
 * preceding bytes.  Both calls synchronise the context's stream.  Errors: DNS_ERR_ARG for an
 * unreadable, truncated or corrupt file or a mismatched grid (the context is left unchanged),
 * DNS_ERR_STATE without a state (save) or for a learned-controller checkpoint without
 * parameters (load). */
DNS_API dns_status dns_save(dns_ctx* ctx, const char* path);
DNS_API dns_status dns_load(dns_ctx* ctx, const char* path);

/* CRC-32 of the checkpoint trailer (reflected polynomial 0xEDB88320, the checksum of zlib and
 * PNG), continued from `crc` (0 to start).  Host-only; needs no GPU. */
DNS_API unsigned int dns_crc32(const void* data, size_t n, unsigned int crc);

/* Fault injection for tests (the paper has no counterpart; no GPU fault is involved): the
 * right-hand side with running index rhs_index (0-based, counted like dns_step_info.n_rhs
 * since dns_set_state) returns NaN in the (0,0,0) mode of its first component, once.  The
 * embedded error of that attempt is then not finite, so the controller rejects it with the
 * smallest factor (Section 2.2.1 reading) and the run goes on; rhs_index < 0 disarms. */
DNS_API dns_status dns_debug_inject(dns_ctx* ctx, long long rhs_index);

/* Test hook for the bounded wait (the paper has no counterpart; no GPU fault is involved):
 * the next z pass enqueued from the host (dns_step, dns_rhs, dns_enqueue_attempts; not the
 * graph of dns_integrate) makes its first CTA wait for 16 bytes that no bulk copy delivers,
 * so that CTA's bounded wait runs out: the attempt ends with DNS_ERR_TIMEOUT and the context
 * stays usable.  One-shot; no effect when the z pass copies element by element. */
DNS_API dns_status dns_debug_stall(dns_ctx* ctx);

/* Debug aid (the paper has no counterpart): with on != 0 both scratch buffers of the passes
 * are filled with all-ones bytes -- a NaN in every element type -- before every right-hand
 * side, so a pass that reads a scratch element that no earlier pass wrote makes the result NaN
 * (a correct build gives results identical to a run without it).  Costs two memsets per
 * right-hand side; takes effect for work enqueued after the call. */
DNS_API dns_status dns_debug_poison(dns_ctx* ctx, int on);

/* Test hook for the FP64-to-FP32 conversion every FP32 kernel uses (the state entering the
 * x-inverse pass, the fp32 form's stage sums, error norm and projection epilogue; integer
 * instructions on the bits, no FP64 arithmetic): y[i] = x[i] rounded to FP32 with the
 * significand rounded to nearest (ties away from zero), magnitudes below the smallest normal
 * float flushed to a signed zero, beyond the largest float an infinity, NaN kept.
 * x_dev: n doubles, y_dev: n floats, both on the device (caller-owned); enqueued on `stream`
 * (NULL: the legacy default stream).  DNS_ERR_ARG for n < 0 or a NULL pointer with n > 0;
 * DNS_ERR_CUDA if the launch fails. */
DNS_API dns_status dns_debug_f32_from_f64(const double* x_dev, float* y_dev, long long n, void* stream);

/* The FP64 pipe's issue rate on the current device, measured: chains of independent DFMA
 * (and, separately, DADD) instructions on every SM, timed with CUDA events on `stream` (NULL:
 * the legacy default stream).  Writes thread instructions per second.  The FP64 form of the
 * passes is bound by this pipe (Section 2.1's transforms in FP64 do about 2 flops per byte of
 * traffic on this part), and its roofline is stated against this rate.  Allocates and frees
 * 8 bytes of device memory; synchronous (about 0.2 s).  DNS_ERR_ARG for NULL outputs,
 * DNS_ERR_CUDA if a launch fails. */
DNS_API dns_status dns_measure_fp64_rate(void* stream, double* dfma_per_s, double* dadd_per_s);

/* Grid facts: retained cut-offs K[3] and the number of device bytes the context holds. */
DNS_API dns_status dns_query(const dns_ctx* ctx, int* K3, size_t* device_bytes);

/* The right-hand side of dns_rhs (same layout, same result) for small grids, without a
 * context and without allocating any device memory.  The paper has no counterpart: this
 * entry point exists for callers that cannot call cudaMalloc -- for instance a host program
 * that hands out all device memory through its own pool or budget, or code on a
 * latency-critical path where cudaMalloc/cudaFree would synchronise the device.
 *
 *   nx, ny, nz  each in {8, 12, 16, 24, 32} (domain [0, 2 pi)^3, no forcing, FP64);
 *               larger sizes return DNS_ERR_UNSUPPORTED before any CUDA call.
 *   nu          viscosity (>= 0);  uhat_dev, f_dev: device pointers as for dns_rhs (no alias).
 *   stream      cudaStream_t as void* (NULL = legacy default stream); asynchronous.
 *
 * Work space: one static __device__ array of about 2.3 MB inside libdns, held by every GPU
 * that loads the library until the process exits.  The first call on a device looks up its
 * address (cudaGetSymbolAddress, with that device current); make that first call before any
 * stream capture.  All calls on a device share the array and each call rewrites every part
 * it reads, so no state carries over; calls that overlap on the GPU (different streams, or
 * different host threads) race on it and must be serialised by the caller.  The looked-up
 * address is cached per device for the life of the process: after cudaDeviceReset on a
 * device the cached address is stale, and this entry point must not be called there again.
 * Returns DNS_ERR_ARG for bad pointers or nu, DNS_ERR_CUDA if a launch fails. */
DNS_API dns_status dns_rhs_noalloc(int nx, int ny, int nz, double nu, const void* uhat_dev, void* f_dev,
                           void* stream);

#ifdef __cplusplus
}
#endif

#endif /* DNS_H */
