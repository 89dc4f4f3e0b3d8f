// C ABI of libdns (include/dns.h): context, device buffers and the orchestration of one
// right-hand-side evaluation (five passes) and of one Runge-Kutta attempt (stage sums, right-
// hand sides, error norm, controller), all enqueued on the context's stream.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/dns.h"
#include "common.cuh"
#include "passes.cuh"
#include "stepper.cuh"
#include "mlp.cuh"

using namespace dns;

namespace {

struct Frac { long long p, q; };

// Bogacki-Shampine 5(4) pair, Appendix A of arXiv:1810.10197 (rows 2..8 of A, b, b-hat).
const Frac kBS5A[8][7] = {
    {},
    {{1, 6}},
    {{2, 27}, {4, 27}},
    {{183, 1372}, {-162, 343}, {1053, 1372}},
    {{68, 297}, {-4, 11}, {42, 143}, {1960, 3861}},
    {{597, 22528}, {81, 352}, {63099, 585728}, {58653, 366080}, {4617, 20480}},
    {{174197, 959244}, {-30942, 79937}, {8152137, 19744439}, {666106, 1039181}, {-29421, 29068},
     {482048, 414219}},
    {{587, 8064}, {0, 1}, {4440339, 15491840}, {24353, 124800}, {387, 44800}, {2152, 5985},
     {7267, 94080}},
};
const Frac kBS5B[8] = {{587, 8064}, {0, 1}, {4440339, 15491840}, {24353, 124800},
                       {387, 44800}, {2152, 5985}, {7267, 94080}, {0, 1}};
const Frac kBS5Bh[8] = {{2479, 34992}, {0, 1}, {123, 416}, {612941, 3411720},
                        {43, 1440}, {2272, 6561}, {79937, 1113912}, {3293, 556956}};
// Dormand-Prince 5(4) pair, Appendix A (rows 2..7 of A, b, b-hat).
const Frac kDP5A[7][6] = {
    {},
    {{1, 5}},
    {{3, 40}, {9, 40}},
    {{44, 45}, {-56, 15}, {32, 9}},
    {{19372, 6561}, {-25360, 2187}, {64448, 6561}, {-212, 729}},
    {{9017, 3168}, {-355, 33}, {46732, 5247}, {49, 176}, {-5103, 18656}},
    {{35, 384}, {0, 1}, {500, 1113}, {125, 192}, {-2187, 6784}, {11, 84}},
};
const Frac kDP5B[7] = {{35, 384}, {0, 1}, {500, 1113}, {125, 192}, {-2187, 6784}, {11, 84}, {0, 1}};
const Frac kDP5Bh[7] = {{5179, 57600}, {0, 1}, {7571, 16695}, {393, 640}, {-92097, 339200}, {187, 2100}, {1, 40}};
// Classical RK4.
const Frac kRK4A[4][3] = {{}, {{1, 2}}, {{0, 1}, {1, 2}}, {{0, 1}, {0, 1}, {1, 1}}};
const Frac kRK4B[4] = {{1, 6}, {1, 3}, {1, 3}, {1, 6}};

long long gcdll(long long a, long long b) {
  a = a < 0 ? -a : a; b = b < 0 ? -b : b;
  while (b) { long long t = a % b; a = b; b = t; }
  return a ? a : 1;
}
// exact difference of two fractions, then one correctly rounded division
double frac_diff(Frac a, Frac b) {
  long long p = a.p * b.q - b.p * a.q, q = a.q * b.q, g = gcdll(p, q);
  return (double)(p / g) / (double)(q / g);
}
double frac_val(Frac a) { return (double)a.p / (double)a.q; }

bool supported(int n) {
  switch (n) {
    case 8: case 12: case 16: case 24: case 32: case 48: case 64: case 96: case 128: case 192:
    case 256: case 384: case 512: case 768: return true;
  }
  return false;
}

const char* kPassNames[] = {"begin_attempt", "stage_sum", "p1_x_inverse_curl", "p2_y_inverse",
                            "p3_z_c2r_cross_r2c", "p4_y_forward", "p5_x_forward_project",
                            "err_norm_partials", "controller", "forcing_coef"};
enum ProfId { PR_BEGIN = 0, PR_STAGE, PR_P1, PR_P2, PR_P3, PR_P4, PR_P5, PR_ERR, PR_CTRL, PR_FORCE, PR_N };

struct ProfRec { int id; cudaEvent_t a, b; };

}  // namespace

struct dns_ctx {
  Geom g{};
  int precision = 0;
  double nu = 0;
  double kappa_d = 0;   // Boussinesq density diffusivity
  double ri = 0;        // Boussinesq Richardson number
  dns_forcing forcing{};
  int device = 0;
  cudaStream_t stream = nullptr;
  double2* uu[2] = {nullptr, nullptr};
  double2* kk[2] = {nullptr, nullptr};
  double2* kfix[9] = {};
  double2* ystage = nullptr;
  double2* rhs_in = nullptr;
  double2* rhs_out = nullptr;
  double2* full_stage = nullptr;   // half-spectrum staging for host copies (lazy)
  void* bufA = nullptr;
  void* bufB = nullptr;
  void* tw[3] = {nullptr, nullptr, nullptr};
  DnsCtrl* ctrl = nullptr;         // integrator
  DnsCtrl* ctrl_rhs = nullptr;     // plain right-hand side
  double* partials = nullptr;
  DnsCtrl* host_ctrl = nullptr;    // pinned mirror
  double* host_partials = nullptr; // pinned
  size_t device_bytes = 0;
  bool failed = false;
  bool has_state = false;
  std::string err;
  double* trace_buf = nullptr;     // attempt records (dns_set_trace)
  int trace_diag = 0;
  float* mlp_buf = nullptr;        // learned-controller parameters (dns_set_controller)
  int var_py = 2, var_p3 = 0;      // tile variants (dns_autotune; y variant 2 runs 0 where it does not apply)
  int p3_bulk = 1;                 // z pass input by bulk copies where possible (dns_autotune)
  int p3_rr = 1;                   // z pass: register-resident FP32 kernel where it applies
  int x_tma = 1;                   // x-inverse pass: tensor-map FP32 kernel where it applies
  bool stall_pending = false;      // dns_debug_stall: the next host-enqueued z pass stalls
  bool capturing = false;          // building dns_integrate's graph
  size_t bytesA = 0, bytesB = 0;   // sizes of the scratch buffers A and B
  bool prof = false;
  std::vector<ProfRec> recs;
  std::vector<cudaEvent_t> pool;
  size_t pool_used = 0;
  // dns_integrate's graph per method: a conditional WHILE node around one attempt
  cudaGraphExec_t gexec[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  cudaGraph_t graph[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  cudaStream_t cap_stream = nullptr;
  unsigned long long* d_iter = nullptr;
  bool poison = false;             // dns_debug_poison: NaN-fill the scratch before each RHS
};

namespace {

dns_status fail(dns_ctx* c, dns_status s, const std::string& msg) {
  if (c) {
    c->err = msg;
    if (s == DNS_ERR_CUDA || s == DNS_ERR_OOM) c->failed = true;
  }
  return s;
}
dns_status cuda_fail(dns_ctx* c, cudaError_t e, const char* what) {
  return fail(c, DNS_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}
#define CK(call, what)                                      \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, what);   \
  } while (0)

cudaEvent_t pool_event(dns_ctx* c) {
  if (c->pool_used == c->pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    c->pool.push_back(e);
  }
  return c->pool[c->pool_used++];
}

// run `launch` bracketed by profiling events when enabled
template <typename F>
cudaError_t timed(dns_ctx* c, int id, F&& launch) {
  if (!c->prof) return launch();
  cudaEvent_t a = pool_event(c), b = pool_event(c);
  if (!a || !b) return cudaErrorMemoryAllocation;
  cudaEventRecord(a, c->stream);
  cudaError_t e = launch();
  cudaEventRecord(b, c->stream);
  c->recs.push_back({id, a, b});
  return e;
}

dns_status alloc(dns_ctx* c, void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(c, DNS_ERR_OOM, std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
  }
  c->device_bytes += bytes;
  return DNS_OK;
}

// twiddle table of one axis (layout: axis_twiddle_turns), each entry rounded once from
// the transforms run in FP32 (both single-precision forms share their kernels and tiles)
static bool fp32_transforms(int p) { return p == DNS_FP32_MIXED || p == DNS_FP32; }

// long double
dns_status make_twiddles(dns_ctx* c, int n, bool zaxis, void** out) {
  const bool f32 = fp32_transforms(c->precision), dwp = c->precision == DNS_FP32X2;
  const size_t esz = f32 ? sizeof(float2) : sizeof(double2);
  const int cnt = std::max(1, axis_twiddle_count(n, zaxis));
  std::vector<unsigned char> host(cnt * esz, 0);
  const long double twopi = 6.283185307179586476925286766559005768L;
  for (int m = 0; m < axis_twiddle_count(n, zaxis); ++m) {
    int num = 0, den = 1;
    axis_twiddle_turns(n, zaxis, m, &num, &den);
    const long double ang = twopi * (long double)num / (long double)den;
    const long double cr = cosl(ang), ci = -sinl(ang);
    if (f32) {
      reinterpret_cast<float2*>(host.data())[m] = make_float2((float)cr, (float)ci);
    } else if (dwp) {   // double-word: high part rounded to FP32, low part the rounded remainder
      const float rh = (float)cr, ih = (float)ci;
      float* q = reinterpret_cast<float*>(host.data()) + 4 * m;
      q[0] = rh; q[1] = (float)(cr - (long double)rh); q[2] = ih; q[3] = (float)(ci - (long double)ih);
    } else {
      reinterpret_cast<double2*>(host.data())[m] = make_double2((double)cr, (double)ci);
    }
  }
  dns_status s = alloc(c, out, cnt * esz);
  if (s != DNS_OK) return s;
  CK(cudaMemcpy(*out, host.data(), cnt * esz, cudaMemcpyHostToDevice), "twiddle upload");
  return DNS_OK;
}

cudaError_t pass(dns_ctx* c, int which, const PassArgs& a) {
  switch (c->precision) {
    case DNS_FP32_MIXED:
    case DNS_FP32: return launch_pass<float>(which, a, c->stream);
    case DNS_FP32X2: return launch_pass<dw>(which, a, c->stream);
    default: return launch_pass<double>(which, a, c->stream);
  }
}

// One evaluation of Eq. (ufdef) on the stage input in `yslot`, result to `kslot`.
dns_status enqueue_rhs(dns_ctx* c, DnsCtrl* ctrl, int yslot, int kslot, int gate_k1) {
  if (c->poison) {   // all-ones bytes are a NaN in every element type
    CK(cudaMemsetAsync(c->bufA, 0xFF, c->bytesA, c->stream), "poison");
    CK(cudaMemsetAsync(c->bufB, 0xFF, c->bytesB, c->stream), "poison");
  }
  if (c->forcing.kind == 1) {
    CK(timed(c, PR_FORCE, [&] {
         return launch_forcing_coef(c->g, ctrl, yslot, c->forcing.kf, c->forcing.power, gate_k1, c->stream);
       }), "forcing coefficient");
  }
  PassArgs a{};
  a.g = c->g;
  a.ctrl = ctrl;
  a.gate_k1 = gate_k1;
  a.yslot = yslot;
  a.kslot = kslot;
  a.nu = c->nu;
  a.epi32 = c->precision == DNS_FP32 ? 1 : 0;
  a.kf2 = c->forcing.kind == 1 ? c->forcing.kf * c->forcing.kf : 0.0;
  a.kappa_d = c->kappa_d;
  a.ri = c->ri;
  a.var_py = c->var_py;
  a.var_p3 = c->var_p3;
  a.p3_bulk = c->p3_bulk;
  a.p3_rr = c->p3_rr;
  a.x_tma = c->x_tma;
  // the buffers the stage-input slot can name (tensor maps of the x-inverse pass)
  if (ctrl == c->ctrl_rhs) {
    a.ycand[0] = c->rhs_in;
  } else if (yslot == SLOT_Y) {
    a.ycand[0] = c->ystage;
    a.ycand_f32 = c->precision == DNS_FP32 ? 1 : 0;
  } else {
    a.ycand[0] = c->uu[0];
    a.ycand[1] = c->uu[1];
  }
  if (c->stall_pending && !c->capturing) {
    a.p3_stall = 16;
    c->stall_pending = false;
  }
  a.out = c->bufA; a.tw = c->tw[0];
  CK(timed(c, PR_P1, [&] { return pass(c, 1, a); }), "pass P1");
  a.in = c->bufA; a.out = c->bufB; a.tw = c->tw[1];
  CK(timed(c, PR_P2, [&] { return pass(c, 2, a); }), "pass P2");
  a.in = c->bufB; a.out = c->bufA; a.tw = c->tw[2];
  CK(timed(c, PR_P3, [&] { return pass(c, 3, a); }), "pass P3");
  a.in = c->bufA; a.out = c->bufB; a.tw = c->tw[1];
  CK(timed(c, PR_P4, [&] { return pass(c, 4, a); }), "pass P4");
  a.in = c->bufB; a.out = nullptr; a.tw = c->tw[0];
  CK(timed(c, PR_P5, [&] { return pass(c, 5, a); }), "pass P5");
  return DNS_OK;
}

dns_status enqueue_stage(dns_ctx* c, int nterms, const int* kslots, const double* coef, int yslot) {
  StageArgs s{};
  s.ctrl = c->ctrl;
  s.gate_k1 = 0;
  s.nterms = nterms;
  for (int j = 0; j < nterms; ++j) { s.kslot[j] = kslots[j]; s.coef[j] = coef[j]; }
  s.uslot = SLOT_U;
  s.yslot = yslot;
  s.n2 = (long long)c->g.nc * c->g.M;
  s.f32 = c->precision == DNS_FP32 ? 1 : 0;
  CK(timed(c, PR_STAGE, [&] { return launch_stage_sum(s, c->stream); }), "stage sum");
  return DNS_OK;
}

// Forcing kind 2 (Section 3.3.1): after an accepted step the band 0 < |kappa| <= kf is
// rescaled so that the step's energy loss is put back (decided on the device).
dns_status enqueue_rescale(dns_ctx* c) {
  if (c->forcing.kind != 2) return DNS_OK;
  CK(timed(c, PR_FORCE, [&] { return launch_rescale(c->g, c->ctrl, c->partials, c->forcing.kf, c->stream); }),
     "band rescale");
  return DNS_OK;
}

// One attempted step (Section 2.2): all stages, error norm and the controller decision.
dns_status enqueue_attempt(dns_ctx* c, int method) {
  dns_status st;
  CK(timed(c, PR_BEGIN, [&] { return launch_begin_attempt(c->ctrl, method, c->stream); }), "begin");
  if (method == DNS_RK4) {
    if ((st = enqueue_rhs(c, c->ctrl, SLOT_U, SLOT_K1, 0)) != DNS_OK) return st;
    for (int i = 1; i < 4; ++i) {
      int ks[3]; double cf[3]; int n = 0;
      for (int j = 0; j < i; ++j)
        if (kRK4A[i][j].p != 0) { ks[n] = SLOT_K1 + j; cf[n] = frac_val(kRK4A[i][j]); ++n; }
      if ((st = enqueue_stage(c, n, ks, cf, SLOT_Y)) != DNS_OK) return st;
      if ((st = enqueue_rhs(c, c->ctrl, SLOT_Y, SLOT_K1 + i, 0)) != DNS_OK) return st;
    }
    int ks[4]; double cf[4];
    for (int j = 0; j < 4; ++j) { ks[j] = SLOT_K1 + j; cf[j] = frac_val(kRK4B[j]); }
    if ((st = enqueue_stage(c, 4, ks, cf, SLOT_UNEW)) != DNS_OK) return st;
    CK(timed(c, PR_CTRL, [&] {
         return launch_controller(c->ctrl, c->partials, 0, 4, c->g.nmodes_half, c->g.nc, c->stream);
       }), "controller");
    if ((st = enqueue_rescale(c)) != DNS_OK) return st;
    if (c->trace_diag) CK(launch_trace_diag(c->g, c->ctrl, c->partials, 0, c->stream), "trace diagnostics");
    return DNS_OK;
  }
  // BS5 / DP5 (first same as last): k_1 only when not carried over
  const bool dp = method >= 3;
  const int S = dp ? 7 : 8;
  auto A = [&](int i, int j) { return dp ? kDP5A[i][j] : kBS5A[i][j]; };
  auto Bw = [&](int j) { return dp ? kDP5B[j] : kBS5B[j]; };
  auto Bh = [&](int j) { return dp ? kDP5Bh[j] : kBS5Bh[j]; };
  if ((st = enqueue_rhs(c, c->ctrl, SLOT_U, SLOT_K1, 1)) != DNS_OK) return st;
  for (int i = 1; i < S; ++i) {
    int ks[7]; double cf[7]; int n = 0;
    for (int j = 0; j < i; ++j)
      if (A(i, j).p != 0) { ks[n] = SLOT_K1 + j; cf[n] = frac_val(A(i, j)); ++n; }
    const int ys = (i == S - 1) ? SLOT_UNEW : SLOT_Y;
    if ((st = enqueue_stage(c, n, ks, cf, ys)) != DNS_OK) return st;
    if ((st = enqueue_rhs(c, c->ctrl, ys, SLOT_K1 + i, 0)) != DNS_OK) return st;
  }
  ErrArgs e{};
  e.ctrl = c->ctrl;
  e.M = c->g.M;
  e.nc = c->g.nc;
  e.partials = c->partials;
  e.f32 = c->precision == DNS_FP32 ? 1 : 0;
  int n = 0;
  for (int j = 0; j < S; ++j) {
    if (Bw(j).p * Bh(j).q == Bh(j).p * Bw(j).q) continue;
    e.kslot[n] = SLOT_K1 + j;
    e.coef[n] = frac_diff(Bw(j), Bh(j));
    ++n;
  }
  e.nterms = n;
  CK(timed(c, PR_ERR, [&] { return launch_err_partials(e, c->stream); }), "error norm");
  CK(timed(c, PR_CTRL, [&] {
       return launch_controller(c->ctrl, c->partials, method, S, c->g.nmodes_half, c->g.nc, c->stream);
     }), "controller");
  if ((st = enqueue_rescale(c)) != DNS_OK) return st;
  if (c->trace_diag) CK(launch_trace_diag(c->g, c->ctrl, c->partials, method, c->stream), "trace diagnostics");
  return DNS_OK;
}

dns_status check_ctx(dns_ctx* c) {
  if (!c) return DNS_ERR_ARG;
  if (c->failed) return DNS_ERR_STATE;
  if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, DNS_ERR_CUDA, "cudaSetDevice");
  return DNS_OK;
}

dns_status read_ctrl(dns_ctx* c) {
  CK(cudaMemcpyAsync(c->host_ctrl, c->ctrl, sizeof(DnsCtrl), cudaMemcpyDeviceToHost, c->stream), "ctrl read");
  CK(cudaStreamSynchronize(c->stream), "synchronize");
  return DNS_OK;
}

void fill_info(dns_ctx* c, dns_step_info* info) {
  if (!info) return;
  const DnsCtrl& h = *c->host_ctrl;
  info->accepted = h.accepted;
  info->status = h.status;
  info->err = h.err;
  info->h_used = h.h_try;
  info->h_next = h.h;
  info->t = h.t;
  info->n_rhs = h.n_rhs;
  info->n_acc = h.n_acc;
  info->n_rej = h.n_rej;
}

dns_status status_from_ctrl(dns_ctx* c) {
  switch (c->host_ctrl->status) {
    case ST_OK: return DNS_OK;
    case ST_NONFINITE: return fail(c, DNS_ERR_NONFINITE, "error estimate not finite through max_rejects retries");
    case ST_UNDERFLOW: return fail(c, DNS_ERR_STEP_UNDERFLOW, "step size underflow");
    case ST_MAX_REJECTS: return fail(c, DNS_ERR_MAX_REJECTS, "too many rejected steps in a row");
    case ST_TIMEOUT: return fail(c, DNS_ERR_TIMEOUT, "a bounded device wait ran out (z-pass bulk copies)");
  }
  return fail(c, DNS_ERR_STATE, "unknown device status");
}

dns_status ensure_stage(dns_ctx* c) {
  if (c->full_stage) return DNS_OK;
  const size_t bytes = (size_t)c->g.nc * c->g.snx * c->g.sny * c->g.snzh * sizeof(double2);
  return alloc(c, (void**)&c->full_stage, bytes);
}

// The captured attempt bakes in the tile variants and whether the trace records diagnostics:
// a change of either drops the cached graphs.
void drop_graphs(dns_ctx* c) {
  for (int m = 0; m < 5; ++m) {
    if (c->gexec[m]) cudaGraphExecDestroy(c->gexec[m]);
    if (c->graph[m]) cudaGraphDestroy(c->graph[m]);
    c->gexec[m] = nullptr;
    c->graph[m] = nullptr;
  }
}

__global__ void k_ctx_continue(cudaGraphConditionalHandle h, const DnsCtrl* c, unsigned long long* iter,
                               unsigned long long max_iter) {
  const unsigned long long it = ++(*iter);
  cudaGraphSetConditional(h, (!c->done && c->status == 0 && it < max_iter) ? 1u : 0u);
}

// Attempts until the controller reports done or a failure (at most 1e8), as one graph launch:
// no host round trip per attempt.
dns_status integrate_graph(dns_ctx* c, int method) {
  if (!c->d_iter) {
    dns_status s = alloc(c, (void**)&c->d_iter, sizeof(unsigned long long));
    if (s != DNS_OK) return s;
  }
  if (!c->cap_stream) CK(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking), "capture stream");
  if (!c->gexec[method]) {
    cudaGraph_t g = nullptr;
    CK(cudaGraphCreate(&g, 0), "graph create");
    cudaGraphConditionalHandle handle;
    cudaGraphNodeParams cp = {};
    cudaGraphNode_t node;
    cudaError_t e = cudaGraphConditionalHandleCreate(&handle, g, 1, cudaGraphCondAssignDefault);
    if (e == cudaSuccess) {
      cp.type = cudaGraphNodeTypeConditional;
      cp.conditional.handle = handle;
      cp.conditional.type = cudaGraphCondTypeWhile;
      cp.conditional.size = 1;
      e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp);
    }
    if (e == cudaSuccess)
      e = cudaStreamBeginCaptureToGraph(c->cap_stream, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                        cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) { cudaGraphDestroy(g); return cuda_fail(c, e, "graph build"); }
    cudaStream_t user = c->stream;
    c->stream = c->cap_stream;
    c->capturing = true;
    dns_status st = enqueue_attempt(c, method);
    c->capturing = false;
    if (st == DNS_OK) {
      k_ctx_continue<<<1, 1, 0, c->cap_stream>>>(handle, c->ctrl, c->d_iter, 100000000ULL);
      e = cudaGetLastError();
    }
    c->stream = user;
    cudaGraph_t captured = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(c->cap_stream, &captured);
    if (st != DNS_OK || e != cudaSuccess || e2 != cudaSuccess) {
      cudaGraphDestroy(g);
      return st != DNS_OK ? st : cuda_fail(c, e != cudaSuccess ? e : e2, "graph capture");
    }
    e = cudaGraphInstantiate(&c->gexec[method], g, 0);
    if (e != cudaSuccess) { cudaGraphDestroy(g); return cuda_fail(c, e, "graph instantiate"); }
    c->graph[method] = g;
  }
  CK(cudaMemsetAsync(c->d_iter, 0, sizeof(unsigned long long), c->stream), "reset counter");
  CK(cudaGraphLaunch(c->gexec[method], c->stream), "graph launch");
  return DNS_OK;
}

}  // namespace

extern "C" {

dns_status dns_create(int nx, int ny, int nz, double nu, const dns_forcing* forcing, int precision,
                      dns_ctx** out) {
  dns_config cfg{};
  cfg.nx = nx; cfg.ny = ny; cfg.nz = nz; cfg.nu = nu; cfg.precision = precision;
  if (forcing) cfg.forcing = *forcing;
  return dns_create_ex(&cfg, out);
}

static dns_status create_impl(const dns_config* cfg, int bouss, double kappa, double ri, dns_ctx** out);

dns_status dns_create_ex(const dns_config* cfg, dns_ctx** out) { return create_impl(cfg, 0, 0.0, 0.0, out); }

dns_status dns_create_boussinesq(const dns_config* cfg, double kappa, double ri, dns_ctx** out) {
  if (!cfg || !out) return DNS_ERR_ARG;
  if (!(kappa >= 0.0) || !std::isfinite(kappa) || !std::isfinite(ri) || cfg->forcing.kind != 0) return DNS_ERR_ARG;
  return create_impl(cfg, 1, kappa, ri, out);
}

static dns_status create_impl(const dns_config* cfg, int bouss, double kappa, double ri, dns_ctx** out) {
  if (!cfg || !out) return DNS_ERR_ARG;
  *out = nullptr;
  if (cfg->dealias != 0 && cfg->dealias != 1) return DNS_ERR_ARG;
  const bool pad = cfg->dealias == 1;
  // 3/2 rule: the state has N frequencies per axis, the transforms run on 3N/2 points
  auto phys = [&](int n) { return pad ? ((n % 4 == 0) ? 3 * n / 2 : -1) : n; };
  if (!supported(phys(cfg->nx)) || !supported(phys(cfg->ny)) || !supported(phys(cfg->nz))) return DNS_ERR_UNSUPPORTED;
  if (cfg->precision != DNS_FP64 && cfg->precision != DNS_FP32_MIXED && cfg->precision != DNS_FP32X2 &&
      cfg->precision != DNS_FP32)
    return DNS_ERR_ARG;
  // the double-word form: transform lengths of 32 and more
  if (cfg->precision == DNS_FP32X2 && (phys(cfg->nx) < 32 || phys(cfg->ny) < 32 || phys(cfg->nz) < 32))
    return DNS_ERR_UNSUPPORTED;
  if (!(cfg->nu >= 0.0) || !std::isfinite(cfg->nu)) return DNS_ERR_ARG;
  if (cfg->forcing.kind < 0 || cfg->forcing.kind > 2) return DNS_ERR_ARG;
  if (cfg->forcing.kind != 0 && !(cfg->forcing.kf > 0.0 && std::isfinite(cfg->forcing.kf))) return DNS_ERR_ARG;
  dns_ctx* c = new dns_ctx();
  c->precision = cfg->precision;
  c->nu = cfg->nu;
  c->kappa_d = kappa;
  c->ri = ri;
  c->forcing = cfg->forcing;
  cudaGetDevice(&c->device);
  Geom& g = c->g;
  g.nx = phys(cfg->nx); g.ny = phys(cfg->ny); g.nz = phys(cfg->nz); g.nzh = g.nz / 2 + 1;
  g.snx = cfg->nx; g.sny = cfg->ny; g.snz = cfg->nz; g.snzh = cfg->nz / 2 + 1;
  g.Kx = (g.nx - 1) / 3; g.Ky = (g.ny - 1) / 3; g.Kz = (g.nz - 1) / 3;
  g.Mx = 2 * g.Kx + 1; g.My = 2 * g.Ky + 1; g.Mz = g.Kz + 1;
  g.MyMz = g.My * g.Mz;
  g.M = (long long)g.Mx * g.MyMz;
  const double twopi = 6.283185307179586476925286766559;
  const double lx = cfg->lx > 0 ? cfg->lx : twopi, ly = cfg->ly > 0 ? cfg->ly : twopi;
  const double lz = cfg->lz > 0 ? cfg->lz : twopi;
  g.sx = cfg->lx > 0 ? twopi / lx : 1.0;
  g.sy = cfg->ly > 0 ? twopi / ly : 1.0;
  g.sz = cfg->lz > 0 ? twopi / lz : 1.0;
  g.inv_n3 = 1.0 / ((double)g.snx * g.sny * g.snz);
  g.nmodes_half = (double)g.snx * g.sny * g.snzh;
  g.fwd_scale = ((double)g.snx * g.sny * g.snz) / ((double)g.nx * g.ny * g.nz);
  g.nc = bouss ? 4 : 3;
  g.bouss = bouss;

  const size_t vbytes = (size_t)g.nc * g.M * sizeof(double2);
  const size_t esz = fp32_transforms(c->precision) ? sizeof(float2) : sizeof(double2);
  // physical-side field counts: inverse (u, omega [, rho]), forward (u x omega [, rho u])
  const size_t fin = g.bouss ? 7 : 6, fout = g.bouss ? 6 : 3;
  const size_t nA = std::max(fin * g.nx * g.My * g.Mz, fout * g.nx * g.ny * g.Mz);
  const size_t nB = std::max(fin * g.nx * g.ny * g.Mz, fout * g.nx * g.My * g.Mz);
  dns_status s = DNS_OK;
  auto A = [&](void** p, size_t b) { if (s == DNS_OK) s = alloc(c, p, b); };
  A((void**)&c->uu[0], vbytes); A((void**)&c->uu[1], vbytes);
  A((void**)&c->kk[0], vbytes); A((void**)&c->kk[1], vbytes);
  for (int i = 2; i <= 7; ++i) A((void**)&c->kfix[i], vbytes);
  A((void**)&c->ystage, vbytes);
  A((void**)&c->rhs_in, vbytes); A((void**)&c->rhs_out, vbytes);
  A(&c->bufA, nA * esz); A(&c->bufB, nB * esz);
  c->bytesA = nA * esz;
  c->bytesB = nB * esz;
  A((void**)&c->ctrl, sizeof(DnsCtrl)); A((void**)&c->ctrl_rhs, sizeof(DnsCtrl));
  A((void**)&c->partials, (size_t)kRedBlocks * kRedStride * sizeof(double));
  if (s == DNS_OK) s = make_twiddles(c, g.nx, false, &c->tw[0]);
  if (s == DNS_OK) s = make_twiddles(c, g.ny, false, &c->tw[1]);
  if (s == DNS_OK) s = make_twiddles(c, g.nz, true, &c->tw[2]);
  if (s == DNS_OK && cudaMallocHost((void**)&c->host_ctrl, sizeof(DnsCtrl)) != cudaSuccess) s = DNS_ERR_OOM;
  if (s == DNS_OK && cudaMallocHost((void**)&c->host_partials, (size_t)kRedBlocks * kRedStride * sizeof(double)) != cudaSuccess)
    s = DNS_ERR_OOM;
  if (s == DNS_OK) {
    DnsCtrl h{};
    h.uu[0] = c->uu[0]; h.uu[1] = c->uu[1];
    h.kk[0] = c->kk[0]; h.kk[1] = c->kk[1];
    for (int i = 2; i <= 7; ++i) h.kfix[i] = c->kfix[i];
    h.slot[SLOT_Y] = c->ystage;
    h.slot[SLOT_U] = c->uu[0];
    h.slot[SLOT_UNEW] = c->uu[1];
    h.slot[SLOT_K1] = c->kk[0];
    for (int i = 2; i <= 7; ++i) h.slot[SLOT_K1 + i - 1] = c->kfix[i];
    h.slot[SLOT_K1 + 7] = c->kk[1];
    h.done = 1; h.max_rejects = 30; h.method = DNS_BS5_ADAPTIVE; h.inject_rhs = -1;
    // DNS_FP32: k_1..k_8 and the stage-input scratch are FP32 (their readers -- stage sums,
    // error norm, the x passes -- use FP32 values of them); dns_rhs and the diagnostics keep
    // FP64 inputs and outputs (ctrl_rhs)
    h.f32_slots = c->precision == DNS_FP32 ? 1 : 0;
    DnsCtrl r{};
    r.slot[SLOT_Y] = c->rhs_in;
    r.slot[SLOT_K1] = c->rhs_out;
    r.need_k1 = 1;
    r.inject_rhs = -1;
    if (cudaMemcpy(c->ctrl, &h, sizeof(h), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(c->ctrl_rhs, &r, sizeof(r), cudaMemcpyHostToDevice) != cudaSuccess)
      s = DNS_ERR_CUDA;
  }
  if (s != DNS_OK) {
    dns_destroy(c);
    return s;
  }
  *out = c;
  return DNS_OK;
}

void dns_destroy(dns_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  drop_graphs(c);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  void* ptrs[] = {c->uu[0], c->uu[1], c->kk[0], c->kk[1], c->ystage, c->rhs_in, c->rhs_out,
                  c->full_stage, c->bufA, c->bufB, c->tw[0], c->tw[1], c->tw[2], c->ctrl,
                  c->ctrl_rhs, c->partials, c->trace_buf, c->mlp_buf, c->d_iter};
  for (void* p : ptrs) if (p) cudaFree(p);
  for (int i = 2; i <= 7; ++i) if (c->kfix[i]) cudaFree(c->kfix[i]);
  if (c->host_ctrl) cudaFreeHost(c->host_ctrl);
  if (c->host_partials) cudaFreeHost(c->host_partials);
  for (cudaEvent_t e : c->pool) cudaEventDestroy(e);
  delete c;
}

const char* dns_last_error(const dns_ctx* c) { return c ? c->err.c_str() : "null context"; }

dns_status dns_set_stream(dns_ctx* c, void* stream) {
  if (!c) return DNS_ERR_ARG;
  c->stream = reinterpret_cast<cudaStream_t>(stream);
  return DNS_OK;
}

dns_status dns_set_state(dns_ctx* c, const void* uhat, int where, double t) {
  dns_status s = check_ctx(c);
  if (s != DNS_OK) return s;
  if (!uhat || (where != 0 && where != 1) || !std::isfinite(t)) return fail(c, DNS_ERR_ARG, "dns_set_state: bad argument");
  if (where == 1) {
    // only the retained box crosses the bus (M / (snx sny snzh) of the array: 0.30 at the 2/3
    // rule): one pitched copy per component and sign quadrant of (kx, ky), straight into the
    // state buffer -- the mapping of the gather kernel
    const Geom& g = c->g;
    const int xb[2][3] = {{0, 0, g.Kx + 1}, {g.Kx + 1, g.snx - (g.Mx - g.Kx - 1), g.Mx - g.Kx - 1}};
    const int yb[2][3] = {{0, 0, g.Ky + 1}, {g.Ky + 1, g.sny - (g.My - g.Ky - 1), g.My - g.Ky - 1}};
    for (int q = 0; q < g.nc; ++q)
      for (int bx = 0; bx < 2; ++bx)
        for (int by = 0; by < 2; ++by) {
          if (xb[bx][2] <= 0 || yb[by][2] <= 0) continue;
          cudaMemcpy3DParms p = {};
          p.srcPtr = make_cudaPitchedPtr(const_cast<void*>(uhat), (size_t)g.snzh * sizeof(double2),
                                         (size_t)g.snzh * sizeof(double2), (size_t)g.sny);
          p.dstPtr = make_cudaPitchedPtr(c->uu[0], (size_t)g.Mz * sizeof(double2), (size_t)g.Mz * sizeof(double2),
                                         (size_t)g.My);
          p.srcPos = make_cudaPos(0, (size_t)yb[by][1], (size_t)q * g.snx + xb[bx][1]);
          p.dstPos = make_cudaPos(0, (size_t)yb[by][0], (size_t)q * g.Mx + xb[bx][0]);
          p.extent = make_cudaExtent((size_t)g.Mz * sizeof(double2), (size_t)yb[by][2], (size_t)xb[bx][2]);
          p.kind = cudaMemcpyHostToDevice;
          CK(cudaMemcpy3DAsync(&p, c->stream), "state upload");
        }
  } else {
    CK(launch_gather(c->g, reinterpret_cast<const double2*>(uhat), c->uu[0], c->stream), "gather");
  }
  CK(launch_ctrl_reset(c->ctrl, t, c->stream), "controller reset");
  if (where == 1) CK(cudaStreamSynchronize(c->stream), "synchronize");
  c->has_state = true;
  return DNS_OK;
}

dns_status dns_get_state(dns_ctx* c, void* uhat, int where) {
  dns_status s = check_ctx(c);
  if (s != DNS_OK) return s;
  if (!uhat || (where != 0 && where != 1)) return fail(c, DNS_ERR_ARG, "dns_get_state: bad argument");
  if (!c->has_state) return fail(c, DNS_ERR_STATE, "no state set");
  const size_t bytes = (size_t)c->g.nc * c->g.snx * c->g.sny * c->g.snzh * sizeof(double2);
  double2* dst = reinterpret_cast<double2*>(uhat);
  if (where == 1) {
    if ((s = ensure_stage(c)) != DNS_OK) return s;
    dst = c->full_stage;
  }
  CK(cudaMemsetAsync(dst, 0, bytes, c->stream), "memset");
  s = read_ctrl(c);
  if (s != DNS_OK) return s;
  const double2* cur = c->uu[c->host_ctrl->parity];
  CK(launch_scatter(c->g, cur, dst, c->stream), "scatter");
  if (where == 1) CK(cudaMemcpyAsync(uhat, c->full_stage, bytes, cudaMemcpyDeviceToHost, c->stream), "state download");
  CK(cudaStreamSynchronize(c->stream), "synchronize");
  return DNS_OK;
}

dns_status dns_rhs(dns_ctx* c, const void* uhat_dev, void* f_dev) {
  dns_status s = check_ctx(c);
  if (s != DNS_OK) return s;
  if (!uhat_dev || !f_dev || uhat_dev == f_dev) return fail(c, DNS_ERR_ARG, "dns_rhs: bad pointers");
  const size_t bytes = (size_t)c->g.nc * c->g.snx * c->g.sny * c->g.snzh * sizeof(double2);
  CK(launch_gather(c->g, reinterpret_cast<const double2*>(uhat_dev), c->rhs_in, c->stream), "gather");
  if ((s = enqueue_rhs(c, c->ctrl_rhs, SLOT_Y, SLOT_K1, 0)) != DNS_OK) return s;
  CK(cudaMemsetAsync(f_dev, 0, bytes, c->stream), "memset");
  CK(launch_scatter(c->g, c->rhs_out, reinterpret_cast<double2*>(f_dev), c->stream), "scatter");
  return DNS_OK;
}

static dns_status config(dns_ctx* c, double t_end, int method, double rtol, double atol, double h0,
                         int max_rejects) {
  if (method < 0 || method > 4) return fail(c, DNS_ERR_ARG, "unknown method");
  if (!(t_end == t_end)) return fail(c, DNS_ERR_ARG, "t_end is NaN");
  if (method != DNS_RK4 && (!(rtol >= 0) || !(atol >= 0) || (rtol == 0 && atol == 0)))
    return fail(c, DNS_ERR_ARG, "tolerances must be >= 0 and not both 0");
  // A purely relative tolerance has no usable norm on these fields: the divergence-free
  // constraint makes some components of some modes zero up to rounding (u_x at kappa =
  // (kx, 0, 0), for one), so their error and scale are both rounding noise and their ratio
  // is arbitrary.  Adaptive control needs an absolute part.
  if ((method == DNS_BS5_ADAPTIVE || method == DNS_DP5_ADAPTIVE) && !(atol > 0))
    return fail(c, DNS_ERR_ARG, "adaptive methods need atol > 0 (a purely relative error norm is "
                                "undefined on modes that are zero up to rounding)");
  if (!(h0 == h0)) return fail(c, DNS_ERR_ARG, "h0 is NaN");
  CK(launch_ctrl_config(c->ctrl, t_end, method, rtol, atol, h0, max_rejects > 0 ? max_rejects : 30,
                        c->stream), "controller config");
  return DNS_OK;
}

dns_status dns_step(dns_ctx* c, int method, double h, double rtol, double atol, double t_end,
                    dns_step_info* info) {
  dns_status s = check_ctx(c);
  if (s != DNS_OK) return s;
  if (!c->has_state) return fail(c, DNS_ERR_STATE, "no state set");
  if (!(h > 0)) return fail(c, DNS_ERR_ARG, "h must be > 0");
  if ((s = read_ctrl(c)) != DNS_OK) return s;
  if (!(t_end > c->host_ctrl->t)) t_end = INFINITY;
  if ((s = config(c, t_end, method, rtol, atol, h, 0)) != DNS_OK) return s;
  if ((s = enqueue_attempt(c, method)) != DNS_OK) return s;
  if ((s = read_ctrl(c)) != DNS_OK) return s;
  fill_info(c, info);
  return status_from_ctrl(c);
}

dns_status dns_integrate(dns_ctx* c, double t_end, int method, double rtol, double atol, double h0,
                         int max_rejects, dns_step_info* info) {
  dns_status s = check_ctx(c);
  if (s != DNS_OK) return s;
  if (!c->has_state) return fail(c, DNS_ERR_STATE, "no state set");
  if ((s = read_ctrl(c)) != DNS_OK) return s;
  if (!(h0 > 0) && !(c->host_ctrl->h > 0)) return fail(c, DNS_ERR_ARG, "no step size: pass h0 > 0");
  if ((s = config(c, t_end, method, rtol, atol, h0, max_rejects)) != DNS_OK) return s;
  if (!c->prof) {
    // one graph launch runs every attempt (per-kernel profiling needs the host loop below)
    if ((s = integrate_graph(c, method)) != DNS_OK) return s;
    if ((s = read_ctrl(c)) != DNS_OK) return s;
    if (!c->host_ctrl->done && c->host_ctrl->status == 0) return fail(c, DNS_ERR_STATE, "step limit reached");
    fill_info(c, info);
    return status_from_ctrl(c);
  }
  const double cells = (double)c->g.nx * c->g.ny * c->g.nz;
  int chunk = (int)std::max(1.0, std::min(32.0, 4.0 * 1048576.0 / cells));
  long long guard = 0;
  for (;;) {
    for (int i = 0; i < chunk; ++i)
      if ((s = enqueue_attempt(c, method)) != DNS_OK) return s;
    if ((s = read_ctrl(c)) != DNS_OK) return s;
    if (c->host_ctrl->done || c->host_ctrl->status != 0) break;
    if (++guard > 100000000LL / chunk) return fail(c, DNS_ERR_STATE, "step limit reached");
  }
  fill_info(c, info);
  return status_from_ctrl(c);
}

dns_status dns_enqueue_attempts(dns_ctx* c, int n, int method, double rtol, double atol,
                                double t_end, double h0) {
  dns_status s = check_ctx(c);
  if (s != DNS_OK) return s;
  if (!c->has_state) return fail(c, DNS_ERR_STATE, "no state set");
  if (n < 0) return fail(c, DNS_ERR_ARG, "n < 0");
  if ((s = config(c, t_end, method, rtol, atol, h0, 0)) != DNS_OK) return s;
  for (int i = 0; i < n; ++i)
    if ((s = enqueue_attempt(c, method)) != DNS_OK) return s;
  return DNS_OK;
}

dns_status dns_get_info(dns_ctx* c, dns_step_info* info) {
  dns_status s = check_ctx(c);
  if (s != DNS_OK) return s;
  if ((s = read_ctrl(c)) != DNS_OK) return s;
  fill_info(c, info);
  return status_from_ctrl(c);
}

dns_status dns_diagnostics(dns_ctx* c, double* E, double* Omega, double* eps) {
  dns_status s = check_ctx(c);
  if (s != DNS_OK) return s;
  if (!c->has_state) return fail(c, DNS_ERR_STATE, "no state set");
  if ((s = read_ctrl(c)) != DNS_OK) return s;
  const double2* cur = c->uu[c->host_ctrl->parity];
  CK(cudaMemcpyAsync(c->rhs_in, cur, (size_t)c->g.nc * c->g.M * sizeof(double2), cudaMemcpyDeviceToDevice,
                     c->stream), "copy");
  if ((s = enqueue_rhs(c, c->ctrl_rhs, SLOT_Y, SLOT_K1, 0)) != DNS_OK) return s;
  CK(launch_diag_partials(c->g, c->rhs_in, c->rhs_out, c->partials, c->stream), "diagnostics");
  CK(cudaMemcpyAsync(c->host_partials, c->partials, (size_t)kRedBlocks * kRedStride * sizeof(double),
                     cudaMemcpyDeviceToHost, c->stream), "read partials");
  CK(cudaStreamSynchronize(c->stream), "synchronize");
  double v[3] = {0, 0, 0};
  for (int b = 0; b < kRedBlocks; ++b)
    for (int q = 0; q < 3; ++q) v[q] += c->host_partials[b * kRedStride + q];
  const double n6 = c->g.inv_n3 * c->g.inv_n3;
  if (E) *E = 0.5 * v[0] * n6;
  if (Omega) *Omega = 0.5 * v[1] * n6;
  if (eps) *eps = -v[2] * n6;
  return DNS_OK;
}

dns_status dns_profile_enable(dns_ctx* c, int enable) {
  if (!c) return DNS_ERR_ARG;
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  c->recs.clear();
  c->pool_used = 0;
  c->prof = enable != 0;
  return DNS_OK;
}

int dns_profile_count(dns_ctx* c) { return c ? PR_N : 0; }

dns_status dns_profile_get(dns_ctx* c, int i, const char** name, long long* launches, double* total_ms) {
  if (!c || i < 0 || i >= PR_N) return DNS_ERR_ARG;
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  long long n = 0;
  double ms = 0.0;
  for (const ProfRec& r : c->recs) {
    if (r.id != i) continue;
    float t = 0.f;
    if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) ms += t;
    ++n;
  }
  if (name) *name = kPassNames[i];
  if (launches) *launches = n;
  if (total_ms) *total_ms = ms;
  return DNS_OK;
}

dns_status dns_spectrum(dns_ctx* c, double* out, int cap, int* nshells) {
  dns_status s = check_ctx(c);
  if (s != DNS_OK) return s;
  if (!c->has_state) return fail(c, DNS_ERR_STATE, "no state set");
  const Geom& g = c->g;
  const double kmax = std::sqrt(std::pow(g.sx * g.Kx, 2) + std::pow(g.sy * g.Ky, 2) + std::pow(g.sz * g.Kz, 2));
  const int ns = (int)std::floor(kmax + 0.5) + 1;
  if (nshells) *nshells = ns;
  if (!out || cap <= 0) return DNS_OK;
  if ((s = read_ctrl(c)) != DNS_OK) return s;
  double* dev = nullptr;
  // scratch: the error-norm partials buffer is too small; use the staging buffer of host copies
  if ((s = ensure_stage(c)) != DNS_OK) return s;
  const size_t need = (size_t)(152 + 1) * ns * sizeof(double);
  const size_t have = (size_t)g.nc * g.snx * g.sny * g.snzh * sizeof(double2);
  if (need > have) return fail(c, DNS_ERR_UNSUPPORTED, "spectrum scratch too small");
  dev = reinterpret_cast<double*>(c->full_stage);
  CK(launch_spectrum(g, c->uu[c->host_ctrl->parity], dev + ns, ns, dev, c->stream), "spectrum");
  std::vector<double> h(ns);
  CK(cudaMemcpyAsync(h.data(), dev, ns * sizeof(double), cudaMemcpyDeviceToHost, c->stream), "read");
  CK(cudaStreamSynchronize(c->stream), "synchronize");
  for (int i = 0; i < std::min(ns, cap); ++i) out[i] = h[i];
  return DNS_OK;
}

dns_status dns_set_trace(dns_ctx* c, long long capacity, int diagnostics) {
  dns_status s = check_ctx(c);
  if (s != DNS_OK) return s;
  if (capacity < 0) return fail(c, DNS_ERR_ARG, "negative trace capacity");
  CK(cudaStreamSynchronize(c->stream), "synchronize");
  if (c->trace_buf) { cudaFree(c->trace_buf); c->trace_buf = nullptr; }
  if (capacity > 0 && (s = alloc(c, (void**)&c->trace_buf, (size_t)capacity * kTraceCols * sizeof(double))) != DNS_OK)
    return s;
  c->trace_diag = capacity > 0 && diagnostics != 0;
  drop_graphs(c);
  CK(launch_ctrl_set_trace(c->ctrl, c->trace_buf, capacity, c->trace_diag, c->stream), "trace set");
  return DNS_OK;
}

dns_status dns_trace(dns_ctx* c, double* out, long long cap, long long* n) {
  dns_status s = check_ctx(c);
  if (s != DNS_OK) return s;
  if ((s = read_ctrl(c)) != DNS_OK) return s;
  const long long have = c->host_ctrl->trace_n;
  if (n) *n = have;
  const long long m = std::min(have, cap);
  if (out && m > 0 && c->trace_buf)
    CK(cudaMemcpy(out, c->trace_buf, (size_t)m * kTraceCols * sizeof(double), cudaMemcpyDeviceToHost), "trace read");
  return DNS_OK;
}

dns_status dns_set_controller(dns_ctx* c, int kind, const float* mlp_params_dev) {
  dns_status s = check_ctx(c);
  if (s != DNS_OK) return s;
  if (kind < 0 || kind > 2 || (kind == 2 && !mlp_params_dev)) return fail(c, DNS_ERR_ARG, "bad controller");
  if (kind == 2) {
    if (!c->mlp_buf && (s = alloc(c, (void**)&c->mlp_buf, kMlpParams * sizeof(float))) != DNS_OK) return s;
    CK(cudaMemcpyAsync(c->mlp_buf, mlp_params_dev, kMlpParams * sizeof(float), cudaMemcpyDeviceToDevice,
                       c->stream), "copy network");
  }
  CK(launch_ctrl_set_controller(c->ctrl, kind, kind == 2 ? c->mlp_buf : nullptr, c->stream), "controller set");
  return DNS_OK;
}

}  // extern "C"

// ---- checkpoint and resume (dns_save / dns_load) ------------------------------------------
#if !defined(__BYTE_ORDER__) || __BYTE_ORDER__ != __ORDER_LITTLE_ENDIAN__
#error "the checkpoint format is little-endian; this host is not"
#endif

namespace {

// CRC-32 with the reflected polynomial 0xEDB88320, pre- and post-inverted (zlib's crc32).
uint32_t crc32_update(uint32_t crc, const void* data, size_t n) {
  static uint32_t table[256];
  static std::once_flag once;
  std::call_once(once, [] {
    for (uint32_t i = 0; i < 256; ++i) {
      uint32_t v = i;
      for (int k = 0; k < 8; ++k) v = (v & 1u) ? (0xEDB88320u ^ (v >> 1)) : (v >> 1);
      table[i] = v;
    }
  });
  const unsigned char* p = static_cast<const unsigned char*>(data);
  crc = ~crc;
  for (size_t i = 0; i < n; ++i) crc = table[(crc ^ p[i]) & 0xFFu] ^ (crc >> 8);
  return ~crc;
}

constexpr char kCkptMagic[8] = {'D', 'N', 'S', 'C', 'K', 'P', 'T', '1'};
constexpr uint32_t kCkptVersion = 1;

// Sequential little-endian writer/reader over a FILE*, keeping a running CRC-32.
struct CkptOut {
  FILE* f;
  uint32_t crc = 0;
  bool ok = true;
  void put(const void* p, size_t n) {
    crc = crc32_update(crc, p, n);
    ok = ok && std::fwrite(p, 1, n, f) == n;
  }
  template <typename T> void v(T x) { put(&x, sizeof(T)); }
};
struct CkptIn {
  FILE* f;
  uint32_t crc = 0;
  bool ok = true;
  void get(void* p, size_t n) {
    if (!ok || std::fread(p, 1, n, f) != n) { ok = false; std::memset(p, 0, n); return; }
    crc = crc32_update(crc, p, n);
  }
  template <typename T> T v() { T x; get(&x, sizeof(T)); return x; }
};

// The controller fields a checkpoint carries, in file order.
template <typename D, typename I, typename L>
void ckpt_ctrl_fields(DnsCtrl& h, D&& d, I&& i, L&& l) {
  d(h.t); d(h.h); d(h.h_try); d(h.err); d(h.err_prev); d(h.rtol); d(h.atol);
  for (int q = 0; q < 4; ++q) d(h.errc[q]);
  i(h.method); i(h.k1_valid); i(h.after_reject); i(h.accepted); i(h.clipped); i(h.ctrl_kind);
  i(h.hist_n); i(h.rej_since);
  for (int q = 0; q < 5; ++q) i(h.hist_rej[q]);
  for (int q = 0; q < 5; ++q) d(h.hist_err[q]);
  for (int q = 0; q < 5; ++q) d(h.hist_h[q]);
  l(h.n_rhs); l(h.n_acc); l(h.n_rej); l(h.n_attempts); l(h.rejects_in_row);
}

}  // namespace

extern "C" {

unsigned int dns_crc32(const void* data, size_t n, unsigned int crc) {
  if (!data && n) return crc;
  return crc32_update(crc, data, n);
}

dns_status dns_save(dns_ctx* c, const char* path) {
  dns_status s = check_ctx(c);
  if (s != DNS_OK) return s;
  if (!path) return fail(c, DNS_ERR_ARG, "dns_save: null path");
  if (!c->has_state) return fail(c, DNS_ERR_STATE, "dns_save: no state set");
  if ((s = read_ctrl(c)) != DNS_OK) return s;
  DnsCtrl h = *c->host_ctrl;
  const Geom& g = c->g;
  const size_t n = (size_t)g.nc * g.M;
  std::vector<double2> u(n), k1;
  CK(cudaMemcpy(u.data(), c->uu[h.parity], n * sizeof(double2), cudaMemcpyDeviceToHost), "state download");
  if (h.k1_valid) {
    k1.resize(n);
    if (h.f32_slots) {   // FP32 k slots: widen (exact) so that the file layout is the same in every form
      std::vector<float2> k32(n);
      CK(cudaMemcpy(k32.data(), c->kk[h.parity], n * sizeof(float2), cudaMemcpyDeviceToHost), "k1 download");
      for (size_t i = 0; i < n; ++i) k1[i] = make_double2(k32[i].x, k32[i].y);
    } else {
      CK(cudaMemcpy(k1.data(), c->kk[h.parity], n * sizeof(double2), cudaMemcpyDeviceToHost), "k1 download");
    }
  }
  FILE* f = std::fopen(path, "wb");
  if (!f) return fail(c, DNS_ERR_ARG, std::string("dns_save: cannot open ") + path);
  CkptOut o{f};
  o.put(kCkptMagic, sizeof(kCkptMagic));
  o.v<uint32_t>(kCkptVersion);
  o.v<int32_t>(g.snx); o.v<int32_t>(g.sny); o.v<int32_t>(g.snz);
  o.v<int32_t>(g.nx != g.snx ? 1 : 0); o.v<int32_t>(g.nc); o.v<int32_t>(c->precision);
  o.v<double>(g.sx); o.v<double>(g.sy); o.v<double>(g.sz);
  o.v<double>(c->nu); o.v<double>(c->kappa_d); o.v<double>(c->ri);
  o.v<int32_t>(c->forcing.kind); o.v<double>(c->forcing.kf); o.v<double>(c->forcing.power);
  ckpt_ctrl_fields(h, [&](double& x) { o.v<double>(x); }, [&](int& x) { o.v<int32_t>(x); },
                            [&](long long& x) { o.v<int64_t>(x); });
  o.v<int64_t>(g.M);
  o.put(u.data(), n * sizeof(double2));
  if (h.k1_valid) o.put(k1.data(), n * sizeof(double2));
  const uint32_t crc = o.crc;
  o.ok = o.ok && std::fwrite(&crc, 1, sizeof(crc), f) == sizeof(crc);
  const bool closed = std::fclose(f) == 0;
  if (!o.ok || !closed) return fail(c, DNS_ERR_ARG, std::string("dns_save: write failed: ") + path);
  return DNS_OK;
}

dns_status dns_load(dns_ctx* c, const char* path) {
  dns_status s = check_ctx(c);
  if (s != DNS_OK) return s;
  if (!path) return fail(c, DNS_ERR_ARG, "dns_load: null path");
  FILE* f = std::fopen(path, "rb");
  if (!f) return fail(c, DNS_ERR_ARG, std::string("dns_load: cannot open ") + path);
  CkptIn in{f};
  const Geom& g = c->g;
  char magic[8];
  in.get(magic, sizeof(magic));
  const uint32_t version = in.v<uint32_t>();
  const int nx = in.v<int32_t>(), ny = in.v<int32_t>(), nz = in.v<int32_t>();
  const int dealias = in.v<int32_t>(), nc = in.v<int32_t>();
  (void)in.v<int32_t>();                       // precision of the saving context
  for (int q = 0; q < 6; ++q) (void)in.v<double>();   // domain scales, nu, kappa, Ri
  (void)in.v<int32_t>(); (void)in.v<double>(); (void)in.v<double>();   // forcing
  std::string why;
  if (!in.ok) why = "truncated header";
  else if (std::memcmp(magic, kCkptMagic, sizeof(magic)) != 0) why = "not a checkpoint";
  else if (version != kCkptVersion) why = "unknown version";
  else if (nx != g.snx || ny != g.sny || nz != g.snz || dealias != (g.nx != g.snx ? 1 : 0) || nc != g.nc)
    why = "grid, dealiasing rule or component count differs from the context";
  DnsCtrl h{};
  ckpt_ctrl_fields(h, [&](double& x) { x = in.v<double>(); }, [&](int& x) { x = in.v<int32_t>(); },
                           [&](long long& x) { x = in.v<int64_t>(); });
  const long long M = in.v<int64_t>();
  if (why.empty() && (!in.ok || M != g.M)) why = in.ok ? "retained box differs" : "truncated header";
  const size_t n = (size_t)g.nc * g.M;
  std::vector<double2> u, k1;
  if (why.empty()) {
    u.resize(n);
    in.get(u.data(), n * sizeof(double2));
    if (h.k1_valid) { k1.resize(n); in.get(k1.data(), n * sizeof(double2)); }
    const uint32_t want = in.crc;
    uint32_t crc = 0;
    if (!in.ok || std::fread(&crc, 1, sizeof(crc), f) != sizeof(crc)) why = "truncated data";
    else if (crc != want) why = "CRC-32 mismatch";
  }
  std::fclose(f);
  if (!why.empty()) return fail(c, DNS_ERR_ARG, std::string("dns_load: ") + why + ": " + path);
  if ((s = read_ctrl(c)) != DNS_OK) return s;
  DnsCtrl& d = *c->host_ctrl;
  if (h.ctrl_kind == 2 && !d.mlp)
    return fail(c, DNS_ERR_STATE, "dns_load: the checkpoint uses the learned controller; set its parameters first");
  CK(cudaMemcpy(c->uu[0], u.data(), n * sizeof(double2), cudaMemcpyHostToDevice), "state upload");
  if (h.k1_valid) {
    if (d.f32_slots) {
      std::vector<float2> k32(n);
      for (size_t i = 0; i < n; ++i) k32[i] = make_float2((float)k1[i].x, (float)k1[i].y);
      CK(cudaMemcpy(c->kk[0], k32.data(), n * sizeof(float2), cudaMemcpyHostToDevice), "k1 upload");
    } else {
      CK(cudaMemcpy(c->kk[0], k1.data(), n * sizeof(double2), cudaMemcpyHostToDevice), "k1 upload");
    }
  }
  d.t = h.t; d.h = h.h; d.h_try = h.h_try; d.err = h.err; d.err_prev = h.err_prev; d.rtol = h.rtol; d.atol = h.atol;
  for (int q = 0; q < 4; ++q) d.errc[q] = h.errc[q];
  d.method = h.method; d.k1_valid = h.k1_valid ? 1 : 0; d.after_reject = h.after_reject; d.accepted = h.accepted;
  d.clipped = h.clipped; d.ctrl_kind = h.ctrl_kind; d.hist_n = h.hist_n; d.rej_since = h.rej_since;
  for (int q = 0; q < 5; ++q) { d.hist_rej[q] = h.hist_rej[q]; d.hist_err[q] = h.hist_err[q]; d.hist_h[q] = h.hist_h[q]; }
  d.n_rhs = h.n_rhs; d.n_acc = h.n_acc; d.n_rej = h.n_rej; d.n_attempts = h.n_attempts; d.rejects_in_row = h.rejects_in_row;
  d.parity = 0; d.t_end = h.t; d.done = 1; d.status = 0; d.skip = 0; d.need_k1 = !d.k1_valid; d.trace_n = 0;
  CK(cudaMemcpyAsync(c->ctrl, c->host_ctrl, sizeof(DnsCtrl), cudaMemcpyHostToDevice, c->stream), "ctrl write");
  CK(cudaStreamSynchronize(c->stream), "synchronize");
  c->has_state = true;
  return DNS_OK;
}

}  // extern "C"

namespace {
using TuneKey = std::tuple<int, int, int, int, int>;   // nx, ny, nz, precision, boussinesq
std::mutex g_tune_mu;
std::map<TuneKey, std::pair<int, int>> g_tune;
bool g_tune_loaded = false;

void tune_load_file() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const char* path = std::getenv("DNS_TUNE_CACHE");
  if (!path) return;
  FILE* f = std::fopen(path, "r");
  if (!f) return;
  int v[7];
  while (std::fscanf(f, "%d %d %d %d %d %d %d", &v[0], &v[1], &v[2], &v[3], &v[4], &v[5], &v[6]) == 7)
    g_tune[TuneKey(v[0], v[1], v[2], v[3], v[4])] = {v[5], v[6]};
  std::fclose(f);
}

void tune_save(const TuneKey& k, std::pair<int, int> v) {
  const char* path = std::getenv("DNS_TUNE_CACHE");
  if (!path) return;
  FILE* f = std::fopen(path, "a");
  if (!f) return;
  std::fprintf(f, "%d %d %d %d %d %d %d\n", std::get<0>(k), std::get<1>(k), std::get<2>(k), std::get<3>(k),
               std::get<4>(k), v.first, v.second);
  std::fclose(f);
}
}  // namespace

extern "C" {

dns_status dns_autotune(dns_ctx* c, int reps, int* variants) {
  dns_status s = check_ctx(c);
  if (s != DNS_OK) return s;
  if (reps < 1) reps = 3;
  const TuneKey key(c->g.nx, c->g.ny, c->g.nz, c->precision, c->g.bouss);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_load_file();
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      const int z = it->second.second;
      const int y = it->second.first;
      if (c->var_py != (y & 3) || c->x_tma != ((y & 4) != 0) || c->var_p3 != (z & 1) ||
          c->p3_bulk != !(z & 2) || c->p3_rr != ((z & 4) != 0))
        drop_graphs(c);
      c->var_py = y & 3;
      c->x_tma = (y & 4) != 0;
      c->var_p3 = z & 1;
      c->p3_bulk = !(z & 2);
      c->p3_rr = (z & 4) != 0;
      if (variants) { variants[0] = y; variants[1] = z; }
      return DNS_OK;
    }
  }
  CK(cudaMemsetAsync(c->bufA, 0, c->bytesA, c->stream), "zero");
  CK(cudaMemsetAsync(c->bufB, 0, c->bytesB, c->stream), "zero");
  PassArgs a{};
  a.g = c->g;
  a.ctrl = c->ctrl_rhs;
  a.yslot = SLOT_Y;
  a.kslot = SLOT_K1;
  a.nu = c->nu;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0), "event");
  CK(cudaEventCreate(&e1), "event");
  // y pass: tile variants 0, 1 and, where it applies, 2 (tensor-map tile copies and
  // register-resident transforms, FP32 forms); z pass: codes 0..3 (bit 0 tile variant, bit 1
  // per-element copies instead of bulk copies) and, where it applies, 4 and 5 (the
  // register-resident FP32 kernel with its two tile variants)
  a.p3_rr = 1;
  const bool f32 = c->precision == DNS_FP32_MIXED || c->precision == DNS_FP32;
  const bool rr_ok = f32 && p3_rr_applies(a);
  const bool yb_ok = f32 && ytma_supported(c->g.ny, c->g.Mz);
  // x-inverse pass, where the tensor-map FP32 kernel applies: k_p1 (0) or that one (1)
  a.x_tma = 1;
  a.ycand[0] = c->rhs_in;
  const bool xt_ok = f32 && x_tma_applies(a);
  float best[3][6] = {{0, 0, 1e30f, 1e30f, 1e30f, 1e30f}, {0, 0, 0, 0, 1e30f, 1e30f},
                      {0, 1e30f, 1e30f, 1e30f, 1e30f, 1e30f}};
  for (int which = 0; which < 3; ++which) {        // 0: y pass (P2), 1: z pass (P3), 2: x pass (P1)
    const int nv = which == 0 ? (yb_ok ? 3 : 2) : (which == 1 ? (rr_ok ? 6 : 4) : (xt_ok ? 2 : 0));
    for (int v = 0; v < nv; ++v) {
      a.var_py = which == 0 ? v : 0;
      a.var_p3 = which == 1 ? (v & 1) : 0;
      a.p3_bulk = which == 1 ? !(v & 2) : 1;
      a.p3_rr = which == 1 && (v & 4) != 0;
      a.x_tma = which == 2 && v == 1;
      if (which == 0) { a.in = c->bufA; a.out = c->bufB; a.tw = c->tw[1]; }
      else if (which == 1) { a.in = c->bufB; a.out = c->bufA; a.tw = c->tw[2]; }
      else { a.in = nullptr; a.out = c->bufA; a.tw = c->tw[0]; }   // stage input: the rhs_in slot
      const int pass_id = which == 0 ? 2 : (which == 1 ? 3 : 1);
      CK(pass(c, pass_id, a), "tune launch");
      CK(cudaEventRecord(e0, c->stream), "event");
      for (int r = 0; r < reps; ++r) CK(pass(c, pass_id, a), "tune launch");
      CK(cudaEventRecord(e1, c->stream), "event");
      CK(cudaEventSynchronize(e1), "event sync");
      CK(cudaEventElapsedTime(&best[which][v], e0, e1), "elapsed");
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  drop_graphs(c);
  c->var_py = 0;
  for (int v = 1; v < 3; ++v) if (best[0][v] < best[0][c->var_py]) c->var_py = v;
  c->x_tma = best[2][1] < best[2][0] ? 1 : 0;
  int z = 0;
  for (int v = 1; v < 6; ++v) if (best[1][v] < best[1][z]) z = v;
  c->var_p3 = z & 1;
  c->p3_bulk = !(z & 2);
  c->p3_rr = (z & 4) != 0;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key] = {c->var_py | (c->x_tma ? 4 : 0), z};
    tune_save(key, {c->var_py | (c->x_tma ? 4 : 0), z});
  }
  if (variants) { variants[0] = c->var_py | (c->x_tma ? 4 : 0); variants[1] = z; }
  return DNS_OK;
}

dns_status dns_debug_inject(dns_ctx* c, long long rhs_index) {
  dns_status s = check_ctx(c);
  if (s != DNS_OK) return s;
  CK(launch_ctrl_inject(c->ctrl, rhs_index < 0 ? -1 : rhs_index, c->stream), "inject");
  return DNS_OK;
}

dns_status dns_debug_stall(dns_ctx* c) {
  if (!c) return DNS_ERR_ARG;
  c->stall_pending = true;
  return DNS_OK;
}

dns_status dns_debug_poison(dns_ctx* c, int on) {
  if (!c) return DNS_ERR_ARG;
  if (c->poison != (on != 0)) drop_graphs(c);
  c->poison = on != 0;
  return DNS_OK;
}

dns_status dns_debug_f32_from_f64(const double* x, float* y, long long n, void* stream) {
  if (n < 0 || (n > 0 && (!x || !y))) return DNS_ERR_ARG;
  return launch_f32_from_f64(x, y, n, (cudaStream_t)stream) == cudaSuccess ? DNS_OK : DNS_ERR_CUDA;
}

dns_status dns_set_tiles(dns_ctx* c, int var_py, int var_p3) {
  if (!c || var_py < 0 || var_py > 6 || (var_py & 3) == 3 || var_p3 < 0 || var_p3 > 5) return DNS_ERR_ARG;
  if (c->var_py != (var_py & 3) || c->x_tma != ((var_py & 4) != 0) || c->var_p3 != (var_p3 & 1) ||
      c->p3_bulk != !(var_p3 & 2) || c->p3_rr != ((var_p3 & 4) != 0))
    drop_graphs(c);
  c->var_py = var_py & 3;
  c->x_tma = (var_py & 4) != 0;
  c->var_p3 = var_p3 & 1;
  c->p3_bulk = !(var_p3 & 2);
  c->p3_rr = (var_p3 & 4) != 0;
  return DNS_OK;
}

dns_status dns_query(const dns_ctx* c, int* K3, size_t* device_bytes) {
  if (!c) return DNS_ERR_ARG;
  if (K3) { K3[0] = c->g.Kx; K3[1] = c->g.Ky; K3[2] = c->g.Kz; }
  if (device_bytes) *device_bytes = c->device_bytes;
  return DNS_OK;
}

}  // extern "C"


// ------------------------------------------------------------------------------------------
// Batched ensembles: independent contexts advanced by one graph launch.  The graph holds one
// conditional WHILE node per instance, side by side with no dependencies between them; the
// body of instance i is one attempt of that instance and a kernel that keeps its own loop
// going while it is unfinished (hard cap on its iterations).  The instances loop
// independently: one that has finished, or whose attempts are short, does not wait for the
// others, and the GPU runs the attempts of all unfinished instances concurrently.
// ------------------------------------------------------------------------------------------
struct dns_batch {
  std::vector<dns_ctx*> ctx;
  std::vector<cudaStream_t> streams;   // one capture stream per instance
  cudaStream_t stream = nullptr;       // launch stream
  unsigned long long* d_iter = nullptr;   // per-instance loop counters
  cudaGraphExec_t exec[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  cudaGraph_t graph[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  int device = 0;
  std::string err;
};

extern "C" {

void dns_destroy_batch(dns_batch* b) {
  if (!b) return;
  cudaSetDevice(b->device);
  if (b->stream) cudaStreamSynchronize(b->stream);
  for (int m = 0; m < 5; ++m) {
    if (b->exec[m]) cudaGraphExecDestroy(b->exec[m]);
    if (b->graph[m]) cudaGraphDestroy(b->graph[m]);
  }
  for (dns_ctx* c : b->ctx) dns_destroy(c);
  for (cudaStream_t s : b->streams) if (s) cudaStreamDestroy(s);
  if (b->stream) cudaStreamDestroy(b->stream);
  if (b->d_iter) cudaFree(b->d_iter);
  delete b;
}

dns_status dns_create_batch(int count, const dns_config* cfgs, dns_batch** out) {
  if (!out || !cfgs || count < 1) return DNS_ERR_ARG;
  *out = nullptr;
  dns_batch* b = new dns_batch();
  cudaGetDevice(&b->device);
  dns_status s = DNS_OK;
  for (int i = 0; i < count && s == DNS_OK; ++i) {
    dns_ctx* c = nullptr;
    s = dns_create_ex(&cfgs[i], &c);
    if (s == DNS_OK) b->ctx.push_back(c);
  }
  if (s == DNS_OK) {
    bool ok = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) == cudaSuccess &&
              cudaMalloc((void**)&b->d_iter, count * sizeof(unsigned long long)) == cudaSuccess;
    b->streams.assign(count, nullptr);
    for (int i = 0; ok && i < count; ++i)
      ok = cudaStreamCreateWithFlags(&b->streams[i], cudaStreamNonBlocking) == cudaSuccess;
    for (int i = 0; ok && i < count; ++i) b->ctx[i]->stream = b->stream;
    // tile variants per distinct grid from the autotuner (timed once per shape, cached)
    for (int i = 0; ok && i < count; ++i) ok = dns_autotune(b->ctx[i], 3, nullptr) == DNS_OK;
    if (!ok) { cudaGetLastError(); s = DNS_ERR_CUDA; }
  }
  if (s != DNS_OK) { dns_destroy_batch(b); return s; }
  *out = b;
  return DNS_OK;
}

const char* dns_batch_last_error(const dns_batch* b) { return b ? b->err.c_str() : "null batch"; }

dns_status dns_batch_context(dns_batch* b, int i, dns_ctx** out) {
  if (!b || !out || i < 0 || i >= (int)b->ctx.size()) return DNS_ERR_ARG;
  *out = b->ctx[i];
  return DNS_OK;
}

dns_status dns_integrate_batch(dns_batch* b, int method, const double* t_end, const double* rtol,
                               const double* atol, const double* h0, dns_step_info* info) {
  if (!b || !t_end || !rtol || !atol || !h0 || method < 0 || method > 4) return DNS_ERR_ARG;
  if (cudaSetDevice(b->device) != cudaSuccess) return DNS_ERR_CUDA;
  const int n = (int)b->ctx.size();
  dns_status s;
  for (int i = 0; i < n; ++i) {
    dns_ctx* c = b->ctx[i];
    if ((s = check_ctx(c)) != DNS_OK) { b->err = "instance failed"; return s; }
    if (!c->has_state) { b->err = "instance without state"; return DNS_ERR_STATE; }
    c->stream = b->stream;
    c->prof = false;
    if ((s = config(c, t_end[i], method, rtol[i], atol[i], h0[i], 0)) != DNS_OK) { b->err = c->err; return s; }
  }
  auto cuda = [&](cudaError_t e, const char* what) {
    if (e != cudaSuccess) { b->err = std::string(what) + ": " + cudaGetErrorString(e); return false; }
    return true;
  };
  if (!b->exec[method]) {
    cudaGraph_t g = nullptr;
    if (!cuda(cudaGraphCreate(&g, 0), "graph create")) return DNS_ERR_CUDA;
    bool ok = true;
    for (int i = 0; ok && i < n; ++i) {
      dns_ctx* c = b->ctx[i];
      cudaGraphConditionalHandle handle;
      ok = cuda(cudaGraphConditionalHandleCreate(&handle, g, 1, cudaGraphCondAssignDefault), "conditional handle");
      cudaGraphNodeParams cp = {};
      cp.type = cudaGraphNodeTypeConditional;
      cp.conditional.handle = handle;
      cp.conditional.type = cudaGraphCondTypeWhile;
      cp.conditional.size = 1;
      cudaGraphNode_t node;
      ok = ok && cuda(cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp), "conditional node");
      ok = ok && cuda(cudaStreamBeginCaptureToGraph(b->streams[i], cp.conditional.phGraph_out[0], nullptr, nullptr,
                                                     0, cudaStreamCaptureModeRelaxed), "begin capture");
      if (!ok) break;
      c->stream = b->streams[i];
      c->capturing = true;
      if (enqueue_attempt(c, method) != DNS_OK) { b->err = c->err; ok = false; }
      c->capturing = false;
      if (ok) {
        k_ctx_continue<<<1, 1, 0, b->streams[i]>>>(handle, c->ctrl, b->d_iter + i, 10000000ULL);
        ok = cuda(cudaGetLastError(), "continue kernel");
      }
      c->stream = b->stream;
      cudaGraph_t captured = nullptr;
      ok = cuda(cudaStreamEndCapture(b->streams[i], &captured), "end capture") && ok;
    }
    if (!ok) { cudaGraphDestroy(g); return DNS_ERR_CUDA; }
    if (!cuda(cudaGraphInstantiate(&b->exec[method], g, 0), "instantiate")) { cudaGraphDestroy(g); return DNS_ERR_CUDA; }
    b->graph[method] = g;
  }
  if (!cuda(cudaMemsetAsync(b->d_iter, 0, n * sizeof(unsigned long long), b->stream), "reset counters") ||
      !cuda(cudaGraphLaunch(b->exec[method], b->stream), "graph launch") ||
      !cuda(cudaStreamSynchronize(b->stream), "synchronize"))
    return DNS_ERR_CUDA;
  dns_status worst = DNS_OK;
  for (int i = 0; i < n; ++i) {
    dns_ctx* c = b->ctx[i];
    if ((s = read_ctrl(c)) != DNS_OK) return s;
    if (info) fill_info(c, &info[i]);
    if (c->host_ctrl->status != 0 && worst == DNS_OK) worst = status_from_ctrl(c);
  }
  return worst;
}

}  // extern "C"
