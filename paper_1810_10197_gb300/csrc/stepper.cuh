// Kernels around the right-hand side: Runge-Kutta stage sums, the embedded error norm, the
// device-resident step controller, half-spectrum <-> retained-box copies, diagnostics.
#pragma once

#include "common.cuh"

namespace dns {

constexpr int kMaxTerms = 8;
constexpr int kRedBlocks = 1216;   // 8 x 152 SMs: partial sums of the error norm / diagnostics
constexpr int kRedThreads = 256;

struct StageArgs {
  const DnsCtrl* ctrl;
  int gate_k1;
  int nterms;
  int kslot[kMaxTerms];
  double coef[kMaxTerms];
  int uslot, yslot;
  long long n2;          // complex elements per field set (3 M)
  int f32;               // 1: increment formed in FP32, k read as FP32 (fp32 form)
};

struct ErrArgs {
  const DnsCtrl* ctrl;
  int nterms;
  int kslot[kMaxTerms];
  double coef[kMaxTerms];   // b_j - bhat_j
  long long M;              // modes per component
  int nc;                   // state components (3 or 4)
  double* partials;         // [kRedBlocks][4]
  int f32;                  // 1: e, sc and the ratio in FP32, k read as FP32 (fp32 form)
};

// Host launchers (stepper.cu).  All enqueue on stream s and return the launch status.
cudaError_t launch_stage_sum(const StageArgs& a, cudaStream_t s);
cudaError_t launch_err_partials(const ErrArgs& a, cudaStream_t s);
cudaError_t launch_f32_from_f64(const double* x, float* y, long long n, cudaStream_t s);
cudaError_t launch_begin_attempt(DnsCtrl* c, int method, cudaStream_t s);
cudaError_t launch_controller(DnsCtrl* c, const double* partials, int method, int nstages,
                              double nmodes, int nc, cudaStream_t s);
cudaError_t launch_ctrl_reset(DnsCtrl* c, double t, cudaStream_t s);
cudaError_t launch_ctrl_inject(DnsCtrl* c, long long rhs_index, cudaStream_t s);
cudaError_t launch_trace_diag(const Geom& g, DnsCtrl* c, double* partials, int method, cudaStream_t s);
cudaError_t launch_ctrl_set_controller(DnsCtrl* c, int kind, const float* mlp, cudaStream_t s);
cudaError_t launch_ctrl_set_trace(DnsCtrl* c, double* trace, long long cap, int diag, cudaStream_t s);
cudaError_t launch_ctrl_config(DnsCtrl* c, double t_end, int method, double rtol, double atol,
                               double h0, int max_rejects, cudaStream_t s);
cudaError_t launch_gather(const Geom& g, const double2* full, double2* compact, cudaStream_t s);
cudaError_t launch_scatter(const Geom& g, const double2* compact, double2* full, cudaStream_t s);
cudaError_t launch_copy_slot(DnsCtrl* c, int slot, double2* dst, long long n2, cudaStream_t s);
cudaError_t launch_forcing_coef(const Geom& g, DnsCtrl* c, int yslot, double kf, double power,
                                int gate_k1, cudaStream_t s);
// band rescale forcing after an accepted step (partials: kRedBlocks x kRedStride scratch)
cudaError_t launch_rescale(const Geom& g, DnsCtrl* c, double* partials, double kf, cudaStream_t s);
constexpr int kRedStride = 4;      // partial sums per block (components)
// energy spectrum: partials[152][nshell] doubles of scratch, out[nshell]
cudaError_t launch_spectrum(const Geom& g, const double2* u, double* partials, int nshell, double* out,
                            cudaStream_t s);
cudaError_t launch_diag_partials(const Geom& g, const double2* u, const double2* f,
                                 double* partials, cudaStream_t s);

}  // namespace dns
