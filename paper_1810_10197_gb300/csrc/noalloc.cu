// dns_rhs_noalloc: the right-hand side of dns_rhs for small grids without any device
// allocation.  Its work space is one file-scope __device__ array that every GPU loading the
// library holds until the process exits (2.3 MB); nothing is allocated per call.
#include <cmath>
#include <mutex>

#include "../../include/dns.h"
#include "common.cuh"
#include "passes.cuh"
#include "stepper.cuh"

using namespace dns;

namespace {

constexpr int kNaMaxN = 32;                         // largest nx, ny, nz accepted
constexpr int kNaK = (kNaMaxN - 1) / 3;             // 2/3-rule cut-off at that size
constexpr int kNaMxy = 2 * kNaK + 1;
constexpr int kNaMz = kNaK + 1;
constexpr long long kNaCompact = 3LL * kNaMxy * kNaMxy * kNaMz;                  // double2
constexpr long long kNaBufA = 6LL * kNaMaxN * kNaMxy * kNaMz;                     // >= 3 nx ny Mz
constexpr long long kNaBufB = 6LL * kNaMaxN * kNaMaxN * kNaMz;                    // >= 3 nx My Mz
constexpr long long kNaTw = 3LL * kNaMaxN;   // >= twiddle_count_z(32) = 17 + 15 and xy counts
constexpr long long kNaCtrl = (sizeof(DnsCtrl) + sizeof(double2) - 1) / sizeof(double2);
// layout in double2 units: in | out | bufA | bufB | tw[3][32] | ctrl
constexpr long long kOffIn = 0, kOffOut = kOffIn + kNaCompact, kOffA = kOffOut + kNaCompact;
constexpr long long kOffB = kOffA + kNaBufA, kOffTw = kOffB + kNaBufB, kOffCtrl = kOffTw + kNaTw;
constexpr long long kNaTotal = kOffCtrl + kNaCtrl;
static_assert(6LL * kNaMaxN * kNaMxy * kNaMz >= 3LL * kNaMaxN * kNaMaxN * kNaMz, "bufA size");

// The shared work space (about 2.3 MB).  Host code must not take the address of this
// symbol directly: its host-side name is only a stand-in.  The device address comes from
// cudaGetSymbolAddress, once per device.
static __device__ __align__(256) double2 g_noalloc_scratch[kNaTotal];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

bool na_size(int n) {
  return n == 8 || n == 12 || n == 16 || n == 24 || n == 32;
}

// Per call: clear the work-space controller record, point it at the work-space fields and
// write the twiddle tables exp(-2 pi i m / n) for the three axes.  The whole record is
// zeroed first, so that every field the passes read (f32_slots among them) is defined by
// this call and not by an earlier one or the array's initial contents.
__global__ void k_na_setup(double2* base, int nx, int ny, int nz) {
  DnsCtrl* c = reinterpret_cast<DnsCtrl*>(base + kOffCtrl);
  static_assert(sizeof(DnsCtrl) % sizeof(unsigned long long) == 0, "controller record size");
  unsigned long long* words = reinterpret_cast<unsigned long long*>(c);
  for (int i = threadIdx.x; i < (int)(sizeof(DnsCtrl) / sizeof(unsigned long long)); i += blockDim.x) words[i] = 0ull;
  __syncthreads();
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    c->slot[SLOT_Y] = base + kOffIn;
    c->slot[SLOT_K1] = base + kOffOut;
    c->skip = 0;
    c->need_k1 = 1;
    c->forcing_coef = 0.0;
    c->inject_rhs = -1;
  }
  const int n3[3] = {nx, ny, nz};
  for (int a = 0; a < 3; ++a) {
    const int cnt = axis_twiddle_count(n3[a], a == 2);
    for (int m = threadIdx.x; m < cnt; m += blockDim.x) {
      int num = 0, den = 1;
      axis_twiddle_turns(n3[a], a == 2, m, &num, &den);
      double s, co;
      sincospi(2.0 * (double)num / (double)den, &s, &co);
      base[kOffTw + a * kNaMaxN + m] = make_double2(co, -s);
    }
  }
}

}  // namespace

extern "C" dns_status dns_rhs_noalloc(int nx, int ny, int nz, double nu, const void* uhat_dev,
                                      void* f_dev, void* stream) {
  if (!na_size(nx) || !na_size(ny) || !na_size(nz)) return DNS_ERR_UNSUPPORTED;
  if (!(nu >= 0.0) || !std::isfinite(nu) || !uhat_dev || !f_dev || uhat_dev == f_dev) return DNS_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return DNS_ERR_CUDA;
  double2* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return DNS_ERR_CUDA;
      }
      g_addr[dev] = p;
    }
    base = reinterpret_cast<double2*>(g_addr[dev]);
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  Geom g{};
  g.nx = nx; g.ny = ny; g.nz = nz; g.nzh = nz / 2 + 1;
  g.Kx = (nx - 1) / 3; g.Ky = (ny - 1) / 3; g.Kz = (nz - 1) / 3;
  g.Mx = 2 * g.Kx + 1; g.My = 2 * g.Ky + 1; g.Mz = g.Kz + 1;
  g.MyMz = g.My * g.Mz;
  g.M = (long long)g.Mx * g.MyMz;
  g.sx = g.sy = g.sz = 1.0;
  g.inv_n3 = 1.0 / ((double)nx * ny * nz);
  g.nmodes_half = (double)nx * ny * g.nzh;
  g.nc = 3;
  g.bouss = 0;
  g.snx = nx; g.sny = ny; g.snz = nz; g.snzh = g.nzh;
  g.fwd_scale = 1.0;
  DnsCtrl* ctrl = reinterpret_cast<DnsCtrl*>(base + kOffCtrl);

  k_na_setup<<<1, 64, 0, s>>>(base, nx, ny, nz);
  if (cudaGetLastError() != cudaSuccess) return DNS_ERR_CUDA;
  if (launch_gather(g, reinterpret_cast<const double2*>(uhat_dev), base + kOffIn, s) != cudaSuccess)
    return DNS_ERR_CUDA;
  PassArgs a{};
  a.g = g;
  a.ctrl = ctrl;
  a.gate_k1 = 0;
  a.yslot = SLOT_Y;
  a.kslot = SLOT_K1;
  a.nu = nu;
  a.kf2 = 0.0;
  void* A = base + kOffA;
  void* B = base + kOffB;
  const double2* tw = base + kOffTw;
  a.out = A; a.tw = tw;
  if (launch_pass<double>(1, a, s) != cudaSuccess) return DNS_ERR_CUDA;
  a.in = A; a.out = B; a.tw = tw + kNaMaxN;
  if (launch_pass<double>(2, a, s) != cudaSuccess) return DNS_ERR_CUDA;
  a.in = B; a.out = A; a.tw = tw + 2 * kNaMaxN;
  if (launch_pass<double>(3, a, s) != cudaSuccess) return DNS_ERR_CUDA;
  a.in = A; a.out = B; a.tw = tw + kNaMaxN;
  if (launch_pass<double>(4, a, s) != cudaSuccess) return DNS_ERR_CUDA;
  a.in = B; a.out = nullptr; a.tw = tw;
  if (launch_pass<double>(5, a, s) != cudaSuccess) return DNS_ERR_CUDA;
  const size_t fbytes = (size_t)3 * nx * ny * g.nzh * sizeof(double2);
  if (cudaMemsetAsync(f_dev, 0, fbytes, s) != cudaSuccess) return DNS_ERR_CUDA;
  if (launch_scatter(g, base + kOffOut, reinterpret_cast<double2*>(f_dev), s) != cudaSuccess)
    return DNS_ERR_CUDA;
  return DNS_OK;
}
