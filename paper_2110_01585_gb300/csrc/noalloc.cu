// Prior-site pass that allocates nothing.
//
// Some callers cannot call cudaMalloc at the point where they run a sweep:
// code that must not allocate after start-up (real-time loops, fixed memory
// budgets), allocators that own the whole device and hand out only the buffers
// they were asked for, or plug-ins whose host does not let them touch the
// device allocator.  They pass in every input and output buffer; the only
// scratch this pass needs (one FP64 partial sum of E|u| per work unit, a status
// word and counters) lives in the file-scope array below, of fixed size.
//
// Every GPU that loads the library holds this array until the process exits.
// All calls on a device share it and it keeps the last call's contents, so
// calls that overlap on the GPU (different streams, or host threads) race on
// it; serialise them.  The first call on a device looks up the array's device
// address with that device current; make that first call before any stream
// capture begins, and do not use the entry point across cudaDeviceReset: the
// cached address belongs to the context it was looked up in.
#include <cuda_runtime.h>
#include <string.h>

#include <mutex>

#include "internal.cuh"

namespace eptv {
namespace {

// One work unit is 16 row pairs of a 60-column strip, so 65536 units hold images
// of up to about 65536 * 32 * 60 = 126 M pixels.
constexpr int kNoAllocMaxBlocks = 65536;
constexpr int kNoAllocDoubles = kNoAllocMaxBlocks + 8;
constexpr int kMaxDevices = 64;

// [0, kNoAllocMaxBlocks): per-unit partial sums of E|u|
// [kNoAllocMaxBlocks + DS_*]: FP64 scalars written by the reduction
// [kNoAllocMaxBlocks + 4, +8): status word and counters (bytes reinterpreted)
static __device__ __align__(256) double g_scratch[kNoAllocDoubles];

std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of g_scratch on the current device (looked up once per device).
void* scratch_address(ep_tv_status* st) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    *st = EP_TV_ERR_CUDA;
    return nullptr;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_scratch) != cudaSuccess || !ptr) {
      *st = EP_TV_ERR_CUDA;
      return nullptr;
    }
    g_addr[dev] = ptr;
  }
  *st = EP_TV_OK;
  return g_addr[dev];
}

}  // namespace
}  // namespace eptv

using namespace eptv;

extern "C" ep_tv_status ep_tv_prior_sweep_noalloc(int32_t height, int32_t width,
                                                  const ep_tv_params* p, const double* beta,
                                                  const float* y, const float* tau0,
                                                  const float* nu0, const float* tau_in,
                                                  const float* nu_in, float* tau_out, float* nu_out,
                                                  const int8_t* k_order, double* abar_out,
                                                  uint32_t* flags_out, void* cuda_stream) {
  if (!p || !beta || !tau_in || !nu_in || !tau_out || !nu_out || !abar_out) return EP_TV_ERR_ARG;
  if (height < 1 || width < 1) return EP_TV_ERR_ARG;
  if ((long long)height * width > (1ll << 31)) return EP_TV_ERR_ARG;
  if (!y && (!tau0 || !nu0)) return EP_TV_ERR_ARG;
  if (p->precision != 0 && p->precision != 1) return EP_TV_ERR_ARG;
  if (!prior_params_ok(p)) return EP_TV_ERR_ARG;
  if (p->periodic != 0 && p->periodic != 1) return EP_TV_ERR_ARG;
  if (p->periodic && ((height % 2) || (width % 2))) return EP_TV_ERR_ARG;
  if (!(p->damping > 0.0 && p->damping <= 1.0) || !(p->var_cap > 0.0)) return EP_TV_ERR_ARG;
  if (y && !(p->xi > 0.0)) return EP_TV_ERR_ARG;
  if (tau_in == tau_out || nu_in == nu_out) return EP_TV_ERR_ARG;
  // Work units in 64-bit: ceil(width / 60) * ceil(((height + 1) / 2 + 1) / 16), the
  // count prior_sweep_blocks returns, without its int overflow for huge sizes.
  const long long units = ((long long)width + 59) / 60 * ((((long long)height + 1) / 2 + 1 + 15) / 16);
  if (units > kNoAllocMaxBlocks) return EP_TV_ERR_ARG;  // image larger than the fixed scratch
  const int nblk = prior_sweep_blocks(height, width);
  if (nblk != units) return EP_TV_ERR_ARG;
  int order = 0x4321;
  if (k_order) {
    int seen = 0;
    order = 0;
    for (int u = 0; u < 4; ++u) {
      const int k = k_order[u];
      if (k < 1 || k > 4 || (seen & (1 << k))) return EP_TV_ERR_ARG;
      seen |= 1 << k;
      order |= k << (4 * u);
    }
  }
  ep_tv_status st;
  double* scratch = (double*)scratch_address(&st);
  if (!scratch) return st;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  double* dscal = scratch + kNoAllocMaxBlocks;
  unsigned* status = (unsigned*)(dscal + 4);
  unsigned long long* counters = (unsigned long long*)(dscal + 5);
  // status and counters start at zero on every call; the partial sums are all
  // overwritten by the pass itself
  if (cudaMemsetAsync(dscal + 4, 0, 4 * sizeof(double), s) != cudaSuccess) return EP_TV_ERR_CUDA;
  SweepArgs a;
  a.tau0 = tau0;
  a.nu0 = nu0;
  a.tin = tau_in;
  a.nin = nu_in;
  a.tout = tau_out;
  a.nout = nu_out;
  a.y = y;
  a.inv_xi = y ? (float)(1.0 / p->xi) : 0.f;
  a.height = height;
  a.width = width;
  a.n = (long long)height * width;
  a.periodic = p->periodic;
  a.periodic_rows = p->periodic;
  a.count_lo = 0;
  a.count_hi = height;
  a.damping = (float)p->damping;
  a.min_tau = (float)(1.0 / p->var_cap);
  a.beta = beta;
  a.order = order;
  a.fp64_tail = p->precision == 0;
  set_prior_args(a, p);
  a.abar_partial = scratch;
  a.status = status;
  a.counters = counters;
  launch_prior_sweep(a, y != nullptr, s);
  launch_abar_reduce(scratch, nblk, dscal, (double)a.n, 0, s);
  if (cudaMemcpyAsync(abar_out, dscal + DS_ABAR, sizeof(double), cudaMemcpyDeviceToDevice, s) !=
      cudaSuccess)
    return EP_TV_ERR_CUDA;
  if (flags_out &&
      cudaMemcpyAsync(flags_out, status, sizeof(unsigned), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return EP_TV_ERR_CUDA;
  return cudaGetLastError() == cudaSuccess ? EP_TV_OK : EP_TV_ERR_CUDA;
}
