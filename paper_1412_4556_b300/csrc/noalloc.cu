// ara_pml_tvar_noalloc: PML and TVaR without any device allocation.
//
// Who needs it: callers that must not call cudaMalloc/cudaFree -- a service
// whose pooling allocator already holds the device memory it is allowed to
// use, or a latency-critical request path that forbids allocation after
// start-up because cudaMalloc and cudaFree can block on, or synchronise with,
// the whole device.  Such callers may not be able to create a context either
// (ara_create allocates), so this entry point takes none.
//
// The selection workspace lives in one file-scope __device__ array of
// kNoAllocScratchBytes (about 33 KB) that every GPU loading the library holds
// until the process exits.  Host code only sees a host-side stand-in for the
// array's name, so the device address is looked up with
// cudaGetSymbolAddress once per device (on the first call on that device,
// with that device current) and passed to the kernels.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>

#include "ara.h"
#include "ara_internal.cuh"

namespace {

constexpr size_t kOutOffset = ara::kSelectWorkspaceMax;                     // 2*R doubles
constexpr size_t kErrOffset = kOutOffset + 2 * ara::kMaxReturnPeriods * 8;  // one uint
constexpr size_t kNoAllocScratchBytes = kErrOffset + 256;
constexpr int kMaxDevices = 64;

std::mutex g_setup_mutex;
unsigned char *g_scratch_addr[kMaxDevices] = {};

}  // namespace

static __device__ __align__(256) unsigned char g_pml_scratch[kNoAllocScratchBytes];

namespace {

ara_status noalloc_fail(ara_status st, const char *msg) {
  ara::set_context_free_error(msg);
  return st;
}

// Device address of the scratch array on the current device (looked up once).
ara_status scratch_for_current_device(unsigned char **out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return noalloc_fail(ARA_E_CUDA, "ara_pml_tvar_noalloc: no current CUDA device");
  }
  if (dev < 0 || dev >= kMaxDevices)
    return noalloc_fail(ARA_E_CUDA, "ara_pml_tvar_noalloc: device index beyond 63");
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_pml_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return noalloc_fail(ARA_E_CUDA, "ara_pml_tvar_noalloc: cudaGetSymbolAddress of the scratch failed");
    }
    g_scratch_addr[dev] = static_cast<unsigned char *>(p);
  }
  *out = g_scratch_addr[dev];
  return ARA_OK;
}

}  // namespace

extern "C" ara_status ara_pml_tvar_noalloc(const double *ylt, int64_t n, const double *return_periods,
                                           int32_t n_rp, double *pml_out, double *tvar_out,
                                           void *cuda_stream) {
  char msg[256];
  if (n < 1 || !ylt) return noalloc_fail(ARA_E_INVALID_ARG, "ara_pml_tvar_noalloc: need n >= 1 trial losses");
  if (n_rp < 1 || n_rp > ara::kMaxReturnPeriods || !return_periods || !pml_out || !tvar_out) {
    snprintf(msg, sizeof(msg),
             "ara_pml_tvar_noalloc: %d return periods requested; the fixed scratch holds 1..%d",
             (int)n_rp, ara::kMaxReturnPeriods);
    return noalloc_fail(ARA_E_INVALID_ARG, msg);
  }
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return noalloc_fail(ARA_E_CUDA, "ara_pml_tvar_noalloc: no current CUDA device");
  }
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, ylt) != cudaSuccess ||
      (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged)) {
    cudaGetLastError();
    return noalloc_fail(ARA_E_INVALID_ARG,
                        "ara_pml_tvar_noalloc: ylt must be device memory (a host copy would need a buffer)");
  }
  // The selection kernels run on the current device and read ylt directly:
  // another GPU's memory is not readable there, so it is refused before any
  // launch.
  if (attr.type == cudaMemoryTypeDevice && attr.device != dev) {
    snprintf(msg, sizeof(msg),
             "ara_pml_tvar_noalloc: ylt is memory of device %d but the current device is %d", attr.device, dev);
    return noalloc_fail(ARA_E_INVALID_ARG, msg);
  }
  int64_t k[ara::kMaxReturnPeriods];
  for (int32_t r = 0; r < n_rp; ++r) {
    if (!(return_periods[r] >= 1.0))
      return noalloc_fail(ARA_E_INVALID_ARG, "ara_pml_tvar_noalloc: return periods must be >= 1");
    const double kk = std::floor((double)n / return_periods[r]);
    if (kk < 1.0)
      return noalloc_fail(ARA_E_INVALID_ARG, "ara_pml_tvar_noalloc: a return period exceeds the trial count");
    k[r] = (int64_t)kk;
  }
  unsigned char *scratch = nullptr;
  ara_status st = scratch_for_current_device(&scratch);
  if (st != ARA_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  double *d_out = reinterpret_cast<double *>(scratch + kOutOffset);
  unsigned int *d_err = reinterpret_cast<unsigned int *>(scratch + kErrOffset);
  // The array keeps the previous call's contents: the error word is cleared
  // here and the selection state by the first kernel of launch_pml_tvar.
  cudaError_t e = cudaMemsetAsync(d_err, 0, sizeof(unsigned int), s);
  if (e == cudaSuccess) e = ara::launch_pml_tvar(ylt, n, k, n_rp, scratch, d_out, d_err, dev, s);
  unsigned int bad = 0;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(pml_out, d_out, (size_t)n_rp * sizeof(double), cudaMemcpyDefault, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(tvar_out, d_out + n_rp, (size_t)n_rp * sizeof(double), cudaMemcpyDefault, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, d_err, sizeof(bad), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    snprintf(msg, sizeof(msg), "ara_pml_tvar_noalloc: %s", cudaGetErrorString(e));
    cudaGetLastError();
    return noalloc_fail(e == cudaErrorMemoryAllocation ? ARA_E_NOMEM : ARA_E_CUDA, msg);
  }
  if (bad) return noalloc_fail(ARA_E_INVALID_ARG, "ara_pml_tvar_noalloc: trial losses must be finite and >= 0");
  return ARA_OK;
}
