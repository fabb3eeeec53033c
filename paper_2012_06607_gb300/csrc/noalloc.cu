// Allocation-free variant of the block Toeplitz solve (md_linsolve_series).
//
// Some callers cannot allocate device memory for a workspace: applications
// whose device memory is owned by another allocator or pre-reserved to the
// last byte, latency-critical code where cudaMalloc / cudaFree would
// synchronise the device, and plug-in or callback contexts that forbid
// allocation.  This entry point takes only inputs and outputs.  Its scratch
// space is a file-scope device array of MD_STATIC_WS_BYTES that lives in the
// library's own module: every GPU that loads the module holds it until the
// process exits.  With lazy module loading the module, and so the array, is
// loaded on a device at its first use there, which may be the first call of
// this entry point.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/mdnewton.h"

// The scratch array.  In host code this name is only a host-side stand-in for
// the symbol; its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_md_static_ws[MD_STATIC_WS_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
void *g_static_addr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device, looked up once
// per device with that device current and kept: it is the address in the
// context current at that first call (the runtime's primary context).
md_status static_ws_address(void **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MD_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!g_static_addr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_md_static_ws) != cudaSuccess || p == nullptr) return MD_ERR_CUDA;
    g_static_addr[dev] = p;
  }
  *out = g_static_addr[dev];
  return MD_OK;
}

}  // namespace

extern "C" md_status md_linsolve_series_static(int limbs, int is_complex, int n, int degree, const double *A,
                                               const double *b, double *dx, int flags, void *stream) {
  const size_t need = md_linsolve_workspace_bytes(limbs, is_complex, n, degree, flags);
  if (need == 0 || !A || !b || !dx) return MD_ERR_ARG;
  if (need > (size_t)MD_STATIC_WS_BYTES) return MD_ERR_WORKSPACE;
  void *ws = nullptr;
  const md_status st = static_ws_address(&ws);
  if (st != MD_OK) return st;
  return md_linsolve_series(limbs, is_complex, n, degree, A, b, dx, ws, (size_t)MD_STATIC_WS_BYTES, flags, stream);
}
