// eps_vjp_static: the fused forward + adjoint call of eps_vjp, for callers
// that cannot hand the library a device workspace.
//
// Some host programs cannot allocate device memory at the point where they
// need the gradient: a framework whose memory pool has already reserved the
// whole device leaves no room for a separate cudaMalloc, and a real-time
// optimisation loop may forbid allocations after start-up because
// cudaMalloc/cudaFree can synchronise the device and take milliseconds.
// This entry point allocates nothing.  Its scratch is one file-scope device
// array of EPS_STATIC_WS_BYTES, created when the library's device code is
// loaded on a GPU and kept by that GPU until the process exits.
#include <cstdint>
#include <mutex>

#include "epschain.h"

// Scratch shared by every call of eps_vjp_static on a given device.
static __device__ __align__(256) unsigned char g_eps_static_ws[EPS_STATIC_WS_BYTES];

namespace {

constexpr int MAX_DEVICES = 64;
std::mutex g_static_mu;
void *g_static_addr[MAX_DEVICES];   // device address of the array, per device

// Device address of the scratch array on the current device.  The host-side
// name of a __device__ array is only a stand-in, so the address is looked up
// once per device with that device current and cached for the rest of the
// process (valid in the device's primary context; a cudaDeviceReset() would
// leave a stale entry, which the header rules out).
eps_status_t static_scratch(void **out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return EPS_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!g_static_addr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_eps_static_ws) != cudaSuccess || !p) return EPS_ERR_CUDA;
    g_static_addr[dev] = p;
  }
  *out = g_static_addr[dev];
  return EPS_OK;
}

}  // namespace

extern "C" eps_status_t eps_vjp_static(const eps_problem_t *prob, const float *C, int32_t n_lambda,
                                       int32_t field_type, const void *const *EF,
                                       const void *const *EA, const float *field_scales,
                                       float scale, float *dJdC, float *eps_out,
                                       eps_stream_t stream) {
  size_t need = 0;
  eps_status_t st = eps_workspace_size(prob, n_lambda, &need);
  if (st != EPS_OK) return st;
  if (need > (size_t)EPS_STATIC_WS_BYTES) return EPS_ERR_WORKSPACE;
  void *ws = nullptr;
  if ((st = static_scratch(&ws)) != EPS_OK) return st;
  // every scratch element the kernels read is written earlier in the same
  // call, so the array needs no clearing between calls
  return eps_vjp(prob, C, n_lambda, field_type, EF, EA, field_scales, scale, dJdC, eps_out, ws,
                 (size_t)EPS_STATIC_WS_BYTES, stream);
}
