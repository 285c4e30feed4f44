// static_workspace.cu -- qmc_integrate_static: batched integration for callers
// that cannot allocate device memory.
//
// Some callers cannot provide a workspace: a plug-in running inside a host
// application that owns every byte of GPU memory, a real-time frame loop where
// cudaMalloc's implicit device synchronisation would stall the frame, or code
// that must run under a fixed memory budget decided at start-up.  For them this
// file keeps the integration scratch in a fixed device array that exists on
// every GPU that loads the library and stays there until the process exits.
//
// Host code cannot use the array's name as a device address (in host code it is
// only a stand-in symbol), so the first call on each device looks the address
// up with cudaGetSymbolAddress while that device is current and caches it.
// That lookup is also what makes the runtime load this file's device code, and
// with it place the array, on a device whose modules load lazily; a call with
// no integrals does only that, so callers can do it at start-up.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "../../include/qmc.h"
#include "qmc_host.h"

namespace {

// The scratch shared by every qmc_integrate_static call on a device.
static __device__ __align__(256) unsigned char g_static_workspace[QMC_STATIC_WORKSPACE_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_address_mutex;
void* g_address[kMaxDevices];  // device address of g_static_workspace, per device id

qmc_status static_workspace_address(void** out) {
  int dev = -1;
  const cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return qmc::cuda_status(e);
  if (dev < 0 || dev >= kMaxDevices) return qmc::cuda_status(cudaErrorInvalidDevice);
  std::lock_guard<std::mutex> lock(g_address_mutex);
  if (!g_address[dev]) {
    void* p = nullptr;
    const cudaError_t es = cudaGetSymbolAddress(&p, g_static_workspace);
    if (es != cudaSuccess) return qmc::cuda_status(es);
    if (p == nullptr) return qmc::cuda_status(cudaErrorInvalidSymbol);
    g_address[dev] = p;
  }
  *out = g_address[dev];
  return QMC_OK;
}

}  // namespace

extern "C" qmc_status qmc_integrate_static(const qmc_problem* p, uint32_t n_integrals,
                                           const uint32_t* d_counts, const float* d_theta,
                                           double* d_estimate, qmc_stream_t stream) {
  if (!p || p->max_count == 0) return QMC_ERR_INVALID_ARG;
  // Worst-case forward workspace for counts <= max_count (sized for the smallest
  // chunk the library may pick, so it covers the chunk actually used).
  qmc_problem forward = *p;
  forward.with_gradient = 0;
  const size_t need = qmc_integrate_workspace_bytes(&forward, n_integrals, nullptr);
  if (need == 0) return QMC_ERR_INVALID_ARG;
  if (need > (size_t)QMC_STATIC_WORKSPACE_BYTES) return QMC_ERR_WORKSPACE;
  if (qmc::launch_fault_injected()) return qmc::injected_fault();
  void* ws = nullptr;
  const qmc_status st = static_workspace_address(&ws);
  if (st != QMC_OK || n_integrals == 0) return st;  // no integrals: the start-up call
  return qmc_integrate(p, n_integrals, d_counts, d_theta, d_estimate, ws,
                       (size_t)QMC_STATIC_WORKSPACE_BYTES, stream);
}
