// qmc_host.h -- host-side error reporting, fault injection and NVTX ranges
// shared by the entry points of libqmc_gb300.so (api.cu, runtime.cu,
// static_workspace.cu); no kernel includes it.
#pragma once

#include <cuda_runtime.h>

#include "../../include/qmc.h"

namespace qmc {

// QMC_OK for cudaSuccess; otherwise records e as the calling thread's last CUDA
// error (qmc_last_cuda_error) and returns QMC_ERR_CUDA.
qmc_status cuda_status(cudaError_t e);
// True when QMC_FAULT_INJECT=launch is set: entry points then fail their launch
// on the host, recording QMC_INJECTED_FAULT, and enqueue nothing.
bool launch_fault_injected();
qmc_status injected_fault();

// An NVTX range in the "qmc" domain for the lifetime of the object.
class NvtxRange {
 public:
  explicit NvtxRange(const char* name);
  ~NvtxRange();
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Runs launch() (returning a cudaError_t) inside an NVTX range named `name`,
// unless a launch fault is injected; maps the result to a qmc_status.
template <class F>
qmc_status enqueue(const char* name, F&& launch) {
  if (launch_fault_injected()) return injected_fault();
  const NvtxRange range(name);
  return cuda_status(launch());
}

}  // namespace qmc
