// runtime.cu -- host runtime around the integration kernels: an autotuner for
// the work split (samples per work item, threads per CTA) with a process-wide
// cache consulted by later calls, and CUDA-graph capture of qmc_* call sequences
// so that a batched integration replays as one graph launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "../../include/qmc.h"
#include "qmc_internal.h"

namespace qmc {
namespace {

// A problem class: results of one tuning run apply to every later call of the
// same class on the same device.
using TuneKey = std::tuple<int, uint32_t, uint32_t, uint32_t, uint32_t, uint32_t, uint32_t, uint32_t>;

std::mutex g_tune_mutex;
std::map<TuneKey, std::pair<uint32_t, uint32_t>> g_tuned;  // -> (chunk, block)

uint32_t size_class(uint32_t n) {
  uint32_t c = 0;
  while (c < 32 && (1u << c) < n) ++c;
  return c;  // ceil(log2 n)
}

TuneKey make_key(const qmc_problem* p, uint32_t n, bool grad) {
  int dev = 0;
  cudaGetDevice(&dev);
  const uint32_t scr = p->d_seeds ? p->randomize : 0u;
  return TuneKey{dev, p->source, p->integrand, p->s, scr, p->seeds_per_integral, grad ? 1u : 0u, size_class(n)};
}

}  // namespace

bool tuned_lookup(const qmc_problem* p, uint32_t n, bool grad, uint32_t* chunk, uint32_t* block) {
  const TuneKey k = make_key(p, n, grad);
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  auto it = g_tuned.find(k);
  if (it == g_tuned.end()) return false;
  *chunk = it->second.first;
  *block = it->second.second;
  return true;
}

}  // namespace qmc

using namespace qmc;

struct qmc_graph_st {
  cudaGraph_t graph;
  cudaGraphExec_t exec;
};

extern "C" {

qmc_status qmc_tune_integrate(const qmc_problem* p, uint32_t n_integrals, const uint32_t* d_counts,
                              const float* d_theta, const double* d_target, double* d_estimate,
                              float* d_grad_theta, double* d_loss, void* d_workspace,
                              size_t workspace_bytes, qmc_stream_t stream, qmc_tuning* h_best) {
  if (!p || !h_best || !d_estimate || n_integrals == 0) return QMC_ERR_INVALID_ARG;
  const bool grad = d_grad_theta != nullptr;
  if (grad && (!d_target || !d_loss)) return QMC_ERR_INVALID_ARG;
  static const uint32_t kChunks[] = {1024, 2048, 4096, 8192};
  static const uint32_t kBlocks[] = {128, 256};
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return QMC_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return QMC_ERR_CUDA;
  }
  qmc_tuning best{0, 0, 0.0f};
  qmc_status status = QMC_OK;
  for (uint32_t chunk : kChunks) {
    for (uint32_t block : kBlocks) {
      qmc_problem q = *p;
      q.chunk = chunk;
      q.block = block;
      auto run = [&]() -> qmc_status {
        return grad ? qmc_integrate_fwd_bwd(&q, n_integrals, d_counts, d_theta, d_target, d_estimate, d_grad_theta,
                                            d_loss, d_workspace, workspace_bytes, stream)
                    : qmc_integrate(&q, n_integrals, d_counts, d_theta, d_estimate, d_workspace,
                                    workspace_bytes, stream);
      };
      if ((status = run()) != QMC_OK) break;  // warm-up (also validates the split)
      std::vector<float> times;
      for (int rep = 0; rep < 3 && status == QMC_OK; ++rep) {
        cudaEventRecord(e0, s);
        status = run();
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) status = QMC_ERR_CUDA;
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        times.push_back(ms);
      }
      if (status != QMC_OK) break;
      std::sort(times.begin(), times.end());
      const float ms = times[times.size() / 2];
      if (best.chunk == 0 || ms < best.ms) best = qmc_tuning{chunk, block, ms};
    }
    if (status != QMC_OK) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (status != QMC_OK) return status;
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tuned[make_key(p, n_integrals, grad)] = {best.chunk, best.block};
  }
  *h_best = best;
  return QMC_OK;
}

qmc_status qmc_tune_clear(void) {
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  g_tuned.clear();
  return QMC_OK;
}

qmc_status qmc_graph_begin(qmc_stream_t stream) {
  if (!stream) return QMC_ERR_INVALID_ARG;  // the legacy default stream cannot be captured
  return cudaStreamBeginCapture((cudaStream_t)stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess
             ? QMC_OK
             : QMC_ERR_CUDA;
}

qmc_status qmc_graph_end(qmc_stream_t stream, qmc_graph_t* out_graph) {
  if (!stream || !out_graph) return QMC_ERR_INVALID_ARG;
  cudaGraph_t graph = nullptr;
  if (cudaStreamEndCapture((cudaStream_t)stream, &graph) != cudaSuccess || !graph) return QMC_ERR_CUDA;
  cudaGraphExec_t exec = nullptr;
  if (cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
    cudaGraphDestroy(graph);
    return QMC_ERR_CUDA;
  }
  *out_graph = new qmc_graph_st{graph, exec};
  return QMC_OK;
}

qmc_status qmc_graph_launch(qmc_graph_t graph, qmc_stream_t stream) {
  if (!graph) return QMC_ERR_INVALID_ARG;
  return cudaGraphLaunch(graph->exec, (cudaStream_t)stream) == cudaSuccess ? QMC_OK : QMC_ERR_CUDA;
}

qmc_status qmc_graph_destroy(qmc_graph_t graph) {
  if (!graph) return QMC_ERR_INVALID_ARG;
  cudaGraphExecDestroy(graph->exec);
  cudaGraphDestroy(graph->graph);
  delete graph;
  return QMC_OK;
}

}  // extern "C"
