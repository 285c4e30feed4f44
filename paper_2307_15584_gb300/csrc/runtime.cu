// runtime.cu -- host runtime around the integration kernels: an autotuner for
// the work split (samples per work item, threads per CTA) with a process-wide
// cache consulted by later calls and, optionally, kept in a JSON file across
// processes (QMC_AUTOTUNE_CACHE); and CUDA-graph capture of qmc_* call
// sequences so that a batched integration replays as one graph launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/qmc.h"
#include "qmc_host.h"
#include "qmc_internal.h"

namespace qmc {
namespace {

// A problem class: results of one tuning run apply to every later call of the
// same class on a device of the same kind (name and SM count, so that a cache
// file written on one GPU model is not applied to another).
struct TuneKey {
  std::string device;
  uint32_t sms, source, integrand, s, randomize, per_integral, grad, size_class;
  bool operator<(const TuneKey& o) const {
    return std::tie(device, sms, source, integrand, s, randomize, per_integral, grad, size_class) <
           std::tie(o.device, o.sms, o.source, o.integrand, o.s, o.randomize, o.per_integral, o.grad,
                    o.size_class);
  }
};

std::mutex g_tune_mutex;
std::map<TuneKey, std::pair<uint32_t, uint32_t>> g_tuned;  // -> (chunk, block)

uint32_t size_class(uint32_t n) {
  uint32_t c = 0;
  while (c < 32 && (1u << c) < n) ++c;
  return c;  // ceil(log2 n)
}

// Name and SM count of the current device ("" and 0 when there is none).
std::pair<std::string, uint32_t> device_identity() {
  static std::mutex mu;
  static std::map<int, std::pair<std::string, uint32_t>> cache;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return {"", 0u};
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find(dev);
  if (it != cache.end()) return it->second;
  cudaDeviceProp prop{};
  std::pair<std::string, uint32_t> id{"", 0u};
  if (cudaGetDeviceProperties(&prop, dev) == cudaSuccess) id = {prop.name, (uint32_t)prop.multiProcessorCount};
  cache[dev] = id;
  return id;
}

TuneKey make_key(const qmc_problem* p, uint32_t n, bool grad) {
  const auto id = device_identity();
  const uint32_t scr = p->d_seeds ? p->randomize : 0u;
  return TuneKey{id.first, id.second, p->source, p->integrand, p->s, scr, p->seeds_per_integral,
                 grad ? 1u : 0u, size_class(n)};
}

bool split_ok(uint32_t chunk, uint32_t block) {
  return chunk >= 32 && chunk <= 8192 && (chunk & (chunk - 1)) == 0 && block >= 32 && block <= 256 &&
         block % 32 == 0;
}

// --- the cache file: a small JSON document, one object per tuned class ----------------
const char* const kFields[] = {"sms", "source", "integrand", "s", "randomize",
                               "seeds_per_integral", "gradient", "size_class", "chunk", "block"};
constexpr int kNumFields = 10;

qmc_status save_locked(const char* path) {
  const std::string tmp = std::string(path) + ".tmp";
  FILE* f = std::fopen(tmp.c_str(), "w");
  if (!f) return QMC_ERR_IO;
  std::fprintf(f, "{\n \"qmc_autotune_cache\": 1,\n \"entries\": [");
  bool first = true;
  for (const auto& kv : g_tuned) {
    const TuneKey& k = kv.first;
    std::string name;
    for (char c : k.device)
      if (c != '"' && c != '\\' && (unsigned char)c >= 32) name += c;
    std::fprintf(f,
                 "%s\n  {\"device\": \"%s\", \"sms\": %u, \"source\": %u, \"integrand\": %u, \"s\": %u, "
                 "\"randomize\": %u, \"seeds_per_integral\": %u, \"gradient\": %u, \"size_class\": %u, "
                 "\"chunk\": %u, \"block\": %u}",
                 first ? "" : ",", name.c_str(), k.sms, k.source, k.integrand, k.s, k.randomize,
                 k.per_integral, k.grad, k.size_class, kv.second.first, kv.second.second);
    first = false;
  }
  std::fprintf(f, "\n ]\n}\n");
  const bool ok = std::fflush(f) == 0;
  std::fclose(f);
  if (!ok || std::rename(tmp.c_str(), path) != 0) {
    std::remove(tmp.c_str());
    return QMC_ERR_IO;
  }
  return QMC_OK;
}

// Parses the objects of the "entries" array: string "device", unsigned integer
// fields; objects with a missing field, a value out of range or an invalid
// split are skipped.  Returns the number of entries taken.
uint32_t parse_entries(const std::string& text) {
  size_t pos = text.find("\"entries\"");
  if (pos == std::string::npos) return 0;
  uint32_t taken = 0;
  while ((pos = text.find('{', pos)) != std::string::npos) {
    const size_t end = text.find('}', pos);
    if (end == std::string::npos) break;
    const std::string obj = text.substr(pos + 1, end - pos - 1);
    pos = end + 1;
    std::string device;
    bool have_device = false;
    uint64_t v[kNumFields];
    bool have[kNumFields] = {};
    size_t q = 0;
    while ((q = obj.find('"', q)) != std::string::npos) {
      const size_t ke = obj.find('"', q + 1);
      if (ke == std::string::npos) break;
      const std::string key = obj.substr(q + 1, ke - q - 1);
      size_t c = obj.find(':', ke);
      if (c == std::string::npos) break;
      ++c;
      while (c < obj.size() && (obj[c] == ' ' || obj[c] == '\t' || obj[c] == '\n' || obj[c] == '\r')) ++c;
      if (c < obj.size() && obj[c] == '"') {
        const size_t ve = obj.find('"', c + 1);
        if (ve == std::string::npos) break;
        if (key == "device") {
          device = obj.substr(c + 1, ve - c - 1);
          have_device = true;
        }
        q = ve + 1;
        continue;
      }
      uint64_t x = 0;
      size_t d = c;
      while (d < obj.size() && obj[d] >= '0' && obj[d] <= '9' && x <= 0xFFFFFFFFull) x = x * 10 + (uint64_t)(obj[d++] - '0');
      const bool number = d > c && x <= 0xFFFFFFFFull;
      for (int i = 0; i < kNumFields; ++i)
        if (number && key == kFields[i]) v[i] = x, have[i] = true;
      q = d > c ? d : c;
    }
    bool complete = have_device;
    for (int i = 0; i < kNumFields; ++i) complete = complete && have[i];
    if (!complete || !split_ok((uint32_t)v[8], (uint32_t)v[9]) || v[6] > 1 || v[5] > 1 || v[7] > 32) continue;
    const TuneKey k{device, (uint32_t)v[0], (uint32_t)v[1], (uint32_t)v[2], (uint32_t)v[3],
                    (uint32_t)v[4], (uint32_t)v[5], (uint32_t)v[6], (uint32_t)v[7]};
    g_tuned[k] = {(uint32_t)v[8], (uint32_t)v[9]};
    ++taken;
  }
  return taken;
}

qmc_status load_locked(const char* path, uint32_t* loaded) {
  FILE* f = std::fopen(path, "r");
  if (!f) return QMC_ERR_IO;
  std::string text;
  char buf[4096];
  size_t n;
  while ((n = std::fread(buf, 1, sizeof buf, f)) > 0) text.append(buf, n);
  const bool bad = std::ferror(f) != 0;
  std::fclose(f);
  if (bad) return QMC_ERR_IO;
  const uint32_t k = parse_entries(text);
  if (loaded) *loaded = k;
  return QMC_OK;
}

// QMC_AUTOTUNE_CACHE: read once, before the first lookup or tuning in the process.
const char* cache_path() {
  const char* p = std::getenv("QMC_AUTOTUNE_CACHE");
  return (p && *p) ? p : nullptr;
}

void load_env_cache_locked() {
  static bool done = false;
  if (done) return;
  done = true;
  if (const char* path = cache_path()) load_locked(path, nullptr);  // a missing file is an empty cache
}

}  // namespace

bool tuned_lookup(const qmc_problem* p, uint32_t n, bool grad, uint32_t* chunk, uint32_t* block) {
  const TuneKey k = make_key(p, n, grad);
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  load_env_cache_locked();
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
  if (launch_fault_injected()) return injected_fault();
  static const uint32_t kChunks[] = {1024, 2048, 4096, 8192};
  static const uint32_t kBlocks[] = {128, 256};
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  cudaError_t ce = cudaEventCreate(&e0);
  if (ce != cudaSuccess) return cuda_status(ce);
  if ((ce = cudaEventCreate(&e1)) != cudaSuccess) {
    cudaEventDestroy(e0);
    return cuda_status(ce);
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
        const cudaError_t se = cudaEventSynchronize(e1);
        if (se != cudaSuccess) status = cuda_status(se);
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
    const TuneKey key = make_key(p, n_integrals, grad);
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    load_env_cache_locked();
    g_tuned[key] = {best.chunk, best.block};
    // a cache file that cannot be written leaves the result in memory only
    if (const char* path = cache_path()) save_locked(path);
  }
  *h_best = best;
  return QMC_OK;
}

qmc_status qmc_tune_clear(void) {
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  g_tuned.clear();
  return QMC_OK;
}

qmc_status qmc_tune_save(const char* path) {
  if (!path || !*path) return QMC_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  return save_locked(path);
}

qmc_status qmc_tune_load(const char* path, uint32_t* h_loaded) {
  if (!path || !*path) return QMC_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  return load_locked(path, h_loaded);
}

qmc_status qmc_tune_lookup(const qmc_problem* p, uint32_t n_integrals, uint32_t with_gradient,
                           qmc_tuning* h_out) {
  if (!p || !h_out || with_gradient > 1) return QMC_ERR_INVALID_ARG;
  uint32_t chunk = 0, block = 0;
  if (!tuned_lookup(p, n_integrals, with_gradient != 0, &chunk, &block)) chunk = block = 0;
  *h_out = qmc_tuning{chunk, block, 0.0f};
  return QMC_OK;
}

qmc_status qmc_graph_begin(qmc_stream_t stream) {
  if (!stream) return QMC_ERR_INVALID_ARG;  // the legacy default stream cannot be captured
  return cuda_status(cudaStreamBeginCapture((cudaStream_t)stream, cudaStreamCaptureModeThreadLocal));
}

qmc_status qmc_graph_end(qmc_stream_t stream, qmc_graph_t* out_graph) {
  if (!stream || !out_graph) return QMC_ERR_INVALID_ARG;
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture((cudaStream_t)stream, &graph);
  if (e != cudaSuccess) return cuda_status(e);
  if (!graph) return cuda_status(cudaErrorStreamCaptureInvalidated);
  cudaGraphExec_t exec = nullptr;
  const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
  if (ei != cudaSuccess) {
    cudaGraphDestroy(graph);
    return cuda_status(ei);
  }
  *out_graph = new qmc_graph_st{graph, exec};
  return QMC_OK;
}

qmc_status qmc_graph_launch(qmc_graph_t graph, qmc_stream_t stream) {
  if (!graph) return QMC_ERR_INVALID_ARG;
  return enqueue("qmc_graph_launch", [&] { return cudaGraphLaunch(graph->exec, (cudaStream_t)stream); });
}

qmc_status qmc_graph_destroy(qmc_graph_t graph) {
  if (!graph) return QMC_ERR_INVALID_ARG;
  cudaGraphExecDestroy(graph->exec);
  cudaGraphDestroy(graph->graph);
  delete graph;
  return QMC_OK;
}

}  // extern "C"
