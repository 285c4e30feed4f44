// api.cu -- the C-ABI of include/qmc.h: argument validation, the host-side
// construction of Sobol' generator matrices, and kernel dispatch.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/qmc.h"
#include "halton_points.h"
#include "qmc_integrate.h"
#include "qmc_host.h"
#include "qmc_internal.h"

namespace qmc {

const DeviceInfo& device_info() {
  static std::mutex mu;
  static std::vector<DeviceInfo> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(mu);
  for (const DeviceInfo& d : cache)
    if (d.device == dev) return d;
  DeviceInfo d{};
  d.device = dev;
  cudaDeviceGetAttribute(&d.sm_count, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&d.cc_major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&d.cc_minor, cudaDevAttrComputeCapabilityMinor, dev);
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  d.smem_per_block_optin = (size_t)optin;
  if (d.sm_count <= 0) d.sm_count = 1;
  cache.reserve(64);
  cache.push_back(d);
  return cache.back();
}

// The checked build's error word (qmc_checked_error); unused in the normal build.
__device__ uint32_t g_check_word;

namespace {
thread_local int t_last_cuda_error = 0;

// Device address of g_check_word on the current device (null on failure).
uint32_t* check_word_address() {
  static std::mutex mu;
  static void* addr[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev] && cudaGetSymbolAddress(&addr[dev], g_check_word) != cudaSuccess) {
    cudaGetLastError();
    addr[dev] = nullptr;
  }
  return static_cast<uint32_t*>(addr[dev]);
}

nvtxDomainHandle_t nvtx_domain() {
  static const nvtxDomainHandle_t d = nvtxDomainCreateA("qmc");
  return d;
}
}  // namespace

CheckCtx check_ctx(uint64_t limit) {
  if (!kChecked) return CheckCtx{nullptr, limit};
  const char* v = std::getenv("QMC_CHECK_SLACK");  // test hook: pretend the outputs end earlier
  const uint64_t slack = v ? std::strtoull(v, nullptr, 10) : 0;
  return CheckCtx{check_word_address(), limit > slack ? limit - slack : 0};
}

qmc_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return QMC_OK;
  t_last_cuda_error = (int)e;
  return QMC_ERR_CUDA;
}

bool launch_fault_injected() {
  const char* v = std::getenv("QMC_FAULT_INJECT");
  return v != nullptr && std::strcmp(v, "launch") == 0;
}

qmc_status injected_fault() {
  t_last_cuda_error = QMC_INJECTED_FAULT;
  return QMC_ERR_CUDA;
}

NvtxRange::NvtxRange(const char* name) {
  nvtxEventAttributes_t at{};
  at.version = NVTX_VERSION;
  at.size = NVTX_EVENT_ATTRIB_STRUCT_SIZE;
  at.messageType = NVTX_MESSAGE_TYPE_ASCII;
  at.message.ascii = name;
  nvtxDomainRangePushEx(nvtx_domain(), &at);
}

NvtxRange::~NvtxRange() { nvtxDomainRangePop(nvtx_domain()); }

WsLayout workspace_layout(uint32_t n, uint64_t capacity_items, uint32_t values_per_item) {
  auto up = [](size_t v) { return (v + 255) / 256 * 256; };
  const size_t nb = ((size_t)n + 1024) / 1024;
  WsLayout L{};
  size_t off = 0;
  L.header = off;
  off += up(sizeof(WsHeader));
  L.item_off = off;
  off += up(((size_t)n + 1) * 4);
  L.row_off = off;
  off += up(((size_t)n + 1) * 8);
  L.block_items = off;
  off += up(nb * 8);
  L.block_rows = off;
  off += up(nb * 8);
  L.loss_terms = off;
  off += up(((size_t)n + 256) * 8);  // per-integral terms, then the loss kernel's block sums
  L.partials = off;
  off += up((size_t)capacity_items * values_per_item * 2 * sizeof(float));
  L.total = off;
  return L;
}

namespace {

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// --- Sobol' matrices (Sec. 2.3).  Polynomials over GF(2) are bit masks, bit k
// holding the coefficient of x^k. ---------------------------------------------

uint32_t gf2_mulmod(uint32_t a, uint32_t b, uint32_t p, uint32_t d) {
  uint32_t r = 0;
  while (b) {
    if (b & 1u) r ^= a;
    b >>= 1;
    a <<= 1;
    if ((a >> d) & 1u) a ^= p;
  }
  return r;
}

// x^e mod p by square-and-multiply.
uint32_t gf2_pow_x(uint64_t e, uint32_t p, uint32_t d) {
  uint32_t base = 2u;
  if ((base >> d) & 1u) base ^= p;
  uint32_t r = 1u;
  while (e) {
    if (e & 1u) r = gf2_mulmod(r, base, p, d);
    base = gf2_mulmod(base, base, p, d);
    e >>= 1;
  }
  return r;
}

// Primitive <=> x has order exactly 2^d - 1 modulo p: x^(2^d-1) = 1 and
// x^((2^d-1)/q) != 1 for every prime q dividing 2^d - 1.
bool is_primitive(uint32_t p, uint32_t d) {
  const uint64_t order = (1ull << d) - 1;
  if (gf2_pow_x(order, p, d) != 1u) return false;
  uint64_t n = order;
  for (uint64_t q = 2; n > 1; ++q) {  // distinct prime factors by trial division
    if (n % q) continue;
    if (gf2_pow_x(order / q, p, d) == 1u) return false;
    while (n % q == 0) n /= q;
  }
  return true;
}

std::vector<uint32_t> primitive_polynomials_deg7() {
  std::vector<uint32_t> out;
  for (uint32_t d = 1; d <= 7; ++d)
    for (uint32_t p = (1u << d) + 1u; p < (1u << (d + 1)); p += 2u)
      if (is_primitive(p, d)) out.push_back(p);
  return out;
}

}  // namespace
}  // namespace qmc

using namespace qmc;

extern "C" {

uint32_t qmc_abi_version(void) { return 5u; }

int qmc_last_cuda_error(void) { return t_last_cuda_error; }

const char* qmc_status_string(qmc_status st) {
  switch (st) {
    case QMC_OK: return "QMC_OK";
    case QMC_ERR_INVALID_ARG: return "QMC_ERR_INVALID_ARG: invalid argument";
    case QMC_ERR_RANGE: return "QMC_ERR_RANGE: index or count range exceeded";
    case QMC_ERR_ALIGN: return "QMC_ERR_ALIGN: device buffer misaligned";
    case QMC_ERR_CUDA: return "QMC_ERR_CUDA: CUDA runtime error";
    case QMC_ERR_TIMEOUT: return "QMC_ERR_TIMEOUT: bounded device wait expired";
    case QMC_ERR_UNSUPPORTED: return "QMC_ERR_UNSUPPORTED: combination not implemented";
    case QMC_ERR_WORKSPACE: return "QMC_ERR_WORKSPACE: workspace missing, misaligned or too small";
    case QMC_ERR_IO: return "QMC_ERR_IO: file could not be read or written";
  }
  return "unknown qmc_status";
}

qmc_status qmc_sobol_matrices_wide(uint32_t s, uint32_t m, const uint32_t* h_raw_init,
                                   uint32_t* h_matrices) {
  static const std::vector<uint32_t> polys = primitive_polynomials_deg7();
  if (s == 0 || s > polys.size() + 1 || !h_matrices || m < 32 || m > 64) return QMC_ERR_INVALID_ARG;
  if (s > 1 && !h_raw_init) return QMC_ERR_INVALID_ARG;
  for (uint32_t j = 0; j < s; ++j) {
    uint32_t* V = h_matrices + (size_t)m * j;  // V[k-1] = first 32 digits of v_k
    if (j == 0) {
      for (uint32_t k = 1; k <= m; ++k) V[k - 1] = k <= 32 ? 0x80000000u >> (k - 1) : 0u;
      continue;
    }
    const uint32_t p = polys[j - 1];
    uint32_t d = 0;
    while (p >> (d + 1)) ++d;
    for (uint32_t k = 1; k <= d; ++k) {
      const uint32_t mk = (uint32_t)(h_raw_init[7 * j + k - 1] & ((1ull << k) - 1)) | 1u;
      V[k - 1] = mk << (32 - k);
    }
    // Bratley-Fox form of the recurrence on direction integers:
    // v_k = v_{k-d} ^ (v_{k-d} >> d) ^ XOR_{l=1}^{d-1} a_l v_{k-l}.  XOR and the
    // right shift commute with truncation to the first 32 digits, so the
    // truncated words obey it for every k, also beyond the 32nd column.
    for (uint32_t k = d + 1; k <= m; ++k) {
      uint32_t v = V[k - d - 1] ^ (V[k - d - 1] >> d);
      for (uint32_t l = 1; l < d; ++l)
        if ((p >> (d - l)) & 1u) v ^= V[k - l - 1];
      V[k - 1] = v;
    }
  }
  return QMC_OK;
}

qmc_status qmc_sobol_matrices(uint32_t s, const uint32_t* h_raw_init, uint32_t* h_matrices) {
  return qmc_sobol_matrices_wide(s, 32, h_raw_init, h_matrices);
}

// [begin, begin + count) lies inside [0, 2^bits) (bits <= 64).
static bool index_range_ok(uint64_t begin, uint64_t count, uint32_t bits) {
  const uint64_t limit_m1 = bits >= 64 ? ~0ull : (1ull << bits) - 1;  // 2^bits - 1
  if (count == 0) return bits >= 64 || begin <= limit_m1 + 1;
  const uint64_t last = begin + (count - 1);
  return last >= begin && last <= limit_m1;
}

// Bit reversal of the q low bits of p.
static uint64_t reverse_bits(uint64_t p, uint32_t q) {
  uint64_t c = 0;
  for (uint32_t k = 0; k < q; ++k) c |= ((p >> k) & 1ull) << (q - 1 - k);
  return c;
}

static qmc_status check_outputs(uint32_t s, uint64_t count, const void* out_u32, const void* out_f32) {
  if (count == 0) return QMC_OK;  // nothing to write: outputs may be null (empty tensors)
  if (count > (1ull << 62) / s) return QMC_ERR_RANGE;  // element offsets stay far below 2^64
  if (!out_u32 && !out_f32) return QMC_ERR_INVALID_ARG;
  if (((uintptr_t)out_u32 & 3u) || ((uintptr_t)out_f32 & 3u)) return QMC_ERR_ALIGN;
  return QMC_OK;
}

// Arguments of the 32-bit-index point entries: the range ends at 2^32 at most.
static qmc_status check_points_args(uint32_t s, uint64_t index_begin, uint64_t count,
                                    const void* out_u32, const void* out_f32) {
  if (s == 0 || s > 1024) return QMC_ERR_INVALID_ARG;
  if (!index_range_ok(index_begin, count, 32)) return QMC_ERR_RANGE;
  return check_outputs(s, count, out_u32, out_f32);
}

qmc_status qmc_sobol_points(const uint32_t* d_matrices, uint32_t s, uint64_t index_begin,
                            uint64_t count, uint32_t scramble, const uint32_t* d_seeds,
                            uint32_t* d_out_u32, float* d_out_f32, qmc_stream_t stream) {
  if (!d_matrices) return QMC_ERR_INVALID_ARG;
  if (scramble > QMC_SCRAMBLE_NESTED_XOR) return QMC_ERR_INVALID_ARG;
  if (scramble != QMC_SCRAMBLE_NONE && !d_seeds) return QMC_ERR_INVALID_ARG;
  qmc_status st = check_points_args(s, index_begin, count, d_out_u32, d_out_f32);
  if (st != QMC_OK || count == 0) return st;
  PointsArgs a{};
  a.matrices = d_matrices;
  a.seeds = d_seeds;
  a.out_u32 = d_out_u32;
  a.out_f32 = d_out_f32;
  a.count = count;
  a.s = s;
  a.index_begin = index_begin;
  a.m = 32;
  a.scramble = scramble;
  a.chk = check_ctx(count * s);
  return enqueue("qmc_sobol_points", [&] { return launch_sobol_points(a, (cudaStream_t)stream); });
}

qmc_status qmc_sobol_points_wide(const uint32_t* d_matrices, uint32_t m, uint32_t s,
                                 uint64_t index_begin, uint64_t count, uint32_t scramble,
                                 const uint32_t* d_seeds, uint32_t* d_out_u32, float* d_out_f32,
                                 qmc_stream_t stream) {
  if (!d_matrices || m < 32 || m > 64 || s == 0 || s > 1024) return QMC_ERR_INVALID_ARG;
  if (scramble > QMC_SCRAMBLE_NESTED_XOR) return QMC_ERR_INVALID_ARG;
  if (scramble != QMC_SCRAMBLE_NONE && !d_seeds) return QMC_ERR_INVALID_ARG;
  if (!index_range_ok(index_begin, count, m)) return QMC_ERR_RANGE;
  const qmc_status st = check_outputs(s, count, d_out_u32, d_out_f32);
  if (st != QMC_OK || count == 0) return st;
  PointsArgs a{};
  a.matrices = d_matrices;
  a.seeds = d_seeds;
  a.out_u32 = d_out_u32;
  a.out_f32 = d_out_f32;
  a.count = count;
  a.index_begin = index_begin;
  a.s = s;
  a.m = m;
  a.scramble = scramble;
  a.chk = check_ctx(count * s);
  return enqueue("qmc_sobol_points_wide", [&] { return launch_sobol_points(a, (cudaStream_t)stream); });
}

qmc_status qmc_sobol_points_partitioned(const uint32_t* d_matrices, uint32_t m, uint32_t s,
                                        uint32_t q, uint64_t p, uint64_t j_begin, uint64_t count,
                                        uint32_t scramble, const uint32_t* d_seeds,
                                        uint32_t* d_out_u32, float* d_out_f32, qmc_stream_t stream) {
  if (!d_matrices || m < 32 || m > 64 || s == 0 || s > 1024 || q >= m) return QMC_ERR_INVALID_ARG;
  if (p >> q) return QMC_ERR_INVALID_ARG;  // element p of 2^q
  if (scramble > QMC_SCRAMBLE_NESTED_XOR) return QMC_ERR_INVALID_ARG;
  if (scramble != QMC_SCRAMBLE_NONE && !d_seeds) return QMC_ERR_INVALID_ARG;
  if (!index_range_ok(j_begin, count, m - q)) return QMC_ERR_RANGE;
  const qmc_status st = check_outputs(s, count, d_out_u32, d_out_f32);
  if (st != QMC_OK || count == 0) return st;
  PointsArgs a{};
  a.matrices = d_matrices + m;  // dimensions 1..s; dimension 0 selects the element
  a.seeds = d_seeds;
  a.out_u32 = d_out_u32;
  a.out_f32 = d_out_f32;
  a.count = count;
  a.index_begin = j_begin;
  a.pconst = reverse_bits(p, q);
  a.s = s;
  a.m = m;
  a.col0 = q;
  a.scramble = scramble;
  a.chk = check_ctx(count * s);
  return enqueue("qmc_sobol_points_partitioned",
                 [&] { return launch_sobol_points(a, (cudaStream_t)stream); });
}

// Fills the Halton arguments shared by the plain and partitioned entries;
// output dimension j is Halton dimension dim0 + j.
static qmc_status halton_args(uint32_t s, uint32_t dim0, uint32_t mode, const uint32_t* h_multipliers,
                              HaltonArgs& a) {
  if (s == 0 || dim0 + s > kHaltonMaxDims || mode > QMC_HALTON_LINEAR) return QMC_ERR_INVALID_ARG;
  if (mode == QMC_HALTON_LINEAR && !h_multipliers) return QMC_ERR_INVALID_ARG;
  a.s = s;
  a.dim0 = dim0;
  a.mode = mode;
  for (uint32_t j = 0; j < s; ++j) {
    const uint32_t b = halton_base(dim0 + j);
    if (mode == QMC_HALTON_LINEAR) {
      const uint32_t m = h_multipliers[j];
      if (b > 2 && (m == 0 || m >= b)) return QMC_ERR_INVALID_ARG;  // must permute the digits
      a.mult[j] = b > 2 ? m : 1u;
    }
  }
  return QMC_OK;
}

qmc_status qmc_halton_points(uint32_t s, uint32_t mode, const uint32_t* h_multipliers, uint64_t index_begin,
                             uint64_t count, uint32_t* d_out_u32, float* d_out_f32, qmc_stream_t stream) {
  HaltonArgs a{};
  qmc_status st = halton_args(s, 0, mode, h_multipliers, a);
  if (st != QMC_OK) return st;
  st = check_points_args(1, index_begin, count, d_out_u32, d_out_f32);
  if (st != QMC_OK || count == 0) return st;
  a.out_u32 = d_out_u32;
  a.out_f32 = d_out_f32;
  a.count = count;
  a.index_begin = index_begin;
  a.chk = check_ctx(count * s);
  return enqueue("qmc_halton_points", [&] { return launch_halton_points(a, (cudaStream_t)stream); });
}

qmc_status qmc_halton_points_partitioned(uint32_t s, uint32_t mode, const uint32_t* h_multipliers,
                                         uint32_t q, uint64_t p, uint64_t j_begin, uint64_t count,
                                         uint32_t* d_out_u32, float* d_out_f32, qmc_stream_t stream) {
  if (q > 63 || (p >> q)) return QMC_ERR_INVALID_ARG;
  HaltonArgs a{};
  qmc_status st = halton_args(s, 1, mode, h_multipliers, a);
  if (st != QMC_OK) return st;
  if (!index_range_ok(j_begin, count, 64 - q)) return QMC_ERR_RANGE;
  st = check_outputs(s, count, d_out_u32, d_out_f32);
  if (st != QMC_OK || count == 0) return st;
  a.out_u32 = d_out_u32;
  a.out_f32 = d_out_f32;
  a.count = count;
  a.index_begin = j_begin;
  a.q = q;
  a.pconst = reverse_bits(p, q);
  a.chk = check_ctx(count * s);
  return enqueue("qmc_halton_points_partitioned",
                 [&] { return launch_halton_points(a, (cudaStream_t)stream); });
}

qmc_status qmc_pixel_lattice_points(const uint32_t* d_g, uint32_t s, uint32_t image_width,
                                    uint32_t image_height, uint64_t pixel_begin, uint64_t n_pixels,
                                    uint32_t spp, uint32_t* d_out_u32, float* d_out_f32,
                                    qmc_stream_t stream) {
  if (!d_g || s == 0 || s > 1024 || image_width == 0 || image_height == 0 || spp == 0)
    return QMC_ERR_INVALID_ARG;
  const uint64_t pixels = (uint64_t)image_width * image_height;
  if (pixel_begin > pixels || n_pixels > pixels - pixel_begin) return QMC_ERR_RANGE;
  if (n_pixels == 0) return QMC_OK;
  if (!d_out_u32 && !d_out_f32) return QMC_ERR_INVALID_ARG;
  if (((uintptr_t)d_out_u32 & 3u) || ((uintptr_t)d_out_f32 & 3u)) return QMC_ERR_ALIGN;
  PixelPointsArgs a{};
  a.g = d_g;
  a.out_u32 = d_out_u32;
  a.out_f32 = d_out_f32;
  a.pixel_begin = pixel_begin;
  a.n_pixels = n_pixels;
  a.spp = spp;
  a.s = s;
  a.width = image_width;
  uint32_t k = 0;
  const uint32_t side = image_width > image_height ? image_width : image_height;
  while (((uint64_t)1 << k) < side) ++k;
  a.grid_log2 = k;
  a.chk = check_ctx(n_pixels * spp * s);
  return enqueue("qmc_pixel_lattice_points",
                 [&] { return launch_pixel_lattice_points(a, (cudaStream_t)stream); });
}

qmc_status qmc_lattice_points(const uint32_t* d_g, const uint32_t* d_shift, uint32_t s,
                              uint64_t index_begin, uint64_t count, uint32_t flags,
                              uint32_t* d_out_u32, float* d_out_f32, qmc_stream_t stream) {
  if (!d_g || (flags & ~QMC_LATTICE_BACKWARD)) return QMC_ERR_INVALID_ARG;
  qmc_status st = check_points_args(s, index_begin, count, d_out_u32, d_out_f32);
  if (st != QMC_OK || count == 0) return st;
  PointsArgs a{};
  a.matrices = d_g;
  a.seeds = d_shift;
  a.out_u32 = d_out_u32;
  a.out_f32 = d_out_f32;
  a.count = count;
  a.s = s;
  a.index_begin = index_begin;
  a.scramble = flags;
  a.chk = check_ctx(count * s);
  return enqueue("qmc_lattice_points", [&] { return launch_lattice_points(a, (cudaStream_t)stream); });
}


// --------------------------------------------------------------------------
// Integration (Sec. 2.5)
// --------------------------------------------------------------------------
namespace {

constexpr uint32_t kDefaultChunk = 4096;
constexpr uint32_t kMinTunedChunk = 1024;
constexpr uint32_t kDefaultBlock = 256;

uint32_t ilog2(uint32_t v) {
  uint32_t l = 0;
  while ((1u << (l + 1)) <= v) ++l;
  return l;
}

// kind (QMC_RLAT_HASH or _LFSR) in the low byte, 1, 2, 4, 8 or 16 instances above.
bool rlat_randomize_ok(uint32_t r) {
  const uint32_t kind = r & 0xFFu, inst = r >> 8;
  return kind <= QMC_RLAT_LFSR && inst >= 1 && inst <= 16 && (inst & (inst - 1)) == 0;
}

qmc_status validate_problem(const qmc_problem* p, bool need_source) {
  if (!p) return QMC_ERR_INVALID_ARG;
  if (p->integrand > QMC_F_SCENE4D || p->source > QMC_SOURCE_RANDOM_LATTICE) return QMC_ERR_INVALID_ARG;
  const uint32_t s = p->s;
  if (p->integrand == QMC_F_BILINEAR2D && s != 2) return QMC_ERR_INVALID_ARG;
  if (p->integrand == QMC_F_GAUSSMIX4_6D && s != 6) return QMC_ERR_INVALID_ARG;
  if (p->integrand == QMC_F_SCENE4D && s != 4) return QMC_ERR_INVALID_ARG;
  if ((p->integrand == QMC_F_GENZ_PRODUCT_PEAK || p->integrand == QMC_F_GENZ_OSCILLATORY) &&
      (s == 0 || s > 16))
    return QMC_ERR_INVALID_ARG;
  if (p->seeds_per_integral > 1) return QMC_ERR_INVALID_ARG;
  if (p->source == QMC_SOURCE_SOBOL) {  // Sec. 2.5.1: J < 2^32 and q index bits below 32 + q <= m
    const uint32_t m = p->index_bits ? p->index_bits : 32u;
    if (m < 32 || m > 64 || p->partition_log2 > 32 || m < 32 + p->partition_log2) return QMC_ERR_INVALID_ARG;
  } else if (p->index_bits || p->partition_log2) {
    return QMC_ERR_INVALID_ARG;
  }
  if (p->chunk != 0 && (p->chunk < 32 || p->chunk > 8192 || (p->chunk & (p->chunk - 1))))
    return QMC_ERR_INVALID_ARG;
  if (p->block != 0 && (p->block % 32 || p->block > 256)) return QMC_ERR_INVALID_ARG;
  if (need_source) {
    if (p->source == QMC_SOURCE_SOBOL) {
      if (!p->d_matrices || p->randomize > QMC_SCRAMBLE_NESTED_XOR) return QMC_ERR_INVALID_ARG;
      if (p->randomize != QMC_SCRAMBLE_NONE && !p->d_seeds) return QMC_ERR_INVALID_ARG;
    } else if (p->source == QMC_SOURCE_LATTICE) {
      if (!p->d_g || (p->randomize & ~QMC_LATTICE_BACKWARD)) return QMC_ERR_INVALID_ARG;
    } else if (p->source == QMC_SOURCE_PIXEL_LATTICE) {  // generator words and an image width
      if (!p->d_g || p->randomize != 0 || p->image_width == 0) return QMC_ERR_INVALID_ARG;
    } else {  // random lattice per pixel: kind | (instances << 8), the seed, an image width
      if (!rlat_randomize_ok(p->randomize) || !p->d_seeds) return QMC_ERR_INVALID_ARG;
      if (p->image_width == 0 || p->image_width > (1u << 20)) return QMC_ERR_INVALID_ARG;
    }
  }
  return QMC_OK;
}

// Order k of the smallest 2^k x 2^k Hilbert grid covering an image of n pixels,
// image_width per row.
uint32_t image_grid_log2(uint32_t n, uint32_t width) {
  const uint64_t rows = width ? ((uint64_t)n + width - 1) / width : 0;
  const uint64_t side = rows > width ? rows : width;
  uint32_t k = 0;
  while (((uint64_t)1 << k) < side) ++k;
  return k;
}

uint32_t values_per_item(const qmc_problem* p, bool grad) {
  return grad ? 17u : 1u;
}


struct Prepared {
  IntegrateArgs a;
  uint32_t block;
};

qmc_status prepare(const qmc_problem* p, uint32_t n, const uint32_t* d_counts, const float* d_theta,
                   void* ws, size_t ws_bytes, bool grad, bool need_source, Prepared& out) {
  qmc_status st = validate_problem(p, need_source);
  if (st != QMC_OK) return st;
  if (!d_counts) return QMC_ERR_INVALID_ARG;
  if (p->integrand != QMC_F_BILINEAR2D && !d_theta) return QMC_ERR_INVALID_ARG;
  if ((p->integrand == QMC_F_GAUSSMIX4_6D || p->integrand == QMC_F_SCENE4D) && !aligned16(d_theta))
    return QMC_ERR_ALIGN;
  if (!ws || ((uintptr_t)ws & 255u)) return QMC_ERR_WORKSPACE;
  const uint32_t vpi = values_per_item(p, grad);
  const WsLayout L0 = workspace_layout(n, 0, vpi);
  if (ws_bytes < L0.total) return QMC_ERR_WORKSPACE;
  const uint64_t capacity = (ws_bytes - L0.partials) / ((size_t)vpi * 2 * sizeof(float));
  const WsLayout L = workspace_layout(n, capacity, vpi);
  char* base = static_cast<char*>(ws);
  IntegrateArgs& a = out.a;
  a = IntegrateArgs{};
  a.source = p->source;
  a.integrand = p->integrand;
  a.s = p->s;
  a.randomize = p->randomize;
  a.matrices = p->d_matrices;
  a.g = p->d_g;
  a.seeds = p->d_seeds;
  a.seeds_per_integral = p->seeds_per_integral;
  if (p->source == QMC_SOURCE_PIXEL_LATTICE) {
    a.seeds = nullptr;
    a.image_width = p->image_width;
    a.grid_log2 = image_grid_log2(n, p->image_width);
  }
  if (p->source == QMC_SOURCE_SOBOL) {
    a.sobol_m = p->index_bits ? p->index_bits : 32u;
    a.part_log2 = p->partition_log2;
    if (a.part_log2 && a.matrices) a.matrices += a.sobol_m;  // dimensions 1..s; dimension 0 partitions
  }
  if (p->source == QMC_SOURCE_RANDOM_LATTICE) {
    if (((uint64_t)n + p->image_width - 1) / p->image_width > (1u << 20)) return QMC_ERR_INVALID_ARG;
    a.image_width = p->image_width;
    a.rlat_log2 = ilog2(p->randomize >> 8);
  }
  // work split: explicit values, else the tuner's record for this problem class, else defaults
  uint32_t chunk = p->chunk, block = p->block;
  if (chunk == 0 || block == 0) {
    uint32_t tc = 0, tb = 0;
    if (tuned_lookup(p, n, grad, &tc, &tb)) {
      if (chunk == 0) chunk = tc;
      if (block == 0) block = tb;
    }
  }
  a.chunk_log2 = ilog2(chunk ? chunk : kDefaultChunk);
  a.n = n;
  a.counts = d_counts;
  a.theta = d_theta;
  a.theta_stride = (p->integrand == QMC_F_GAUSSMIX4_6D || p->integrand == QMC_F_SCENE4D) ? 16u
                   : p->integrand == QMC_F_BILINEAR2D                                    ? 0u
                                                                                         : 2u * p->s;
  a.hdr = reinterpret_cast<WsHeader*>(base + L.header);
  a.item_off = reinterpret_cast<uint32_t*>(base + L.item_off);
  a.row_off = nullptr;
  a.ws_block_items = reinterpret_cast<uint64_t*>(base + L.block_items);
  a.ws_block_rows = reinterpret_cast<uint64_t*>(base + L.block_rows);
  a.ws_loss_terms = reinterpret_cast<double*>(base + L.loss_terms);
  a.partials = reinterpret_cast<float*>(base + L.partials);
  a.capacity_items = capacity;
  a.check_word = check_ctx(0).word;
  (void)L.row_off;
  out.block = block ? block : kDefaultBlock;
  return QMC_OK;
}

}  // namespace

qmc_status qmc_random_lattice_points(uint32_t kind, uint32_t seed, uint32_t instances, uint32_t s,
                                     uint32_t image_width, uint32_t image_height, uint64_t pixel_begin,
                                     uint64_t n_pixels, uint32_t spp, uint32_t* d_out_u32, float* d_out_f32,
                                     qmc_stream_t stream) {
  if (!rlat_randomize_ok(kind | (instances << 8)) || instances > 16) return QMC_ERR_INVALID_ARG;
  if (s == 0 || s > 1024 || spp == 0) return QMC_ERR_INVALID_ARG;
  if (image_width == 0 || image_height == 0 || image_width > (1u << 20) || image_height > (1u << 20))
    return QMC_ERR_INVALID_ARG;
  const uint64_t pixels = (uint64_t)image_width * image_height;
  if (pixel_begin > pixels || n_pixels > pixels - pixel_begin) return QMC_ERR_RANGE;
  if (n_pixels == 0) return QMC_OK;
  const qmc_status st = check_outputs(s, n_pixels * spp, d_out_u32, d_out_f32);
  if (st != QMC_OK) return st;
  RandomPointsArgs a{};
  a.out_u32 = d_out_u32;
  a.out_f32 = d_out_f32;
  a.pixel_begin = pixel_begin;
  a.n_pixels = n_pixels;
  a.spp = spp;
  a.s = s;
  a.width = image_width;
  a.kind = kind;
  a.seed = seed;
  a.r_log2 = ilog2(instances);
  a.chk = check_ctx(n_pixels * spp * s);
  return enqueue("qmc_random_lattice_points",
                 [&] { return launch_random_lattice_points(a, (cudaStream_t)stream); });
}

size_t qmc_integrate_workspace_bytes(const qmc_problem* p, uint32_t n_integrals,
                                     const uint32_t* h_counts) {
  if (validate_problem(p, false) != QMC_OK) return 0;
  const bool grad = p->with_gradient != 0;
  const uint32_t C = p->chunk ? p->chunk : kMinTunedChunk;
  uint64_t items = 0;
  if (h_counts) {
    for (uint32_t i = 0; i < n_integrals; ++i) items += ((uint64_t)h_counts[i] + C - 1) / C;
  } else {
    items = (uint64_t)n_integrals * (((uint64_t)p->max_count + C - 1) / C);
  }
  if (items >= 0xFFFFFFFFull) return 0;
  return workspace_layout(n_integrals, items, values_per_item(p, grad)).total;
}

qmc_status qmc_integrate(const qmc_problem* p, uint32_t n_integrals, const uint32_t* d_counts,
                         const float* d_theta, double* d_estimate, void* d_workspace,
                         size_t workspace_bytes, qmc_stream_t stream) {
  if (!d_estimate) return QMC_ERR_INVALID_ARG;
  Prepared pr;
  qmc_status st = prepare(p, n_integrals, d_counts, d_theta, d_workspace, workspace_bytes, false, true, pr);
  if (st != QMC_OK || n_integrals == 0) return st;
  pr.a.estimate = d_estimate;
  return enqueue("qmc_integrate",
                 [&] { return launch_integrate(pr.a, pr.block, false, (cudaStream_t)stream); });
}

qmc_status qmc_integrate_backward(const qmc_problem* p, uint32_t n_integrals,
                                  const uint32_t* d_counts, const float* d_theta,
                                  const double* d_grad_estimate, float* d_grad_theta,
                                  void* d_workspace, size_t workspace_bytes, qmc_stream_t stream) {
  if (!d_grad_estimate || !d_grad_theta) return QMC_ERR_INVALID_ARG;
  if (p && p->integrand != QMC_F_GAUSSMIX4_6D) return QMC_ERR_UNSUPPORTED;
  Prepared pr;
  qmc_status st = prepare(p, n_integrals, d_counts, d_theta, d_workspace, workspace_bytes, true, true, pr);
  if (st != QMC_OK || n_integrals == 0) return st;
  pr.a.grad_est = d_grad_estimate;
  pr.a.grad_theta = d_grad_theta;
  return enqueue("qmc_integrate_backward",
                 [&] { return launch_integrate(pr.a, pr.block, true, (cudaStream_t)stream); });
}

qmc_status qmc_integrate_fwd_bwd(const qmc_problem* p, uint32_t n_integrals,
                                 const uint32_t* d_counts, const float* d_theta,
                                 const double* d_target, double* d_estimate, float* d_grad_theta,
                                 double* d_loss, void* d_workspace, size_t workspace_bytes,
                                 qmc_stream_t stream) {
  if (!d_target || !d_estimate || !d_grad_theta || !d_loss) return QMC_ERR_INVALID_ARG;
  if (p && p->integrand != QMC_F_GAUSSMIX4_6D) return QMC_ERR_UNSUPPORTED;
  Prepared pr;
  qmc_status st = prepare(p, n_integrals, d_counts, d_theta, d_workspace, workspace_bytes, true, true, pr);
  if (st != QMC_OK) return st;
  if (n_integrals == 0)
    return enqueue("qmc_integrate_fwd_bwd",
                   [&] { return cudaMemsetAsync(d_loss, 0, sizeof(double), (cudaStream_t)stream); });
  pr.a.target = d_target;
  pr.a.estimate = d_estimate;
  pr.a.grad_theta = d_grad_theta;
  pr.a.loss = d_loss;
  return enqueue("qmc_integrate_fwd_bwd",
                 [&] { return launch_integrate(pr.a, pr.block, true, (cudaStream_t)stream); });
}

qmc_status qmc_integrate_points(const qmc_problem* p, uint32_t n_integrals,
                                const uint32_t* d_counts, const float* d_points,
                                uint32_t points_shared, const float* d_theta,
                                double* d_estimate, void* d_workspace, size_t workspace_bytes,
                                qmc_stream_t stream) {
  if (!d_points || !d_estimate || points_shared > 1) return QMC_ERR_INVALID_ARG;
  Prepared pr;
  qmc_status st = prepare(p, n_integrals, d_counts, d_theta, d_workspace, workspace_bytes, false, false, pr);
  if (st != QMC_OK || n_integrals == 0) return st;
  const WsLayout L = workspace_layout(n_integrals, 0, 1);
  pr.a.points = d_points;
  pr.a.points_shared = points_shared;
  pr.a.row_off = reinterpret_cast<uint64_t*>(static_cast<char*>(d_workspace) + L.row_off);
  pr.a.estimate = d_estimate;
  return enqueue("qmc_integrate_points",
                 [&] { return launch_integrate(pr.a, pr.block, false, (cudaStream_t)stream); });
}

qmc_status qmc_checked_error(uint32_t* h_bits, uint32_t reset) {
  if (!h_bits || reset > 1) return QMC_ERR_INVALID_ARG;
  *h_bits = 0;
  if (!kChecked) return QMC_ERR_UNSUPPORTED;
  uint32_t* word = check_word_address();
  if (!word) return cuda_status(cudaErrorInvalidSymbol);
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(h_bits, word, sizeof(uint32_t), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && reset) e = cudaMemset(word, 0, sizeof(uint32_t));
  return cuda_status(e);
}

qmc_status qmc_read_device_error(const void* d_workspace, uint32_t* h_error_bits,
                                 qmc_stream_t stream) {
  if (!d_workspace || !h_error_bits || ((uintptr_t)d_workspace & 255u)) return QMC_ERR_INVALID_ARG;
  WsHeader h{};
  const qmc_status st = enqueue("qmc_read_device_error", [&] {
    const cudaError_t e =
        cudaMemcpyAsync(&h, d_workspace, sizeof(h), cudaMemcpyDeviceToHost, (cudaStream_t)stream);
    return e != cudaSuccess ? e : cudaStreamSynchronize((cudaStream_t)stream);
  });
  if (st == QMC_OK) *h_error_bits = h.error_bits;
  return st;
}

}  // extern "C"
