// noalloc.cu — run a rectangular nest without allocating any memory.
//
// Some callers cannot allocate device memory at run time: a latency-critical
// serving loop (cudaMalloc / cudaFree synchronise the whole device and stall
// every other stream), a service that handed its whole device-memory budget out
// at start-up, or code that runs while a framework holds its allocator.  For
// them hp_nest_run_static runs the same kernels as hp_nest_run, but the
// partial results of a reduction split over grid parts live in one file-scope
// device array of fixed size instead of per-nest scratch.
//
// The array is shared by every call in the process and keeps the contents the
// last call left; nothing in it has to start at zero, because the first pass
// writes every partial it uses before the second pass reads it.  Two calls
// whose work overlaps on the GPU (different streams, or different host
// threads) race on the array.  Each GPU that loads the library holds the array
// until the process exits.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "api_internal.h"
#include "rect_launch.cuh"

namespace hp {

constexpr size_t kStaticScratchBytes = size_t(8) << 20;  // 8 MiB per device
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

namespace {
std::mutex g_static_mu;
void* g_static_addr[kMaxDevices] = {};

// Device address of the array on the current device, looked up once per device
// with that device current.  In host code the array's name only stands in for
// the symbol; its device address must come from cudaGetSymbolAddress.
hp_status static_scratch_address(int dev, void** out) {
  if (dev < 0 || dev >= kMaxDevices) return fail(HP_EUNSUPPORTED, "device index beyond the static scratch table");
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || p == nullptr)
      return fail(HP_ECUDA, std::string("cudaGetSymbolAddress (static scratch): ") + cudaGetErrorString(e));
    g_static_addr[dev] = p;
  }
  *out = g_static_addr[dev];
  return HP_OK;
}
}  // namespace

}  // namespace hp

using namespace hp;

extern "C" hp_status hp_nest_run_static(hp_nest* n, const void* const* in_dev, void* out_dev, void* stream) {
  if (!n) return fail(HP_EINVAL, "nest is NULL");
  if (n->kind != NEST_RECT) return fail(HP_EUNSUPPORTED, "hp_nest_run_static takes rectangular nests");
  const NestPlan& p = n->plan;
  if (p.body == HP_BODY_GEOMETRIC)
    return fail(HP_EUNSUPPORTED, "hp_nest_run_static: the GEOMETRIC body needs a device table; use hp_nest_run");
  const RectPlan& rp = p.rp;
  const size_t need = rp.G > 1 ? static_cast<size_t>(rp.items) * partial_bytes(p.prec, p.op) : 0;
  if (need > kStaticScratchBytes)
    return fail(HP_EINVAL, "hp_nest_run_static: the plan needs " + std::to_string(need) +
                               " bytes of grid-part scratch, more than the static maximum of " +
                               std::to_string(kStaticScratchBytes) + " bytes");
  for (int i = 0; i < p.n_inputs; ++i) {
    if (!in_dev || !in_dev[i]) return fail(HP_EINVAL, "missing device input " + std::to_string(i));
    if (rp.V == 4 && (reinterpret_cast<uintptr_t>(in_dev[i]) & 15u))
      return fail(HP_EINVAL, "input " + std::to_string(i) + " must be 16-byte aligned (plan uses 128-bit loads)");
  }
  if (!out_dev && rp.O > 0) return fail(HP_EINVAL, "out_dev is NULL");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "no CUDA device");
  if (n->device >= 0 && n->device != dev) return fail(HP_EINVAL, "nest was first run on another device");
  if (n->cfg.ready && n->cfg.device != dev) return fail(HP_EINVAL, "nest was first run on another device");
  void* scratch = nullptr;
  hp_status st = static_scratch_address(dev, &scratch);
  if (st != HP_OK) return st;
  if (!n->cfg.ready) {
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "device query");
    n->cfg.sms = sms;
    n->cfg.device = dev;
  }
  RectArgs a{in_dev, out_dev, scratch, nullptr, static_cast<cudaStream_t>(stream)};
  const bool fp = p.prec == HP_F32 || p.prec == HP_F32_COMP;
  switch (p.op) {
    case HP_RED_SUM:
      if (p.prec == HP_F32) return launch_rect_f32_sum(p, n->cfg, a);
      if (p.prec == HP_F32_COMP) return launch_rect_f32_comp(p, n->cfg, a);
      if (p.prec == HP_I32) return launch_rect_i32_sum(p, n->cfg, a);
      return launch_rect_i64_sum(p, n->cfg, a);
    case HP_RED_MAX:
      if (fp) return launch_rect_f32_max(p, n->cfg, a);
      if (p.prec == HP_I32) return launch_rect_i32_max(p, n->cfg, a);
      return launch_rect_i64_max(p, n->cfg, a);
    case HP_RED_MIN:
      if (fp) return launch_rect_f32_min(p, n->cfg, a);
      if (p.prec == HP_I32) return launch_rect_i32_min(p, n->cfg, a);
      return launch_rect_i64_min(p, n->cfg, a);
    default:
      return fail(HP_EINVAL, "bad op");
  }
}
