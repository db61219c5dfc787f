// api.cu — the C ABI (include/hp.h): nest objects, device state, dispatch.
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstring>
#include <new>
#include <string>

#include "api_internal.h"
#include "rect_launch.cuh"

using namespace hp;

namespace hp {
const std::string& last_error_string();

uint64_t next_plan_id() {
  static std::atomic<uint64_t> counter{0};
  return ++counter;
}

hp_status ensure_device(hp_nest* n) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "no CUDA device");
  if (n->device >= 0) {
    if (dev != n->device) return fail(HP_EINVAL, "nest was first run on another device");
    return HP_OK;
  }
  // hp_nest_run_static sizes the launch (and sets the kernels' attributes) on
  // its own device without taking the nest's device: that launch
  // configuration belongs to that device
  if (n->cfg.ready && n->cfg.device != dev) return fail(HP_EINVAL, "nest was first run on another device");
  int sms = 0;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_fail(e, "device query");
  n->sms = sms;
  n->cfg.sms = sms;
  n->cfg.device = dev;
  e = cudaMalloc(&n->err, sizeof(int32_t));
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc (error word)");
  e = cudaMemset(n->err, 0, sizeof(int32_t));
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemset (error word)");
  if (n->kind == NEST_RECT) {
    const RectPlan& rp = n->plan.rp;
    if (rp.G > 1 && rp.items > 0) {
      n->part_bytes = static_cast<size_t>(rp.items) * partial_bytes(n->plan.prec, n->plan.op);
      e = cudaMalloc(&n->part, n->part_bytes);
      if (e != cudaSuccess) return fail(HP_ENOMEM, std::string("cudaMalloc (grid partials): ") + cudaGetErrorString(e));
    }
    if (!n->plan.geo_table.empty()) {
      const size_t b = n->plan.geo_table.size() * sizeof(float);
      e = cudaMalloc(&n->geo, b);
      if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc (geometric table)");
      e = cudaMemcpy(n->geo, n->plan.geo_table.data(), b, cudaMemcpyHostToDevice);
      if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy (geometric table)");
    }
  } else if (n->kind == NEST_ORDERED) {
    hp_status st = ordered_prepare(n);
    if (st != HP_OK) return st;
  } else if (n->kind == NEST_NARROW) {
    hp_status st = narrow_prepare(n);
    if (st != HP_OK) return st;
  } else {
    hp_status st = csr_prepare(n);
    if (st != HP_OK) return st;
  }
  n->device = dev;
  return HP_OK;
}

hp_status run_rect(hp_nest* n, const void* const* in_dev, void* out_dev, cudaStream_t st) {
  return run_rect_with(n, in_dev, out_dev, n->part, st);
}

// run with caller-provided grid-part scratch (a server's per-request scratch)
// and, for compensated sums, an optional residual output
hp_status run_rect_with(hp_nest* n, const void* const* in_dev, void* out_dev, void* part, cudaStream_t st,
                        float* comp) {
  const NestPlan& p = n->plan;
  for (int i = 0; i < p.n_inputs; ++i) {
    if (!in_dev || !in_dev[i]) return fail(HP_EINVAL, "missing device input " + std::to_string(i));
    if (p.rp.V == 4 && (reinterpret_cast<uintptr_t>(in_dev[i]) & 15u))
      return fail(HP_EINVAL, "input " + std::to_string(i) + " must be 16-byte aligned (plan uses 128-bit loads)");
  }
  if (!out_dev && p.rp.O > 0) return fail(HP_EINVAL, "out_dev is NULL");
  if (p.rp.G > 1 && p.rp.items > 0 && !part) return fail(HP_EINVAL, "grid-split plan without partial scratch");
  RectArgs a{in_dev, out_dev, part, n->geo, st, comp};
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

double error_bound(const hp_nest* n) {
  if (n->kind == NEST_RECT) return error_bound_rect(n->plan);
  if (n->kind == NEST_NARROW) return 0.0;   // integers: exact
  if (n->kind == NEST_ORDERED) {
    if (n->ord.op == HP_RED_LAST_VALID) return 0.0;   // values are copied, never computed
    // gamma_{2k}, k = R - 1: a product of R maps (or matrices) makes R - 1 combines
    // in any tree, each rounding twice, and the relative errors of all of them add;
    // no finite bound once 2k u reaches 1
    const double u = std::ldexp(1.0, -24), k2 = 2.0 * static_cast<double>(std::max<int64_t>(n->ord.R - 1, 0));
    return k2 * u < 1.0 ? k2 * u / (1.0 - k2 * u) : INFINITY;
  }
  if (n->csr.op != HP_RED_SUM || n->csr.prec != HP_F32_COMP) return n->csr.op == HP_RED_SUM ? 1e-5 : 0.0;
  return 1e-6;
}

// free a rectangular nest's device scratch so that the next run re-plans its
// launch and re-allocates for a new plan
hp_status tune_release_device(hp_nest* n) {
  if (n->device < 0) return HP_OK;
  if (n->part) cudaFree(n->part);
  if (n->geo) cudaFree(n->geo);
  if (n->err) cudaFree(n->err);
  n->part = nullptr;
  n->geo = nullptr;
  n->err = nullptr;
  n->part_bytes = 0;
  n->device = -1;
  n->cfg = LaunchCfg();
  return HP_OK;
}

size_t out_bytes(const hp_nest* n) {
  if (n->kind == NEST_RECT) return static_cast<size_t>(n->plan.rp.O) * n->plan.out_elem_bytes;
  if (n->kind == NEST_ORDERED) return ordered_out_bytes(n->ord);
  if (n->kind == NEST_NARROW) return static_cast<size_t>(n->nar.O) * sizeof(int32_t);
  return csr_out_bytes(n);
}

}  // namespace hp

extern "C" {

int hp_version(void) { return 100; }

hp_status hp_set_option(const char* name, int64_t value) {
  if (!name) return fail(HP_EINVAL, "option name is NULL");
  const std::string n(name);
  if (n == "pipeline") {
    options().pipeline = value;
    return HP_OK;
  }
  if (n == "serve_batching") {
    if (value < 0 || value > 2) return fail(HP_EINVAL, "serve_batching is 0 (plain), 1 (batched) or 2 (resident)");
    options().serve_batching = value;
    return HP_OK;
  }
  if (n == "tune_log") {
    options().tune_log = value;
    return HP_OK;
  }
  if (n == "host_zero_copy") {
    options().host_zero_copy = value;
    return HP_OK;
  }
  return fail(HP_EINVAL, "unknown option " + n);
}

hp_status hp_get_option(const char* name, int64_t* value) {
  if (!name || !value) return fail(HP_EINVAL, "NULL argument");
  const std::string n(name);
  if (n == "pipeline") {
    *value = options().pipeline;
    return HP_OK;
  }
  if (n == "serve_batching") {
    *value = options().serve_batching;
    return HP_OK;
  }
  if (n == "tune_log") {
    *value = options().tune_log;
    return HP_OK;
  }
  if (n == "host_zero_copy") {
    *value = options().host_zero_copy;
    return HP_OK;
  }
  return fail(HP_EINVAL, "unknown option " + n);
}

const char* hp_last_error(void) { return last_error_string().c_str(); }

hp_status hp_nest_create(int depth, const int64_t* extents, const int64_t* csr_offsets, int64_t n_rows,
                         const hp_level_map* map, hp_red_op op, int red_level, hp_prec prec, hp_body body,
                         const void* body_params, hp_nest** out) {
  if (!out) return fail(HP_EINVAL, "out is NULL");
  *out = nullptr;
  hp_nest* n = new (std::nothrow) hp_nest();
  if (!n) return fail(HP_ENOMEM, "host allocation failed");
  std::string why;
  hp_status st;
  if (prec == HP_I8 || prec == HP_I16) {
    n->kind = NEST_NARROW;
    st = plan_narrow(depth, extents, map, op, red_level, prec, body, &n->nar, &why);
  } else if (op == HP_RED_AFFINE_COMPOSE || op == HP_RED_MAT2_PRODUCT || op == HP_RED_LAST_VALID) {
    n->kind = NEST_ORDERED;
    st = plan_ordered(depth, extents, map, op, red_level, prec, body, &n->ord, &why);
  } else if (csr_offsets != nullptr || body == HP_BODY_CSR_GATHER || op == HP_RED_HIST_COUNT) {
    n->kind = NEST_CSR;
    st = plan_csr(depth, n_rows, map, op, red_level, prec, body, body_params, &n->csr, &why);
  } else {
    n->kind = NEST_RECT;
    st = plan_rect(depth, extents, map, op, red_level, prec, body, body_params, &n->plan, &why);
  }
  if (st != HP_OK) {
    delete n;
    return fail(st, why);
  }
  n->plan_id = next_plan_id();
  *out = n;
  set_error("");
  return HP_OK;
}

hp_status hp_nest_run(hp_nest* n, const void* const* in_dev, void* out_dev, void* stream) {
  if (!n) return fail(HP_EINVAL, "nest is NULL");
  hp_status st = ensure_device(n);
  if (st != HP_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (n->kind == NEST_RECT) return run_rect(n, in_dev, out_dev, s);
  if (n->kind == NEST_ORDERED) return run_ordered(n, in_dev, out_dev, s);
  if (n->kind == NEST_NARROW) return run_narrow(n, in_dev, out_dev, s);
  return run_csr(n, in_dev, out_dev, s);
}

hp_status hp_nest_run_comp(hp_nest* n, const void* const* in_dev, void* out_dev, void* comp_dev, void* stream) {
  if (!n) return fail(HP_EINVAL, "nest is NULL");
  if (n->kind != NEST_RECT || n->plan.prec != HP_F32_COMP || n->plan.op != HP_RED_SUM)
    return fail(HP_EUNSUPPORTED, "hp_nest_run_comp takes rectangular compensated FP32 sums (HP_F32_COMP, HP_RED_SUM)");
  const RectPlan& rp = n->plan.rp;
  if (!comp_dev && rp.O > 0) return fail(HP_EINVAL, "comp_dev is NULL");
  hp_status st = ensure_device(n);
  if (st != HP_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return run_rect_with(n, in_dev, out_dev, n->part, s, static_cast<float*>(comp_dev));
}

hp_status hp_nest_run_host(hp_nest* n, const void* const* in_host, void* out_host, void* stream) {
  if (!n) return fail(HP_EINVAL, "nest is NULL");
  if (n->kind != NEST_RECT) return fail(HP_EUNSUPPORTED, "hp_nest_run_host takes rectangular nests");
  hp_status st = ensure_device(n);
  if (st != HP_OK) return st;
  const NestPlan& p = n->plan;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  const void* dev_in[2] = {nullptr, nullptr};
  for (int i = 0; i < p.n_inputs; ++i) {
    if (!in_host || !in_host[i]) return fail(HP_EINVAL, "missing host input " + std::to_string(i));
    const size_t b = static_cast<size_t>(p.in_elems[i]) * p.in_elem_bytes;
    // The streamed input (every element read once per run) may be read by the
    // kernel straight from page-locked host memory that the device maps: on a
    // Grace-Blackwell node the kernel's own loads cross the chip-to-chip link
    // faster than a copy-engine transfer, and no staging copy precedes the run.
    // The broadcast operand is re-read by every output, so it is staged.
    if (i == 0 && options().host_zero_copy) {
      cudaPointerAttributes at{};
      if (cudaPointerGetAttributes(&at, in_host[i]) == cudaSuccess && at.type == cudaMemoryTypeHost &&
          at.devicePointer != nullptr && (p.rp.V != 4 || (reinterpret_cast<uintptr_t>(at.devicePointer) & 15u) == 0)) {
        dev_in[i] = at.devicePointer;
        continue;
      }
      cudaGetLastError();   // a pointer CUDA does not know is not an error here
    }
    if (n->stage_in_bytes[i] < b) {
      if (n->stage_in[i]) cudaFree(n->stage_in[i]);
      n->stage_in[i] = nullptr;
      n->stage_in_bytes[i] = 0;
      e = cudaMalloc(&n->stage_in[i], b ? b : 16);
      if (e != cudaSuccess) return fail(HP_ENOMEM, "cudaMalloc (staging input)");
      n->stage_in_bytes[i] = b;
    }
    if (b) {
      e = cudaMemcpyAsync(n->stage_in[i], in_host[i], b, cudaMemcpyHostToDevice, s);
      if (e != cudaSuccess) return cuda_fail(e, "H2D copy");
    }
    dev_in[i] = n->stage_in[i];
  }
  const size_t ob = out_bytes(n);
  if (ob && !out_host) return fail(HP_EINVAL, "out_host is NULL");
  if (n->stage_out_bytes < ob) {
    if (n->stage_out) cudaFree(n->stage_out);
    n->stage_out = nullptr;
    n->stage_out_bytes = 0;
    e = cudaMalloc(&n->stage_out, ob);
    if (e != cudaSuccess) return fail(HP_ENOMEM, "cudaMalloc (staging output)");
    n->stage_out_bytes = ob;
  }
  st = run_rect(n, dev_in, n->stage_out, s);
  if (st != HP_OK) return st;
  if (ob) {
    e = cudaMemcpyAsync(out_host, n->stage_out, ob, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_fail(e, "D2H copy");
  }
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
  return HP_OK;
}

hp_status hp_nest_error_bound(const hp_nest* n, double* rel_bound) {
  if (!n || !rel_bound) return fail(HP_EINVAL, "NULL argument");
  *rel_bound = error_bound(n);
  return HP_OK;
}

hp_status hp_nest_describe(const hp_nest* n, char* buf, size_t len) {
  if (!n || !buf || len == 0) return fail(HP_EINVAL, "NULL argument");
  const std::string s = n->kind == NEST_RECT      ? describe_plan(n->plan)
                        : n->kind == NEST_ORDERED ? describe_ordered(n->ord)
                        : n->kind == NEST_NARROW  ? describe_narrow(n->nar)
                                                  : describe_csr(n->csr);
  const size_t k = s.size() < len - 1 ? s.size() : len - 1;
  std::memcpy(buf, s.data(), k);
  buf[k] = 0;
  return HP_OK;
}

hp_status hp_nest_check(hp_nest* n, void* stream, int32_t* device_error) {
  if (!n) return fail(HP_EINVAL, "nest is NULL");
  if (device_error) *device_error = 0;
  if (n->device < 0 || !n->err) return HP_OK;  // never ran
  cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
  int32_t v = 0;
  e = cudaMemcpy(&v, n->err, sizeof(v), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "read error word");
  if (device_error) *device_error = v;
  if (v != 0)
    return fail(HP_ETIMEOUT, "device error word set (code " + std::to_string(v) +
                                 (v == 2   ? ": CSR offsets or columns outside the declared sizes)"
                                  : v == 3 ? ": a batched stage wait ran out of time)"
                                           : ")"));
  return HP_OK;
}

void hp_nest_destroy(hp_nest* n) {
  if (!n) return;
  batch_forget(n);
  if (n->device >= 0) {
    if (n->part) cudaFree(n->part);
    if (n->geo) cudaFree(n->geo);
    if (n->err) cudaFree(n->err);
    for (int i = 0; i < 2; ++i)
      if (n->stage_in[i]) cudaFree(n->stage_in[i]);
    if (n->stage_out) cudaFree(n->stage_out);
    if (n->tickets) cudaFree(n->tickets);
    csr_release(n);
  }
  delete n;
}

}  // extern "C"
