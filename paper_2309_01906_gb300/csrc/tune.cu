// tune.cu — the autotuner: pick the level -> hardware binding of a nest's shape
// class by timing legal candidates on the caller's buffers (Sec. 3.2 selects
// levels by what they provide and Sec. 3.3 compiles a region for several
// candidate levels and picks one at run time; here the pick is measured).
//
// With flags bit 1 every candidate (and the planner's own map) is timed in the
// batched executor, on as many copies of the nest as give about 2^24
// iterations, and the planner's map is kept unless another one is 3% faster.
//
// Candidates keep the outputs on the grid and put every reduced level on one
// hardware level: a CTA of 2 (single runs), 4 or 8 warps, a warp, a sub-warp group of 2..16
// lanes, the 4 vector slots of one thread, one thread sequentially, or a split
// of the reduction over several grid parts.  Long reductions also get cluster
// teams of 2, 4 or 8 CTAs (single runs only: the batched executor runs single
// CTAs), and nests with several reduced levels per-level bindings (a CTA's
// warps over the first reduced level and each warp's lanes over the inner
// ones; grid parts over the first and a CTA over the rest).  The winner is stored per shape
// class (log2 of outputs and of the reduced size, 128-bit divisibility, body,
// precision, operator); nests created later with an automatic map take it.
#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>
#include <cstdio>
#include <string>
#include <vector>

#include "api_internal.h"

namespace hp {

hp_status tune_release_device(hp_nest* n);
const std::string& last_error_string();

namespace {

std::vector<TuneChoice> candidates(const NestPlan& p, int sms, bool with_auto, bool batched) {
  int64_t O = 1, R = 1;
  for (int l = 0; l < p.red_level; ++l) O *= p.ext[l];
  for (int l = p.red_level; l < p.depth; ++l) R *= p.ext[l];
  const int d = p.depth, r = p.red_level;
  std::vector<TuneChoice> c;
  if (with_auto) c.push_back(TuneChoice{});   // the planner's own map first
  auto add = [&](int hw, int sub, int64_t parts) {
    TuneChoice t;
    t.red_hw = hw;
    t.sub = sub;
    t.split_parts = parts;
    c.push_back(t);
  };
  // a per-level binding: the first reduced level on (hw, sub) (or split over
  // `parts` grid parts), the inner reduced levels on (ihw, isub)
  auto add_map = [&](int hw, int sub, int64_t parts, int ihw, int isub) {
    TuneChoice t;
    t.red_hw = hw;
    t.sub = sub;
    t.split_parts = parts;
    t.inner_hw = ihw;
    t.inner_sub = isub;
    c.push_back(t);
  };
  if (!batched && R >= 8192) {
    // cluster teams (DSMEM combine): the batched executor runs single CTAs only
    for (int C : {2, 4, 8}) {
      if (R / C < 2048) continue;
      if (d - r >= 2) {
        for (int W : {4, 8})
          if (R / (static_cast<int64_t>(C) * W * 32) >= 8) add_map(HP_HW_CLUSTER, C, 0, HP_HW_CTA, W);
      } else {
        add(HP_HW_CLUSTER, C, 0);
      }
    }
  }
  if (!batched && d - r >= 2 && R >= 1024) {
    // mixed per-level bindings: the warps of a CTA over the first reduced
    // level, the lanes of each warp over the inner ones (single runs only: the
    // batched executor streams a nest through its ring only when the reduced
    // levels collapse into one)
    for (int W : {4, 8}) add_map(HP_HW_CTA, W, 0, HP_HW_WARP, 0);
    if (R >= 65536 && O < 8 * sms) {
      // the first reduced level split over grid parts, a CTA over the rest
      const int64_t n0 = p.ext[r];
      const int64_t parts = std::max<int64_t>(2, (2 * static_cast<int64_t>(sms) + O - 1) / std::max<int64_t>(O, 1));
      if (n0 >= 2 * parts) add_map(HP_HW_GRID, 0, parts, HP_HW_CTA, 8);
    }
  }
  if (R <= 64) add(HP_HW_SEQ, 0, 0);
  if (R % 4 == 0 && R <= 256) add(HP_HW_LANE, 4, 0);
  for (int w : {2, 4, 8, 16})
    if (R >= 2 * w && R <= 256 * w) add(HP_HW_SUBWARP, w, 0);
  if (R >= 32) add(HP_HW_WARP, 0, 0);
  if (R >= 512) {
    // a CTA of 2 warps puts one short output on more SMs at once (single runs:
    // in the batched executor it would leave 6 of its 8 consumer warps idle)
    if (!batched) add(HP_HW_CTA, 2, 0);
    add(HP_HW_CTA, 4, 0);
    add(HP_HW_CTA, 8, 0);
  }
  if (R >= 16384 && O < 8 * sms) {
    for (int64_t want : {int64_t(sms), int64_t(2) * sms, int64_t(4) * sms}) {
      const int64_t parts = std::max<int64_t>(2, (want + O - 1) / O);
      if (R / parts >= 2048) add(HP_HW_GRID, 0, parts);
    }
  }
  return c;
}

// mean time of `reps` back-to-back runs between two events
hp_status time_runs(hp_nest* tmp, const void* const* in_dev, void* out_dev, cudaStream_t st, int reps, float* ms) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  hp_status s = HP_OK;
  cudaEventRecord(e0, st);
  for (int i = 0; i < reps && s == HP_OK; ++i) s = run_rect(tmp, in_dev, out_dev, st);
  cudaEventRecord(e1, st);
  const cudaError_t e = cudaEventSynchronize(e1);
  float t = 0.0f;
  if (e == cudaSuccess) cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s != HP_OK) return s;
  if (e != cudaSuccess) return fail(HP_ECUDA, std::string("tuning run: ") + cudaGetErrorString(e));
  *ms = t / reps;
  return HP_OK;
}

// mean device time of `reps` runs captured back to back in one CUDA graph on
// the private stream cs (the host's launch rate does not enter)
hp_status time_runs_graph(hp_nest* tmp, const void* const* in_dev, void* out_dev, cudaStream_t cs, int reps,
                          float* ms) {
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return fail(HP_ECUDA, std::string("tuning capture: ") + cudaGetErrorString(e));
  hp_status s = HP_OK;
  for (int i = 0; i < reps && s == HP_OK; ++i) s = run_rect(tmp, in_dev, out_dev, cs);
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(cs, &g);
  if (s != HP_OK || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return s != HP_OK ? s : fail(HP_ECUDA, std::string("tuning capture: ") + cudaGetErrorString(e));
  }
  cudaGraphExec_t x = nullptr;
  e = cudaGraphInstantiate(&x, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(HP_ECUDA, std::string("tuning graph: ") + cudaGetErrorString(e));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  e = cudaGraphLaunch(x, cs);   // warm
  cudaEventRecord(e0, cs);
  if (e == cudaSuccess) e = cudaGraphLaunch(x, cs);
  cudaEventRecord(e1, cs);
  const cudaError_t es = cudaEventSynchronize(e1);
  float t = 0.0f;
  if (e == cudaSuccess && es == cudaSuccess) cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaGraphExecDestroy(x);
  if (e != cudaSuccess || es != cudaSuccess)
    return fail(HP_ECUDA, std::string("tuning run: ") + cudaGetErrorString(e != cudaSuccess ? e : es));
  *ms = t / reps;
  return HP_OK;
}

// Time one candidate: a warm-up run on the caller's stream (it also sizes the
// launch), then three trials, the best kept.  A trial replays a CUDA graph of
// enough back-to-back runs for about 0.3 ms of device time (3 to 256 runs), so
// that microsecond kernels are timed on the device, not by the host's launch
// rate or the event resolution.
hp_status time_plan(hp_nest* tmp, const void* const* in_dev, void* out_dev, cudaStream_t st, float* ms) {
  hp_status s = ensure_device(tmp);
  if (s != HP_OK) return s;
  if ((s = run_rect(tmp, in_dev, out_dev, st)) != HP_OK) return s;  // warm-up (and launch configuration)
  float est = 0.0f;
  if ((s = time_runs(tmp, in_dev, out_dev, st, 3, &est)) != HP_OK) return s;
  cudaError_t e = cudaStreamSynchronize(st);   // the capture stream takes over the caller's buffers
  if (e != cudaSuccess) return fail(HP_ECUDA, std::string("tuning: ") + cudaGetErrorString(e));
  cudaStream_t cs = nullptr;
  e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e != cudaSuccess) return fail(HP_ECUDA, std::string("tuning stream: ") + cudaGetErrorString(e));
  const int reps = est > 0.0f ? std::max(3, std::min(256, static_cast<int>(0.3f / est))) : 256;
  float best = FLT_MAX;
  for (int trial = 0; trial < 3 && s == HP_OK; ++trial) {
    float t = 0.0f;
    s = time_runs_graph(tmp, in_dev, out_dev, cs, reps, &t);
    best = std::min(best, t);
  }
  cudaStreamDestroy(cs);
  if (s != HP_OK) return s;
  *ms = best;
  return HP_OK;
}

// the same, in the batched executor: `copies` instances of the nest in one
// hp_nest_run_batch (they read the same inputs and write the same, identical
// outputs), so that a small nest is timed at the throughput it gets there
hp_status time_plan_batched(hp_nest* tmp, const void* const* in_dev, void* out_dev, cudaStream_t st, int copies,
                            float* ms) {
  hp_status s = ensure_device(tmp);
  if (s != HP_OK) return s;
  std::vector<hp_nest*> ns(copies, tmp);
  std::vector<const void* const*> ins(copies, in_dev);
  std::vector<void*> outs(copies, out_dev);
  if ((s = hp_nest_run_batch(ns.data(), ins.data(), outs.data(), copies, st)) != HP_OK) return s;  // builds the batch
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  constexpr int kReps = 3;
  cudaEventRecord(e0, st);
  for (int i = 0; i < kReps && s == HP_OK; ++i) s = hp_nest_run_batch(ns.data(), ins.data(), outs.data(), copies, st);
  cudaEventRecord(e1, st);
  const cudaError_t e = cudaEventSynchronize(e1);
  float t = 0.0f;
  if (e == cudaSuccess) cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s != HP_OK) return s;
  if (e != cudaSuccess) return fail(HP_ECUDA, std::string("tuning run: ") + cudaGetErrorString(e));
  *ms = t / kReps;
  return HP_OK;
}

}  // namespace
}  // namespace hp

using namespace hp;

namespace hp {
namespace {

// FNV-1a over the requirement triples: the cache key of choices made under them
uint64_t req_hash(int depth, const hp_level_req* req) {
  uint64_t h = 1469598103934665603ull;
  auto mix = [&](uint64_t v) {
    for (int i = 0; i < 8; ++i) {
      h ^= (v >> (8 * i)) & 0xffu;
      h *= 1099511628211ull;
    }
  };
  mix(static_cast<uint64_t>(depth));
  for (int l = 0; l < depth; ++l) {
    mix(req[l].sync);
    mix(req[l].reserve);
    mix(static_cast<uint64_t>(req[l].min_num));
  }
  return h | 1u;   // never 0 (0 = no requirements)
}

hp_status tune_impl(hp_nest* n, const hp_level_req* req, const void* const* in_dev, void* out_dev, void* stream,
                    int32_t flags) {
  if (!n) return fail(HP_EINVAL, "nest is NULL");
  if (n->kind != NEST_RECT) return fail(HP_EUNSUPPORTED, "only rectangular nests are tuned");
  NestPlan& p = n->plan;
  if (p.red_level == p.depth) {   // nothing is reduced: nothing to bind, only the map to check
    std::string why;
    if (req && !map_meets(p.depth, req, p.map, &why)) return fail(HP_EINVAL, "the nest's map: " + why);
    return HP_OK;
  }
  if (req) {   // host check first: unsatisfiable requirements need no device
    bool any = false;
    hp_level_map m[HP_MAX_DEPTH];
    any = hp_level_select(p.depth, req, m) == HP_OK;
    std::string why;
    for (const TuneChoice& c : candidates(p, n->sms > 0 ? n->sms : 152, true, false)) {   // GB300 before the first run
      if (any) break;
      tune_apply(p, c, m);
      any = map_meets(p.depth, req, m, &why);
    }
    if (!any) return fail(HP_EINVAL, "no candidate map meets the level requirements (" + why + ")");
  }
  hp_status s = ensure_device(n);
  if (s != HP_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  TuneKey key = tune_key(p);
  if (req) key.req = req_hash(p.depth, req);
  TuneChoice best;
  const bool reuse = (flags & 1) == 0;
  const bool batched = (flags & 2) != 0;
  // batched timing: enough copies for about 2^24 iterations (at most 64)
  const int copies = static_cast<int>(std::min<int64_t>(64, std::max<int64_t>(1, ((int64_t(1) << 24) + p.total - 1) /
                                                                                   std::max<int64_t>(1, p.total))));
  bool have = reuse && tune_lookup(key, &best);
  if (!have) {
    float best_ms = FLT_MAX;
    float auto_ms = -1.0f;
    std::vector<TuneChoice> cand = candidates(p, n->sms, batched || req, batched);
    if (req) {
      // Sec. 3.2: the requirements are the constraint language; only maps that
      // meet them are timed, and the map chosen from them comes first
      std::vector<TuneChoice> kept;
      TuneChoice sel;
      if (hp_level_select(p.depth, req, sel.map) == HP_OK) {
        sel.n_map = p.depth;
        kept.push_back(sel);
      }
      for (const TuneChoice& c : cand) {
        hp_level_map m[HP_MAX_DEPTH];
        tune_apply(p, c, m);
        std::string why;
        if (map_meets(p.depth, req, m, &why)) kept.push_back(c);
      }
      if (kept.empty()) {
        std::string why;
        hp_level_map m[HP_MAX_DEPTH];
        tune_apply(p, TuneChoice{}, m);
        map_meets(p.depth, req, m, &why);
        return fail(HP_EINVAL, "no candidate map meets the level requirements (" + why + ")");
      }
      cand.swap(kept);
    }
    for (const TuneChoice& c : cand) {
      hp_level_map m[HP_MAX_DEPTH];
      tune_apply(p, c, m);
      hp_nest* tmp = nullptr;
      const void* params = nullptr;
      hp_affine_params ap;
      if (p.body == HP_BODY_AFFINE) {
        ap = {p.rp.aff_a, p.rp.aff_b, p.rp.aff_m};
        params = &ap;
      }
      if (p.body == HP_BODY_GEOMETRIC) continue;  // table-driven test body: not tuned
      if (hp_nest_create(p.depth, p.ext, nullptr, 0, m, p.op, p.red_level, p.prec, p.body, params, &tmp) != HP_OK)
        continue;  // illegal for this shape
      float ms = 0.0f;
      const hp_status ts = batched ? time_plan_batched(tmp, in_dev, out_dev, st, copies, &ms)
                                   : time_plan(tmp, in_dev, out_dev, st, &ms);
      if (options().tune_log) {
        std::string mp;
        for (int l = 0; l < p.depth; ++l)
          mp += std::string(l ? "," : "") + std::to_string(m[l].hw) + ":" + std::to_string(m[l].sub_width) + ":" +
                std::to_string(m[l].tile);
        std::fprintf(stderr, "hp tune: map [%s] %s %.4f ms%s\n", mp.c_str(), tmp->plan.kernel.c_str(), ms,
                     ts == HP_OK ? "" : (" failed: " + last_error_string()).c_str());
      }
      hp_nest_destroy(tmp);
      if (ts != HP_OK) {
        if (ts == HP_ECUDA) return ts;
        continue;
      }
      if (c.red_hw == HP_HW_AUTO && c.n_map == 0) auto_ms = ms;
      if (ms < best_ms) {
        best_ms = ms;
        best = c;
        have = true;
      }
    }
    // batched: keep the planner's map unless another one is clearly faster
    if (batched && auto_ms >= 0.0f && best_ms > 0.97f * auto_ms) best = TuneChoice{};
    if (!have) return fail(req ? HP_EINVAL : HP_EUNSUPPORTED, req ? "no map that meets the level requirements runs for this shape"
                                                                 : "no candidate binding runs for this shape");
    tune_store(key, best);
  }
  // install the winner in this nest (its device scratch is sized per plan)
  hp_level_map m[HP_MAX_DEPTH];
  tune_apply(p, best, m);
  NestPlan np;
  std::string why;
  const void* params = nullptr;
  hp_affine_params ap;
  if (p.body == HP_BODY_AFFINE) {
    ap = {p.rp.aff_a, p.rp.aff_b, p.rp.aff_m};
    params = &ap;
  }
  s = plan_rect(p.depth, p.ext, m, p.op, p.red_level, p.prec, p.body, params, &np, &why);
  if (s != HP_OK) return fail(s, why);
  np.tuned = true;
  s = tune_release_device(n);
  if (s != HP_OK) return s;
  n->plan = np;
  n->plan_id = next_plan_id();   // cached batches built with the old plan no longer match
  s = ensure_device(n);
  if (s != HP_OK) return s;
  return run_rect(n, in_dev, out_dev, st);  // the outputs hold the installed plan's result
}

}  // namespace
}  // namespace hp

extern "C" hp_status hp_nest_tune(hp_nest* n, const void* const* in_dev, void* out_dev, void* stream, int32_t flags) {
  return tune_impl(n, nullptr, in_dev, out_dev, stream, flags);
}

extern "C" hp_status hp_nest_tune_req(hp_nest* n, const hp_level_req* req, const void* const* in_dev, void* out_dev,
                                      void* stream, int32_t flags) {
  if (!req) return fail(HP_EINVAL, "req is NULL (use hp_nest_tune)");
  return tune_impl(n, req, in_dev, out_dev, stream, flags);
}
