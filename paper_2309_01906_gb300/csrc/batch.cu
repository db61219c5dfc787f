// batch.cu — hp_nest_run_batch: many independent nests in one persistent
// launch per arithmetic, replayed from a cached CUDA graph.
//
// Per distinct list of nests a context is built once: a tile table (each
// nest's work items cut into tiles of similar size, ordered largest first so
// that the dynamic tile queue ends with small tiles), device arrays for the
// nest descriptors, per-output tickets of grid-split nests, tile counters, and
// two CUDA graphs (upload of the descriptors from one of two pinned host
// buffers, counter reset, the persistent kernels of the arithmetics on parallel
// branches).  A call refills the pinned
// buffer the previous-but-one call used (after waiting for that call's event)
// and replays its graph, so consecutive calls overlap.
#include <cuda_runtime.h>

#include <algorithm>
#include <list>
#include <memory>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "api_internal.h"
#include "batch_kernels.cuh"

namespace hp {

namespace {

struct BatchCtx {
  std::vector<hp_nest*> key;
  std::vector<uint64_t> ids;                   // plan id of each nest when built
  int device = -1;
  BatchNest* d_nests = nullptr;
  BatchNest* h_nests[2] = {nullptr, nullptr};   // pinned
  BatchTile* d_tiles = nullptr;
  int32_t* d_tickets = nullptr;
  unsigned long long* d_counters = nullptr;
  std::vector<int64_t> ticket_off;             // per nest (G > 1): offset into d_tickets
  struct Group {
    int combo;
    int64_t first, n_tiles;
    int grid;
  };
  std::vector<Group> groups;
  cudaStream_t cap = nullptr;
  std::vector<cudaStream_t> side;              // capture branches of the second and later arithmetics
  std::vector<cudaEvent_t> fork_join;          // capture-time dependencies (fork, then one join per branch)
  cudaGraphExec_t exec[2] = {nullptr, nullptr};
  cudaEvent_t done[2] = {nullptr, nullptr};
  bool used[2] = {false, false};
  bool filled[2] = {false, false};   // plans written into pinned buffer b
  int parity = 0;
  int64_t n_tiles = 0;

  ~BatchCtx() {
    for (int b = 0; b < 2; ++b) {
      if (done[b]) {
        cudaEventSynchronize(done[b]);
        cudaEventDestroy(done[b]);
      }
      if (exec[b]) cudaGraphExecDestroy(exec[b]);
      if (h_nests[b]) cudaFreeHost(h_nests[b]);
    }
    if (cap) cudaStreamDestroy(cap);
    for (cudaStream_t st : side) cudaStreamDestroy(st);
    for (cudaEvent_t ev : fork_join) cudaEventDestroy(ev);
    cudaFree(d_nests);
    cudaFree(d_tiles);
    cudaFree(d_tickets);
    cudaFree(d_counters);
  }
};

std::mutex g_batch_mu;
std::list<std::unique_ptr<BatchCtx>> g_batch_ctx;   // most recently used first
constexpr size_t kMaxBatchCtx = 4;

// Can the persistent kernel run this plan?  Its CTA has 8 consumer warps and
// no cluster: block teams of clusters (or of more warps) run with their own
// launches instead.
bool batch_runs(const RectPlan& rp) { return !(rp.team == TEAM_BLOCK && (rp.C > 1 || rp.W > kBatchThreads / 32)); }

hp_status cuda_err(cudaError_t e, const char* what) {
  return fail(HP_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// tiles of one nest: items cut into ranges of about `target` elements of work
void make_tiles(int nest, const RectPlan& rp, int64_t target, std::vector<BatchTile>& out,
                std::vector<int64_t>& work) {
  if (rp.items == 0) return;
  int64_t per_item;
  if (rp.team == TEAM_MAP) per_item = 1;
  else if (rp.split) per_item = std::max<int64_t>(1, rp.R / std::max<int64_t>(1, rp.vn[0]) * rp.tile);
  else per_item = std::max<int64_t>(1, rp.R);
  int64_t k = std::max<int64_t>(1, target / per_item);
  if (rp.team == TEAM_LANES) {
    const int64_t teams = (kBatchThreads / 32) * (32 / rp.L);
    k = (k + teams - 1) / teams * teams;   // whole CTAs of teams
  }
  if (rp.team == TEAM_MAP) k = std::max<int64_t>(k, kBatchThreads);
  k = std::min<int64_t>(k, int64_t(1) << 30);
  for (int64_t i0 = 0; i0 < rp.items; i0 += k) {
    const int64_t c = std::min<int64_t>(k, rp.items - i0);
    out.push_back({nest, static_cast<int32_t>(c), i0});
    work.push_back(c * per_item);
  }
}

hp_status build_ctx(BatchCtx& ctx, hp_nest* const* nests, int count, int dev, int sms) {
  ctx.device = dev;
  cudaError_t e;
  // tickets of grid-split nests
  int64_t tickets = 0;
  ctx.ticket_off.assign(count, -1);
  for (int i = 0; i < count; ++i) {
    const RectPlan& rp = nests[i]->plan.rp;
    if (rp.G > 1) {
      ctx.ticket_off[i] = tickets;
      tickets += rp.O;
    }
  }
  // tile target: about 4 tiles per resident CTA over the whole batch
  int64_t total = 0;
  for (int i = 0; i < count; ++i) {
    const RectPlan& rp = nests[i]->plan.rp;
    total += rp.team == TEAM_MAP ? rp.O : rp.O * std::max<int64_t>(1, rp.R);
  }
  const int64_t resident = static_cast<int64_t>(sms) * 8;
  const int64_t target = std::max<int64_t>(1 << 14, total / (4 * resident));
  // tiles grouped by arithmetic, each group largest first
  std::vector<std::vector<BatchTile>> per(kBatchCombos);
  std::vector<std::vector<int64_t>> per_work(kBatchCombos);
  for (int i = 0; i < count; ++i) {
    const NestPlan& p = nests[i]->plan;
    if (!batch_runs(p.rp)) continue;   // runs alone, after the persistent kernels
    const int c = batch_combo(p.prec, p.op);
    make_tiles(i, p.rp, target, per[c], per_work[c]);
  }
  std::vector<BatchTile> all;
  for (int c = 0; c < kBatchCombos; ++c) {
    if (per[c].empty()) continue;
    std::vector<size_t> idx(per[c].size());
    std::iota(idx.begin(), idx.end(), 0);
    std::stable_sort(idx.begin(), idx.end(), [&](size_t a, size_t b) { return per_work[c][a] > per_work[c][b]; });
    BatchCtx::Group g;
    g.combo = c;
    g.first = static_cast<int64_t>(all.size());
    g.n_tiles = static_cast<int64_t>(idx.size());
    g.grid = batch_combo_blocks_per_sm(c) * sms;
    for (size_t k : idx) all.push_back(per[c][k]);
    ctx.groups.push_back(g);
  }
  ctx.n_tiles = static_cast<int64_t>(all.size());
  if ((e = cudaMalloc(&ctx.d_nests, sizeof(BatchNest) * std::max(count, 1))) != cudaSuccess ||
      (e = cudaMalloc(&ctx.d_tiles, sizeof(BatchTile) * std::max<size_t>(all.size(), 1))) != cudaSuccess ||
      (e = cudaMalloc(&ctx.d_tickets, sizeof(int32_t) * std::max<int64_t>(tickets, 1))) != cudaSuccess ||
      (e = cudaMalloc(&ctx.d_counters, sizeof(unsigned long long) * kBatchCombos)) != cudaSuccess)
    return fail(HP_ENOMEM, std::string("cudaMalloc (batch context): ") + cudaGetErrorString(e));
  for (int b = 0; b < 2; ++b)
    if ((e = cudaMallocHost(&ctx.h_nests[b], sizeof(BatchNest) * std::max(count, 1))) != cudaSuccess)
      return fail(HP_ENOMEM, "cudaMallocHost (batch descriptors)");
  if (!all.empty() && (e = cudaMemcpy(ctx.d_tiles, all.data(), sizeof(BatchTile) * all.size(),
                                      cudaMemcpyHostToDevice)) != cudaSuccess)
    return cuda_err(e, "upload tile table");
  if ((e = cudaMemset(ctx.d_tickets, 0, sizeof(int32_t) * std::max<int64_t>(tickets, 1))) != cudaSuccess)
    return cuda_err(e, "zero tickets");
  if ((e = cudaStreamCreateWithFlags(&ctx.cap, cudaStreamNonBlocking)) != cudaSuccess)
    return cuda_err(e, "capture stream");
  // the persistent kernels of different arithmetics are independent (own tile
  // ranges and counters, shared read-only descriptors): they go on parallel
  // branches of the graph, so the CTAs of one start as the other's drain
  const size_t n_groups = ctx.groups.size();
  for (size_t gi = 1; gi < n_groups; ++gi) {
    cudaStream_t st = nullptr;
    if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess)
      return cuda_err(e, "capture branch stream");
    ctx.side.push_back(st);
  }
  for (size_t k = 0; k < n_groups; ++k) {   // [0]: fork, [gi]: join of branch gi
    cudaEvent_t ev = nullptr;
    if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess)
      return cuda_err(e, "capture branch event");
    ctx.fork_join.push_back(ev);
  }
  // two graphs: descriptors from pinned buffer b, counters reset, one persistent kernel per arithmetic
  for (int b = 0; b < 2; ++b) {
    if ((e = cudaEventCreateWithFlags(&ctx.done[b], cudaEventDisableTiming)) != cudaSuccess)
      return cuda_err(e, "batch event");
    if ((e = cudaStreamBeginCapture(ctx.cap, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
      return cuda_err(e, "begin capture");
    cudaError_t ce = cudaMemcpyAsync(ctx.d_nests, ctx.h_nests[b], sizeof(BatchNest) * std::max(count, 1),
                                     cudaMemcpyHostToDevice, ctx.cap);
    if (ce == cudaSuccess)
      ce = cudaMemsetAsync(ctx.d_counters, 0, sizeof(unsigned long long) * kBatchCombos, ctx.cap);
    if (ce == cudaSuccess && n_groups > 1) ce = cudaEventRecord(ctx.fork_join[0], ctx.cap);
    for (size_t gi = 0; ce == cudaSuccess && gi < n_groups; ++gi) {
      const BatchCtx::Group& g = ctx.groups[gi];
      cudaStream_t st = gi == 0 ? ctx.cap : ctx.side[gi - 1];
      if (gi > 0) ce = cudaStreamWaitEvent(st, ctx.fork_join[0], 0);
      BatchLaunch L{ctx.d_nests, ctx.d_tiles + g.first, g.n_tiles, ctx.d_counters + gi, g.grid};
      if (ce == cudaSuccess) ce = launch_batch_combo(g.combo, L, st);
      if (ce == cudaSuccess && gi > 0) ce = cudaEventRecord(ctx.fork_join[gi], st);
    }
    for (size_t gi = 1; ce == cudaSuccess && gi < n_groups; ++gi) ce = cudaStreamWaitEvent(ctx.cap, ctx.fork_join[gi], 0);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(ctx.cap, &graph);
    if (ce != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return cuda_err(ce, "capture batch graph");
    }
    if (e != cudaSuccess) return cuda_err(e, "end capture");
    e = cudaGraphInstantiate(&ctx.exec[b], graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_err(e, "instantiate batch graph");
  }
  return HP_OK;
}

}  // namespace

// A destroyed nest's address can be reused by a new nest: drop every cached
// context that refers to it.
void batch_forget(const hp_nest* n) {
  std::lock_guard<std::mutex> lock(g_batch_mu);
  for (auto it = g_batch_ctx.begin(); it != g_batch_ctx.end();) {
    const auto& key = (*it)->key;
    if (std::find(key.begin(), key.end(), n) != key.end()) it = g_batch_ctx.erase(it);
    else ++it;
  }
}

}  // namespace hp

using namespace hp;

extern "C" hp_status hp_nest_run_batch(hp_nest* const* nests, const void* const* const* in_dev, void* const* out_dev,
                                       int count, void* stream) {
  if (count < 0) return fail(HP_EINVAL, "count must be >= 0");
  if (count == 0) return HP_OK;
  if (!nests || !in_dev || !out_dev) return fail(HP_EINVAL, "NULL argument");
  for (int i = 0; i < count; ++i) {
    hp_nest* n = nests[i];
    if (!n) return fail(HP_EINVAL, "nest " + std::to_string(i) + " is NULL");
    if (n->kind != NEST_RECT) return fail(HP_EUNSUPPORTED, "batched nests must be rectangular");
    const NestPlan& p = n->plan;
    const RectPlan& rp = p.rp;
    if (p.body == HP_BODY_GEOMETRIC) return fail(HP_EUNSUPPORTED, "the GEOMETRIC body is not batched");
    hp_status st = ensure_device(n);
    if (st != HP_OK) return st;
    for (int k = 0; k < p.n_inputs; ++k) {
      if (!in_dev[i] || !in_dev[i][k]) return fail(HP_EINVAL, "nest " + std::to_string(i) + ": missing input");
      if (rp.V == 4 && (reinterpret_cast<uintptr_t>(in_dev[i][k]) & 15u))
        return fail(HP_EINVAL, "nest " + std::to_string(i) + ": inputs must be 16-byte aligned");
    }
    if (!out_dev[i] && rp.O > 0) return fail(HP_EINVAL, "nest " + std::to_string(i) + ": out is NULL");
  }
  int dev = nests[0]->device;
  std::lock_guard<std::mutex> lock(g_batch_mu);
  // find (or build) the context of this exact list of nests
  BatchCtx* ctx = nullptr;
  for (auto it = g_batch_ctx.begin(); it != g_batch_ctx.end(); ++it) {
    bool same = (*it)->device == dev && (*it)->key.size() == static_cast<size_t>(count) &&
                std::equal((*it)->key.begin(), (*it)->key.end(), nests);
    for (int i = 0; same && i < count; ++i) same = (*it)->ids[i] == nests[i]->plan_id;
    if (same) {
      g_batch_ctx.splice(g_batch_ctx.begin(), g_batch_ctx, it);
      ctx = g_batch_ctx.front().get();
      break;
    }
  }
  if (!ctx) {
    auto c = std::make_unique<BatchCtx>();
    c->key.assign(nests, nests + count);
    for (int i = 0; i < count; ++i) c->ids.push_back(nests[i]->plan_id);
    hp_status st = build_ctx(*c, nests, count, dev, nests[0]->sms);
    if (st != HP_OK) return st;
    g_batch_ctx.push_front(std::move(c));
    while (g_batch_ctx.size() > kMaxBatchCtx) g_batch_ctx.pop_back();
    ctx = g_batch_ctx.front().get();
  }
  const int b = ctx->parity;
  cudaError_t e;
  if (ctx->used[b] && (e = cudaEventSynchronize(ctx->done[b])) != cudaSuccess)
    return cuda_err(e, "wait for the previous use of the descriptor buffer");
  BatchNest* h = ctx->h_nests[b];
  const bool first_fill = !ctx->filled[b];
  for (int i = 0; i < count; ++i) {
    const hp_nest* n = nests[i];
    if (first_fill) h[i].rp = n->plan.rp;   // plans are fixed; later calls only rewrite the pointers
    h[i].in0 = n->plan.n_inputs > 0 ? in_dev[i][0] : nullptr;
    h[i].in1 = n->plan.n_inputs > 1 ? in_dev[i][1] : nullptr;
    h[i].out = out_dev[i];
    h[i].part = n->part;
    h[i].tickets = ctx->ticket_off[i] >= 0 ? ctx->d_tickets + ctx->ticket_off[i] : nullptr;
    h[i].err = n->err;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if ((e = cudaGraphLaunch(ctx->exec[b], s)) != cudaSuccess) return cuda_err(e, "batch graph launch");
  // nests the persistent kernel cannot run (cluster teams): their own kernels, same stream
  for (int i = 0; i < count; ++i) {
    if (batch_runs(nests[i]->plan.rp)) continue;
    const hp_status st = run_rect(nests[i], in_dev[i], out_dev[i], s);
    if (st != HP_OK) return st;
  }
  if ((e = cudaEventRecord(ctx->done[b], s)) != cudaSuccess) return cuda_err(e, "batch event record");
  ctx->used[b] = true;
  ctx->filled[b] = true;
  ctx->parity ^= 1;
  return HP_OK;
}
