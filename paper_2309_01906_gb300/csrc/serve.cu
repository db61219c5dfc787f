// serve.cu — continuous batching of nest requests under a device-memory budget.
//
// A scheduler thread owns the GPU side of a server.  Submitted requests wait in
// a queue; the scheduler admits them while a slot is free and the admitted
// requests' inputs, outputs and scratch stay within the budget, packs every
// admitted request that is not yet running into one step, and launches the step
// on a free stream with the batched persistent kernels (one per arithmetic).
// With several streams, steps overlap on the device and requests that arrive
// while others run join the next step.  Completion is observed by querying the
// step's event; the scheduler then frees the slots, memory and scratch and
// admits more.  While steps are in flight, and for 2 ms after the last
// activity, the scheduler polls without sleeping (it owns one host core);
// idle longer, it waits on a condition variable that hp_serve_submit signals.
// In these launched forms no device code waits on anything.
//
// Resident form (serve_batching 2): instead of launching steps, the scheduler
// keeps one instance of the batched persistent kernel running while there is
// work (resident_kernels.cuh) and hands it each admitted request through
// mapped page-locked host memory: a slot descriptor, the request's tiles in a
// ring, then the instance's tail.  The kernel writes each finished request's
// sequence number to the slot's completion word, which the scheduler polls.
// Instances take new tiles for one epoch of host time and are stopped and
// replaced on a second stream; their device waits are bounded.
//
// Every request runs its nest's own plan with the single-run reduction tree
// (the batched kernels are bit-identical to hp_nest_run), so a result does not
// depend on what else was in its step.  Grid-split plans take their partials
// and tickets from server-owned pools, so concurrent requests on one nest never
// share scratch.  With hp_set_option("serve_batching", 0) a server launches
// every request alone with the single-nest kernels instead (the plain
// per-request baseline).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "api_internal.h"
#include "batch_kernels.cuh"
#include "rect_launch.cuh"
#include "resident_kernels.cuh"

namespace hp {

const std::string& last_error_string();

namespace {

double now_us() {
  return std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// first-fit allocator of byte ranges inside one device block
class RangeAlloc {
 public:
  void reset(size_t cap) {
    free_.clear();
    if (cap) free_[0] = cap;
  }
  bool alloc(size_t n, size_t* off) {
    n = (n + 255) & ~size_t(255);
    if (n == 0) {
      *off = 0;
      return true;
    }
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= n) {
        *off = it->first;
        const size_t rest = it->second - n, start = it->first + n;
        free_.erase(it);
        if (rest) free_[start] = rest;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t n) {
    n = (n + 255) & ~size_t(255);
    if (n == 0) return;
    auto it = free_.emplace(off, n).first;
    auto next = std::next(it);
    if (next != free_.end() && it->first + it->second == next->first) {
      it->second += next->second;
      free_.erase(next);
    }
    if (it != free_.begin()) {
      auto prev = std::prev(it);
      if (prev->first + prev->second == it->first) {
        prev->second += it->second;
        free_.erase(it);
      }
    }
  }

 private:
  std::map<size_t, size_t> free_;
};

enum ReqState : uint8_t { RQ_QUEUED = 0, RQ_RUNNING = 1, RQ_DONE = 2, RQ_FAILED = 3 };

struct Request {
  uint64_t ticket;
  hp_nest* nest;
  const void* in[2];
  void* out;
  double t_submit;       // arrival: scheduled (hp_serve_submit_at) or the submit call
  size_t bytes;          // inputs + outputs + scratch counted against the budget
  size_t part_bytes, ticket_bytes;
  size_t part_off, ticket_off;
  uint8_t state;
};

struct Step {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  bool busy = false;
  std::vector<Request*> reqs;     // admitted into this step (stable deque elements)
  BatchNest* h_nests = nullptr;   // pinned staging
  BatchTile* h_tiles = nullptr;
  size_t cap_nests = 0, cap_tiles = 0;      // pinned capacities
  BatchNest* d_nests = nullptr;
  BatchTile* d_tiles = nullptr;
  size_t dcap_nests = 0, dcap_tiles = 0;    // device capacities
  unsigned long long* d_counters = nullptr;
};

// resident mode: one kernel instance at a time takes new tiles (two alternate)
struct ResidentInst {
  cudaStream_t stream = nullptr;
  cudaEvent_t ended = nullptr;
  unsigned long long* d_dev = nullptr;   // claim counter and mirrored tail / stop words
  bool running = false;                  // launched; its end not yet observed
  bool stopped = false;                  // its stop flag is written
  uint64_t base = 0;                     // ring index of its first tile
  double t_start = 0.0;
};

struct ResidentLive {
  Request* r;
  int slot;
  uint32_t seq;
  uint64_t t0;         // ring index of the request's first tile
  double t_admit;      // host time of its admission
};

struct Resident {
  int combo = -1;                        // the arithmetic (batch_combo), fixed by the first request
  int grid = 0;
  ResidentReq* h_reqs = nullptr;         // mapped page-locked host memory, with device aliases
  ResidentReq* d_reqs = nullptr;
  BatchTile* h_ring = nullptr;
  BatchTile* d_ring = nullptr;
  ResidentCtl* h_ctl = nullptr;
  ResidentCtl* d_ctl = nullptr;
  uint32_t* h_done = nullptr;
  uint32_t* d_done = nullptr;
  int32_t* h_status = nullptr;
  int32_t* d_status = nullptr;
  int32_t* d_counts = nullptr;           // device memory
  int32_t* d_err = nullptr;              // device error word of every served request
  ResidentInst inst[2];
  int cur = 0;
  uint64_t ring_next = 0;                // ring index of the next tile written
  double t_query = 0.0;                  // host time of the last event query
  std::vector<int> free_slots;
  std::vector<uint32_t> seq;
  std::vector<ResidentLive> live;
  std::vector<BatchTile> tiles;          // scratch
};

}  // namespace
}  // namespace hp

struct hp_server {
  size_t budget = 0;
  int max_slots = 0;
  int max_step = 4096;               // requests per step
  bool batching = true;
  bool resident = false;             // serve_batching 2: a resident kernel takes the tiles
  hp::Resident res;
  int device = 0, sms = 0;
  std::mutex mu;
  std::condition_variable cv_done;
  std::condition_variable cv_work;   // wakes an idle scheduler when a request arrives
  std::deque<uint64_t> queue;
  std::deque<hp::Request> reqs;      // ticket t is reqs[t - 1]; elements never move
  size_t bytes_in_flight = 0;
  int slots_used = 0;
  std::vector<hp::Step> steps;
  // scratch pools of grid-split plans
  void* part_pool = nullptr;
  int32_t* ticket_pool = nullptr;    // kept all-zero between uses
  size_t part_cap = 0, ticket_cap = 0;
  hp::RangeAlloc part_alloc, ticket_alloc;
  // statistics
  std::vector<double> lat_us;        // reserved and touched at creation: no copy or page fault under the lock
  double t_first = 0.0, t_last = 0.0;
  uint64_t n_done = 0;
  uint64_t n_steps = 0;
  size_t peak_bytes = 0;
  int peak_slots = 0;
  std::string error;
  std::atomic<bool> stop{false};
  std::thread th;
};

namespace hp {
namespace {

size_t request_bytes(const hp_nest* n, size_t* part_bytes, size_t* ticket_bytes) {
  const NestPlan& p = n->plan;
  const RectPlan& rp = p.rp;
  size_t b = 0;
  for (int i = 0; i < p.n_inputs; ++i) b += static_cast<size_t>(p.in_elems[i]) * p.in_elem_bytes;
  b += static_cast<size_t>(rp.O) * p.out_elem_bytes;
  *part_bytes = rp.G > 1 ? static_cast<size_t>(rp.items) * partial_bytes(p.prec, p.op) : 0;
  *ticket_bytes = rp.G > 1 ? static_cast<size_t>(rp.O) * sizeof(int32_t) : 0;
  return b + *part_bytes + *ticket_bytes;
}

// tiles of one request's nest (work items cut into ranges of about `target` elements)
void step_tiles(int nest, const RectPlan& rp, int64_t target, std::vector<BatchTile>& out) {
  if (rp.items == 0) return;
  int64_t per_item = rp.team == TEAM_MAP ? 1
                   : rp.split ? std::max<int64_t>(1, rp.R / std::max<int64_t>(1, rp.vn[0]) * rp.tile)
                              : std::max<int64_t>(1, rp.R);
  int64_t k = std::max<int64_t>(1, target / per_item);
  if (rp.team == TEAM_LANES) {
    const int64_t teams = (kBatchThreads / 32) * (32 / rp.L);
    k = (k + teams - 1) / teams * teams;
  }
  if (rp.team == TEAM_MAP) k = std::max<int64_t>(k, kBatchThreads);
  k = std::min<int64_t>(k, int64_t(1) << 30);
  for (int64_t i0 = 0; i0 < rp.items; i0 += k)
    out.push_back({nest, static_cast<int32_t>(std::min<int64_t>(k, rp.items - i0)), i0});
}

}  // namespace
}  // namespace hp

namespace hp {
namespace {

bool grow_pinned(void** p, size_t* cap, size_t need, size_t elem) {
  if (*cap >= need) return true;
  size_t n = std::max(need, *cap * 2 + 64);
  if (*p) cudaFreeHost(*p);
  *p = nullptr;
  *cap = 0;
  if (cudaMallocHost(p, n * elem) != cudaSuccess) return false;
  *cap = n;
  return true;
}

bool grow_device(void** p, size_t* cap, size_t need, size_t elem) {
  if (*cap >= need) return true;
  size_t n = std::max(need, *cap * 2 + 64);
  if (*p) cudaFree(*p);
  *p = nullptr;
  if (cudaMalloc(p, n * elem) != cudaSuccess) return false;
  *cap = n;
  return true;
}

// launch one step: all its requests in one persistent kernel per arithmetic
hp_status launch_batched(hp_server* s, Step& st) {
  const size_t n = st.reqs.size();
  std::vector<BatchTile> tiles[kBatchCombos];
  int64_t total = 0;
  for (const Request* r : st.reqs) {
    const RectPlan& rp = r->nest->plan.rp;
    total += rp.team == TEAM_MAP ? rp.O : rp.O * std::max<int64_t>(1, rp.R);
  }
  const int64_t target = std::max<int64_t>(1 << 14, total / (4 * static_cast<int64_t>(s->sms) * 8));
  if (!grow_pinned(reinterpret_cast<void**>(&st.h_nests), &st.cap_nests, n, sizeof(BatchNest)))
    return fail(HP_ENOMEM, "pinned step descriptors");
  for (size_t i = 0; i < n; ++i) {
    const Request& r = *st.reqs[i];
    const NestPlan& p = r.nest->plan;
    BatchNest& bn = st.h_nests[i];
    bn.rp = p.rp;
    bn.in0 = r.in[0];
    bn.in1 = r.in[1];
    bn.out = r.out;
    bn.part = r.part_bytes ? static_cast<char*>(s->part_pool) + r.part_off : nullptr;
    bn.tickets = r.ticket_bytes ? reinterpret_cast<int32_t*>(reinterpret_cast<char*>(s->ticket_pool) + r.ticket_off)
                                : nullptr;
    bn.err = r.nest->err;
    step_tiles(static_cast<int>(i), p.rp, target, tiles[batch_combo(p.prec, p.op)]);
  }
  size_t n_tiles = 0;
  for (auto& v : tiles) n_tiles += v.size();
  if (!grow_pinned(reinterpret_cast<void**>(&st.h_tiles), &st.cap_tiles, n_tiles, sizeof(BatchTile)))
    return fail(HP_ENOMEM, "pinned step tiles");
  if (!grow_device(reinterpret_cast<void**>(&st.d_nests), &st.dcap_nests, n, sizeof(BatchNest)) ||
      !grow_device(reinterpret_cast<void**>(&st.d_tiles), &st.dcap_tiles, n_tiles, sizeof(BatchTile)))
    return fail(HP_ENOMEM, "device step tables");
  size_t off = 0;
  int64_t first[kBatchCombos];
  for (int c = 0; c < kBatchCombos; ++c) {
    first[c] = static_cast<int64_t>(off);
    std::copy(tiles[c].begin(), tiles[c].end(), st.h_tiles + off);
    off += tiles[c].size();
  }
  cudaError_t e = cudaMemcpyAsync(st.d_nests, st.h_nests, n * sizeof(BatchNest), cudaMemcpyHostToDevice, st.stream);
  if (e == cudaSuccess && n_tiles)
    e = cudaMemcpyAsync(st.d_tiles, st.h_tiles, n_tiles * sizeof(BatchTile), cudaMemcpyHostToDevice, st.stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(st.d_counters, 0, kBatchCombos * sizeof(unsigned long long), st.stream);
  for (int c = 0; e == cudaSuccess && c < kBatchCombos; ++c) {
    if (tiles[c].empty()) continue;
    const int grid = static_cast<int>(std::min<int64_t>(static_cast<int64_t>(tiles[c].size()),
                                                        static_cast<int64_t>(batch_combo_blocks_per_sm(c)) * s->sms));
    BatchLaunch L{st.d_nests, st.d_tiles + first[c], static_cast<int64_t>(tiles[c].size()), st.d_counters + c, grid};
    e = launch_batch_combo(c, L, st.stream);
  }
  if (e == cudaSuccess) e = cudaEventRecord(st.done, st.stream);
  if (e != cudaSuccess) return fail(HP_ECUDA, std::string("serve step launch: ") + cudaGetErrorString(e));
  return HP_OK;
}

// plain mode: every request of the step launched alone with the single-nest kernels
hp_status launch_plain(hp_server* s, Step& st) {
  for (Request* r : st.reqs) {
    void* part = r->part_bytes ? static_cast<char*>(s->part_pool) + r->part_off : nullptr;
    const hp_status h = run_rect_with(r->nest, r->in, r->out, part, st.stream);
    if (h != HP_OK) return h;
  }
  const cudaError_t e = cudaEventRecord(st.done, st.stream);
  return e == cudaSuccess ? HP_OK : fail(HP_ECUDA, "serve event record");
}

// a request leaves the server (caller holds the lock)
void finish_req(hp_server* s, Request* r, bool ok, double t) {
  r->state = ok ? RQ_DONE : RQ_FAILED;
  s->bytes_in_flight -= r->bytes;
  s->slots_used -= 1;
  if (r->part_bytes) s->part_alloc.release(r->part_off, r->part_bytes);
  if (r->ticket_bytes) s->ticket_alloc.release(r->ticket_off, r->ticket_bytes);
  if (ok) {
    s->lat_us.push_back(t - r->t_submit);
    s->n_done += 1;
    s->t_last = t;
  }
}

void finish_step(hp_server* s, Step& st, bool ok) {
  const double t = now_us();
  std::lock_guard<std::mutex> lock(s->mu);
  for (Request* r : st.reqs) finish_req(s, r, ok, t);
  st.reqs.clear();
  st.busy = false;
  s->cv_done.notify_all();
}

// the device descriptor of an admitted request
BatchNest batch_nest_of(const hp_server* s, const Request& r) {
  BatchNest bn;
  bn.rp = r.nest->plan.rp;
  bn.in0 = r.in[0];
  bn.in1 = r.in[1];
  bn.out = r.out;
  bn.part = r.part_bytes ? static_cast<char*>(s->part_pool) + r.part_off : nullptr;
  bn.tickets = r.ticket_bytes ? reinterpret_cast<int32_t*>(reinterpret_cast<char*>(s->ticket_pool) + r.ticket_off)
                              : nullptr;
  bn.err = s->resident ? s->res.d_err : r.nest->err;
  return bn;
}

// how long an idle scheduler keeps polling before it sleeps on the condition variable
constexpr double kServeSpinUs = 2000.0;

// ---------------------------------------------------------------- resident mode
#ifndef HP_RESIDENT_CTAS_PER_SM
#define HP_RESIDENT_CTAS_PER_SM 0                             // resident CTAs per SM (0: one fewer than fit)
#endif
constexpr double kResidentEpochUs = 100000.0;                 // host time an instance takes new tiles
constexpr unsigned long long kResidentCapNs = 2000000000ull;  // device bound of one tile wait
constexpr uint64_t kResidentRing = uint64_t(1) << 16;         // tile ring entries
#ifndef HP_RESIDENT_TILE_ITERS
#define HP_RESIDENT_TILE_ITERS 4096                   // 2048: p50 15.3 us, 4096: 15.3, 8192: 15.9, 16384: 17.4
#endif
constexpr int64_t kResidentTileIters = HP_RESIDENT_TILE_ITERS; // iterations per tile, at least
constexpr int64_t kResidentMaxTiles = 1024;                   // tiles per request, about at most
constexpr double kResidentLateUs = 10e6;                      // a request not done 10 s after admission fails the server

template <class T>
bool alloc_mapped(T** h, T** d, size_t n) {
  *h = nullptr;
  *d = nullptr;
  if (cudaHostAlloc(reinterpret_cast<void**>(h), n * sizeof(T), cudaHostAllocMapped) != cudaSuccess) return false;
  std::memset(static_cast<void*>(*h), 0, n * sizeof(T));
  return cudaHostGetDevicePointer(reinterpret_cast<void**>(d), *h, 0) == cudaSuccess;
}

hp_status resident_init(hp_server* s) {
  Resident& R = s->res;
  if (!alloc_mapped(&R.h_reqs, &R.d_reqs, s->max_slots) || !alloc_mapped(&R.h_ring, &R.d_ring, kResidentRing) ||
      !alloc_mapped(&R.h_ctl, &R.d_ctl, 2) || !alloc_mapped(&R.h_done, &R.d_done, s->max_slots) ||
      !alloc_mapped(&R.h_status, &R.d_status, 2))
    return fail(HP_ENOMEM, "mapped page-locked memory (resident server tables)");
  if (cudaMalloc(&R.d_counts, sizeof(int32_t) * s->max_slots) != cudaSuccess ||
      cudaMemset(R.d_counts, 0, sizeof(int32_t) * s->max_slots) != cudaSuccess ||
      cudaMalloc(&R.d_err, sizeof(int32_t)) != cudaSuccess || cudaMemset(R.d_err, 0, sizeof(int32_t)) != cudaSuccess)
    return fail(HP_ENOMEM, "cudaMalloc (resident tile counts)");
  for (ResidentInst& I : R.inst) {
    if (cudaStreamCreateWithFlags(&I.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&I.ended, cudaEventDisableTiming) != cudaSuccess ||
        cudaMalloc(&I.d_dev, sizeof(unsigned long long) * kResidentDevWords) != cudaSuccess)
      return fail(HP_ECUDA, "resident server streams");
  }
  R.free_slots.resize(s->max_slots);
  for (int i = 0; i < s->max_slots; ++i) R.free_slots[i] = s->max_slots - 1 - i;
  R.seq.assign(s->max_slots, 0u);
  return HP_OK;
}

void resident_free(hp_server* s) {
  Resident& R = s->res;
  for (ResidentInst& I : R.inst) {
    if (I.stream) cudaStreamSynchronize(I.stream);
    if (I.ended) cudaEventDestroy(I.ended);
    if (I.stream) cudaStreamDestroy(I.stream);
    if (I.d_dev) cudaFree(I.d_dev);
  }
  if (R.d_counts) cudaFree(R.d_counts);
  if (R.d_err) cudaFree(R.d_err);
  if (R.h_reqs) cudaFreeHost(R.h_reqs);
  if (R.h_ring) cudaFreeHost(R.h_ring);
  if (R.h_ctl) cudaFreeHost(R.h_ctl);
  if (R.h_done) cudaFreeHost(R.h_done);
  if (R.h_status) cudaFreeHost(R.h_status);
}

void resident_stop(Resident& R, int i) {
  if (!R.inst[i].running || R.inst[i].stopped) return;
  __atomic_store_n(&R.h_ctl[i].stop, 1ull, __ATOMIC_RELEASE);   // after every tail store to it
  R.inst[i].stopped = true;
}

hp_status resident_launch(hp_server* s, int i) {
  Resident& R = s->res;
  ResidentInst& I = R.inst[i];
  if (R.grid == 0) {
    // one CTA per SM fewer than fit: other kernels keep room on every SM
    const int per_sm = resident_combo_blocks_per_sm(R.combo);
    const int use = HP_RESIDENT_CTAS_PER_SM > 0 ? std::min(HP_RESIDENT_CTAS_PER_SM, per_sm) : per_sm - 1;
    R.grid = std::max(1, use) * s->sms;
  }
  R.h_ctl[i].tail = 0;
  R.h_ctl[i].stop = 0;
  R.h_status[i] = 0;
  ResidentSource src{R.d_reqs, R.d_ring, kResidentRing - 1, R.ring_next, R.d_ctl + i, I.d_dev,
                     R.d_counts, R.d_done, R.d_status + i, kResidentCapNs};
  cudaError_t e = cudaMemsetAsync(I.d_dev, 0, sizeof(unsigned long long) * kResidentDevWords, I.stream);
  if (e == cudaSuccess) e = launch_resident_combo(R.combo, src, R.grid, I.stream);
  if (e == cudaSuccess) e = cudaEventRecord(I.ended, I.stream);
  if (e != cudaSuccess) return fail(HP_ECUDA, std::string("resident kernel launch: ") + cudaGetErrorString(e));
  I.running = true;
  I.stopped = false;
  I.base = R.ring_next;
  I.t_start = now_us();
  std::lock_guard<std::mutex> lock(s->mu);
  s->n_steps += 1;
  return HP_OK;
}

// every live request fails (an instance ended early or reported an error)
void resident_fail_all(hp_server* s, const std::string& why) {
  Resident& R = s->res;
  const double t = now_us();
  std::lock_guard<std::mutex> lock(s->mu);
  if (s->error.empty()) s->error = why;
  for (const ResidentLive& L : R.live) {
    finish_req(s, L.r, false, t);
    R.free_slots.push_back(L.slot);
  }
  R.live.clear();
  s->cv_done.notify_all();
}

// one pass of the resident scheduler; true when something happened
bool resident_pass(hp_server* s, double& last_active) {
  Resident& R = s->res;
  bool progress = false;
  // completions, read from the host words the kernel writes
  if (!R.live.empty()) {
    const double t = now_us();
    std::unique_lock<std::mutex> lock(s->mu, std::defer_lock);
    for (size_t j = 0; j < R.live.size();) {
      const ResidentLive L = R.live[j];
      if (__atomic_load_n(&R.h_done[L.slot], __ATOMIC_ACQUIRE) == L.seq) {
        if (!lock.owns_lock()) lock.lock();
        finish_req(s, L.r, true, t);
        R.free_slots.push_back(L.slot);
        R.live[j] = R.live.back();
        R.live.pop_back();
        progress = true;
      } else {
        ++j;
      }
    }
    if (progress) s->cv_done.notify_all();
  }
  // a device error word, or a request far past any plausible run time: the
  // server fails its live requests (and refuses new ones)
  if (!R.live.empty()) {
    bool bad = false;
    for (int i = 0; i < 2; ++i)
      if (R.inst[i].running && __atomic_load_n(&R.h_status[i], __ATOMIC_ACQUIRE) != 0) bad = true;
    if (bad) {
      resident_fail_all(s, "resident kernel reported a wait that gave up");
      progress = true;
    } else {
      const double t = now_us();
      for (const ResidentLive& L : R.live)
        if (t - L.t_admit > kResidentLateUs) {
          resident_fail_all(s, "a resident request did not complete within 10 s");
          progress = true;
          break;
        }
    }
  }
  // instances that ended: expected after a stop; otherwise every live request
  // fails (queried every 20 us: an event query costs about a microsecond)
  const double t_q = now_us();
  if (t_q - R.t_query >= 20.0) {
    R.t_query = t_q;
    for (int i = 0; i < 2; ++i) {
      ResidentInst& I = R.inst[i];
      if (!I.running) continue;
      const cudaError_t q = cudaEventQuery(I.ended);
      if (q == cudaErrorNotReady) continue;
      I.running = false;
      const int32_t st = __atomic_load_n(&R.h_status[i], __ATOMIC_ACQUIRE);
      if (q != cudaSuccess || st != 0 || !I.stopped)
        resident_fail_all(s, q != cudaSuccess ? std::string("resident kernel: ") + cudaGetErrorString(q)
                                              : "resident kernel ended early (device status " + std::to_string(st) +
                                                    ")");
      progress = true;
    }
  }
  bool queued;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    queued = !s->queue.empty() && s->error.empty();
  }
  if (queued) {
    // the instance that takes new tiles: the current one unless it is stopped
    if (R.inst[R.cur].stopped || !R.inst[R.cur].running) {
      const int nxt = R.inst[R.cur].stopped ? R.cur ^ 1 : R.cur;
      if (!R.inst[nxt].running) {
        R.cur = nxt;
        if (resident_launch(s, nxt) != HP_OK) {
          resident_fail_all(s, last_error_string());
          return true;
        }
        progress = true;
      }
    }
    ResidentInst& I = R.inst[R.cur];
    if (I.running && !I.stopped) {
      uint64_t low = R.ring_next;
      for (const ResidentLive& L : R.live) low = std::min(low, L.t0);
      int admitted = 0;
      std::vector<Request*> empty;
      {
        std::lock_guard<std::mutex> lock(s->mu);
        while (!s->queue.empty() && s->slots_used < s->max_slots && !R.free_slots.empty()) {
          Request& r = s->reqs[s->queue.front() - 1];
          if (s->bytes_in_flight + r.bytes > s->budget) break;
          const RectPlan& rp = r.nest->plan.rp;
          const int64_t total = rp.team == TEAM_MAP ? rp.O : rp.O * std::max<int64_t>(1, rp.R);
          R.tiles.clear();
          const int slot = R.free_slots.back();
          step_tiles(slot, rp, std::max(kResidentTileIters, total / kResidentMaxTiles), R.tiles);
          if (R.ring_next + R.tiles.size() - low > kResidentRing) break;
          if (r.part_bytes && !s->part_alloc.alloc(r.part_bytes, &r.part_off)) break;
          if (r.ticket_bytes && !s->ticket_alloc.alloc(r.ticket_bytes, &r.ticket_off)) {
            if (r.part_bytes) s->part_alloc.release(r.part_off, r.part_bytes);
            break;
          }
          s->queue.pop_front();
          s->bytes_in_flight += r.bytes;
          s->slots_used += 1;
          s->peak_bytes = std::max(s->peak_bytes, s->bytes_in_flight);
          s->peak_slots = std::max(s->peak_slots, s->slots_used);
          r.state = RQ_RUNNING;
          R.free_slots.pop_back();
          if (R.tiles.empty()) {   // no work items: done at once
            empty.push_back(&r);
            R.free_slots.push_back(slot);
            continue;
          }
          const uint32_t sq = ++R.seq[slot] == 0 ? ++R.seq[slot] : R.seq[slot];
          ResidentReq& d = R.h_reqs[slot];
          d.bn = batch_nest_of(s, r);
          d.n_tiles = static_cast<int32_t>(R.tiles.size());
          d.seq = sq;
          R.live.push_back({&r, slot, sq, R.ring_next, now_us()});
          for (const BatchTile& t : R.tiles) R.h_ring[R.ring_next++ & (kResidentRing - 1)] = t;
          admitted += 1;
        }
        const double t = now_us();
        for (Request* r : empty) finish_req(s, r, true, t);
        if (!empty.empty()) s->cv_done.notify_all();
      }
      if (admitted) {
        // publish: descriptors and tiles above are written before the tail
        __atomic_store_n(&R.h_ctl[R.cur].tail, R.ring_next - I.base, __ATOMIC_RELEASE);
      }
      if (admitted || !empty.empty()) progress = true;
    }
  }
  if (progress) last_active = now_us();
  // the current instance stops after its epoch (the next one starts at once
  // while work is pending) or once the server has been idle for a while
  ResidentInst& I = R.inst[R.cur];
  if (I.running && !I.stopped) {
    const double t = now_us();
    bool pending;
    {
      std::lock_guard<std::mutex> lock(s->mu);
      pending = !s->queue.empty();
    }
    const bool work = !R.live.empty() || pending;
    if (!work && t - last_active > kServeSpinUs) {
      resident_stop(R, R.cur);
    } else if (t - I.t_start > kResidentEpochUs && !R.inst[R.cur ^ 1].running) {
      resident_stop(R, R.cur);
      if (work) {   // without work the next admission starts the next instance
        R.cur ^= 1;
        if (resident_launch(s, R.cur) != HP_OK) resident_fail_all(s, last_error_string());
      }
    }
  }
  return progress;
}


void scheduler(hp_server* s) {
  cudaSetDevice(s->device);
  double last_active = now_us();
  while (!s->stop.load(std::memory_order_relaxed)) {
    bool progress = false;
    if (s->resident) {
      progress = resident_pass(s, last_active);
      if (!progress) {
        if (!s->res.live.empty() || now_us() - last_active < kServeSpinUs) {
          std::this_thread::yield();
        } else {
          std::unique_lock<std::mutex> lock(s->mu);
          s->cv_work.wait_for(lock, std::chrono::milliseconds(1),
                              [&] { return !s->queue.empty() || s->stop.load(std::memory_order_relaxed); });
        }
      }
      continue;
    }
    for (Step& st : s->steps) {
      if (!st.busy) continue;
      const cudaError_t q = cudaEventQuery(st.done);
      if (q == cudaSuccess || q != cudaErrorNotReady) {
        if (q != cudaSuccess) {
          std::lock_guard<std::mutex> lock(s->mu);
          s->error = std::string("step failed: ") + cudaGetErrorString(q);
        }
        finish_step(s, st, q == cudaSuccess);
        progress = true;
      }
    }
    for (Step& st : s->steps) {
      if (st.busy) continue;
      {
        // admit queued requests while a slot, the budget and scratch allow
        std::lock_guard<std::mutex> lock(s->mu);
        while (!s->queue.empty() && s->slots_used < s->max_slots &&
               static_cast<int>(st.reqs.size()) < s->max_step) {
          Request& r = s->reqs[s->queue.front() - 1];
          if (s->bytes_in_flight + r.bytes > s->budget) break;
          if (r.part_bytes && !s->part_alloc.alloc(r.part_bytes, &r.part_off)) break;
          if (r.ticket_bytes && !s->ticket_alloc.alloc(r.ticket_bytes, &r.ticket_off)) {
            if (r.part_bytes) s->part_alloc.release(r.part_off, r.part_bytes);
            break;
          }
          s->queue.pop_front();
          s->bytes_in_flight += r.bytes;
          s->slots_used += 1;
          s->peak_bytes = std::max(s->peak_bytes, s->bytes_in_flight);
          s->peak_slots = std::max(s->peak_slots, s->slots_used);
          r.state = RQ_RUNNING;
          st.reqs.push_back(&r);
        }
      }
      if (st.reqs.empty()) break;
      // a step of one request goes straight to the single-nest kernels (same
      // result bits, fewer API calls); larger steps run batched
      const hp_status h = (s->batching && st.reqs.size() > 1) ? launch_batched(s, st) : launch_plain(s, st);
      if (h != HP_OK) {
        {
          std::lock_guard<std::mutex> lock(s->mu);
          s->error = last_error_string();
        }
        finish_step(s, st, false);
      } else {
        st.busy = true;
        std::lock_guard<std::mutex> lock(s->mu);
        s->n_steps += 1;
      }
      progress = true;
    }
    if (progress) last_active = now_us();
    if (!progress) {
      // work on the GPU, or activity in the last kServeSpinUs: query again at
      // once (the scheduler owns a host core); idle longer: sleep until a
      // request arrives (a wake-up costs tens of microseconds)
      bool busy = false;
      for (const Step& st : s->steps) busy = busy || st.busy;
      if (busy || now_us() - last_active < kServeSpinUs) {
        std::this_thread::yield();
      } else {
        std::unique_lock<std::mutex> lock(s->mu);
        s->cv_work.wait_for(lock, std::chrono::milliseconds(1),
                            [&] { return !s->queue.empty() || s->stop.load(std::memory_order_relaxed); });
      }
    }
  }
}

}  // namespace
}  // namespace hp

using namespace hp;

extern "C" {

hp_status hp_serve_create(size_t mem_budget_bytes, int max_slots, int n_streams, hp_server** out) {
  if (!out) return fail(HP_EINVAL, "out is NULL");
  *out = nullptr;
  if (mem_budget_bytes == 0 || max_slots < 1 || n_streams < 1 || n_streams > 64)
    return fail(HP_EINVAL, "budget must be > 0, max_slots >= 1, n_streams in [1, 64]");
  hp_server* s = new (std::nothrow) hp_server();
  if (!s) return fail(HP_ENOMEM, "host allocation failed");
  s->budget = mem_budget_bytes;
  s->max_slots = max_slots;
  try {
    s->lat_us.resize(size_t(1) << 21);   // 16 MB: 2M latencies before the vector must grow
    s->lat_us.clear();
  } catch (...) {
    delete s;
    return fail(HP_ENOMEM, "host allocation failed");
  }
  s->batching = options().serve_batching != 0;
  s->resident = options().serve_batching == 2;
  cudaError_t e = cudaGetDevice(&s->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, s->device);
  if (e != cudaSuccess) {
    delete s;
    return fail(HP_ECUDA, std::string("no CUDA device: ") + cudaGetErrorString(e));
  }
  // scratch pools for grid-split plans: partials and (always zero) tickets
  s->part_cap = std::min<size_t>(mem_budget_bytes / 8 + (1 << 20), size_t(1) << 30);
  s->ticket_cap = std::min<size_t>(mem_budget_bytes / 64 + (1 << 20), size_t(64) << 20);
  if (cudaMalloc(&s->part_pool, s->part_cap) != cudaSuccess ||
      cudaMalloc(reinterpret_cast<void**>(&s->ticket_pool), s->ticket_cap) != cudaSuccess ||
      cudaMemset(s->ticket_pool, 0, s->ticket_cap) != cudaSuccess) {
    hp_serve_destroy(s);
    return fail(HP_ENOMEM, "cudaMalloc (serving scratch pools)");
  }
  s->part_alloc.reset(s->part_cap);
  s->ticket_alloc.reset(s->ticket_cap);
  s->steps.resize(n_streams);
  for (Step& st : s->steps) {
    if (cudaStreamCreateWithFlags(&st.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&st.done, cudaEventDisableTiming) != cudaSuccess ||
        cudaMalloc(&st.d_counters, kBatchCombos * sizeof(unsigned long long)) != cudaSuccess) {
      hp_serve_destroy(s);
      return fail(HP_ECUDA, "serving streams");
    }
  }
  if (s->resident) {
    const hp_status h = resident_init(s);
    if (h != HP_OK) {
      const std::string why = last_error_string();
      hp_serve_destroy(s);
      return fail(h, why);
    }
  }
  // load the persistent kernels now (their attributes and occupancy queries
  // load the code): a first launch that loads them took about 3 ms, which the
  // first requests would wait for
  if (s->resident) {
    for (int c = 0; c < kBatchCombos; ++c)
      if (resident_combo_ok(c)) (void)resident_combo_blocks_per_sm(c);
  } else if (s->batching) {
    for (int c = 0; c < kBatchCombos; ++c) (void)batch_combo_blocks_per_sm(c);
  }
  s->th = std::thread(scheduler, s);
  *out = s;
  return HP_OK;
}

namespace {

// arrival_us < 0: the request arrives now (latency counted from the call)
hp_status submit(hp_server* s, const hp_nest* shape, const void* const* in_dev, void* out_dev, double arrival_us,
                 uint64_t* ticket) {
  if (!s || !shape || !ticket) return fail(HP_EINVAL, "NULL argument");
  hp_nest* n = const_cast<hp_nest*>(shape);
  if (n->kind != NEST_RECT) return fail(HP_EUNSUPPORTED, "served nests must be rectangular");
  const RectPlan& rp = n->plan.rp;
  if (s->batching && rp.team == TEAM_BLOCK && (rp.C > 1 || rp.W > kBatchThreads / 32))
    return fail(HP_EUNSUPPORTED, "served block teams are single CTAs of at most 8 warps");
  if (n->plan.body == HP_BODY_GEOMETRIC) return fail(HP_EUNSUPPORTED, "the GEOMETRIC body is not served");
  const int combo = batch_combo(n->plan.prec, n->plan.op);
  if (s->resident && !resident_combo_ok(combo))
    return fail(HP_EUNSUPPORTED, "a resident server runs FP32 and int32 nests");
  if (s->resident) {
    // nothing of the nest is prepared on the device: a resident request needs
    // only its host plan (its error word is the server's), and allocating
    // here could wait for the running resident kernel
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != s->device || (n->device >= 0 && n->device != s->device))
      return fail(HP_EINVAL, "the nest, the calling thread and the server must share one device");
  } else {
    const hp_status st = ensure_device(n);
    if (st != HP_OK) return st;
  }
  for (int i = 0; i < n->plan.n_inputs; ++i)
    if (!in_dev || !in_dev[i]) return fail(HP_EINVAL, "missing device input");
  if (!out_dev && rp.O > 0) return fail(HP_EINVAL, "out_dev is NULL");
  Request r{};
  r.nest = n;
  r.in[0] = n->plan.n_inputs > 0 ? in_dev[0] : nullptr;
  r.in[1] = n->plan.n_inputs > 1 ? in_dev[1] : nullptr;
  r.out = out_dev;
  r.bytes = request_bytes(n, &r.part_bytes, &r.ticket_bytes);
  if (r.bytes > s->budget) return fail(HP_ENOMEM, "request alone exceeds the server's memory budget");
  if (r.part_bytes > s->part_cap || r.ticket_bytes > s->ticket_cap)
    return fail(HP_ENOMEM, "request's grid-split scratch exceeds the server's scratch pool");
  r.state = RQ_QUEUED;
  std::lock_guard<std::mutex> lock(s->mu);
  if (!s->error.empty()) return fail(HP_ECUDA, s->error);
  if (s->resident) {
    if (s->res.combo < 0) s->res.combo = combo;
    if (s->res.combo != combo)
      return fail(HP_EUNSUPPORTED, "a resident server runs one arithmetic: its first request's precision and op");
  }
  const double t = now_us();
  if (arrival_us > t) return fail(HP_EINVAL, "hp_serve_submit_at: the arrival time lies in the future");
  r.t_submit = arrival_us >= 0.0 ? arrival_us : t;
  if (s->reqs.empty()) s->t_first = r.t_submit;
  r.ticket = s->reqs.size() + 1;
  s->reqs.push_back(r);
  *ticket = r.ticket;
  s->queue.push_back(*ticket);
  s->cv_work.notify_one();
  return HP_OK;
}

}  // namespace

hp_status hp_serve_submit(hp_server* s, const hp_nest* shape, const void* const* in_dev, void* out_dev,
                          uint64_t* ticket) {
  return submit(s, shape, in_dev, out_dev, -1.0, ticket);
}

hp_status hp_serve_submit_at(hp_server* s, const hp_nest* shape, const void* const* in_dev, void* out_dev,
                             double arrival_us, uint64_t* ticket) {
  if (!(arrival_us >= 0.0)) return fail(HP_EINVAL, "hp_serve_submit_at: arrival time must be >= 0");
  return submit(s, shape, in_dev, out_dev, arrival_us, ticket);
}

double hp_serve_clock_us(void) { return now_us(); }

hp_status hp_serve_poll(hp_server* s, uint64_t ticket, int timeout_us) {
  if (!s) return fail(HP_EINVAL, "server is NULL");
  std::unique_lock<std::mutex> lock(s->mu);
  if (ticket == 0 || ticket > s->reqs.size()) return fail(HP_EINVAL, "unknown ticket");
  auto state = [&] { return s->reqs[ticket - 1].state; };
  if (state() < RQ_DONE && timeout_us != 0) {
    auto done = [&] { return state() >= RQ_DONE; };
    if (timeout_us < 0) s->cv_done.wait(lock, done);
    else s->cv_done.wait_for(lock, std::chrono::microseconds(timeout_us), done);
  }
  const uint8_t st = state();
  if (st == RQ_DONE) return HP_OK;
  if (st == RQ_FAILED) return fail(HP_ECUDA, "request failed: " + s->error);
  return timeout_us == 0 ? HP_EAGAIN : HP_ETIMEOUT;
}

hp_status hp_serve_stats(const hp_server* cs, double* p50, double* p99, double* p999, double* nps) {
  if (!cs) return fail(HP_EINVAL, "server is NULL");
  hp_server* s = const_cast<hp_server*>(cs);
  std::vector<double> v;
  double t0, t1;
  uint64_t n;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    v = s->lat_us;
    t0 = s->t_first;
    t1 = s->t_last;
    n = s->n_done;
  }
  auto pct = [&](double q) {
    if (v.empty()) return 0.0;
    const size_t k = std::min(v.size() - 1, static_cast<size_t>(q * static_cast<double>(v.size() - 1) + 0.5));
    std::nth_element(v.begin(), v.begin() + static_cast<long>(k), v.end());
    return v[k];
  };
  if (p50) *p50 = pct(0.5);
  if (p99) *p99 = pct(0.99);
  if (p999) *p999 = pct(0.999);
  if (nps) *nps = (n > 0 && t1 > t0) ? static_cast<double>(n) / ((t1 - t0) * 1e-6) : 0.0;
  return HP_OK;
}

hp_status hp_serve_counters(const hp_server* cs, uint64_t* completed, uint64_t* steps, size_t* peak_bytes,
                            int32_t* peak_slots) {
  if (!cs) return fail(HP_EINVAL, "server is NULL");
  hp_server* s = const_cast<hp_server*>(cs);
  std::lock_guard<std::mutex> lock(s->mu);
  if (completed) *completed = s->n_done;
  if (steps) *steps = s->n_steps;
  if (peak_bytes) *peak_bytes = s->peak_bytes;
  if (peak_slots) *peak_slots = s->peak_slots;
  return HP_OK;
}

void hp_serve_destroy(hp_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stop.store(true);
  }
  s->cv_work.notify_all();
  if (s->th.joinable()) s->th.join();
  if (s->resident) {
    resident_stop(s->res, 0);
    resident_stop(s->res, 1);
    resident_free(s);
  }
  for (Step& st : s->steps) {
    if (st.stream) cudaStreamSynchronize(st.stream);
    if (st.done) cudaEventDestroy(st.done);
    if (st.stream) cudaStreamDestroy(st.stream);
    if (st.h_nests) cudaFreeHost(st.h_nests);
    if (st.h_tiles) cudaFreeHost(st.h_tiles);
    if (st.d_nests) cudaFree(st.d_nests);
    if (st.d_tiles) cudaFree(st.d_tiles);
    if (st.d_counters) cudaFree(st.d_counters);
  }
  if (s->part_pool) cudaFree(s->part_pool);
  if (s->ticket_pool) cudaFree(s->ticket_pool);
  delete s;
}

}  // extern "C"
