// batch_kernels.cuh — one persistent launch over the tiles of many nests.
//
// Every CTA runs a dynamic schedule at grid level (Sec. 3.5): tiles are taken
// from an atomic counter until the table is exhausted.  A tile is a range of
// work items of one nest; it runs with that nest's own plan and with exactly
// the per-thread fold order and team tree of rect_block_kernel /
// rect_lanes_kernel, so every nest's outputs equal those of hp_nest_run on it,
// bit for bit.  Nests split over grid parts fold their parts with
// rect_combine_kernel's combine (combine_parts) once the last part of an
// output has arrived (a per-output ticket counter; nobody waits on it).
//
// The CTA is warp-specialised.  One producer warp takes the tiles, copies each
// tile's nest descriptor into a small tile queue in shared memory and, when
// the tile's inputs form one contiguous range (a single reduced virtual level
// of stride 1: every planner map), streams that range through a ring of
// shared-memory stages with 1-D bulk copies (cp.async.bulk, completion counted
// in bytes on one mbarrier per stage).  The range is widened to 16-byte
// granules, so any alignment of the nest's data streams at full width.  Eight
// consumer warps fold from the ring in phases: a phase waits for the stages
// that cover its window of iterations, folds them in the order fold_item
// would, and releases the stages below its end.  The producer runs up to a
// ring ahead, across item and tile boundaries, so HBM reads never drain at a
// reduction.  Tiles that cannot stream (GEOMETRIC / AFFINE bodies, several
// reduced virtual levels, maps without reduction) fold from global memory.
//
// Every wait is bounded in time: one that runs out sets the nest's device
// error word (code 3, read by hp_nest_check) and a CTA-wide abort flag, after
// which the CTA skips the remaining waits, leaves at the next tile boundary
// and lets its bulk copies land before it exits.
#pragma once

#include "rect_kernels.cuh"

namespace hp {

constexpr int kBatchThreads = 256;                       // consumer threads: block teams of up to 8 warps
constexpr int kBatchWarps = kBatchThreads / 32;
constexpr int kBatchAllThreads = kBatchThreads + 32;     // + the producer warp
#ifndef HP_BATCH_STAGE_BYTES
#define HP_BATCH_STAGE_BYTES 16384
#endif
#ifndef HP_BATCH_STAGES
#define HP_BATCH_STAGES 4
#endif
constexpr int kStageBytes = HP_BATCH_STAGE_BYTES;        // one ring stage
constexpr int kStages = HP_BATCH_STAGES;
constexpr int kRingBytes = kStages * kStageBytes;        // a power of two (ring offsets are masked)
static_assert((kStageBytes & (kStageBytes - 1)) == 0 && (kStages & (kStages - 1)) == 0 && kStageBytes >= 1024,
              "ring stages: powers of two");
constexpr int kTileQueue = 4;                            // tiles the producer may run ahead
constexpr int kLanesWindowBytes = kRingBytes / 2 - 16;   // largest window of a lanes-team phase
constexpr int kBlockPhaseBytes = 2 * kStageBytes;        // window of a block-team phase (whole steps)
constexpr unsigned long long kBatchWaitNs = 1000000000ull;  // a wait gives up after 1 s
constexpr int32_t kErrStageWait = 3;                     // device error code of a wait that gave up
#ifndef HP_BATCH_MIN_BLOCKS
#define HP_BATCH_MIN_BLOCKS 3                            // resident CTAs per SM the registers are sized for
#endif

// one nest of a batch, as the device sees it
struct BatchNest {
  RectPlan rp;
  const void* in0;
  const void* in1;
  void* out;
  void* part;          // grid-part partials (G > 1)
  int32_t* tickets;    // per output (G > 1)
  int32_t* err;        // the nest's device error word
};

struct BatchTile {
  int32_t nest;
  int32_t count;       // items
  int64_t item0;
};

// a tile as the producer hands it to the consumers
struct BatchQueued {
  BatchNest bn;
  BatchTile t;
  int64_t k0;          // ring stage (running count) holding the first byte of the stream
  uint64_t a0;         // stream start: the tile's first input byte rounded down to 16 bytes
  uint64_t gA;         // address of the nest's input A
  int32_t nst;         // stages of the stream (0: the tile folds from global memory)
  int32_t end;         // 1: no more tiles
  int32_t req_tiles;   // resident executor: tiles of the tile's request
  uint32_t req_seq;    // resident executor: the request's sequence number in its slot
};

// Can a nest's tiles stream through the ring?  One reduced virtual level of
// stride 1 makes every item (and every tile: consecutive items are adjacent)
// one contiguous range of A; a lanes-team phase must hold at least one item.
__host__ __device__ inline bool batch_streams(const RectPlan& p) {
  if (p.team == TEAM_MAP || p.nv != 1 || p.vstride[0] != 1 || p.R < 1) return false;
  if (p.body != HP_BODY_LOAD && p.body != HP_BODY_DOT_BCAST) return false;
  if (p.team == TEAM_LANES && p.R * 4 > kLanesWindowBytes) return false;
  return true;
}

// iterations [base + lo, base + hi) of A that work item `item` folds (one reduced level)
__host__ __device__ inline void batch_item_span(const RectPlan& p, int64_t item, int64_t& base, int64_t& lo,
                                                int64_t& hi) {
  if (p.G == 1) {
    base = item * p.R;
    lo = 0;
    hi = p.vn[0];
    return;
  }
  const int64_t o = item / p.G, g = item - o * p.G;
  base = o * p.R;
  lo = 0;
  hi = p.vn[0];
  if (p.split) {
    lo = g * p.tile;
    hi = (lo + p.tile < p.vn[0]) ? lo + p.tile : p.vn[0];
  }
}

// where a nest's results go (copied to registers for the streamed paths)
struct EmitTo {
  void* out;
  void* part;          // grid-part partials (G > 1)
  int32_t* tickets;    // per output (G > 1)
  int32_t G;
};

// the last part of an output to arrive combines them all (the combine of
// rect_combine_kernel, so results equal hp_nest_run's); out of line, so that
// its registers do not weigh on the streaming loops that call batch_emit
template <class Op>
__device__ __forceinline__ void batch_combine(const typename Op::Acc* pp, int32_t G, typename Op::Out* out) {
  *out = combine_parts<Op>(pp, G, nullptr);
}

template <class Op>
__device__ __forceinline__ void batch_emit(const EmitTo& to, int64_t item, typename Op::Acc a) {
  using Acc = typename Op::Acc;
  if (to.G == 1) {
    static_cast<typename Op::Out*>(to.out)[item] = Op::finish(a);
    return;
  }
  Acc* part = static_cast<Acc*>(to.part);
  const int64_t o = item / to.G;
  part[item] = a;
  __threadfence();  // publish the partial before taking the ticket
  if (atomicAdd(&to.tickets[o], 1) == to.G - 1) {
    __threadfence();  // all parts of this output are visible
    batch_combine<Op>(part + o * to.G, to.G, static_cast<typename Op::Out*>(to.out) + o);
    to.tickets[o] = 0;  // ready for the next run
  }
}
template <class Op>
__device__ __forceinline__ void batch_emit(const RectPlan& p, const BatchNest& bn, int64_t item, typename Op::Acc a) {
  batch_emit<Op>(EmitTo{bn.out, bn.part, bn.tickets, p.G}, item, a);
}

// ---------------------------------------------------------------- mbarrier / bulk-copy primitives
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile(
      "{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(bar)
      : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint32_t bar, uint32_t bytes) {
  asm volatile(
      "{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(bar), "r"(bytes)
      : "memory");
}
__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
  return t;
}
__device__ __forceinline__ int ld_abort(uint32_t at) {
  int v;
  asm volatile("ld.volatile.shared.s32 %0, [%1];\n" : "=r"(v) : "r"(at) : "memory");
  return v;
}
__device__ __forceinline__ void st_abort(uint32_t at) {
  asm volatile("st.volatile.shared.s32 [%0], 1;\n" ::"r"(at) : "memory");
}
// the slow part of a wait: poll until the phase of parity `parity` completes;
// false when the CTA's abort flag (shared address abort_at, 0 = none) is set
// or the wait ran out of time
static __device__ __noinline__ bool mbar_wait_slow(uint32_t bar, uint32_t parity, uint32_t abort_at,
                                                   unsigned long long limit_ns) {
  const unsigned long long t0 = global_ns();
  for (uint32_t i = 1;; ++i) {
    if (mbar_test(bar, parity)) return true;
    if ((i & 31u) == 0) {
      if (abort_at && ld_abort(abort_at)) return false;
      if (global_ns() - t0 > limit_ns) return false;
    }
  }
}
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint32_t abort_at,
                                          unsigned long long limit_ns = kBatchWaitNs) {
  return mbar_test(bar, parity) || mbar_wait_slow(bar, parity, abort_at, limit_ns);
}
// 1-D bulk copy global -> shared, completion counted on `bar` in bytes
// (both addresses 16-byte aligned, bytes a multiple of 16)
__device__ __forceinline__ void bulk_g2s(uint32_t dst, uint64_t src, uint32_t bytes, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}
// barrier of the consumer warps only (the producer warp never joins it)
__device__ __forceinline__ void consumer_sync() {
  asm volatile("bar.sync 1, %0;\n" ::"n"(kBatchThreads) : "memory");
}
// the same barrier, returning to every consumer thread the OR of `flag` over
// all of them (one decision even when the producer changes a flag meanwhile)
__device__ __forceinline__ bool consumer_sync_or(int flag) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred pa, pr;\n setp.ne.s32 pa, %1, 0;\n bar.red.or.pred pr, 1, %2, pa;\n"
      " selp.u32 %0, 1, 0, pr;\n}\n"
      : "=r"(r)
      : "r"(flag), "n"(kBatchThreads)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ void lds4(uint32_t a, float (&r)[4]) {
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];\n"
               : "=f"(r[0]), "=f"(r[1]), "=f"(r[2]), "=f"(r[3])
               : "r"(a));
}
__device__ __forceinline__ void lds4(uint32_t a, int32_t (&r)[4]) {
  asm volatile("ld.shared.v4.s32 {%0, %1, %2, %3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}
__device__ __forceinline__ void lds1(uint32_t a, float& r) {
  asm volatile("ld.shared.f32 %0, [%1];\n" : "=f"(r) : "r"(a));
}
__device__ __forceinline__ void lds1(uint32_t a, int32_t& r) {
  asm volatile("ld.shared.s32 %0, [%1];\n" : "=r"(r) : "r"(a));
}

// ---------------------------------------------------------------- folding from the ring
// Iteration e of A sits at ring byte (4 e + shift) mod kRingBytes (32-bit
// arithmetic suffices: only the low bits survive the mask); the broadcast
// operand of DOT_BCAST still comes from global memory (L1/L2-resident).
template <class Op, bool DOT>
struct RingFold {
  using In = typename Op::In;
  uint32_t ring;      // shared address of the ring
  uint32_t shift;
  const In* w;
  template <int V>
  __device__ __forceinline__ Vals<Op, V> load(uint32_t off, const In* wp, int32_t x) const {
    Vals<Op, V> v;
    const uint32_t a = ring + ((off + 4u * static_cast<uint32_t>(x)) & static_cast<uint32_t>(kRingBytes - 1));
    if constexpr (V == 4) {
      lds4(a, v.a);
    } else {
#pragma unroll
      for (int i = 0; i < V; ++i) lds1(a + 4u * i, v.a[i]);
    }
    if constexpr (DOT) {
      if constexpr (V == 4) {
        const auto r = ld_keep4(wp + x);
        v.b[0] = r.x;
        v.b[1] = r.y;
        v.b[2] = r.z;
        v.b[3] = r.w;
      } else {
#pragma unroll
        for (int i = 0; i < V; ++i) v.b[i] = ld_keep(wp + x + i);
      }
    }
    return v;
  }
  template <int V>
  __device__ __forceinline__ void apply(typename Op::Acc (&acc)[V], const Vals<Op, V>& v) const {
    if constexpr (DOT) fold_vals_dot<Op, V>(acc, v.a, v.b);
    else fold_vals_load<Op, V>(acc, v.a);
  }
  // the thread's iterations lo + x for x = x0, x0 + P, ... < x1 of the item
  // whose reduced level starts at flat iteration `first` (= base + lo), in
  // the order fold_item visits them, several loads in flight before their folds
  template <int V>
  __device__ __forceinline__ void run(int64_t first, int64_t lo, int32_t x0, int32_t x1, int32_t P,
                                      typename Op::Acc (&acc)[V]) const {
    run_at<V>(static_cast<uint32_t>(first) * 4u + shift, DOT ? w + lo : nullptr, x0, x1, P, acc);
  }
  // the same with the ring byte (before the mask) of iteration lo and the
  // broadcast operand at lo given
  template <int V>
  __device__ __forceinline__ void run_at(uint32_t off, const In* wp, int32_t x0, int32_t x1, int32_t P,
                                         typename Op::Acc (&acc)[V]) const {
    int32_t x = x0;
    if constexpr (V == 1) {
      for (; x + 3 * P < x1; x += 4 * P) {
        const auto v0 = load<V>(off, wp, x);
        const auto v1 = load<V>(off, wp, x + P);
        const auto v2 = load<V>(off, wp, x + 2 * P);
        const auto v3 = load<V>(off, wp, x + 3 * P);
        apply<V>(acc, v0);
        apply<V>(acc, v1);
        apply<V>(acc, v2);
        apply<V>(acc, v3);
      }
    } else {
      for (; x + P < x1; x += 2 * P) {
        const auto v0 = load<V>(off, wp, x);
        const auto v1 = load<V>(off, wp, x + P);
        apply<V>(acc, v0);
        apply<V>(acc, v1);
      }
    }
    for (; x < x1; x += P) apply<V>(acc, load<V>(off, wp, x));
  }

  // Fold two items together: the same iterations x = x0, x0 + P, ... < x1
  // of items A and B, whose iteration 0 sits at ring bytes (before the mask)
  // offA and offA + dist.  Each item sees exactly the operation sequence of
  // run_at; the two chains are independent (twice the work in flight per
  // thread) and, for FP32 sums of one slot, advance as packed FP32x2 pairs.
  template <int V>
  __device__ __forceinline__ void run_pair(uint32_t offA, uint32_t dist, int32_t x0, int32_t x1, int32_t P,
                                           typename Op::Acc (&A)[V], typename Op::Acc (&B)[V]) const {
    const uint32_t a0 = (offA + 4u * static_cast<uint32_t>(x0)) & static_cast<uint32_t>(kRingBytes - 1);
    const In* wp = DOT ? w : nullptr;
    if (x0 >= x1) return;
    if (a0 + dist + 4u * static_cast<uint32_t>(x1 - x0) <= static_cast<uint32_t>(kRingBytes)) {
      // neither item wraps around the end of the ring: linear addresses
      const uint32_t step = 4u * static_cast<uint32_t>(P);
      uint32_t pa = ring + a0;
      for (int32_t x = x0; x < x1; x += P, pa += step) {
        Vals<Op, V> va, vb;
        if constexpr (V == 4) {
          lds4(pa, va.a);
          lds4(pa + dist, vb.a);
        } else {
#pragma unroll
          for (int i = 0; i < V; ++i) {
            lds1(pa + 4u * i, va.a[i]);
            lds1(pa + dist + 4u * i, vb.a[i]);
          }
        }
        if constexpr (DOT) load_w<V>(wp, x, va, vb);
        apply2<V>(A, B, va, vb);
      }
    } else {
      for (int32_t x = x0; x < x1; x += P) {
        Vals<Op, V> va = load<V>(offA, wp, x), vb = load<V>(offA + dist, wp, x);
        apply2<V>(A, B, va, vb);
      }
    }
  }
  template <int V>
  __device__ __forceinline__ void load_w(const In* wp, int32_t x, Vals<Op, V>& va, Vals<Op, V>& vb) const {
    if constexpr (V == 4) {
      const auto r = ld_keep4(wp + x);
      va.b[0] = vb.b[0] = r.x;
      va.b[1] = vb.b[1] = r.y;
      va.b[2] = vb.b[2] = r.z;
      va.b[3] = vb.b[3] = r.w;
    } else {
#pragma unroll
      for (int i = 0; i < V; ++i) va.b[i] = vb.b[i] = ld_keep(wp + x + i);
    }
  }
  template <int V>
  __device__ __forceinline__ void apply2(typename Op::Acc (&A)[V], typename Op::Acc (&B)[V], const Vals<Op, V>& va,
                                         const Vals<Op, V>& vb) const {
    if constexpr (V == 1 && std::is_same<Op, OpF32Comp>::value) {
      float2 sp = make_float2(A[0].s, B[0].s), cp = make_float2(A[0].c, B[0].c);
      if constexpr (DOT) comp_prod_pair(sp, cp, make_float2(va.a[0], vb.a[0]), make_float2(va.b[0], vb.b[0]));
      else comp_add_pair(sp, cp, make_float2(va.a[0], vb.a[0]));
      A[0] = {sp.x, cp.x};
      B[0] = {sp.y, cp.y};
    } else if constexpr (V == 1 && std::is_same<Op, OpF32Sum>::value) {
      float2 sp = make_float2(A[0], B[0]);
      if constexpr (DOT) sp = fma2(make_float2(va.a[0], vb.a[0]), make_float2(va.b[0], vb.b[0]), sp);
      else sp = add2(sp, make_float2(va.a[0], vb.a[0]));
      A[0] = sp.x;
      B[0] = sp.y;
    } else {
      apply<V>(A, va);
      apply<V>(B, vb);
    }
  }
};

// geometry of a streamed nest, in registers
struct RingGeom {
  int64_t R;           // reduced iterations per output
  int64_t vn0;         // extent of the (single) reduced virtual level
  int64_t tile;        // iterations per grid part
  int32_t G;           // grid parts per output
  int32_t P;           // slots of the reduced level: iterations per step
};
__device__ __forceinline__ void ring_span(const RingGeom& g, int64_t item, int64_t& base, int64_t& lo, int64_t& hi) {
  if (g.G == 1) {
    base = item * g.R;
    lo = 0;
    hi = g.vn0;
    return;
  }
  const int64_t o = item / g.G, part = item - o * g.G;
  base = o * g.R;
  lo = part * g.tile;
  hi = (lo + g.tile < g.vn0) ? lo + g.tile : g.vn0;
}

// ---------------------------------------------------------------- tiles folded from global memory
// items [item0, item0 + count) of a block-team nest: one item at a time, the
// plan's W warps fold, the consumer warps combine them in warp order
template <class Op, int V, class Body>
__device__ __forceinline__ void batch_block_items(const RectPlan& p, const Body& body, const BatchNest& bn,
                                                  int64_t item0, int count, typename Op::Acc* wsh) {
  using Acc = typename Op::Acc;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool active = warp < p.W;
  const int grp = lane / p.grp_lanes, lig = lane % p.grp_lanes;
  int32_t slot[kMaxV];
#pragma unroll
  for (int v = 0; v < kMaxV; ++v) slot[v] = warp * p.cw[v] + grp * p.cg[v] + lig * p.cl[v];
  for (int m = 0; m < count; ++m) {
    const int64_t item = item0 + m;
    const int64_t o = item / p.G, g = item - o * p.G;
    Acc acc[V];
#pragma unroll
    for (int i = 0; i < V; ++i) acc[i] = Op::ident();
    if (active) fold_item<Op, V>(p, body, o, g, slot, acc);
    const Acc a = lanes_allreduce<Op>(fold_vec<Op, V>(acc), 32);
    if (lane == 0 && active) wsh[warp] = a;
    consumer_sync();
    if (tid == 0) {
      Acc r = wsh[0];
      for (int w = 1; w < p.W; ++w) r = Op::combine(r, wsh[w]);
      batch_emit<Op>(p, bn, item, r);
    }
    consumer_sync();
  }
}

// items of a lanes-team nest: every group of L lanes of the consumer warps is a team
template <class Op, int V, class Body>
__device__ __forceinline__ void batch_lanes_items(const RectPlan& p, const Body& body, const BatchNest& bn,
                                                  int64_t item0, int count) {
  using Acc = typename Op::Acc;
  const int L = p.L;
  const int tid = threadIdx.x, lane = tid & 31;
  const int lt = lane % L;
  const int grp = lt / p.grp_lanes, lig = lt % p.grp_lanes;
  int32_t slot[kMaxV];
#pragma unroll
  for (int v = 0; v < kMaxV; ++v) slot[v] = grp * p.cg[v] + lig * p.cl[v];
  const int teams = kBatchWarps * (32 / L);
  const int team = tid / L;
  for (int b = 0; b < count; b += teams) {
    const bool valid = b + team < count;
    const int64_t item = item0 + b + team;
    Acc acc[V];
#pragma unroll
    for (int i = 0; i < V; ++i) acc[i] = Op::ident();
    if (valid) {
      const int64_t o = item / p.G, g = item - o * p.G;
      fold_item<Op, V>(p, body, o, g, slot, acc);
    }
    const Acc a = lanes_allreduce<Op>(fold_vec<Op, V>(acc), L);
    if (valid && lt == 0) batch_emit<Op>(p, bn, item, a);
  }
}

// a nest without reduction: one output per iteration
template <class Op, class Body>
__device__ __forceinline__ void batch_map_items(const Body& body, const BatchNest& bn, int64_t item0, int count) {
  for (int k = threadIdx.x; k < count; k += kBatchThreads) {
    typename Op::Acc acc[1] = {Op::ident()};
    body.template fold<1>(acc, item0 + k, 0);
    static_cast<typename Op::Out*>(bn.out)[item0 + k] = Op::finish(acc[0]);
  }
}

// ---------------------------------------------------------------- tiles streamed through the ring
// Consumer-side view of the ring for one tile.  `ready` (stages this thread
// has seen complete) and `rel` (stages this warp has released) run over the
// CTA's whole stage sequence and advance identically in every thread.
struct RingView {
  uint32_t full, empty;   // shared addresses of the stage barriers; the abort flag sits 8 bytes below `full`
  uint32_t errp;          // shared address of the tile's pointer to its nest's error word
  int64_t k0;             // first stage of the tile
  uint64_t off0;          // stream byte of iteration e is 4 e + off0 (mod 2^64; off0 = A - a0)
};

// a stage wait of tile `rv` gave up: abort the CTA, flag the nest
static __device__ __noinline__ void ring_give_up(uint32_t full, uint32_t errp) {
  if (ld_abort(full - 8u)) return;
  st_abort(full - 8u);
  unsigned long long e;
  asm volatile("ld.shared.u64 %0, [%1];\n" : "=l"(e) : "r"(errp) : "memory");
  if (e) atomicExch(reinterpret_cast<int32_t*>(e), kErrStageWait);
}

// ring stage index holding iteration e of the tile's nest
__device__ __forceinline__ int64_t ring_stage(const RingView& r, int64_t e) {
  return r.k0 + static_cast<int64_t>((static_cast<uint64_t>(e) * 4u + r.off0) / kStageBytes);
}
// wait until every stage holding iterations before e_hi has landed
__device__ __forceinline__ void ring_wait(const RingView& r, int64_t e_hi, int64_t& ready) {
  const int64_t last = ring_stage(r, e_hi - 1);
  for (; ready <= last; ++ready) {
    const uint32_t bar = r.full + 8u * static_cast<uint32_t>(ready & (kStages - 1));
    if (!mbar_wait(bar, static_cast<uint32_t>((ready / kStages) & 1), r.full - 8u)) ring_give_up(r.full, r.errp);
  }
}
// release (for this warp) every stage below `lim`
__device__ __forceinline__ void ring_release(const RingView& r, int64_t lim, int64_t& rel) {
  if (rel >= lim) return;
  __syncwarp();   // every lane's reads of these stages are done
  for (; rel < lim; ++rel)
    if ((threadIdx.x & 31) == 0) mbar_arrive(r.empty + 8u * static_cast<uint32_t>(rel & (kStages - 1)));
}

// Reduce the partials of B items (part[r] = item r) over the L lanes of a
// team in one go: recursive halving, each step handing half of the items to
// the xor partner and combining the lower lane's partial first.  Every item
// gets exactly the tree that lanes_allreduce builds at the team's lane 0, at
// about one combine per item instead of log2(L).  On return part[0] of lane
// lt holds item lt / (L / B) (B a power of two, B <= L).
template <class Op, int B>
__device__ __forceinline__ void lanes_reduce_many(typename Op::Acc (&part)[B], int L, int lt) {
  using Acc = typename Op::Acc;
  int m = L >> 1;
#pragma unroll
  for (int cnt = B; cnt > 1; cnt >>= 1, m >>= 1) {
    const bool up = (lt & m) != 0;
#pragma unroll
    for (int i = 0; i < cnt / 2; ++i) {
      const Acc send = up ? part[i] : part[i + cnt / 2];
      const Acc keep = up ? part[i + cnt / 2] : part[i];
      const Acc recv = Op::shfl_xor(send, m, L);
      part[i] = up ? Op::combine(recv, keep) : Op::combine(keep, recv);
    }
  }
  for (; m >= 1; m >>= 1) {
    const Acc o = Op::shfl_xor(part[0], m, L);
    part[0] = (lt & m) ? Op::combine(o, part[0]) : Op::combine(part[0], o);
  }
}
constexpr int kReduceBatch = 4;   // items reduced together

// block team, streamed.  Items go in chunks of up to kMaxM: each item is
// folded in phases of whole steps (about two stages; a short remainder joins
// the last phase), its warp partials are parked in shared memory, and after
// one consumer barrier per chunk the first threads combine and emit the
// chunk's items in parallel (the ticket round trips of split items overlap).
// The partials alternate between two buffers, so nobody waits for the emits.
template <class Op, int V, class Fold>
__device__ __forceinline__ void ring_block_items(const RingGeom& gm, const Fold& fold, const BatchNest& bn, int W,
                                                 int32_t s0, int64_t item0, int count, const RingView& rv,
                                                 int64_t& ready, int64_t& rel,
                                                 typename Op::Acc (*wsh)[kMaxM][kBatchWarps]) {
  using Acc = typename Op::Acc;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool active = warp < W;
  const int32_t P = gm.P;
  const int32_t KP = P * ((kBlockPhaseBytes / 4) / P > 0 ? (kBlockPhaseBytes / 4) / P : 1);
  int buf = 0;
  for (int m0 = 0; m0 < count; m0 += kMaxM, buf ^= 1) {
    const int mc = (count - m0 < kMaxM) ? count - m0 : kMaxM;
    for (int mb = 0; mb < mc; mb += kReduceBatch) {
      Acc part[kReduceBatch];
#pragma unroll
      for (int r = 0; r < kReduceBatch; ++r) {
        Acc acc[V];
#pragma unroll
        for (int i = 0; i < V; ++i) acc[i] = Op::ident();
        if (mb + r < mc) {
          int64_t base, lo, hi;
          ring_span(gm, item0 + m0 + mb + r, base, lo, hi);
          const int32_t n = static_cast<int32_t>(hi - lo);   // at most a part: below 2^31 when streamed
          for (int32_t w0 = 0; w0 < n;) {
            int32_t w1 = (n - w0 > KP) ? w0 + KP : n;
            if (n - w1 < KP / 2) w1 = n;
            ring_wait(rv, base + lo + w1, ready);
            if (active) fold.template run<V>(base + lo, lo, w0 + s0, w1, P, acc);
            ring_release(rv, ring_stage(rv, base + lo + w1), rel);
            w0 = w1;
          }
        }
        part[r] = fold_vec<Op, V>(acc);
      }
      lanes_reduce_many<Op, kReduceBatch>(part, 32, lane);
      const int k = lane / (32 / kReduceBatch);
      if ((lane & (32 / kReduceBatch - 1)) == 0 && active && mb + k < mc) wsh[buf][mb + k][warp] = part[0];
    }
    consumer_sync();
    if (tid < mc) {
      Acc r = wsh[buf][tid][0];
      for (int w = 1; w < W; ++w) r = Op::combine(r, wsh[buf][tid][w]);
      batch_emit<Op>(bn.rp, bn, item0 + m0 + tid, r);
    }
  }
}

// lanes teams, streamed: a phase holds as many consecutive items as fit half
// the ring, in whole rounds of one item per team where possible; each team
// folds the items of its index in every round
template <class Op, int V, class Fold>
__device__ __forceinline__ void ring_lanes_items(const RingGeom& gm, const Fold& fold, const BatchNest& bn, int L,
                                                 int32_t s0, int64_t item0, int count, const RingView& rv,
                                                 int64_t& ready, int64_t& rel) {
  using Acc = typename Op::Acc;
  const int tid = threadIdx.x;
  const int lt = (tid & 31) % L;
  const int teams = kBatchWarps * (32 / L);
  const int team = tid / L;
  const int64_t fit = kLanesWindowBytes / (4 * gm.R);
  const int per = static_cast<int>(fit >= teams ? (fit / teams) * teams : (fit > 0 ? fit : 1));
  if (gm.G == 1) {
    // one item per output, R < 2^13 iterations: phase-relative 32-bit offsets
    typename Op::Out* outp = static_cast<typename Op::Out*>(bn.out) + item0;
    const int32_t R = static_cast<int32_t>(gm.R);
    for (int b = 0; b < count; b += per) {
      const int n = (count - b < per) ? count - b : per;
      const int64_t e0 = (item0 + b) * gm.R;
      const int64_t e1 = e0 + static_cast<int64_t>(n) * R;
      ring_wait(rv, e1, ready);
      const uint32_t off = static_cast<uint32_t>(e0) * 4u + fold.shift;
      const uint32_t dist = 4u * static_cast<uint32_t>(teams * R);   // ring bytes between a team's rounds
      if (L >= kReduceBatch) {
        // kReduceBatch rounds (two pairs), then one batched team reduction
        constexpr int B = kReduceBatch;
        for (int j0 = 0; j0 < n; j0 += B * teams) {   // the same trip count in every lane
          Acc part[B];
#pragma unroll
          for (int r = 0; r < B; r += 2) {
            const int ja = j0 + r * teams + team, jb = ja + teams;
            Acc accA[V], accB[V];
#pragma unroll
            for (int i = 0; i < V; ++i) accA[i] = accB[i] = Op::ident();
            const uint32_t offA = off + 4u * static_cast<uint32_t>(ja * R);
            if (jb < n) fold.template run_pair<V>(offA, dist, s0, R, gm.P, accA, accB);
            else if (ja < n) fold.template run_at<V>(offA, fold.w, s0, R, gm.P, accA);
            part[r] = fold_vec<Op, V>(accA);
            part[r + 1] = fold_vec<Op, V>(accB);
          }
          lanes_reduce_many<Op, B>(part, L, lt);
          const int j = j0 + (lt / (L / B)) * teams + team;
          if ((lt & (L / B - 1)) == 0 && j < n) outp[b + j] = Op::finish(part[0]);
        }
      } else {
        for (int j0 = 0; j0 < n; j0 += 2 * teams) {   // the same trip count in every lane
          const int ja = j0 + team, jb = ja + teams;
          Acc accA[V], accB[V];
#pragma unroll
          for (int i = 0; i < V; ++i) accA[i] = accB[i] = Op::ident();
          const uint32_t offA = off + 4u * static_cast<uint32_t>(ja * R);
          if (jb < n) fold.template run_pair<V>(offA, dist, s0, R, gm.P, accA, accB);
          else if (ja < n) fold.template run_at<V>(offA, fold.w, s0, R, gm.P, accA);
          const Acc a = lanes_allreduce<Op>(fold_vec<Op, V>(accA), L);
          // a thread team (L = 1) has no partner to shuffle with: skip the empty second item
          const Acc c = (L == 1 && jb >= n) ? Op::ident() : lanes_allreduce<Op>(fold_vec<Op, V>(accB), L);
          if (lt == 0) {
            if (ja < n) outp[b + ja] = Op::finish(a);
            if (jb < n) outp[b + jb] = Op::finish(c);
          }
        }
      }
      ring_release(rv, ring_stage(rv, e1), rel);
    }
    return;
  }
  for (int b = 0; b < count; b += per) {
    const int n = (count - b < per) ? count - b : per;
    int64_t base, lo, hi;
    ring_span(gm, item0 + b + n - 1, base, lo, hi);
    const int64_t w_end = base + hi;
    ring_wait(rv, w_end, ready);
    for (int j0 = 0; j0 < n; j0 += teams) {   // the same trip count in every lane
      const int j = j0 + team;
      const bool valid = j < n;
      Acc acc[V];
#pragma unroll
      for (int i = 0; i < V; ++i) acc[i] = Op::ident();
      if (valid) {
        ring_span(gm, item0 + b + j, base, lo, hi);
        fold.template run<V>(base + lo, lo, s0, static_cast<int32_t>(hi - lo), gm.P, acc);
      }
      const Acc a = lanes_allreduce<Op>(fold_vec<Op, V>(acc), L);
      if (valid && lt == 0) batch_emit<Op>(bn.rp, bn, item0 + b + j, a);
    }
    ring_release(rv, ring_stage(rv, w_end), rel);
  }
}

// ---------------------------------------------------------------- one tile, consumer side
template <class Op, class Body>
__device__ __forceinline__ void batch_tile(const RectPlan& p, const Body& body, const BatchNest& bn, const BatchTile& t,
                                           typename Op::Acc* wsh) {
  if (p.team == TEAM_MAP) {
    batch_map_items<Op>(body, bn, t.item0, t.count);
  } else if (p.team == TEAM_BLOCK) {
    if (p.V == 4) batch_block_items<Op, 4>(p, body, bn, t.item0, t.count, wsh);
    else batch_block_items<Op, 1>(p, body, bn, t.item0, t.count, wsh);
  } else {
    if (p.V == 4) batch_lanes_items<Op, 4>(p, body, bn, t.item0, t.count);
    else batch_lanes_items<Op, 1>(p, body, bn, t.item0, t.count);
  }
}

template <class Op, bool DOT>
__device__ __forceinline__ void ring_tile(const BatchQueued& e, uint32_t ring, const RingView& rv, int64_t& ready,
                                          int64_t& rel, typename Op::Acc (*wsh)[kMaxM][kBatchWarps]) {
  const RectPlan& p = e.bn.rp;
  RingFold<Op, DOT> fold;
  fold.ring = ring;
  fold.shift = static_cast<uint32_t>(rv.off0 + static_cast<uint64_t>(rv.k0 & (kStages - 1)) * kStageBytes);
  fold.w = static_cast<const typename Op::In*>(e.bn.in1);
  const RingGeom gm{p.R, p.vn[0], p.tile, p.G, p.vP[0]};
  const int64_t item0 = e.t.item0;
  const int count = e.t.count;
  const int lane = threadIdx.x & 31;
  if (p.team == TEAM_BLOCK) {
    const int W = p.W, warp = threadIdx.x >> 5;
    const int grp = lane / p.grp_lanes, lig = lane % p.grp_lanes;
    const int32_t s0 = warp * p.cw[0] + grp * p.cg[0] + lig * p.cl[0];
    if (p.V == 4) ring_block_items<Op, 4>(gm, fold, e.bn, W, s0, item0, count, rv, ready, rel, wsh);
    else ring_block_items<Op, 1>(gm, fold, e.bn, W, s0, item0, count, rv, ready, rel, wsh);
  } else {
    const int L = p.L;
    const int lt = lane % L;
    const int32_t s0 = (lt / p.grp_lanes) * p.cg[0] + (lt % p.grp_lanes) * p.cl[0];
    if (p.V == 4) ring_lanes_items<Op, 4>(gm, fold, e.bn, L, s0, item0, count, rv, ready, rel);
    else ring_lanes_items<Op, 1>(gm, fold, e.bn, L, s0, item0, count, rv, ready, rel);
  }
}

// ---------------------------------------------------------------- tile sources
// Where the producer warp takes its tiles from.  claim() runs on lane 0 and
// returns the index of the next tile, or -1 when there is none; tile() and
// desc() run on the whole warp after it.

// a tile table in device memory, taken through an atomic counter (one launch)
struct TableSource {
  static constexpr bool kResident = false;
  const BatchNest* __restrict__ nests;
  const BatchTile* __restrict__ tiles;
  int64_t n_tiles;
  unsigned long long* counter;

  __device__ __forceinline__ int64_t claim() const {
    const int64_t k = static_cast<int64_t>(atomicAdd(counter, 1ull));
    return k < n_tiles ? k : -1;
  }
  __device__ __forceinline__ BatchTile tile(int64_t k) const { return tiles[k]; }
  __device__ __forceinline__ void desc(int lane, const BatchTile& t, BatchQueued& e) const {
    const int32_t* src = reinterpret_cast<const int32_t*>(nests + t.nest);
    int32_t* dst = reinterpret_cast<int32_t*>(&e.bn);
    for (int i = lane; i < static_cast<int>(sizeof(BatchNest) / 4); i += 32) dst[i] = src[i];
  }
  // a consumer wait for the next tile that gave up
  __device__ __forceinline__ void report(int32_t code) const {
    if (nests[0].err) atomicExch(nests[0].err, code);
  }
  __device__ __forceinline__ unsigned long long idle_limit_ns() const { return kBatchWaitNs; }
  __device__ __forceinline__ void tile_done(const BatchQueued&, uint32_t) const {}
};

// ---------------------------------------------------------------- producer warp
template <class Src>
__device__ __forceinline__ void batch_producer(const Src& src, BatchQueued* tq, uint32_t ring, uint32_t full,
                                               uint32_t empty, uint32_t tq_full, uint32_t tq_empty,
                                               uint32_t abort_at) {
  const int lane = threadIdx.x & 31;
  int64_t kst = 0;   // stages issued so far
  for (int64_t q = 0;; ++q) {
    const int s = static_cast<int>(q % kTileQueue);
    int ok = 1;
    if (lane == 0) ok = mbar_wait(tq_empty + 8u * s, static_cast<uint32_t>(((q / kTileQueue) & 1) ^ 1), abort_at);
    if (!__shfl_sync(~0u, ok, 0)) break;   // consumers gave up: they leave at their next tile boundary
    long long k = 0;
    if (lane == 0) k = src.claim();
    k = __shfl_sync(~0u, k, 0);
    if constexpr (Src::kResident) __syncwarp();   // lane 0's acquire of the tile orders the warp's reads
    BatchQueued& e = tq[s];
    if (k < 0) {
      if (lane == 0) e.end = 1;
      mbar_arrive(tq_full + 8u * s);
      break;
    }
    const BatchTile t = src.tile(k);
    src.desc(lane, t, e);
    __syncwarp();
    const RectPlan& p = e.bn.rp;
    int64_t nst = 0;
    uint64_t a0 = 0, a1 = 0, gA = 0;
    if (batch_streams(p) && e.bn.in0 != nullptr && t.count > 0) {
      int64_t b0, l0, h0, b1, l1, h1;
      batch_item_span(p, t.item0, b0, l0, h0);
      batch_item_span(p, t.item0 + t.count - 1, b1, l1, h1);
      gA = reinterpret_cast<uint64_t>(e.bn.in0);
      a0 = (gA + 4u * static_cast<uint64_t>(b0 + l0)) & ~uint64_t(15);
      a1 = (gA + 4u * static_cast<uint64_t>(b1 + h1) + 15u) & ~uint64_t(15);
      if (a1 > a0) nst = static_cast<int64_t>((a1 - a0 + kStageBytes - 1) / kStageBytes);
    }
    if (lane == 0) {
      e.t = t;
      e.k0 = kst;
      e.a0 = a0;
      e.gA = gA;
      e.nst = static_cast<int32_t>(nst);
      e.end = 0;
    }
    __syncwarp();
    mbar_arrive(tq_full + 8u * s);   // every lane releases the words it wrote
    if (lane == 0) {
      for (int64_t i = 0; i < nst; ++i) {
        const int64_t kk = kst + i;
        const uint32_t slot = static_cast<uint32_t>(kk % kStages);
        if (!mbar_wait(empty + 8u * slot, static_cast<uint32_t>(((kk / kStages) & 1) ^ 1), abort_at)) {
          if (!ld_abort(abort_at)) {
            st_abort(abort_at);
            if (e.bn.err) atomicExch(e.bn.err, kErrStageWait);
          }
          nst = i;   // stages not issued are never waited for (the CTA is aborting)
          break;
        }
        const uint64_t src_a = a0 + static_cast<uint64_t>(i) * kStageBytes;
        const uint32_t bytes = static_cast<uint32_t>(a1 - src_a < kStageBytes ? a1 - src_a : kStageBytes);
        mbar_arrive_tx(full + 8u * slot, bytes);
        bulk_g2s(ring + slot * kStageBytes, src_a, bytes, full + 8u * slot);
      }
    }
    kst += __shfl_sync(~0u, nst, 0);
    if (ld_abort(abort_at)) break;
  }
  // let the copies in flight land before the warp exits (the last ring of stages)
  if (lane == 0)
    for (int64_t kk = kst > kStages ? kst - kStages : 0; kk < kst; ++kk)
      mbar_wait(full + 8u * static_cast<uint32_t>(kk % kStages), static_cast<uint32_t>((kk / kStages) & 1), 0u);
}

// ---------------------------------------------------------------- the persistent CTA
template <class Op, class Src>
__device__ __forceinline__ void batch_cta(const Src& src) {
  using Acc = typename Op::Acc;
  using In = typename Op::In;
  extern __shared__ __align__(128) unsigned char batch_ring[];
  // bars[0]: the CTA's abort flag; then the stage and tile-queue barriers
  __shared__ __align__(8) unsigned long long bars[1 + 2 * kStages + 2 * kTileQueue];
  __shared__ BatchQueued tq[kTileQueue];
  __shared__ Acc wsh[2][kMaxM][kBatchWarps];
  const uint32_t ring = smem_u32(batch_ring);
  const uint32_t abort_at = smem_u32(&bars[0]);
  const uint32_t full = abort_at + 8u, empty = full + 8u * kStages;
  const uint32_t tq_full = empty + 8u * kStages, tq_empty = tq_full + 8u * kTileQueue;
  if (threadIdx.x == 0) {
    for (int i = 0; i < kStages; ++i) {
      mbar_init(full + 8u * i, 1);
      mbar_init(empty + 8u * i, kBatchWarps);
    }
    for (int i = 0; i < kTileQueue; ++i) {
      mbar_init(tq_full + 8u * i, 32);
      mbar_init(tq_empty + 8u * i, kBatchThreads);
    }
    bars[0] = 0;
  }
  __syncthreads();
  if (threadIdx.x >= kBatchThreads) {
    batch_producer(src, tq, ring, full, empty, tq_full, tq_empty, abort_at);
    return;
  }
  int64_t ready = 0, rel = 0;
  for (int64_t q = 0;; ++q) {
    const int s = static_cast<int>(q % kTileQueue);
    if (!mbar_wait(tq_full + 8u * s, static_cast<uint32_t>((q / kTileQueue) & 1), abort_at, src.idle_limit_ns()) &&
        !ld_abort(abort_at)) {
      st_abort(abort_at);
      src.report(kErrStageWait);
    }
    if (consumer_sync_or(ld_abort(abort_at))) break;   // one decision for all consumer warps
    const BatchQueued& e = tq[s];
    if (e.end) break;
    const RectPlan& p = e.bn.rp;
    if (e.nst > 0) {
      const RingView rv{full, empty, smem_u32(&e.bn.err), e.k0, e.gA - e.a0};
      if (p.body == HP_BODY_DOT_BCAST) ring_tile<Op, true>(e, ring, rv, ready, rel, wsh);
      else ring_tile<Op, false>(e, ring, rv, ready, rel, wsh);
      ring_release(rv, e.k0 + e.nst, rel);
    } else {
      switch (p.body) {
        case HP_BODY_LOAD: {
          BodyLoad<Op> b{static_cast<const In*>(e.bn.in0)};
          batch_tile<Op>(p, b, e.bn, e.t, &wsh[0][0][0]);
          break;
        }
        case HP_BODY_DOT_BCAST: {
          BodyDot<Op> b{static_cast<const In*>(e.bn.in0), static_cast<const In*>(e.bn.in1)};
          batch_tile<Op>(p, b, e.bn, e.t, &wsh[0][0][0]);
          break;
        }
        default: {
          BodyAffine<Op> b;
          b.a = p.aff_a;
          b.b = p.aff_b;
          b.m = p.aff_m;
          batch_tile<Op>(p, b, e.bn, e.t, &wsh[0][0][0]);
          break;
        }
      }
    }
    if constexpr (Src::kResident) src.tile_done(e, abort_at);
    mbar_arrive(tq_empty + 8u * s);   // this thread is done with the entry
  }
}

template <class Op>
__global__ void __launch_bounds__(kBatchAllThreads, HP_BATCH_MIN_BLOCKS)
    batch_kernel(const BatchNest* __restrict__ nests, const BatchTile* __restrict__ tiles, int64_t n_tiles,
                 unsigned long long* counter) {
  batch_cta<Op>(TableSource{nests, tiles, n_tiles, counter});
}

// host-side launch of one arithmetic's persistent kernel (batch_f32.cu, batch_int.cu)
struct BatchLaunch {
  const BatchNest* nests;
  const BatchTile* tiles;
  int64_t n_tiles;
  unsigned long long* counter;
  int grid;
};

template <class Op>
inline cudaError_t batch_prepare() {
  static const cudaError_t e =
      cudaFuncSetAttribute(batch_kernel<Op>, cudaFuncAttributeMaxDynamicSharedMemorySize, kRingBytes);
  return e;
}

template <class Op>
inline cudaError_t launch_batch_op(const BatchLaunch& b, cudaStream_t st) {
  cudaError_t e = batch_prepare<Op>();
  if (e != cudaSuccess) return e;
  batch_kernel<Op><<<b.grid, kBatchAllThreads, kRingBytes, st>>>(b.nests, b.tiles, b.n_tiles, b.counter);
  return cudaPeekAtLastError();
}

template <class Op>
inline int batch_blocks_per_sm() {
  if (batch_prepare<Op>() != cudaSuccess) return 1;
  int n = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_kernel<Op>, kBatchAllThreads, kRingBytes);
  return n < 1 ? 1 : n;
}

// arithmetic index of a nest: 0 f32 sum, 1 compensated sum, 2 f32 max, 3 f32 min,
// 4..6 int32 sum / max / min, 7..9 int64 sum / max / min
inline int batch_combo(hp_prec prec, hp_red_op op) {
  const int o = op == HP_RED_SUM ? 0 : op == HP_RED_MAX ? 1 : 2;
  if (prec == HP_F32 || prec == HP_F32_COMP) return o == 0 ? (prec == HP_F32 ? 0 : 1) : 1 + o;
  return (prec == HP_I32 ? 4 : 7) + o;
}
constexpr int kBatchCombos = 10;

cudaError_t launch_batch_combo(int combo, const BatchLaunch& b, cudaStream_t st);   // batch_f32.cu / batch_int.cu
int batch_combo_blocks_per_sm(int combo);

}  // namespace hp
