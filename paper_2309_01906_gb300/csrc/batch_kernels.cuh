// batch_kernels.cuh — one persistent launch over the tiles of many nests.
//
// Every CTA takes tile after tile from an atomic counter (a dynamic schedule
// at grid level, Sec. 3.5) until the table is exhausted.  A tile is a range of
// work items of one nest; it runs with that nest's own plan and with exactly
// the per-thread fold and team tree of rect_block_kernel / rect_lanes_kernel
// (same fold_item, same lane butterfly, same warp order), so every nest's
// outputs equal those of hp_nest_run on it, bit for bit.  Nests split over
// grid parts fold their parts in part order once the last part of an output
// has arrived (a per-output ticket counter; nobody waits on it).
#pragma once

#include "rect_kernels.cuh"

namespace hp {

constexpr int kBatchThreads = 256;   // CTA size of the persistent kernel (block teams up to 8 warps)

// one nest of a batch, as the device sees it
struct BatchNest {
  RectPlan rp;
  const void* in0;
  const void* in1;
  void* out;
  void* part;          // grid-part partials (G > 1)
  int32_t* tickets;    // per output (G > 1)
};

struct BatchTile {
  int32_t nest;
  int32_t count;       // items
  int64_t item0;
};

template <class Op>
__device__ __forceinline__ void batch_emit(const RectPlan& p, const BatchNest& bn, int64_t item, typename Op::Acc a) {
  using Acc = typename Op::Acc;
  if (p.G == 1) {
    static_cast<typename Op::Out*>(bn.out)[item] = Op::finish(a);
    return;
  }
  Acc* part = static_cast<Acc*>(bn.part);
  const int64_t o = item / p.G;
  part[item] = a;
  __threadfence();  // publish the partial before taking the ticket
  if (atomicAdd(&bn.tickets[o], 1) == p.G - 1) {
    __threadfence();  // all parts of this output are visible
    const Acc* pp = part + o * p.G;
    if constexpr (sizeof(Acc) == 8 && Op::kFp) {
      // compensated partials: the final grid-level combine in FP64, part order
      const volatile float* pv = reinterpret_cast<const volatile float*>(pp);
      double s = 0.0;
      for (int g = 0; g < p.G; ++g) {
        s += static_cast<double>(pv[2 * g]);
        s += static_cast<double>(pv[2 * g + 1]);
      }
      static_cast<typename Op::Out*>(bn.out)[o] = static_cast<float>(s);
    } else {
      const volatile Acc* pv = pp;
      Acc v = pv[0];
      for (int g = 1; g < p.G; ++g) v = Op::combine(v, pv[g]);
      static_cast<typename Op::Out*>(bn.out)[o] = Op::finish(v);
    }
    bn.tickets[o] = 0;  // ready for the next run
  }
}

// items [item0, item0 + count) of a block-team nest: one item at a time, the
// plan's W warps fold, the CTA combines them in warp order
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
    __syncthreads();
    if (tid == 0) {
      Acc r = wsh[0];
      for (int w = 1; w < p.W; ++w) r = Op::combine(r, wsh[w]);
      batch_emit<Op>(p, bn, item, r);
    }
    __syncthreads();
  }
}

// items of a lanes-team nest: every group of L lanes of the CTA is a team
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
  const int teams = (blockDim.x >> 5) * (32 / L);
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
  for (int k = threadIdx.x; k < count; k += blockDim.x) {
    typename Op::Acc acc[1] = {Op::ident()};
    body.template fold<1>(acc, item0 + k, 0);
    static_cast<typename Op::Out*>(bn.out)[item0 + k] = Op::finish(acc[0]);
  }
}

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

template <class Op>
__global__ void __launch_bounds__(kBatchThreads) batch_kernel(const BatchNest* __restrict__ nests,
                                                              const BatchTile* __restrict__ tiles, int64_t n_tiles,
                                                              unsigned long long* counter) {
  using Acc = typename Op::Acc;
  using In = typename Op::In;
  __shared__ BatchNest sn;
  __shared__ BatchTile st;
  __shared__ long long next;
  __shared__ Acc wsh[kBatchThreads / 32];
  while (true) {
    if (threadIdx.x == 0) next = static_cast<long long>(atomicAdd(counter, 1ull));
    __syncthreads();
    const long long k = next;
    if (k >= n_tiles) break;
    if (threadIdx.x == 0) {
      st = tiles[k];
      sn = nests[st.nest];
    }
    __syncthreads();
    const RectPlan& p = sn.rp;
    switch (p.body) {
      case HP_BODY_LOAD: {
        BodyLoad<Op> b{static_cast<const In*>(sn.in0)};
        batch_tile<Op>(p, b, sn, st, wsh);
        break;
      }
      case HP_BODY_DOT_BCAST: {
        BodyDot<Op> b{static_cast<const In*>(sn.in0), static_cast<const In*>(sn.in1)};
        batch_tile<Op>(p, b, sn, st, wsh);
        break;
      }
      default: {
        BodyAffine<Op> b;
        b.a = p.aff_a;
        b.b = p.aff_b;
        b.m = p.aff_m;
        batch_tile<Op>(p, b, sn, st, wsh);
        break;
      }
    }
    __syncthreads();  // the tile's shared state is rewritten next
  }
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
inline cudaError_t launch_batch_op(const BatchLaunch& b, cudaStream_t st) {
  batch_kernel<Op><<<b.grid, kBatchThreads, 0, st>>>(b.nests, b.tiles, b.n_tiles, b.counter);
  return cudaPeekAtLastError();
}

template <class Op>
inline int batch_blocks_per_sm() {
  int n = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_kernel<Op>, kBatchThreads, 0);
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
