// rect_kernels.cuh — the rectangular nest executor (device code).
//
// One output of the nest is combined by a team (plan.cpp decides which):
//   rect_block_kernel  a cluster of C CTAs or a single CTA.  Each thread folds
//                      its share of the reduced levels, then lanes combine by
//                      xor-shuffle (Sec. 3.7), warps through shared memory in
//                      warp order (Sec. 3.7's fallback one level up), CTAs of
//                      a cluster through distributed shared memory in rank
//                      order; items are handled in rounds of M so that one
//                      barrier serves M outputs.
//   rect_lanes_kernel  a group of L lanes of one warp (warp, sub-warp group of
//                      Sec. 3.8, or a single thread): lanes combine by
//                      xor-shuffle with width L.
// When the first reduced level is bound to the grid, every output is cut into
// G parts that write partials; rect_combine_kernel folds them in part order
// (combine_parts; compensated partials as a double-float sum).
// The reduction tree depends only on the plan, never on which SM ran what, so
// runs are bit-reproducible.
#pragma once

#include <cooperative_groups.h>
#include <cstdint>

#include "accum.cuh"
#include "hp_internal.h"

namespace hp {

namespace cg = cooperative_groups;

#ifndef HP_FOLD_LOADS
#define HP_FOLD_LOADS 4   // loads a thread issues before folding them (plain-load kernels)
#endif

// ---------------------------------------------------------------- loads
__device__ __forceinline__ float4 ld_stream4(const float* p) { return __ldcs(reinterpret_cast<const float4*>(p)); }
__device__ __forceinline__ int4 ld_stream4(const int32_t* p) { return __ldcs(reinterpret_cast<const int4*>(p)); }
__device__ __forceinline__ float4 ld_keep4(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }
__device__ __forceinline__ int4 ld_keep4(const int32_t* p) { return __ldg(reinterpret_cast<const int4*>(p)); }
__device__ __forceinline__ float ld_stream(const float* p) { return __ldcs(p); }
__device__ __forceinline__ int32_t ld_stream(const int32_t* p) { return __ldcs(p); }
__device__ __forceinline__ float ld_keep(const float* p) { return __ldg(p); }
__device__ __forceinline__ int32_t ld_keep(const int32_t* p) { return __ldg(p); }

template <class V4>
__device__ __forceinline__ auto v4get(const V4& v, int i) {
  return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w;
}

// ---------------------------------------------------------------- bodies
// fold V consecutive iterations starting at flat (reduced index rflat)
// Memory bodies split a step into load (V consecutive iterations at flat, the
// broadcast operand at rflat) and apply (fold them into the V slots), so that
// fold_item can issue several loads before the first fold.
template <class Op, int V>
struct Vals {
  typename Op::In a[V];
  typename Op::In b[V];
};

template <class Op>
struct BodyLoad {
  static constexpr bool kPipeable = true;
  static constexpr bool kDot = false;
  const typename Op::In* A;
  __host__ __device__ const typename Op::In* wptr() const { return nullptr; }
  template <int V>
  __device__ __forceinline__ Vals<Op, V> load(int64_t flat, int64_t) const {
    Vals<Op, V> v;
    if constexpr (V == 4) {
      const auto q = ld_stream4(A + flat);
      v.a[0] = q.x;
      v.a[1] = q.y;
      v.a[2] = q.z;
      v.a[3] = q.w;
    } else {
#pragma unroll
      for (int i = 0; i < V; ++i) v.a[i] = ld_stream(A + flat + i);
    }
    return v;
  }
  template <int V>
  __device__ __forceinline__ void apply(typename Op::Acc (&acc)[V], const Vals<Op, V>& v) const {
    fold_vals_load<Op, V>(acc, v.a);
  }
  template <int V>
  __device__ __forceinline__ void fold(typename Op::Acc (&acc)[V], int64_t flat, int64_t rflat) const {
    apply<V>(acc, load<V>(flat, rflat));
  }
};

template <class Op>
struct BodyDot {
  static constexpr bool kPipeable = true;
  static constexpr bool kDot = true;
  const typename Op::In* A;
  const typename Op::In* w;
  __host__ __device__ const typename Op::In* wptr() const { return w; }
  template <int V>
  __device__ __forceinline__ Vals<Op, V> load(int64_t flat, int64_t rflat) const {
    Vals<Op, V> v;
    if constexpr (V == 4) {
      const auto q = ld_stream4(A + flat);
      const auto r = ld_keep4(w + rflat);
      v.a[0] = q.x;
      v.a[1] = q.y;
      v.a[2] = q.z;
      v.a[3] = q.w;
      v.b[0] = r.x;
      v.b[1] = r.y;
      v.b[2] = r.z;
      v.b[3] = r.w;
    } else {
#pragma unroll
      for (int i = 0; i < V; ++i) {
        v.a[i] = ld_stream(A + flat + i);
        v.b[i] = ld_keep(w + rflat + i);
      }
    }
    return v;
  }
  template <int V>
  __device__ __forceinline__ void apply(typename Op::Acc (&acc)[V], const Vals<Op, V>& v) const {
    fold_vals_dot<Op, V>(acc, v.a, v.b);
  }
  template <int V>
  __device__ __forceinline__ void fold(typename Op::Acc (&acc)[V], int64_t flat, int64_t rflat) const {
    apply<V>(acc, load<V>(flat, rflat));
  }
};

// a + b * (flat mod m): exact in int64, wrapped for int32, rounded once for FP
template <class Op>
struct BodyAffine {
  static constexpr bool kPipeable = false;
  static constexpr bool kDot = false;
  const typename Op::In* A = nullptr;
  __host__ __device__ const typename Op::In* wptr() const { return nullptr; }
  int64_t a, b, m;
  template <int V>
  __device__ __forceinline__ void fold(typename Op::Acc (&acc)[V], int64_t flat, int64_t) const {
#pragma unroll
    for (int i = 0; i < V; ++i) {
      const int64_t v = a + b * ((flat + i) % m);
      if constexpr (Op::kFp) {
        Op::add_val(acc[i], static_cast<float>(v));
      } else if constexpr (sizeof(typename Op::Out) == 4) {
        Op::add_val(acc[i], static_cast<int32_t>(static_cast<uint32_t>(static_cast<uint64_t>(v))));
      } else {
        Op::add_val(acc[i], static_cast<long long>(v));
      }
    }
  }
};

// fl32(q^(flat mod m)) from a table the planner filled
template <class Op>
struct BodyGeo {
  static constexpr bool kPipeable = false;
  static constexpr bool kDot = false;
  const typename Op::In* A = nullptr;
  __host__ __device__ const typename Op::In* wptr() const { return nullptr; }
  const float* table;
  int64_t m;
  template <int V>
  __device__ __forceinline__ void fold(typename Op::Acc (&acc)[V], int64_t flat, int64_t) const {
#pragma unroll
    for (int i = 0; i < V; ++i) Op::add_val(acc[i], __ldg(table + (flat + i) % m));
  }
};

// ---------------------------------------------------------------- per-thread fold of one item
template <class Op, int V, class Body>
__device__ __forceinline__ void fold_item(const RectPlan& p, const Body& body, int64_t o, int64_t g,
                                          const int32_t (&slot)[kMaxV], typename Op::Acc (&acc)[V]) {
  const int nv = p.nv;
  int64_t lo[kMaxV], hi[kMaxV], x[kMaxV];
#pragma unroll
  for (int v = 0; v < kMaxV; ++v) {
    if (v < nv) {
      lo[v] = 0;
      hi[v] = p.vn[v];
    }
  }
  if (p.split) {
    lo[0] = g * p.tile;
    hi[0] = (lo[0] + p.tile < p.vn[0]) ? lo[0] + p.tile : p.vn[0];
  }
  for (int v = 0; v < nv - 1; ++v) {
    x[v] = lo[v] + slot[v];
    if (x[v] >= hi[v]) return;
  }
  const int64_t obase = o * p.R;
  const int last = nv - 1;
  const int64_t in_lo = lo[last] + slot[last], in_hi = hi[last], P = p.vP[last];
  while (true) {
    int64_t roff = 0;
    for (int v = 0; v < last; ++v) roff += x[v] * p.vstride[v];
    const int64_t base = obase + roff;
    if constexpr (Body::kPipeable) {
      // HP_FOLD_LOADS loads in flight before the first of their folds (same fold order)
      constexpr int NL = HP_FOLD_LOADS;
      int64_t xi = in_lo;
      for (; xi + (NL - 1) * P < in_hi; xi += NL * P) {
        decltype(body.template load<V>(base, roff)) v[NL];
#pragma unroll
        for (int q = 0; q < NL; ++q) v[q] = body.template load<V>(base + xi + q * P, roff + xi + q * P);
#pragma unroll
        for (int q = 0; q < NL; ++q) body.template apply<V>(acc, v[q]);
      }
      for (; xi < in_hi; xi += P) body.template fold<V>(acc, base + xi, roff + xi);
    } else {
      for (int64_t xi = in_lo; xi < in_hi; xi += P) body.template fold<V>(acc, base + xi, roff + xi);
    }
    int v = last - 1;
    for (; v >= 0; --v) {
      x[v] += p.vP[v];
      if (x[v] < hi[v]) break;
      x[v] = lo[v] + slot[v];
    }
    if (v < 0) break;
  }
}

template <class Op, int V>
__device__ __forceinline__ typename Op::Acc fold_vec(const typename Op::Acc (&acc)[V]) {
  if constexpr (V == 4) return Op::combine(Op::combine(acc[0], acc[1]), Op::combine(acc[2], acc[3]));
  else if constexpr (V == 2) return Op::combine(acc[0], acc[1]);
  else return acc[0];
}

template <class Op>
__device__ __forceinline__ typename Op::Acc lanes_allreduce(typename Op::Acc a, int width) {
  for (int m = width >> 1; m >= 1; m >>= 1) a = Op::combine(a, Op::shfl_xor(a, m, width));
  return a;
}

template <class Op>
__device__ __forceinline__ void emit(const RectPlan& p, int64_t item, typename Op::Acc a, typename Op::Out* out,
                                     typename Op::Acc* part) {
  if (p.G == 1) {
    out[item] = Op::finish(a);
    if constexpr (std::is_same_v<typename Op::Acc, f2>) {
      if (p.comp) p.comp[item] = Op::residual(a);
    }
  } else {
    part[item] = a;
  }
}

// ---------------------------------------------------------------- team = cluster or CTA
template <class Op, int V, class Body>
__global__ void __launch_bounds__(1024) rect_block_kernel(RectPlan p, Body body, typename Op::Out* out,
                                                          typename Op::Acc* part) {
  using Acc = typename Op::Acc;
  __shared__ Acc wpart[2][kMaxM][kMaxWarps];
  __shared__ Acc cpart[2][kMaxM];
  const int C = p.C;
  int rank = 0;
  int64_t team = blockIdx.x, n_teams = gridDim.x;
  if (C > 1) {
    rank = static_cast<int>(cg::this_cluster().block_rank());
    team = blockIdx.x / C;
    n_teams = gridDim.x / C;
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int grp = lane / p.grp_lanes, lig = lane % p.grp_lanes;
  int32_t slot[kMaxV];
#pragma unroll
  for (int v = 0; v < kMaxV; ++v)
    slot[v] = rank * p.cr[v] + warp * p.cw[v] + grp * p.cg[v] + lig * p.cl[v];
  const int M = p.M, W = p.W;
  const int64_t n_chunks = (p.items + M - 1) / M;
  int buf = 0;
  for (int64_t chunk = team; chunk < n_chunks; chunk += n_teams) {
    const int64_t item0 = chunk * M;
    const int mcount = static_cast<int>((p.items - item0 < M) ? p.items - item0 : M);
    for (int m = 0; m < mcount; ++m) {
      const int64_t item = item0 + m;
      const int64_t o = item / p.G, g = item - o * p.G;
      Acc acc[V];
#pragma unroll
      for (int i = 0; i < V; ++i) acc[i] = Op::ident();
      fold_item<Op, V>(p, body, o, g, slot, acc);
      Acc a = lanes_allreduce<Op>(fold_vec<Op, V>(acc), 32);
      if (lane == 0) wpart[buf][m][warp] = a;
    }
    __syncthreads();
    if (threadIdx.x < mcount) {
      Acc a = wpart[buf][threadIdx.x][0];
      for (int w = 1; w < W; ++w) a = Op::combine(a, wpart[buf][threadIdx.x][w]);
      cpart[buf][threadIdx.x] = a;
    }
    if (C > 1) {
      cg::cluster_group cl = cg::this_cluster();
      cl.sync();  // release own CTA partials, acquire the peers'
      for (int m = rank + C * static_cast<int>(threadIdx.x); m < mcount; m += C * static_cast<int>(blockDim.x)) {
        Acc a = *cl.map_shared_rank(&cpart[buf][m], 0);
        for (int q = 1; q < C; ++q) a = Op::combine(a, *cl.map_shared_rank(&cpart[buf][m], q));
        emit<Op>(p, item0 + m, a, out, part);
      }
    } else if (threadIdx.x < mcount) {
      emit<Op>(p, item0 + threadIdx.x, cpart[buf][threadIdx.x], out, part);
    }
    buf ^= 1;
  }
  if (C > 1) cg::this_cluster().sync();  // peers may still read this CTA's partials
}

// ---------------------------------------------------------------- team = cluster or CTA, pipelined
// Same plan, same fold order and reduction tree as rect_block_kernel (results
// are bit-identical), but every thread streams its own 128-bit element groups
// through a private ring of D item stages in shared memory filled by cp.async,
// so D items' loads per thread stay in flight across item boundaries and
// across the CTA / cluster barriers of the rounds.  A thread only ever reads
// the slots it filled itself, so the ring needs no barrier: cp.async.wait_group
// orders each read after its own copies, and a stage is refilled only after
// the values read from it have been consumed by the folds.
constexpr int kPatMax = 8;    // element groups per thread per item
constexpr int kPipeMaxThreads = 256;
#ifndef HP_PIPE_MIN_BLOCKS
#define HP_PIPE_MIN_BLOCKS 2   // resident CTAs per SM the register budget is sized for
#endif

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(smem_dst)), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

__device__ __forceinline__ float4 neg4(float4 v) { return make_float4(-v.x, -v.y, -v.z, -v.w); }
__device__ __forceinline__ int4 neg4(int4 v) { return make_int4(-v.x, -v.y, -v.z, -v.w); }

template <class In> struct Vec4Of;
template <> struct Vec4Of<float> { using T = float4; };
template <> struct Vec4Of<int32_t> { using T = int4; };

template <class Op, class V4>
__device__ __forceinline__ void fold4_load(typename Op::Acc (&acc)[4], const V4& a) {
  Op::add_val(acc[0], a.x);
  Op::add_val(acc[1], a.y);
  Op::add_val(acc[2], a.z);
  Op::add_val(acc[3], a.w);
}
template <class Op, class V4>
__device__ __forceinline__ void fold4_dot(typename Op::Acc (&acc)[4], const V4& a, const V4& b) {
  Op::add_prod(acc[0], a.x, b.x);
  Op::add_prod(acc[1], a.y, b.y);
  Op::add_prod(acc[2], a.z, b.z);
  Op::add_prod(acc[3], a.w, b.w);
}

// the element groups (offsets within one output's reduced space) one thread
// folds for any item, in fold_item's order; returns their number
__device__ __forceinline__ int build_pattern(const RectPlan& p, const int32_t (&slot)[kMaxV], int32_t* pat,
                                             int stride) {
  const int nv = p.nv;
  int64_t x[kMaxV];
  int n = 0;
  for (int v = 0; v < nv - 1; ++v) {
    x[v] = slot[v];
    if (x[v] >= p.vn[v]) return 0;
  }
  const int last = nv - 1;
  while (true) {
    int64_t roff = 0;
    for (int v = 0; v < last; ++v) roff += x[v] * p.vstride[v];
    for (int64_t xi = slot[last]; xi < p.vn[last]; xi += p.vP[last]) {
      if (n < kPatMax) pat[n * stride] = static_cast<int32_t>(roff + xi);
      ++n;
    }
    int v = last - 1;
    for (; v >= 0; --v) {
      x[v] += p.vP[v];
      if (x[v] < p.vn[v]) break;
      x[v] = slot[v];
    }
    if (v < 0) break;
  }
  return n < kPatMax ? n : kPatMax;  // the planner only picks this kernel when n <= kPatMax
}

// D items in flight per thread: each stage holds one item's element groups
// (at most kPatMax 16-byte groups per thread), committed as one cp.async group.
template <class Op, bool DOT, int D>
__global__ void __launch_bounds__(kPipeMaxThreads, HP_PIPE_MIN_BLOCKS) rect_block_pipe_kernel(RectPlan p, const typename Op::In* __restrict__ A,
                                                               const typename Op::In* __restrict__ w,
                                                               typename Op::Out* out, typename Op::Acc* part) {
  using Acc = typename Op::Acc;
  using In = typename Op::In;
  using V4 = typename Vec4Of<In>::T;
  extern __shared__ __align__(16) unsigned char pipe_smem[];
  const int nthr = blockDim.x, tid = threadIdx.x;
  const int G = p.groups;                                            // stage width (groups per item)
  V4* ring = reinterpret_cast<V4*>(pipe_smem);                      // [D][G][nthr]
  int32_t* pat = reinterpret_cast<int32_t*>(pipe_smem);             // [kPatMax][nthr], before the ring is used
  __shared__ Acc wpart[2][kMaxM][kPipeMaxThreads / 32];
  __shared__ Acc cpart[2][kMaxM];
  const int C = p.C;
  int rank = 0;
  int64_t team = blockIdx.x, n_teams = gridDim.x;
  if (C > 1) {
    rank = static_cast<int>(cg::this_cluster().block_rank());
    team = blockIdx.x / C;
    n_teams = gridDim.x / C;
  }
  const int warp = tid >> 5, lane = tid & 31;
  const int grp = lane / p.grp_lanes, lig = lane % p.grp_lanes;
  int32_t slot[kMaxV];
#pragma unroll
  for (int v = 0; v < kMaxV; ++v) slot[v] = rank * p.cr[v] + warp * p.cw[v] + grp * p.cg[v] + lig * p.cl[v];
  const int nt = build_pattern(p, slot, pat + tid, nthr);
  int32_t po[kPatMax];
  V4 wv[kPatMax];
#pragma unroll
  for (int k = 0; k < kPatMax; ++k) {
    po[k] = (k < nt) ? pat[k * nthr + tid] : 0;
    if constexpr (DOT) {
      if (k < nt) wv[k] = ld_keep4(w + po[k]);
    }
  }
  __syncthreads();  // every pattern is in registers before the ring (same memory) fills
  const int M = p.M, W = p.W;
  const int64_t R = p.R, items = p.items;
  const int64_t n_chunks = (items + M - 1) / M;
  V4* const ring_t = ring + tid;
  const int stage_stride = G * nthr;

  // producer cursor over this team's items: item pm of chunk pc
  int64_t pc = team;
  int pm = 0;
  int pcount = (pc < n_chunks) ? static_cast<int>((items - pc * M < M) ? items - pc * M : M) : 0;
  bool pvalid = nt > 0 && pc < n_chunks;
  const In* pitem = pvalid ? A + pc * M * R : A;
  auto issue = [&](int stage) {
    if (pvalid) {
      V4* dst = ring_t + stage * stage_stride;
#pragma unroll
      for (int k = 0; k < kPatMax; ++k)
        if (k < nt) cp_async16(dst + k * nthr, pitem + po[k]);
      pitem += R;
      if (++pm == pcount) {
        pm = 0;
        pc += n_teams;
        pvalid = pc < n_chunks;
        pcount = pvalid ? static_cast<int>((items - pc * M < M) ? items - pc * M : M) : 0;
        if (pvalid) pitem = A + pc * M * R;
      }
    }
    cp_async_commit();
  };
#pragma unroll
  for (int s = 0; s < D; ++s) issue(s);

  int rstage = 0;
  int buf = 0;
  for (int64_t chunk = team; chunk < n_chunks; chunk += n_teams) {
    const int64_t item0 = chunk * M;
    const int mcount = static_cast<int>((items - item0 < M) ? items - item0 : M);
    for (int m = 0; m < mcount; ++m) {
      Fold4<Op> f;
      f.init();
      if (nt > 0) {
        cp_async_wait<D - 1>();
        const V4* src = ring_t + rstage * stage_stride;
#pragma unroll
        for (int k = 0; k < kPatMax; ++k) {
          if (k < nt) {
            const V4 a = src[k * nthr];
            if constexpr (DOT) f.dot(a, wv[k], wv[k]);
            else f.load(a);
          }
        }
        issue(rstage);   // the folds above consumed the stage
        rstage = (rstage + 1 == D) ? 0 : rstage + 1;
      }
      Acc acc[4];
      f.get(acc);
      Acc a = lanes_allreduce<Op>(fold_vec<Op, 4>(acc), 32);
      if (lane == 0) wpart[buf][m][warp] = a;
    }
    __syncthreads();
    if (tid < mcount) {
      Acc a = wpart[buf][tid][0];
      for (int q = 1; q < W; ++q) a = Op::combine(a, wpart[buf][tid][q]);
      cpart[buf][tid] = a;
    }
    if (C > 1) {
      cg::cluster_group cl = cg::this_cluster();
      cl.sync();
      for (int m = rank + C * tid; m < mcount; m += C * nthr) {
        Acc a = *cl.map_shared_rank(&cpart[buf][m], 0);
        for (int q = 1; q < C; ++q) a = Op::combine(a, *cl.map_shared_rank(&cpart[buf][m], q));
        emit<Op>(p, item0 + m, a, out, part);
      }
    } else if (tid < mcount) {
      emit<Op>(p, item0 + tid, cpart[buf][tid], out, part);
    }
    buf ^= 1;
  }
  cp_async_wait<0>();
  if (C > 1) cg::this_cluster().sync();
}

// items in flight for a plan with G groups per item
__host__ __device__ constexpr int pipe_depth(int groups) { return groups > 4 ? 2 : 4; }
// largest dynamic shared memory of any pipelined plan: stages of 16-byte groups
// for kPipeMaxThreads threads (D * G <= 16), or the pattern table
constexpr size_t kPipeDynMax = static_cast<size_t>(kPipeMaxThreads) * 16 * 16;

// ---------------------------------------------------------------- team = L lanes of a warp
template <class Op, int V, class Body>
__global__ void __launch_bounds__(1024) rect_lanes_kernel(RectPlan p, Body body, typename Op::Out* out,
                                                          typename Op::Acc* part) {
  using Acc = typename Op::Acc;
  const int L = p.L;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int lt = lane % L;
  const int grp = lt / p.grp_lanes, lig = lt % p.grp_lanes;
  int32_t slot[kMaxV];
#pragma unroll
  for (int v = 0; v < kMaxV; ++v) slot[v] = grp * p.cg[v] + lig * p.cl[v];
  const int teams_per_warp = 32 / L;
  const int64_t warp_global = static_cast<int64_t>(blockIdx.x) * p.W + warp;
  const int64_t n_teams = static_cast<int64_t>(gridDim.x) * p.W * teams_per_warp;
  for (int64_t base = warp_global * teams_per_warp; base < p.items; base += n_teams) {
    const int64_t item = base + lane / L;
    const bool valid = item < p.items;
    Acc acc[V];
#pragma unroll
    for (int i = 0; i < V; ++i) acc[i] = Op::ident();
    if (valid) {
      const int64_t o = item / p.G, g = item - o * p.G;
      fold_item<Op, V>(p, body, o, g, slot, acc);
    }
    Acc a = lanes_allreduce<Op>(fold_vec<Op, V>(acc), L);
    if (valid && lt == 0) emit<Op>(p, item, a, out, part);
  }
}

// ---------------------------------------------------------------- grid parts -> outputs
// A warp per output: the lanes stage up to 256 parts at a time in shared
// memory with coalesced loads, and lane 0 folds them in part order (the steps
// of combine_parts, so the bits equal the batched executors').  256 threads.
constexpr int kCombineWarps = 8;
constexpr int kCombineChunk = 256;
template <class Op>
__global__ void __launch_bounds__(32 * kCombineWarps) rect_combine_kernel(int64_t O, int32_t G,
                                                                        const typename Op::Acc* part,
                                                                        typename Op::Out* out, float* comp) {
  using Acc = typename Op::Acc;
  __shared__ Acc stage[kCombineWarps][kCombineChunk];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int64_t o = blockIdx.x * static_cast<int64_t>(kCombineWarps) + warp; o < O;
       o += static_cast<int64_t>(gridDim.x) * kCombineWarps) {
    const Acc* pp = part + o * G;
    PartFold<Op> f;
    for (int32_t c0 = 0; c0 < G; c0 += kCombineChunk) {
      const int n = G - c0 < kCombineChunk ? G - c0 : kCombineChunk;
      for (int i = lane; i < n; i += 32) stage[warp][i] = pp[c0 + i];
      __syncwarp();
      if (lane == 0) {
        int i = 0;
        if (c0 == 0) {
          f.first(stage[warp][0]);
          i = 1;
        }
        for (; i + 8 <= n; i += 8) {   // eight shared-memory loads before their folds
          Acc v[8];
#pragma unroll
          for (int k = 0; k < 8; ++k) v[k] = stage[warp][i + k];
#pragma unroll
          for (int k = 0; k < 8; ++k) f.add(v[k]);
        }
        for (; i < n; ++i) f.add(stage[warp][i]);
      }
      __syncwarp();
    }
    if (lane == 0) out[o] = f.result(comp ? comp + o : nullptr);
  }
}

// ---------------------------------------------------------------- no reduction: one output per iteration
template <class Op, class Body>
__global__ void rect_map_kernel(RectPlan p, Body body, typename Op::Out* out) {
  for (int64_t f = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; f < p.O;
       f += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    typename Op::Acc acc[1] = {Op::ident()};
    body.template fold<1>(acc, f, 0);
    out[f] = Op::finish(acc[0]);
    if constexpr (std::is_same_v<typename Op::Acc, f2>) {
      if (p.comp) p.comp[f] = Op::residual(acc[0]);
    }
  }
}

}  // namespace hp
