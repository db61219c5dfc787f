// ordered.cu — nests with an ordered, non-commutative reduction.
//
// Sec. 2: a reduction combines on each level the results of its sibling
// tasks; with a non-commutative operator the siblings must be combined in the
// order of the iterations they folded.  The lowering gives every warp a
// contiguous range of iterations and folds it in rounds: in each round lane l
// folds the l-th of 32 consecutive pieces sequentially (so the warp's loads
// are coalesced), a __shfl_down_sync tree at distances 1, 2, ..., 16 joins the
// 32 pieces in order into lane 0 (at each level a lane's own range first, the
// range of the lane at the given distance after it: Sec. 3.7's sibling
// exchange, one combine per level), and the round joins the warp's running
// state.
// Warps of a CTA are combined by rank the same way, and the parts of an output
// are folded in part order by the CTA that takes the last ticket.
//
// The operator is a compile-time parameter of the kernels (the op table):
//   HP_RED_AFFINE_COMPOSE  f_x(y) = a_x y + b_x composed in order; (A1, B1) then
//                          (A2, B2) give (A2 A1, fma(A2, B1, B2));
//   HP_RED_MAT2_PRODUCT    2x2 matrices multiplied in order, the later on the
//                          left: E then L give L E (each entry one product and
//                          one fused multiply-add);
//   HP_RED_LAST_VALID      the value of the last iteration that is not NaN;
//                          E then L give L unless L is NaN.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <sstream>
#include <string>

#include "api_internal.h"

namespace hp {

constexpr int kOrdThreads = 256;

namespace {

int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

}  // namespace

hp_status plan_ordered(int depth, const int64_t* extents, const hp_level_map* map, hp_red_op op, int red_level,
                       hp_prec prec, hp_body body, OrderedPlan* out, std::string* why) {
  auto bad = [&](const std::string& m) {
    *why = m;
    return HP_EINVAL;
  };
  if (op != HP_RED_AFFINE_COMPOSE && op != HP_RED_MAT2_PRODUCT && op != HP_RED_LAST_VALID)
    return bad("not an ordered reduction");
  if (depth < 1 || depth > HP_MAX_DEPTH) return bad("depth must be in [1, HP_MAX_DEPTH]");
  if (!extents) return bad("extents is NULL");
  if (red_level < 0 || red_level >= depth) return bad("red_level must be in [0, depth - 1] (something is reduced)");
  if (prec != HP_F32) return bad("ordered reductions take prec HP_F32");
  if (body != HP_BODY_LOAD) return bad("ordered reductions take body HP_BODY_LOAD (inputs per operator)");
  OrderedPlan p;
  p.depth = depth;
  p.red_level = red_level;
  p.op = op;
  p.ib = op == HP_RED_MAT2_PRODUCT ? 16 : 4;   // bytes of one iteration in each input array
  int64_t O = 1, R = 1, inner = 1;
  for (int l = 0; l < depth; ++l) {
    if (extents[l] < 0) return bad("extents must be >= 0");
    p.ext[l] = extents[l];
    const int64_t e = std::max<int64_t>(extents[l], 1);
    if (l < red_level) O = O * extents[l];
    else R = R * extents[l];
    if (l > red_level) inner *= e;
    if (O > (int64_t(1) << 40) || R > (int64_t(1) << 40)) return bad("nest too large");
  }
  if (O * std::max<int64_t>(R, 1) > (int64_t(1) << 40)) return bad("nest too large (2^40 iterations)");
  p.O = O;
  p.R = R;
  bool all_auto = map == nullptr;
  if (map) {
    all_auto = true;
    for (int l = 0; l < depth; ++l)
      if (map[l].hw != HP_HW_AUTO) all_auto = false;
  }
  p.auto_map = all_auto;
  int red_hw = HP_HW_AUTO, sub = 0;
  int64_t tile = 0;
  if (!all_auto) {
    for (int l = 0; l < red_level; ++l)
      if (map[l].hw != HP_HW_GRID) return bad("ordered reductions keep their output levels on GRID");
    red_hw = map[red_level].hw;
    sub = map[red_level].sub_width;
    tile = map[red_level].tile;
    for (int l = red_level; l < depth; ++l)
      if (map[l].hw != red_hw) return bad("the reduced levels of an ordered reduction share one hardware level");
    if (red_hw != HP_HW_WARP && red_hw != HP_HW_CTA && red_hw != HP_HW_GRID)
      return bad("ordered reductions put their reduced levels on WARP, CTA or GRID");
    if (red_hw == HP_HW_CTA && (sub < 0 || sub > 32)) return bad("CTA sub_width must be in [0, 32]");
    if (tile < 0) return bad("tile must be >= 0");
  } else {
    // a warp per output for short ranges, a CTA for long ones, grid parts when
    // few outputs face a long range
    red_hw = R <= 1024 ? HP_HW_WARP : ((O >= 304 || R <= 65536) ? HP_HW_CTA : HP_HW_GRID);
  }
  if (red_hw == HP_HW_WARP) {
    p.team = 0;
    p.W = 1;
    p.G = 1;
    p.part = R;
  } else {
    p.team = 1;
    p.W = (red_hw == HP_HW_CTA && sub > 0) ? sub : 8;
    if (red_hw == HP_HW_GRID) {
      int64_t part;
      if (tile > 0) {
        part = tile * inner;
      } else {
        // about 8 CTA teams per SM over all parts (2 waves of 4 resident CTAs)
        const int64_t want = std::max<int64_t>(1, ceil_div(8 * 152, std::max<int64_t>(O, 1)));
        part = std::max<int64_t>(16384, ceil_div(R, want));
        // whole iterations of the first reduced level, and parts of whole 256- / 128-bit loads
        // when R allows
        const int64_t al = p.ib == 16 ? (R % 2 == 0 ? 2 : 1) : (R % 8 == 0 ? 8 : (R % 4 == 0 ? 4 : 1));
        const int64_t step = inner * al / std::__gcd<int64_t>(inner, al);
        part = ceil_div(part, step) * step;
      }
      p.part = std::max<int64_t>(1, part);
      p.G = R > 0 ? ceil_div(R, p.part) : 1;
      if (p.G > (int64_t(1) << 30)) return bad("too many grid parts");
    } else {
      p.G = 1;
      p.part = R;
    }
  }
  for (int l = 0; l < depth; ++l)
    p.map[l] = {l < red_level ? HP_HW_GRID : red_hw, l >= red_level && red_hw == HP_HW_CTA ? p.W : 0,
                l == red_level && red_hw == HP_HW_GRID ? p.part / inner : 0};
  if (p.ib == 16)   // a matrix is one 128-bit load; two make one 256-bit load
    p.V = (R % 2 == 0 && p.part % 2 == 0) ? 8 : 4;
  else
    p.V = (R % 8 == 0 && p.part % 8 == 0) ? 8 : ((R % 4 == 0 && p.part % 4 == 0) ? 4 : 1);
  // a lane's piece of each round, measured per operator: 8 affine maps (32 bytes
  // of each input: a warp's load reads 1 KB in one piece), 4 matrices, 32 values
  // (fewer rounds where the butterfly or the round's latency costs more than
  // coalescing gains); a warp's range is a whole number of pieces
  p.piece = op == HP_RED_MAT2_PRODUCT ? 4 : (op == HP_RED_LAST_VALID ? 32 : 8);
  p.chunk = p.team == 0 ? std::max<int64_t>(R, 1) : ceil_div(std::max<int64_t>(p.part, 1), p.W);
  p.chunk = ceil_div(p.chunk, p.piece) * p.piece;
  // longest chain: a piece, 5 lane levels, the rounds, 5 warp levels (CTA teams), the part fold
  const int64_t rounds = ceil_div(p.chunk, 32 * p.piece);
  p.k = static_cast<int32_t>(
      std::min<int64_t>(p.piece + 5 + rounds + (p.team ? 5 : 0) + (p.G - 1), int64_t(1) << 30));
  *out = p;
  return HP_OK;
}

std::string describe_ordered(const OrderedPlan& p) {
  static const char* hw[] = {"grid", "cluster", "cta", "warp", "subwarp", "lane", "seq", "auto"};
  std::ostringstream s;
  const char* op = p.op == HP_RED_MAT2_PRODUCT ? "mat2_product" : (p.op == HP_RED_LAST_VALID ? "last_valid" : "affine_compose");
  s << "{\"kind\":\"ordered\",\"op\":\"" << op << "\",\"depth\":" << p.depth << ",\"red_level\":" << p.red_level
    << ",\"extents\":[";
  for (int l = 0; l < p.depth; ++l) s << (l ? "," : "") << p.ext[l];
  s << "],\"map\":[";
  for (int l = 0; l < p.depth; ++l)
    s << (l ? "," : "") << "{\"hw\":\"" << hw[p.map[l].hw] << "\",\"sub_width\":" << p.map[l].sub_width
      << ",\"tile\":" << p.map[l].tile << "}";
  s << "],\"auto_map\":" << (p.auto_map ? "true" : "false") << ",\"team\":\"" << (p.team ? "block" : "warp")
    << "\",\"outputs\":" << p.O << ",\"reduced\":" << p.R << ",\"warps\":" << p.W << ",\"grid_parts\":" << p.G
    << ",\"part\":" << p.part << ",\"chunk\":" << p.chunk << ",\"piece\":" << p.piece << ",\"vec\":" << p.V
    << ",\"chain\":" << p.k
    << ",\"kernel\":\"ordered_" << (p.team ? "block" : "warp") << "\"}";
  return s.str();
}

namespace {

struct OrdArgs {
  const float* a;     // affine: the a_x; matrices: 4 entries per iteration (row-major); last valid: the values
  const float* b;     // affine: the b_x
  float* out;
  float* part;        // the state of every (output, part) when G > 1
  int32_t* tickets;   // per output, G > 1
  int64_t O, R, G, part_len, chunk;
  int32_t W;
};

// one 256-bit read-only load (a whole 32-byte sector; the address is 32-byte aligned)
__device__ __forceinline__ void ld8(const float* p, float* r) {
  asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
      : "=f"(r[0]), "=f"(r[1]), "=f"(r[2]), "=f"(r[3]), "=f"(r[4]), "=f"(r[5]), "=f"(r[6]), "=f"(r[7])
      : "l"(p));
}

// A lane walks its own block, so its loads do not coalesce across the warp:
// V = 8 takes whole 32-byte sectors with 256-bit loads (each in one request),
// V = 4 128-bit loads, V = 1 scalar loads.  Every fold runs over [s, e) of the
// output whose first iteration is `base`, in order.

struct AffineOp {
  using S = float2;   // (A, B)
  static constexpr int kOut = 2;
  template <int V>
  __device__ static constexpr int64_t piece() { return 8; }   // a lane's iterations per round
  __device__ static S ident() { return make_float2(1.0f, 0.0f); }
  __device__ static S combine(S e, S l) { return make_float2(__fmul_rn(l.x, e.x), __fmaf_rn(l.x, e.y, l.y)); }
  __device__ static S shfl(S v, int m) {
    return make_float2(__shfl_down_sync(0xffffffffu, v.x, m), __shfl_down_sync(0xffffffffu, v.y, m));
  }
  __device__ static void put(float* p, int64_t i, S v) {
    p[2 * i] = v.x;
    p[2 * i + 1] = v.y;
  }
  __device__ static S get(const volatile float* p, int64_t i) { return make_float2(p[2 * i], p[2 * i + 1]); }
  template <int V>
  __device__ static S fold(const OrdArgs& g, int64_t base, int64_t s, int64_t e, S v);
};

template <int V>
__device__ __forceinline__ float2 fold_affine(const float* __restrict__ a, const float* __restrict__ b, int64_t s,
                                            int64_t e, float2 v) {
  if constexpr (V == 8) {
    for (; s + 16 <= e; s += 16) {
      float av[16], bv[16];
      ld8(a + s, av);
      ld8(a + s + 8, av + 8);
      ld8(b + s, bv);
      ld8(b + s + 8, bv + 8);
#pragma unroll
      for (int q = 0; q < 16; ++q) v = AffineOp::combine(v, make_float2(av[q], bv[q]));
    }
    for (; s < e; s += 8) {
      float av[8], bv[8];
      ld8(a + s, av);
      ld8(b + s, bv);
#pragma unroll
      for (int q = 0; q < 8; ++q) v = AffineOp::combine(v, make_float2(av[q], bv[q]));
    }
  } else if constexpr (V == 4) {
    for (; s + 16 <= e; s += 16) {   // four 128-bit loads of each input in flight
      float4 av[4], bv[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        av[q] = __ldg(reinterpret_cast<const float4*>(a + s + 4 * q));
        bv[q] = __ldg(reinterpret_cast<const float4*>(b + s + 4 * q));
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        v = AffineOp::combine(v, make_float2(av[q].x, bv[q].x));
        v = AffineOp::combine(v, make_float2(av[q].y, bv[q].y));
        v = AffineOp::combine(v, make_float2(av[q].z, bv[q].z));
        v = AffineOp::combine(v, make_float2(av[q].w, bv[q].w));
      }
    }
    for (; s < e; s += 4) {
      const float4 a0 = __ldg(reinterpret_cast<const float4*>(a + s));
      const float4 b0 = __ldg(reinterpret_cast<const float4*>(b + s));
      v = AffineOp::combine(v, make_float2(a0.x, b0.x));
      v = AffineOp::combine(v, make_float2(a0.y, b0.y));
      v = AffineOp::combine(v, make_float2(a0.z, b0.z));
      v = AffineOp::combine(v, make_float2(a0.w, b0.w));
    }
  } else {
    for (; s < e; ++s) v = AffineOp::combine(v, make_float2(__ldg(a + s), __ldg(b + s)));
  }
  return v;
}

template <int V>
__device__ __forceinline__ AffineOp::S AffineOp::fold(const OrdArgs& g, int64_t base, int64_t s, int64_t e, S v) {
  return fold_affine<V>(g.a + base, g.b + base, s, e, v);
}

struct Mat2Op {
  using S = float4;   // (m00, m01, m10, m11)
  static constexpr int kOut = 4;
  template <int V>
  __device__ static constexpr int64_t piece() { return 4; }
  __device__ static S ident() { return make_float4(1.0f, 0.0f, 0.0f, 1.0f); }
  __device__ static S combine(S e, S l) {   // L E
    return make_float4(__fmaf_rn(l.x, e.x, __fmul_rn(l.y, e.z)), __fmaf_rn(l.x, e.y, __fmul_rn(l.y, e.w)),
                       __fmaf_rn(l.z, e.x, __fmul_rn(l.w, e.z)), __fmaf_rn(l.z, e.y, __fmul_rn(l.w, e.w)));
  }
  __device__ static S shfl(S v, int m) {
    return make_float4(__shfl_down_sync(0xffffffffu, v.x, m), __shfl_down_sync(0xffffffffu, v.y, m),
                       __shfl_down_sync(0xffffffffu, v.z, m), __shfl_down_sync(0xffffffffu, v.w, m));
  }
  __device__ static void put(float* p, int64_t i, S v) {
    p[4 * i] = v.x;
    p[4 * i + 1] = v.y;
    p[4 * i + 2] = v.z;
    p[4 * i + 3] = v.w;
  }
  __device__ static S get(const volatile float* p, int64_t i) {
    return make_float4(p[4 * i], p[4 * i + 1], p[4 * i + 2], p[4 * i + 3]);
  }
  template <int V>
  __device__ static S fold(const OrdArgs& g, int64_t base, int64_t s, int64_t e, S v) {
    const float* __restrict__ m = g.a + 4 * base;
    if constexpr (V == 8) {   // two matrices per 256-bit load
      for (; s + 8 <= e; s += 8) {
        float r[32];
#pragma unroll
        for (int q = 0; q < 4; ++q) ld8(m + 4 * s + 8 * q, r + 8 * q);
#pragma unroll
        for (int q = 0; q < 8; ++q) v = combine(v, make_float4(r[4 * q], r[4 * q + 1], r[4 * q + 2], r[4 * q + 3]));
      }
      for (; s < e; s += 2) {
        float r[8];
        ld8(m + 4 * s, r);
        v = combine(v, make_float4(r[0], r[1], r[2], r[3]));
        v = combine(v, make_float4(r[4], r[5], r[6], r[7]));
      }
    } else if constexpr (V == 4) {   // one matrix per 128-bit load
      for (; s + 4 <= e; s += 4) {
        float4 q[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) q[u] = __ldg(reinterpret_cast<const float4*>(m + 4 * (s + u)));
#pragma unroll
        for (int u = 0; u < 4; ++u) v = combine(v, q[u]);
      }
      for (; s < e; ++s) v = combine(v, __ldg(reinterpret_cast<const float4*>(m + 4 * s)));
    } else {
      for (; s < e; ++s) {
        const float* x = m + 4 * s;
        v = combine(v, make_float4(__ldg(x), __ldg(x + 1), __ldg(x + 2), __ldg(x + 3)));
      }
    }
    return v;
  }
};

struct LastOp {
  using S = float;    // the last value that is not NaN so far (NaN: none)
  static constexpr int kOut = 1;
  template <int V>
  __device__ static constexpr int64_t piece() { return 32; }
  __device__ static S ident() { return __int_as_float(0x7fc00000); }
  __device__ static S combine(S e, S l) { return l != l ? e : l; }
  __device__ static S shfl(S v, int m) { return __shfl_down_sync(0xffffffffu, v, m); }
  __device__ static void put(float* p, int64_t i, S v) { p[i] = v; }
  __device__ static S get(const volatile float* p, int64_t i) { return p[i]; }
  template <int V>
  __device__ static S fold(const OrdArgs& g, int64_t base, int64_t s, int64_t e, S v) {
    const float* __restrict__ a = g.a + base;
    if constexpr (V == 8) {
      for (; s + 32 <= e; s += 32) {
        float r[32];
#pragma unroll
        for (int q = 0; q < 4; ++q) ld8(a + s + 8 * q, r + 8 * q);
#pragma unroll
        for (int q = 0; q < 32; ++q) v = combine(v, r[q]);
      }
      for (; s < e; s += 8) {
        float r[8];
        ld8(a + s, r);
#pragma unroll
        for (int q = 0; q < 8; ++q) v = combine(v, r[q]);
      }
    } else if constexpr (V == 4) {
      for (; s + 16 <= e; s += 16) {
        float4 q[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) q[u] = __ldg(reinterpret_cast<const float4*>(a + s + 4 * u));
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          v = combine(v, q[u].x);
          v = combine(v, q[u].y);
          v = combine(v, q[u].z);
          v = combine(v, q[u].w);
        }
      }
      for (; s < e; s += 4) {
        const float4 q = __ldg(reinterpret_cast<const float4*>(a + s));
        v = combine(combine(combine(combine(v, q.x), q.y), q.z), q.w);
      }
    } else {
      for (; s < e; ++s) v = combine(v, __ldg(a + s));
    }
    return v;
  }
};

// ranks 0..31 combined in rank order into lane 0: at distance m lane l (a
// multiple of 2m) holds ranks [l, l + m) and takes [l + m, l + 2m) from lane
// l + m, its own range first.  Only lane 0's result is meaningful (the other
// lanes combine ranges that are not adjacent); it is the same tree as an xor
// butterfly's lane 0, with one combine per level and no selects.
template <class Op>
__device__ __forceinline__ typename Op::S lanes_in_order(typename Op::S v, int lane) {
  (void)lane;
#pragma unroll
  for (int m = 1; m < 32; m <<= 1) v = Op::combine(v, Op::shfl(v, m));
  return v;
}

// A warp folds its range [ws, we) in rounds of 32 consecutive pieces of P
// iterations: lane l folds the l-th piece (so one load instruction of the
// warp reads 32 adjacent pieces: coalesced), the lane tree joins the 32 pieces
// in order, and the round joins the running state.  Lane 0 ends with the
// composition of the whole range.
template <class Op, int V>
__device__ __forceinline__ typename Op::S fold_warp(const OrdArgs& g, int64_t base, int64_t ws, int64_t we, int lane) {
  constexpr int64_t P = Op::template piece<V>();
  typename Op::S v = Op::ident();
  for (int64_t r0 = ws; r0 < we; r0 += 32 * P) {
    const int64_t s = std::min<int64_t>(r0 + lane * P, we), e = std::min<int64_t>(s + P, we);
    typename Op::S pc = Op::template fold<V>(g, base, s, e, Op::ident());
    pc = lanes_in_order<Op>(pc, lane);
    v = Op::combine(v, pc);
  }
  return v;
}

template <class Op, int V>
__global__ void __launch_bounds__(kOrdThreads) ordered_warp_kernel(OrdArgs g) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = static_cast<int64_t>(gridDim.x) * (kOrdThreads / 32);
  for (int64_t o = static_cast<int64_t>(blockIdx.x) * (kOrdThreads / 32) + (threadIdx.x >> 5); o < g.O; o += warps) {
    const typename Op::S v = fold_warp<Op, V>(g, o * g.R, 0, g.R, lane);
    if (lane == 0) Op::put(g.out, o, v);
  }
}

template <class Op, int V>
__global__ void __launch_bounds__(1024) ordered_block_kernel(OrdArgs g) {   // W <= 32 warps per team
  __shared__ typename Op::S wp[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t items = g.O * g.G;
  for (int64_t item = blockIdx.x; item < items; item += gridDim.x) {
    const int64_t o = item / g.G, pg = item - o * g.G;
    const int64_t lo = pg * g.part_len, hi = std::min<int64_t>(lo + g.part_len, g.R);
    const int64_t ws = std::min<int64_t>(lo + warp * g.chunk, hi), we = std::min<int64_t>(ws + g.chunk, hi);
    const typename Op::S v = fold_warp<Op, V>(g, o * g.R, ws, we, lane);
    if (lane == 0) wp[warp] = v;
    __syncthreads();
    if (warp == 0) {
      typename Op::S w = lane < g.W ? wp[lane] : Op::ident();   // the identity pads the ranks
      w = lanes_in_order<Op>(w, lane);
      if (lane == 0) {
        if (g.G == 1) {
          Op::put(g.out, o, w);
        } else {
          Op::put(g.part, item, w);
          __threadfence();   // publish the part before taking the ticket
          if (atomicAdd(&g.tickets[o], 1) == g.G - 1) {
            __threadfence();
            const volatile float* pp = g.part;
            typename Op::S r = Op::get(pp, o * g.G);
            for (int64_t q = 1; q < g.G; ++q) r = Op::combine(r, Op::get(pp, o * g.G + q));   // part order
            Op::put(g.out, o, r);
            g.tickets[o] = 0;   // ready for the next run
          }
        }
      }
    }
    __syncthreads();   // wp is rewritten by the next item
  }
}

template <class K>
int blocks_for(K kernel, int threads, int sms) {
  int per = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, 0);
  return std::max(1, per) * sms;
}

// CTAs for `items` work items when `resident` fit at once: the fewest waves,
// with the items spread evenly over them (no short last wave)
int64_t balanced_grid(int64_t items, int64_t resident) {
  if (items <= resident) return std::max<int64_t>(items, 1);
  const int64_t waves = ceil_div(items, resident);
  return ceil_div(items, waves);
}

int out_floats(const OrderedPlan& p) {
  return p.op == HP_RED_MAT2_PRODUCT ? Mat2Op::kOut : (p.op == HP_RED_LAST_VALID ? LastOp::kOut : AffineOp::kOut);
}

template <class Op, int V>
void launch_ordered(const OrderedPlan& p, const OrdArgs& g, int sms, cudaStream_t st) {
  if (p.team == 0) {
    auto k = ordered_warp_kernel<Op, V>;
    const int64_t need = ceil_div(p.O, kOrdThreads / 32);
    const int grid = static_cast<int>(balanced_grid(need, blocks_for(k, kOrdThreads, sms)));
    k<<<grid, kOrdThreads, 0, st>>>(g);
  } else {
    const int threads = 32 * p.W;
    auto go = [&](auto k) {
      const int grid = static_cast<int>(balanced_grid(p.O * p.G, blocks_for(k, threads, sms)));
      k<<<grid, threads, 0, st>>>(g);
    };
    go(ordered_block_kernel<Op, V>);
  }
}

template <class Op>
void launch_ordered_v(const OrderedPlan& p, const OrdArgs& g, int v, int sms, cudaStream_t st) {
  if (v == 8) launch_ordered<Op, 8>(p, g, sms, st);
  else if (v == 4) launch_ordered<Op, 4>(p, g, sms, st);
  else launch_ordered<Op, 1>(p, g, sms, st);
}

}  // namespace

size_t ordered_out_bytes(const OrderedPlan& p) { return static_cast<size_t>(p.O) * out_floats(p) * sizeof(float); }

hp_status ordered_prepare(hp_nest* n) {
  const OrderedPlan& p = n->ord;
  if (p.G > 1 && p.O > 0) {
    n->part_bytes = static_cast<size_t>(p.O * p.G) * out_floats(p) * sizeof(float);
    cudaError_t e = cudaMalloc(&n->part, n->part_bytes);
    if (e != cudaSuccess) return fail(HP_ENOMEM, "cudaMalloc (ordered parts)");
    if ((e = cudaMalloc(&n->tickets, sizeof(int32_t) * p.O)) != cudaSuccess)
      return fail(HP_ENOMEM, "cudaMalloc (ordered tickets)");
    if ((e = cudaMemset(n->tickets, 0, sizeof(int32_t) * p.O)) != cudaSuccess)
      return fail(HP_ECUDA, std::string("cudaMemset (tickets): ") + cudaGetErrorString(e));
  }
  return HP_OK;
}

hp_status run_ordered(hp_nest* n, const void* const* in_dev, void* out_dev, cudaStream_t st) {
  const OrderedPlan& p = n->ord;
  if (p.O == 0) return HP_OK;
  if (!out_dev) return fail(HP_EINVAL, "out is NULL");
  const bool affine = p.op == HP_RED_AFFINE_COMPOSE;
  if (p.R > 0 && (!in_dev || !in_dev[0] || (affine && !in_dev[1])))
    return fail(HP_EINVAL, affine ? "inputs {a, b} expected" : "input array expected");
  OrdArgs g;
  g.a = p.R > 0 ? static_cast<const float*>(in_dev[0]) : nullptr;
  g.b = (p.R > 0 && affine) ? static_cast<const float*>(in_dev[1]) : nullptr;
  g.out = static_cast<float*>(out_dev);
  g.part = static_cast<float*>(n->part);
  g.tickets = n->tickets;
  g.O = p.O;
  g.R = p.R;
  g.G = p.G;
  g.part_len = std::max<int64_t>(p.part, 1);
  g.chunk = p.chunk;
  g.W = p.W;
  if (reinterpret_cast<uintptr_t>(out_dev) % 4 != 0) return fail(HP_EINVAL, "out must be 4-byte aligned");
  // the widest loads the plan and the input alignment allow (blocks start at whole loads)
  const uintptr_t al = reinterpret_cast<uintptr_t>(g.a) | reinterpret_cast<uintptr_t>(g.b);
  const int v = (p.V == 8 && al % 32 == 0) ? 8 : ((p.V >= 4 && al % 16 == 0) ? 4 : 1);
  const int sms = n->sms;
  if (p.op == HP_RED_MAT2_PRODUCT) launch_ordered_v<Mat2Op>(p, g, v, sms, st);
  else if (p.op == HP_RED_LAST_VALID) launch_ordered_v<LastOp>(p, g, v, sms, st);
  else launch_ordered_v<AffineOp>(p, g, v, sms, st);
  const cudaError_t e = cudaPeekAtLastError();
  if (e != cudaSuccess) return fail(HP_ECUDA, std::string("ordered launch: ") + cudaGetErrorString(e));
  return HP_OK;
}

}  // namespace hp
