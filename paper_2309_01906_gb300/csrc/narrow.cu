// narrow.cu — nests on 8- and 16-bit integers with a SIMD-in-register level.
//
// App. A: besides the SIMT lanes, CUDA offers SIMD intrinsics on integers that
// treat a 32-bit register as two 16-bit or four 8-bit lanes; Sec. 3.8: a level
// can be split below the lanes.  Here every 32-bit register of a thread's
// 128-bit load is such a level: sums and int8 dot products go through
// __dp4a / __dp2a_lo into an int32 accumulator (exact modulo 2^32), maxima and
// minima through packed running registers (__vmaxs4 / __vmins4, __vmaxs2 /
// __vmins2) whose sub-lanes are folded once at the end.  Warps combine with
// the warp-reduce instructions (__reduce_add/max/min_sync), CTAs in shared
// memory, grid parts after a ticket.  Integer results do not depend on the
// order, so threads take 16-byte pieces cyclically (coalesced).
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <sstream>
#include <string>

#include "api_internal.h"

namespace hp {

constexpr int kNarThreads = 256;

namespace {
int64_t ceil_div64(int64_t a, int64_t b) { return (a + b - 1) / b; }
int64_t gcd64(int64_t a, int64_t b) { return b == 0 ? a : gcd64(b, a % b); }
}  // namespace

hp_status plan_narrow(int depth, const int64_t* extents, const hp_level_map* map, hp_red_op op, int red_level,
                      hp_prec prec, hp_body body, NarrowPlan* out, std::string* why) {
  auto bad = [&](const std::string& m) {
    *why = m;
    return HP_EINVAL;
  };
  if (prec != HP_I8 && prec != HP_I16) return bad("not an 8- or 16-bit nest");
  if (op != HP_RED_SUM && op != HP_RED_MAX && op != HP_RED_MIN) return bad("HP_I8 / HP_I16 reduce with SUM, MAX or MIN");
  if (body != HP_BODY_LOAD && body != HP_BODY_DOT_BCAST) return bad("HP_I8 / HP_I16 take body LOAD or DOT_BCAST");
  if (body == HP_BODY_DOT_BCAST && (prec != HP_I8 || op != HP_RED_SUM))
    return bad("DOT_BCAST on narrow integers: HP_I8 with SUM (int8 x int8 products)");
  if (depth < 1 || depth > HP_MAX_DEPTH) return bad("depth must be in [1, HP_MAX_DEPTH]");
  if (!extents) return bad("extents is NULL");
  if (red_level < 0 || red_level >= depth) return bad("red_level must be in [0, depth - 1] (something is reduced)");
  NarrowPlan p;
  p.depth = depth;
  p.red_level = red_level;
  p.op = op;
  p.prec = prec;
  p.body = body;
  p.esize = prec == HP_I8 ? 1 : 2;
  int64_t O = 1, R = 1, inner = 1;
  for (int l = 0; l < depth; ++l) {
    if (extents[l] < 0) return bad("extents must be >= 0");
    p.ext[l] = extents[l];
    if (l < red_level) O *= extents[l];
    else R *= extents[l];
    if (l > red_level) inner *= std::max<int64_t>(extents[l], 1);
    if (O > (int64_t(1) << 40) || R > (int64_t(1) << 40)) return bad("nest too large");
  }
  if (O * std::max<int64_t>(R, 1) > (int64_t(1) << 42)) return bad("nest too large (2^42 iterations)");
  p.O = O;
  p.R = R;
  bool all_auto = map == nullptr;
  if (map) {
    all_auto = true;
    for (int l = 0; l < depth; ++l)
      if (map[l].hw != HP_HW_AUTO) all_auto = false;
  }
  p.auto_map = all_auto;
  int red_hw, sub = 0;
  int64_t tile = 0;
  const int64_t bytes = R * p.esize;
  if (all_auto) {
    red_hw = bytes <= 16384 ? HP_HW_WARP : ((O >= 304 || bytes <= (int64_t(1) << 18)) ? HP_HW_CTA : HP_HW_GRID);
  } else {
    for (int l = 0; l < red_level; ++l)
      if (map[l].hw != HP_HW_GRID) return bad("narrow-integer nests keep their output levels on GRID");
    red_hw = map[red_level].hw;
    sub = map[red_level].sub_width;
    tile = map[red_level].tile;
    for (int l = red_level; l < depth; ++l)
      if (map[l].hw != red_hw) return bad("the reduced levels of a narrow-integer nest share one hardware level");
    if (red_hw != HP_HW_WARP && red_hw != HP_HW_CTA && red_hw != HP_HW_GRID)
      return bad("narrow-integer nests put their reduced levels on WARP, CTA or GRID");
    if (red_hw == HP_HW_CTA && (sub < 0 || sub > 32)) return bad("CTA sub_width must be in [0, 32]");
    if (tile < 0) return bad("tile must be >= 0");
  }
  const int64_t piece = 16 / p.esize;   // elements of one 128-bit load
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
        const int64_t want = std::max<int64_t>(1, ceil_div64(8 * 152, std::max<int64_t>(O, 1)));
        part = std::max<int64_t>(65536, ceil_div64(R, want));
        const int64_t step = (R % piece == 0) ? inner * piece / gcd64(inner, piece) : inner;   // whole pieces
        part = ceil_div64(part, step) * step;
      }
      p.part = std::max<int64_t>(1, part);
      p.G = R > 0 ? ceil_div64(R, p.part) : 1;
      if (p.G > (int64_t(1) << 30)) return bad("too many grid parts");
    } else {
      p.G = 1;
      p.part = R;
    }
  }
  for (int l = 0; l < depth; ++l)
    p.map[l] = {l < red_level ? HP_HW_GRID : red_hw, l >= red_level && red_hw == HP_HW_CTA ? p.W : 0,
                l == red_level && red_hw == HP_HW_GRID ? p.part / inner : 0};
  *out = p;
  return HP_OK;
}

std::string describe_narrow(const NarrowPlan& p) {
  static const char* hw[] = {"grid", "cluster", "cta", "warp", "subwarp", "lane", "seq", "auto"};
  static const char* ops[] = {"sum", "max", "min"};
  std::ostringstream s;
  s << "{\"kind\":\"narrow\",\"prec\":\"" << (p.prec == HP_I8 ? "i8" : "i16") << "\",\"op\":\"" << ops[p.op]
    << "\",\"body\":\"" << (p.body == HP_BODY_LOAD ? "load" : "dot_bcast") << "\",\"depth\":" << p.depth
    << ",\"red_level\":" << p.red_level << ",\"extents\":[";
  for (int l = 0; l < p.depth; ++l) s << (l ? "," : "") << p.ext[l];
  s << "],\"map\":[";
  for (int l = 0; l < p.depth; ++l)
    s << (l ? "," : "") << "{\"hw\":\"" << hw[p.map[l].hw] << "\",\"sub_width\":" << p.map[l].sub_width
      << ",\"tile\":" << p.map[l].tile << "}";
  s << "],\"auto_map\":" << (p.auto_map ? "true" : "false") << ",\"team\":\"" << (p.team ? "block" : "warp")
    << "\",\"outputs\":" << p.O << ",\"reduced\":" << p.R << ",\"warps\":" << p.W << ",\"grid_parts\":" << p.G
    << ",\"part\":" << p.part << ",\"vec\":" << 16 / p.esize << ",\"simd\":" << 4 / p.esize << ",\"kernel\":\"narrow_"
    << (p.team ? "block" : "warp") << "\"}";
  return s.str();
}

namespace {

struct NarArgs {
  const void* a;
  const void* w;     // DOT_BCAST: broadcast operand over the reduced levels
  int32_t* out;
  int32_t* part;
  int32_t* tickets;
  int64_t O, R, G, part_len;
  int32_t W;
};

// E: int8_t or int16_t; OP: 0 sum, 1 max, 2 min
template <class E, int OP>
struct NarrowOp {
  static constexpr bool kI8 = sizeof(E) == 1;
  // packed identity of a running max / min register, and the scalar identity
  static constexpr uint32_t packed_ident() {
    return OP == 1 ? (kI8 ? 0x80808080u : 0x80008000u) : (kI8 ? 0x7f7f7f7fu : 0x7fff7fffu);
  }
  static constexpr int32_t ident() { return OP == 0 ? 0 : (OP == 1 ? (kI8 ? -128 : -32768) : (kI8 ? 127 : 32767)); }
  // one 32-bit register of the input: 4 (2) sub-lanes
  __device__ static __forceinline__ void fold_word(uint32_t x, uint32_t wv, int32_t& acc, uint32_t& pk, bool dot) {
    if constexpr (OP == 0) {
      if constexpr (kI8) acc = __dp4a(static_cast<int>(x), dot ? static_cast<int>(wv) : 0x01010101, acc);
      else acc = __dp2a_lo(static_cast<int>(x), 0x0101, acc);
    } else if constexpr (kI8) {
      pk = OP == 1 ? __vmaxs4(pk, x) : __vmins4(pk, x);
    } else if constexpr (OP == 1) {   // packed 16-bit max / min are native instructions from sm_90 on
      asm("max.s16x2 %0, %1, %2;" : "=r"(pk) : "r"(pk), "r"(x));
    } else {
      asm("min.s16x2 %0, %1, %2;" : "=r"(pk) : "r"(pk), "r"(x));
    }
  }
  __device__ static __forceinline__ int32_t unpack(uint32_t pk) {   // fold the sub-lanes of a packed register
    int32_t r = ident();
    const int n = kI8 ? 4 : 2;
    for (int i = 0; i < n; ++i) {
      const int32_t v = kI8 ? static_cast<int32_t>(static_cast<int8_t>(pk >> (8 * i)))
                            : static_cast<int32_t>(static_cast<int16_t>(pk >> (16 * i)));
      r = OP == 1 ? max(r, v) : min(r, v);
    }
    return r;
  }
  __device__ static __forceinline__ int32_t combine(int32_t a, int32_t b) {
    if constexpr (OP == 0) return static_cast<int32_t>(static_cast<uint32_t>(a) + static_cast<uint32_t>(b));
    else if constexpr (OP == 1) return max(a, b);
    else return min(a, b);
  }
  __device__ static __forceinline__ int32_t warp_reduce(int32_t v) {
    if constexpr (OP == 0) return __reduce_add_sync(0xffffffffu, v);
    else if constexpr (OP == 1) return __reduce_max_sync(0xffffffffu, v);
    else return __reduce_min_sync(0xffffffffu, v);
  }
};

// this thread's share of elements [lo, hi) of one output (base = the output's first element)
template <class E, int OP, bool DOT, bool VEC>
__device__ __forceinline__ int32_t fold_range(const E* __restrict__ a, const E* __restrict__ w, int64_t lo, int64_t hi,
                                              int64_t t, int64_t T) {
  using Op = NarrowOp<E, OP>;
  int32_t acc = OP == 0 ? 0 : Op::ident();
  uint32_t pk = Op::packed_ident();
  if constexpr (VEC) {
    constexpr int64_t kP = 16 / sizeof(E);   // elements per 128-bit piece
    const int64_t first = lo / kP + t, pe = hi / kP;
    const uint4* ap = reinterpret_cast<const uint4*>(a) + first;
    const uint4* wq = reinterpret_cast<const uint4*>(w) + first;
    int64_t n = first < pe ? (pe - first + T - 1) / T : 0;   // pieces of this thread
    for (; n >= 4; n -= 4, ap += 4 * T, wq += 4 * T) {       // four pieces in flight
      uint4 q[4], r[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        q[u] = __ldcs(ap + u * T);
        if constexpr (DOT) r[u] = __ldg(wq + u * T);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        Op::fold_word(q[u].x, DOT ? r[u].x : 0u, acc, pk, DOT);
        Op::fold_word(q[u].y, DOT ? r[u].y : 0u, acc, pk, DOT);
        Op::fold_word(q[u].z, DOT ? r[u].z : 0u, acc, pk, DOT);
        Op::fold_word(q[u].w, DOT ? r[u].w : 0u, acc, pk, DOT);
      }
    }
    for (; n > 0; --n, ap += T, wq += T) {
      const uint4 q = __ldcs(ap);
      uint4 r = make_uint4(0u, 0u, 0u, 0u);
      if constexpr (DOT) r = __ldg(wq);
      Op::fold_word(q.x, r.x, acc, pk, DOT);
      Op::fold_word(q.y, r.y, acc, pk, DOT);
      Op::fold_word(q.z, r.z, acc, pk, DOT);
      Op::fold_word(q.w, r.w, acc, pk, DOT);
    }
    if constexpr (OP != 0) acc = Op::unpack(pk);
  } else {
    for (int64_t x = lo + t; x < hi; x += T) {
      const int32_t v = static_cast<int32_t>(a[x]);
      if constexpr (OP == 0) {
        acc = static_cast<int32_t>(static_cast<uint32_t>(acc) +
                                   static_cast<uint32_t>(DOT ? v * static_cast<int32_t>(w[x]) : v));
      } else {
        acc = Op::combine(acc, v);
      }
    }
  }
  return acc;
}

// Teams of up to 256 threads are compiled for 8 resident CTAs per SM (32
// registers): a streaming fold needs the bytes in flight of 2048 threads to
// keep HBM busy.  Larger CTA teams (sub_width up to 32 warps) take a 1024-thread
// variant.
constexpr int kNarMinBlocks = 8;

template <class E, int OP, bool DOT, bool VEC>
__global__ void __launch_bounds__(kNarThreads, kNarMinBlocks) narrow_warp_kernel(NarArgs g) {
  using Op = NarrowOp<E, OP>;
  const int lane = threadIdx.x & 31;
  const int64_t warps = static_cast<int64_t>(gridDim.x) * (kNarThreads / 32);
  for (int64_t o = static_cast<int64_t>(blockIdx.x) * (kNarThreads / 32) + (threadIdx.x >> 5); o < g.O; o += warps) {
    const E* a = static_cast<const E*>(g.a) + o * g.R;
    const E* w = static_cast<const E*>(g.w);
    int32_t v = fold_range<E, OP, DOT, VEC>(a, w, 0, g.R, lane, 32);
    v = Op::warp_reduce(v);
    if (lane == 0) g.out[o] = v;
  }
}

template <class E, int OP, bool DOT, bool VEC, int MAXT>
__global__ void __launch_bounds__(MAXT, MAXT == kNarThreads ? kNarMinBlocks : 1) narrow_block_kernel(NarArgs g) {
  using Op = NarrowOp<E, OP>;
  __shared__ int32_t wp[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t items = g.O * g.G;
  for (int64_t item = blockIdx.x; item < items; item += gridDim.x) {
    const int64_t o = item / g.G, pg = item - o * g.G;
    const int64_t lo = pg * g.part_len, hi = std::min<int64_t>(lo + g.part_len, g.R);
    const E* a = static_cast<const E*>(g.a) + o * g.R;
    int32_t v = fold_range<E, OP, DOT, VEC>(a, static_cast<const E*>(g.w), lo, hi, threadIdx.x, blockDim.x);
    v = Op::warp_reduce(v);
    if (lane == 0) wp[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      int32_t r = wp[0];
      for (int q = 1; q < g.W; ++q) r = Op::combine(r, wp[q]);
      if (g.G == 1) {
        g.out[o] = r;
      } else {
        g.part[item] = r;
        __threadfence();   // publish the part before taking the ticket
        if (atomicAdd(&g.tickets[o], 1) == g.G - 1) {
          __threadfence();
          const volatile int32_t* pp = g.part + o * g.G;
          int32_t s = pp[0];
          for (int64_t q = 1; q < g.G; ++q) s = Op::combine(s, pp[q]);
          g.out[o] = s;
          g.tickets[o] = 0;   // ready for the next run
        }
      }
    }
    __syncthreads();   // wp is rewritten by the next item
  }
}

template <class K>
int nar_blocks(K kernel, int threads, int sms) {
  int per = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, 0);
  return std::max(1, per) * sms;
}

// CTAs for `items` work items when `resident` fit at once: the fewest waves,
// with the items spread evenly over them (no short last wave)
int64_t balanced_grid(int64_t items, int64_t resident) {
  if (items <= resident) return std::max<int64_t>(items, 1);
  const int64_t waves = ceil_div64(items, resident);
  return ceil_div64(items, waves);
}

template <class E, int OP, bool DOT, bool VEC>
cudaError_t launch_narrow(const NarrowPlan& p, const NarArgs& g, int sms, cudaStream_t st) {
  if (p.team == 0) {
    const int64_t need = ceil_div64(p.O, kNarThreads / 32);
    const int grid =
        static_cast<int>(balanced_grid(need, nar_blocks(narrow_warp_kernel<E, OP, DOT, VEC>, kNarThreads, sms)));
    narrow_warp_kernel<E, OP, DOT, VEC><<<grid, kNarThreads, 0, st>>>(g);
  } else {
    const int threads = 32 * p.W;
    if (threads <= kNarThreads) {
      auto k = narrow_block_kernel<E, OP, DOT, VEC, kNarThreads>;
      const int grid = static_cast<int>(balanced_grid(p.O * p.G, nar_blocks(k, threads, sms)));
      k<<<grid, threads, 0, st>>>(g);
    } else {
      auto k = narrow_block_kernel<E, OP, DOT, VEC, 1024>;
      const int grid = static_cast<int>(balanced_grid(p.O * p.G, nar_blocks(k, threads, sms)));
      k<<<grid, threads, 0, st>>>(g);
    }
  }
  return cudaPeekAtLastError();
}

template <class E, int OP, bool DOT>
cudaError_t launch_narrow_v(const NarrowPlan& p, const NarArgs& g, bool vec, int sms, cudaStream_t st) {
  return vec ? launch_narrow<E, OP, DOT, true>(p, g, sms, st) : launch_narrow<E, OP, DOT, false>(p, g, sms, st);
}

}  // namespace

hp_status narrow_prepare(hp_nest* n) {
  const NarrowPlan& p = n->nar;
  if (p.G > 1 && p.O > 0) {
    n->part_bytes = static_cast<size_t>(p.O * p.G) * sizeof(int32_t);
    cudaError_t e = cudaMalloc(&n->part, n->part_bytes);
    if (e != cudaSuccess) return fail(HP_ENOMEM, "cudaMalloc (narrow parts)");
    if ((e = cudaMalloc(&n->tickets, sizeof(int32_t) * p.O)) != cudaSuccess)
      return fail(HP_ENOMEM, "cudaMalloc (narrow tickets)");
    if ((e = cudaMemset(n->tickets, 0, sizeof(int32_t) * p.O)) != cudaSuccess)
      return fail(HP_ECUDA, std::string("cudaMemset (tickets): ") + cudaGetErrorString(e));
  }
  return HP_OK;
}

hp_status run_narrow(hp_nest* n, const void* const* in_dev, void* out_dev, cudaStream_t st) {
  const NarrowPlan& p = n->nar;
  if (p.O == 0) return HP_OK;
  if (!out_dev) return fail(HP_EINVAL, "out is NULL");
  const bool dot = p.body == HP_BODY_DOT_BCAST;
  if (p.R > 0 && (!in_dev || !in_dev[0] || (dot && !in_dev[1]))) return fail(HP_EINVAL, "missing input");
  NarArgs g;
  g.a = p.R > 0 ? in_dev[0] : nullptr;
  g.w = (p.R > 0 && dot) ? in_dev[1] : nullptr;
  g.out = static_cast<int32_t*>(out_dev);
  g.part = static_cast<int32_t*>(n->part);
  g.tickets = n->tickets;
  g.O = p.O;
  g.R = p.R;
  g.G = p.G;
  g.part_len = std::max<int64_t>(p.part, 1);
  g.W = p.W;
  const int64_t piece = 16 / p.esize;
  const bool vec = p.R % piece == 0 && g.part_len % piece == 0 && reinterpret_cast<uintptr_t>(g.a) % 16 == 0 &&
                   (!dot || reinterpret_cast<uintptr_t>(g.w) % 16 == 0);
  cudaError_t e;
  const int sms = n->sms;
  if (p.prec == HP_I8) {
    if (dot) e = launch_narrow_v<int8_t, 0, true>(p, g, vec, sms, st);
    else if (p.op == HP_RED_SUM) e = launch_narrow_v<int8_t, 0, false>(p, g, vec, sms, st);
    else if (p.op == HP_RED_MAX) e = launch_narrow_v<int8_t, 1, false>(p, g, vec, sms, st);
    else e = launch_narrow_v<int8_t, 2, false>(p, g, vec, sms, st);
  } else {
    if (p.op == HP_RED_SUM) e = launch_narrow_v<int16_t, 0, false>(p, g, vec, sms, st);
    else if (p.op == HP_RED_MAX) e = launch_narrow_v<int16_t, 1, false>(p, g, vec, sms, st);
    else e = launch_narrow_v<int16_t, 2, false>(p, g, vec, sms, st);
  }
  if (e != cudaSuccess) return fail(HP_ECUDA, std::string("narrow launch: ") + cudaGetErrorString(e));
  return HP_OK;
}

}  // namespace hp
