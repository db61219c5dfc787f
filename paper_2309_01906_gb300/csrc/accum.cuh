// accum.cuh — accumulation policies of the executor (one per precision x op).
//
// Each policy gives: Acc (the running value a thread, warp, CTA or cluster
// holds), ident(), add_val (fold one body value), add_prod (fold a*b),
// combine (fold another partial: the sibling combine of Sec. 2 / Sec. 3.7),
// shfl_xor (exchange a partial between lanes, Sec. 3.7 __shfl_xor_sync),
// finish (Acc -> output element).
//
// Compensated FP32 (HP_F32_COMP) follows Ogita, Rump and Oishi, "Accurate sum
// and dot product" (SIAM J. Sci. Comput. 26(6), 2005), algorithm Dot2: each
// product is split exactly into p + e (TwoProduct via FMA), each sum into
// s + e (Knuth's TwoSum, 6 flops, branch-free), and the error terms are added
// up in a second FP32 word.  Partials combine by TwoSum of the leading words
// plus the sum of the trailing words.  All operations use explicit
// round-to-nearest intrinsics so that no contraction into FMA can change them.
#pragma once

#include <cstdint>
#include <type_traits>

#include <cuda_runtime.h>

namespace hp {

struct f2 {
  float s, c;
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

struct OpF32Sum {
  using In = float;
  using Acc = float;
  using Out = float;
  static constexpr bool kFp = true;
  __device__ static Acc ident() { return 0.0f; }
  __device__ static void add_val(Acc& a, float x) { a = __fadd_rn(a, x); }
  __device__ static void add_prod(Acc& a, float x, float y) { a = __fmaf_rn(x, y, a); }
  __device__ static Acc combine(Acc a, Acc b) { return __fadd_rn(a, b); }
  __device__ static Acc shfl_xor(Acc a, int m, int w) { return __shfl_xor_sync(0xffffffffu, a, m, w); }
  __device__ static Out finish(Acc a) { return a; }
};

struct OpF32Comp {
  using In = float;
  using Acc = f2;
  using Out = float;
  static constexpr bool kFp = true;
  __device__ static Acc ident() { return {0.0f, 0.0f}; }
  __device__ static void add_val(Acc& a, float x) {
    float s, e;
    two_sum(a.s, x, s, e);
    a.s = s;
    a.c = __fadd_rn(a.c, e);
  }
  __device__ static void add_prod(Acc& a, float x, float y) {
    const float p = __fmul_rn(x, y);
    const float ep = __fmaf_rn(x, y, -p);  // exact: x*y = p + ep
    float s, es;
    two_sum(a.s, p, s, es);
    a.s = s;
    a.c = __fadd_rn(a.c, __fadd_rn(ep, es));
  }
  __device__ static Acc combine(Acc a, Acc b) {
    float s, e;
    two_sum(a.s, b.s, s, e);
    return {s, __fadd_rn(__fadd_rn(a.c, b.c), e)};
  }
  __device__ static Acc shfl_xor(Acc a, int m, int w) {
    return {__shfl_xor_sync(0xffffffffu, a.s, m, w), __shfl_xor_sync(0xffffffffu, a.c, m, w)};
  }
  __device__ static Out finish(Acc a) { return __fadd_rn(a.s, a.c); }
  // exact error of finish(): finish(a) + residual(a) == a.s + a.c (TwoSum)
  __device__ static float residual(Acc a) {
    float s, e;
    two_sum(a.s, a.c, s, e);
    return e;
  }
};

struct OpF32Max {
  using In = float;
  using Acc = float;
  using Out = float;
  static constexpr bool kFp = true;
  __device__ static Acc ident() { return -__int_as_float(0x7f800000); }
  __device__ static void add_val(Acc& a, float x) { a = fmaxf(a, x); }
  __device__ static void add_prod(Acc& a, float x, float y) { a = fmaxf(a, __fmul_rn(x, y)); }
  __device__ static Acc combine(Acc a, Acc b) { return fmaxf(a, b); }
  __device__ static Acc shfl_xor(Acc a, int m, int w) { return __shfl_xor_sync(0xffffffffu, a, m, w); }
  __device__ static Out finish(Acc a) { return a; }
};

struct OpF32Min {
  using In = float;
  using Acc = float;
  using Out = float;
  static constexpr bool kFp = true;
  __device__ static Acc ident() { return __int_as_float(0x7f800000); }
  __device__ static void add_val(Acc& a, float x) { a = fminf(a, x); }
  __device__ static void add_prod(Acc& a, float x, float y) { a = fminf(a, __fmul_rn(x, y)); }
  __device__ static Acc combine(Acc a, Acc b) { return fminf(a, b); }
  __device__ static Acc shfl_xor(Acc a, int m, int w) { return __shfl_xor_sync(0xffffffffu, a, m, w); }
  __device__ static Out finish(Acc a) { return a; }
};

// int32: body values and sums modulo 2^32 (unsigned arithmetic, no UB)
struct OpI32Sum {
  using In = int32_t;
  using Acc = uint32_t;
  using Out = int32_t;
  static constexpr bool kFp = false;
  __device__ static Acc ident() { return 0u; }
  __device__ static void add_val(Acc& a, int32_t x) { a += static_cast<uint32_t>(x); }
  __device__ static void add_prod(Acc& a, int32_t x, int32_t y) {
    a += static_cast<uint32_t>(x) * static_cast<uint32_t>(y);
  }
  __device__ static Acc combine(Acc a, Acc b) { return a + b; }
  __device__ static Acc shfl_xor(Acc a, int m, int w) { return __shfl_xor_sync(0xffffffffu, a, m, w); }
  __device__ static Out finish(Acc a) { return static_cast<int32_t>(a); }
};

struct OpI32Max {
  using In = int32_t;
  using Acc = int32_t;
  using Out = int32_t;
  static constexpr bool kFp = false;
  __device__ static Acc ident() { return INT32_MIN; }
  __device__ static void add_val(Acc& a, int32_t x) { a = max(a, x); }
  __device__ static void add_prod(Acc& a, int32_t x, int32_t y) {
    a = max(a, static_cast<int32_t>(static_cast<uint32_t>(x) * static_cast<uint32_t>(y)));
  }
  __device__ static Acc combine(Acc a, Acc b) { return max(a, b); }
  __device__ static Acc shfl_xor(Acc a, int m, int w) { return __shfl_xor_sync(0xffffffffu, a, m, w); }
  __device__ static Out finish(Acc a) { return a; }
};

struct OpI32Min {
  using In = int32_t;
  using Acc = int32_t;
  using Out = int32_t;
  static constexpr bool kFp = false;
  __device__ static Acc ident() { return INT32_MAX; }
  __device__ static void add_val(Acc& a, int32_t x) { a = min(a, x); }
  __device__ static void add_prod(Acc& a, int32_t x, int32_t y) {
    a = min(a, static_cast<int32_t>(static_cast<uint32_t>(x) * static_cast<uint32_t>(y)));
  }
  __device__ static Acc combine(Acc a, Acc b) { return min(a, b); }
  __device__ static Acc shfl_xor(Acc a, int m, int w) { return __shfl_xor_sync(0xffffffffu, a, m, w); }
  __device__ static Out finish(Acc a) { return a; }
};

// int64 accumulation of int32 inputs (products exact in int64)
struct OpI64Sum {
  using In = int32_t;
  using Acc = unsigned long long;
  using Out = long long;
  static constexpr bool kFp = false;
  __device__ static Acc ident() { return 0ull; }
  __device__ static void add_val(Acc& a, long long x) { a += static_cast<Acc>(x); }
  __device__ static void add_prod(Acc& a, int32_t x, int32_t y) {
    a += static_cast<Acc>(static_cast<long long>(x) * static_cast<long long>(y));
  }
  __device__ static Acc combine(Acc a, Acc b) { return a + b; }
  __device__ static Acc shfl_xor(Acc a, int m, int w) { return __shfl_xor_sync(0xffffffffu, a, m, w); }
  __device__ static Out finish(Acc a) { return static_cast<long long>(a); }
};

struct OpI64Max {
  using In = int32_t;
  using Acc = long long;
  using Out = long long;
  static constexpr bool kFp = false;
  __device__ static Acc ident() { return INT64_MIN; }
  __device__ static void add_val(Acc& a, long long x) { a = max(a, x); }
  __device__ static void add_prod(Acc& a, int32_t x, int32_t y) {
    a = max(a, static_cast<long long>(x) * static_cast<long long>(y));
  }
  __device__ static Acc combine(Acc a, Acc b) { return max(a, b); }
  __device__ static Acc shfl_xor(Acc a, int m, int w) { return __shfl_xor_sync(0xffffffffu, a, m, w); }
  __device__ static Out finish(Acc a) { return a; }
};

struct OpI64Min {
  using In = int32_t;
  using Acc = long long;
  using Out = long long;
  static constexpr bool kFp = false;
  __device__ static Acc ident() { return INT64_MAX; }
  __device__ static void add_val(Acc& a, long long x) { a = min(a, x); }
  __device__ static void add_prod(Acc& a, int32_t x, int32_t y) {
    a = min(a, static_cast<long long>(x) * static_cast<long long>(y));
  }
  __device__ static Acc combine(Acc a, Acc b) { return min(a, b); }
  __device__ static Acc shfl_xor(Acc a, int m, int w) { return __shfl_xor_sync(0xffffffffu, a, m, w); }
  __device__ static Out finish(Acc a) { return a; }
};

// ---------------------------------------------------------------------------
// Packed FP32x2 arithmetic (PTX add/sub/mul/fma .rn.f32x2, sm_100 and later):
// each half is an IEEE round-to-nearest FP32 operation, so a pair of
// independent accumulators advanced by one packed instruction gives exactly
// the results of two scalar instructions.
#define HP_F32X2_OP2(name, op)                                                                   \
  __device__ __forceinline__ float2 name(float2 a, float2 b) {                                    \
    float2 r;                                                                                    \
    asm("{\n .reg .b64 ra, rb, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n " op     \
        " rd, ra, rb;\n mov.b64 {%0, %1}, rd;\n}"                                              \
        : "=f"(r.x), "=f"(r.y)                                                                   \
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));                                               \
    return r;                                                                                    \
  }
HP_F32X2_OP2(add2, "add.rn.f32x2")
HP_F32X2_OP2(sub2, "sub.rn.f32x2")
HP_F32X2_OP2(mul2, "mul.rn.f32x2")
#undef HP_F32X2_OP2

__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
  float2 r;
  asm("{\n .reg .b64 ra, rb, rc, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n"
      " mov.b64 rc, {%6, %7};\n fma.rn.f32x2 rd, ra, rb, rc;\n mov.b64 {%0, %1}, rd;\n}"
      : "=f"(r.x), "=f"(r.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return r;
}

// TwoSum on two lanes at once
__device__ __forceinline__ void two_sum2(float2 a, float2 b, float2& s, float2& e) {
  s = add2(a, b);
  const float2 bb = sub2(s, a);
  e = add2(sub2(a, sub2(s, bb)), sub2(b, bb));
}

// compensated fold of one value / one product into two slots at once
__device__ __forceinline__ void comp_add_pair(float2& s, float2& c, float2 v) {
  float2 t, e;
  two_sum2(s, v, t, e);
  s = t;
  c = add2(c, e);
}
// the exact product errors come from two scalar FMAs (free operand negation)
__device__ __forceinline__ void comp_prod_pair(float2& s, float2& c, float2 x, float2 w) {
  const float2 p = mul2(x, w);
  const float2 ep = make_float2(__fmaf_rn(x.x, w.x, -p.x), __fmaf_rn(x.y, w.y, -p.y));
  float2 t, e;
  two_sum2(s, p, t, e);
  s = t;
  c = add2(c, add2(ep, e));
}

// Fold state of the 4 vector slots of one thread.  The generic version uses
// the policy's scalar operations; FP32 sums use packed pairs (slots 0,1 and
// 2,3) with the same per-slot operation sequence, hence identical results.
template <class Op>
struct Fold4 {
  typename Op::Acc a[4];
  __device__ __forceinline__ void init() {
#pragma unroll
    for (int i = 0; i < 4; ++i) a[i] = Op::ident();
  }
  template <class V4>
  __device__ __forceinline__ void load(const V4& x) {
    Op::add_val(a[0], x.x);
    Op::add_val(a[1], x.y);
    Op::add_val(a[2], x.z);
    Op::add_val(a[3], x.w);
  }
  template <class V4>
  __device__ __forceinline__ void dot(const V4& x, const V4& w, const V4&) {
    Op::add_prod(a[0], x.x, w.x);
    Op::add_prod(a[1], x.y, w.y);
    Op::add_prod(a[2], x.z, w.z);
    Op::add_prod(a[3], x.w, w.w);
  }
  __device__ __forceinline__ void get(typename Op::Acc (&out)[4]) const {
#pragma unroll
    for (int i = 0; i < 4; ++i) out[i] = a[i];
  }
};

template <>
struct Fold4<OpF32Comp> {
  float2 s01, s23, c01, c23;   // leading and trailing words of slots (0,1) and (2,3)
  __device__ __forceinline__ void init() { s01 = s23 = c01 = c23 = make_float2(0.0f, 0.0f); }
  __device__ __forceinline__ void load(const float4& x) {
    comp_add_pair(s01, c01, make_float2(x.x, x.y));
    comp_add_pair(s23, c23, make_float2(x.z, x.w));
  }
  __device__ __forceinline__ void dot(const float4& x, const float4& w, const float4&) {
    comp_prod_pair(s01, c01, make_float2(x.x, x.y), make_float2(w.x, w.y));
    comp_prod_pair(s23, c23, make_float2(x.z, x.w), make_float2(w.z, w.w));
  }
  __device__ __forceinline__ void get(f2 (&out)[4]) const {
    out[0] = {s01.x, c01.x};
    out[1] = {s01.y, c01.y};
    out[2] = {s23.x, c23.x};
    out[3] = {s23.y, c23.y};
  }
};

template <>
struct Fold4<OpF32Sum> {
  float2 s01, s23;
  __device__ __forceinline__ void init() { s01 = s23 = make_float2(0.0f, 0.0f); }
  __device__ __forceinline__ void load(const float4& x) {
    s01 = add2(s01, make_float2(x.x, x.y));
    s23 = add2(s23, make_float2(x.z, x.w));
  }
  __device__ __forceinline__ void dot(const float4& x, const float4& w, const float4&) {
    s01 = fma2(make_float2(x.x, x.y), make_float2(w.x, w.y), s01);
    s23 = fma2(make_float2(x.z, x.w), make_float2(w.z, w.w), s23);
  }
  __device__ __forceinline__ void get(float (&out)[4]) const {
    out[0] = s01.x;
    out[1] = s01.y;
    out[2] = s23.x;
    out[3] = s23.y;
  }
};

// Fold V loaded values (and products with V broadcast values) into the V slot
// accumulators acc[0..V-1]: slot i takes value i.  FP32 sums of 4 slots use the
// packed pairs (0,1), (2,3); the per-slot operation sequence is unchanged.
template <class Op, int V, class In>
__device__ __forceinline__ void fold_vals_load(typename Op::Acc (&acc)[V], const In (&a)[V]) {
  if constexpr (V == 4 && std::is_same<Op, OpF32Comp>::value) {
    float2 s01 = make_float2(acc[0].s, acc[1].s), c01 = make_float2(acc[0].c, acc[1].c);
    float2 s23 = make_float2(acc[2].s, acc[3].s), c23 = make_float2(acc[2].c, acc[3].c);
    comp_add_pair(s01, c01, make_float2(a[0], a[1]));
    comp_add_pair(s23, c23, make_float2(a[2], a[3]));
    acc[0] = {s01.x, c01.x};
    acc[1] = {s01.y, c01.y};
    acc[2] = {s23.x, c23.x};
    acc[3] = {s23.y, c23.y};
  } else if constexpr (V == 4 && std::is_same<Op, OpF32Sum>::value) {
    const float2 s01 = add2(make_float2(acc[0], acc[1]), make_float2(a[0], a[1]));
    const float2 s23 = add2(make_float2(acc[2], acc[3]), make_float2(a[2], a[3]));
    acc[0] = s01.x;
    acc[1] = s01.y;
    acc[2] = s23.x;
    acc[3] = s23.y;
  } else {
#pragma unroll
    for (int i = 0; i < V; ++i) Op::add_val(acc[i], a[i]);
  }
}

template <class Op, int V, class In>
__device__ __forceinline__ void fold_vals_dot(typename Op::Acc (&acc)[V], const In (&a)[V], const In (&b)[V]) {
  if constexpr (V == 4 && std::is_same<Op, OpF32Comp>::value) {
    float2 s01 = make_float2(acc[0].s, acc[1].s), c01 = make_float2(acc[0].c, acc[1].c);
    float2 s23 = make_float2(acc[2].s, acc[3].s), c23 = make_float2(acc[2].c, acc[3].c);
    comp_prod_pair(s01, c01, make_float2(a[0], a[1]), make_float2(b[0], b[1]));
    comp_prod_pair(s23, c23, make_float2(a[2], a[3]), make_float2(b[2], b[3]));
    acc[0] = {s01.x, c01.x};
    acc[1] = {s01.y, c01.y};
    acc[2] = {s23.x, c23.x};
    acc[3] = {s23.y, c23.y};
  } else if constexpr (V == 4 && std::is_same<Op, OpF32Sum>::value) {
    const float2 s01 = fma2(make_float2(a[0], a[1]), make_float2(b[0], b[1]), make_float2(acc[0], acc[1]));
    const float2 s23 = fma2(make_float2(a[2], a[3]), make_float2(b[2], b[3]), make_float2(acc[2], acc[3]));
    acc[0] = s01.x;
    acc[1] = s01.y;
    acc[2] = s23.x;
    acc[3] = s23.y;
  } else {
#pragma unroll
    for (int i = 0; i < V; ++i) Op::add_prod(acc[i], a[i], b[i]);
  }
}

// ---------------------------------------------------------------- grid parts
// L2 loads of partials (other SMs of the same launch may have written them)
__device__ __forceinline__ f2 ld_part(const f2* p) {
  const float2 v = __ldcg(reinterpret_cast<const float2*>(p));
  return f2{v.x, v.y};
}
__device__ __forceinline__ float ld_part(const float* p) { return __ldcg(p); }
__device__ __forceinline__ uint32_t ld_part(const uint32_t* p) { return __ldcg(p); }
__device__ __forceinline__ int32_t ld_part(const int32_t* p) { return __ldcg(p); }
__device__ __forceinline__ unsigned long long ld_part(const unsigned long long* p) { return __ldcg(p); }
__device__ __forceinline__ long long ld_part(const long long* p) { return __ldcg(p); }

// The final combine of one output's G partials (the second pass of Sec. 2's
// recursive reduction when a reduced level is split over the grid), shared by
// every executor so that their results agree bit for bit.  Parts are folded
// in part order.  Compensated partials (s_g, c_g) are added as double-float
// numbers: TwoSum carries s_g into the running sum exactly, and its error and
// c_g go to a second FP32 word (the cascaded summation of Ogita, Rump and
// Oishi, "Accurate sum and dot product", 2005); the result is the rounded sum
// of the two words and rem (may be null) its exact rounding error.  Its error
// is at most gamma_2G (gamma_G + 2 gamma_k) sum|t| beyond the parts' own (k
// the parts' chain length), far below the FP32 result's rounding.  FP64 is
// not used: a dependent FP64 operation costs about 63 SM cycles on this GPU
// (FP32: 4.5), and a chain of 2G of them took about 40 us for G = 304.
// one fold step of that combine; every executor folds the same steps in the
// same order
template <class Op, bool COMP = std::is_same_v<typename Op::Acc, f2>>
struct PartFold;
template <class Op>
struct PartFold<Op, true> {
  float S = 0.0f, C = 0.0f;
  __device__ __forceinline__ void first(const f2& v) { add(v); }
  __device__ __forceinline__ void add(const f2& v) {
    float s2, e;
    two_sum(S, v.s, s2, e);
    S = s2;
    C = __fadd_rn(C, e);
    C = __fadd_rn(C, v.c);
  }
  __device__ __forceinline__ float result(float* rem) const {
    float r, e;
    two_sum(S, C, r, e);
    if (rem) *rem = e;
    return r;
  }
};
template <class Op>
struct PartFold<Op, false> {
  typename Op::Acc a;
  __device__ __forceinline__ void first(const typename Op::Acc& v) { a = v; }
  __device__ __forceinline__ void add(const typename Op::Acc& v) { a = Op::combine(a, v); }
  __device__ __forceinline__ typename Op::Out result(float*) const { return Op::finish(a); }
};

// the combine by one thread, loading 8 parts at a time from L2
template <class Op>
__device__ __forceinline__ typename Op::Out combine_parts(const typename Op::Acc* pp, int32_t G, float* rem) {
  using Acc = typename Op::Acc;
  constexpr int K = 8;
  PartFold<Op> f;
  f.first(ld_part(pp));
  int32_t g = 1;
  for (; g + K <= G; g += K) {
    Acc v[K];
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = ld_part(pp + g + k);
#pragma unroll
    for (int k = 0; k < K; ++k) f.add(v[k]);
  }
  for (; g < G; ++g) f.add(ld_part(pp + g));
  return f.result(rem);
}

}  // namespace hp
