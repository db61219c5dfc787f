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

}  // namespace hp
