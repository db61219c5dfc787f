// csr.cu — ragged (CSR) nests: out[i] = OP_{e in [off[i], off[i+1])} val[e] * x[col[e]]
// and the count histogram hist[b] = #{e : col[e] >> shift == b}.
//
// The inner level is ragged, so its binding to hardware is chosen per row
// (Sec. 3.3: a region compiled for several candidate levels, one picked at run
// time; Sec. 3.8: sub-warp partitions for short rows).  Each run bins the rows
// by length into classes and runs one kernel per class:
//   class 0  len <= 4      one thread per row            (SEQ)
//   class 1  len <= 64     a group of 8 lanes per row     (SUBWARP(8))
//   class 2  len <= 2048   a warp per row                 (WARP)
//   class 3  len <= 16384  a CTA of 256 threads per row   (CTA)
//   class 4  longer        chunks of 16384 entries, a CTA per chunk writing
//                          its partial to the chunk's slot; a second kernel
//                          folds each row's partials in chunk order (GRID,
//                          two-pass; double-float for compensated sums).
// Within a class, lane t of a row's team folds entries start + t + k*L (L the
// team's lanes) into 4 accumulators (k mod 4), then the team combines them in
// a fixed tree; the tree depends on the row's length only, never on which
// team ran it or where the row sits in the class list, so results are
// reproducible although the class lists are filled with atomics.
// The histogram is counted in shared memory per CTA and flushed with 64-bit
// integer atomics (exact in any order), fused into the same sweep or alone.
// An explicit map for the entry level (SEQ, SUBWARP(w), WARP, CTA) puts every
// row into that one class instead.
// The x gathers are random 4-byte reads that L1 almost never serves again, so
// they are cached in L2 only (__ldcg): no L1 line fills for single use.
#include <cuda_runtime.h>

#include <algorithm>
#include <new>
#include <sstream>
#include <string>

#include "accum.cuh"
#include "api_internal.h"

namespace hp {

constexpr int kCsrClasses = 5;
#ifndef HP_CSR_LIMIT1
#define HP_CSR_LIMIT1 64                                  // longest row of an 8-lane team (32: 6.44 ms, 64: 6.40, 128: 6.42 on the Zipf workload)
#endif
#ifndef HP_CSR_LIMIT2
#define HP_CSR_LIMIT2 2048                                // longest row of a warp team (1024: 6.42 ms, 2048: 6.37, 4096: 6.37)
#endif
#ifndef HP_CSR_LIMIT3
#define HP_CSR_LIMIT3 16384                               // longest row of a CTA team
#endif
#ifndef HP_CSR_CHUNK
#define HP_CSR_CHUNK 16384                                // entries per chunk of a longer row
#endif
constexpr int64_t kCsrLimit0 = 4, kCsrLimit1 = HP_CSR_LIMIT1, kCsrLimit2 = HP_CSR_LIMIT2, kCsrLimit3 = HP_CSR_LIMIT3;  // class bounds (inclusive)
constexpr int64_t kCsrChunk = HP_CSR_CHUNK;
static_assert(kCsrLimit3 >= kCsrChunk, "split rows must be longer than one chunk (bounds the chunk slots)");
constexpr int kCsrCtaThreads = 256;                       // the chunk kernel's CTA
#ifndef HP_CSR_ROW_CTA_THREADS
#define HP_CSR_ROW_CTA_THREADS 256                         // the CTA-per-row kernel's CTA
#endif
constexpr int kCsrRowCtaThreads = HP_CSR_ROW_CTA_THREADS;
constexpr int kCsrBinThreads = 256;
constexpr int kCsrHistSmemMax = 12288;                   // bins counted in shared memory
#ifndef HP_CSR_GROUPS
#define HP_CSR_GROUPS 2                                   // 128-bit groups of col / val loaded before their folds
#endif
#ifndef HP_CSR_MIN_BLOCKS
#define HP_CSR_MIN_BLOCKS 5                               // resident CTAs per SM the wide-team kernels' registers allow (48 registers)
#endif

struct CsrState {
  int64_t* counters = nullptr;   // [0..4] rows per class, [5] chunk slots, [6..10] scatter cursors
  int32_t* rows = nullptr;       // row ids grouped by class
  int32_t* chunk_row = nullptr;  // per chunk slot: row id
  int32_t* chunk_idx = nullptr;  // per chunk slot: chunk index within its row
  int32_t* chunk_cnt = nullptr;  // per chunk slot: chunks of its row
  void* part = nullptr;          // per chunk slot: partial accumulator
  int64_t max_chunks = 0;
  int grid_rows = 0;             // persistent grid sizes
  int grid_cta = 0;
  int grid_row_cta = 0;
};

// ---------------------------------------------------------------- planning
hp_status plan_csr(int depth, int64_t n_rows, const hp_level_map* map, hp_red_op op, int red_level, hp_prec prec,
                   hp_body body, const void* body_params, CsrPlan* out, std::string* why) {
  auto bad = [&](const std::string& s) {
    *why = s;
    return HP_EINVAL;
  };
  if (depth != 2) return bad("CSR nests have depth 2 (rows, entries)");
  if (n_rows < 0 || n_rows >= (int64_t(1) << 31)) return bad("CSR n_rows must be in [0, 2^31)");
  if (!body_params) return bad("CSR nests need hp_csr_params");
  const hp_csr_params* cp = static_cast<const hp_csr_params*>(body_params);
  if (cp->nnz < 0) return bad("CSR nnz must be >= 0");
  if (cp->n_cols < 0 || cp->n_cols >= (int64_t(1) << 31)) return bad("CSR n_cols must be in [0, 2^31)");
  if (op == HP_RED_HIST_COUNT || cp->fuse_hist) {
    if (cp->n_bins < 1 || cp->n_bins >= (int64_t(1) << 31)) return bad("histogram n_bins must be in [1, 2^31)");
    if (cp->hist_shift < 0 || cp->hist_shift > 30) return bad("histogram shift must be in [0, 30]");
  }
  if (op == HP_RED_HIST_COUNT) {
    if (red_level != 0) return bad("a count histogram reduces over all levels (red_level 0)");
    if (cp->fuse_hist) return bad("fuse_hist applies to SUM / MAX / MIN nests");
  } else {
    if (op != HP_RED_SUM && op != HP_RED_MAX && op != HP_RED_MIN) return bad("unknown reduction op");
    if (red_level != 1) return bad("CSR nests reduce the entries of each row (red_level 1)");
    if (body != HP_BODY_CSR_GATHER) return bad("CSR nests take the CSR_GATHER body");
    if (prec != HP_F32 && prec != HP_F32_COMP) return bad("CSR nests compute in FP32 (plain or compensated)");
  }
  CsrPlan p;
  p.n_rows = n_rows;
  p.nnz = cp->nnz;
  p.n_cols = cp->n_cols;
  p.hist_shift = cp->hist_shift;
  p.fuse_hist = cp->fuse_hist;
  p.n_bins = cp->n_bins;
  p.op = op;
  p.prec = prec;
  p.fixed_class = -1;
  if (map) {
    if (map[0].hw != HP_HW_GRID && map[0].hw != HP_HW_AUTO) return bad("CSR rows are bound to the grid");
    const int hw = map[1].hw;
    if (hw == HP_HW_AUTO) p.fixed_class = -1;
    else if (hw == HP_HW_SEQ || hw == HP_HW_LANE) p.fixed_class = 0;
    else if (hw == HP_HW_SUBWARP) {
      if (map[1].sub_width != 8 && map[1].sub_width != 0) return bad("CSR sub-warp rows use groups of 8 lanes");
      p.fixed_class = 1;
    } else if (hw == HP_HW_WARP) p.fixed_class = 2;
    else if (hw == HP_HW_CTA) p.fixed_class = 3;
    else if (hw == HP_HW_GRID) p.fixed_class = 4;
    else return bad("CSR entries bind to SEQ, SUBWARP(8), WARP, CTA, GRID or AUTO");
  }
  *out = p;
  return HP_OK;
}

std::string describe_csr(const CsrPlan& p) {
  std::ostringstream s;
  s << "{\"kind\":\"csr\",\"rows\":" << p.n_rows << ",\"nnz\":" << p.nnz << ",\"cols\":" << p.n_cols
    << ",\"op\":" << static_cast<int>(p.op) << ",\"fuse_hist\":" << p.fuse_hist << ",\"bins\":" << p.n_bins
    << ",\"shift\":" << p.hist_shift << ",\"fixed_class\":" << p.fixed_class
    << ",\"class_limits\":[" << kCsrLimit0 << "," << kCsrLimit1 << "," << kCsrLimit2 << "," << kCsrLimit3
    << "],\"chunk\":" << kCsrChunk << "}";
  return s.str();
}

// ---------------------------------------------------------------- device code
namespace {

__device__ __forceinline__ int row_class(int64_t len, int fixed) {
  if (fixed >= 0) return fixed;
  if (len <= kCsrLimit0) return 0;
  if (len <= kCsrLimit1) return 1;
  if (len <= kCsrLimit2) return 2;
  if (len <= kCsrLimit3) return 3;
  return 4;
}

__device__ __forceinline__ int64_t n_chunks_of(int64_t len) { return len > 0 ? (len + kCsrChunk - 1) / kCsrChunk : 1; }

__global__ void csr_zero_kernel(int64_t* counters, int n, long long* hist, int64_t n_bins) {
  const int64_t i0 = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  if (i0 < n) counters[i0] = 0;
  if (hist)
    for (int64_t i = i0; i < n_bins; i += stride) hist[i] = 0;
}

// pass 1: rows per class and chunk slots of long rows (warp ballots, one
// shared-memory add per warp and class, one global add per block and class)
__global__ void csr_bin_count_kernel(const int64_t* __restrict__ off, int64_t n_rows, int fixed, int64_t* counters) {
  __shared__ unsigned long long cnt[kCsrClasses + 1];
  if (threadIdx.x <= kCsrClasses) cnt[threadIdx.x] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t tile = blockIdx.x * static_cast<int64_t>(blockDim.x); tile < n_rows; tile += stride) {
    const int64_t i = tile + threadIdx.x;
    int c = -1;
    int64_t len = 0;
    if (i < n_rows) {
      len = off[i + 1] - off[i];
      c = row_class(len, fixed);
    }
#pragma unroll
    for (int k = 0; k < kCsrClasses; ++k) {
      const unsigned m = __ballot_sync(0xffffffffu, c == k);
      if (lane == 0 && m) atomicAdd(&cnt[k], static_cast<unsigned long long>(__popc(m)));
    }
    if (c == 4) atomicAdd(&cnt[kCsrClasses], static_cast<unsigned long long>(n_chunks_of(len)));
  }
  __syncthreads();
  if (threadIdx.x <= kCsrClasses && cnt[threadIdx.x])
    atomicAdd(reinterpret_cast<unsigned long long*>(&counters[threadIdx.x]), cnt[threadIdx.x]);
}

// pass 2: scatter row ids into their class's range (tile by tile: warp ballots
// give each row its rank, one global add per block and class reserves the
// tile's range); reserve chunk slots of long rows
__global__ void __launch_bounds__(kCsrBinThreads) csr_bin_scatter_kernel(
    const int64_t* __restrict__ off, int64_t n_rows, int fixed, int64_t* counters, int32_t* rows, int32_t* chunk_row,
    int32_t* chunk_idx, int32_t* chunk_cnt, int64_t max_chunks, int32_t* err) {
  constexpr int kWarps = kCsrBinThreads / 32;
  __shared__ int wpos[kWarps][kCsrClasses];
  __shared__ long long bbase[kCsrClasses];
  // class c occupies rows[start_c .. start_c + count_c); cursors live in counters[6 + c]
  int64_t start[kCsrClasses];
  int64_t acc = 0;
#pragma unroll
  for (int c = 0; c < kCsrClasses; ++c) {
    start[c] = acc;
    acc += counters[c];
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt_mask = (1u << lane) - 1u;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t tile = blockIdx.x * static_cast<int64_t>(blockDim.x); tile < n_rows; tile += stride) {
    const int64_t i = tile + threadIdx.x;
    int c = -1;
    int64_t len = 0;
    if (i < n_rows) {
      len = off[i + 1] - off[i];
      c = row_class(len, fixed);
    }
    int rank = 0;
#pragma unroll
    for (int k = 0; k < kCsrClasses; ++k) {
      const unsigned m = __ballot_sync(0xffffffffu, c == k);
      if (lane == 0) wpos[warp][k] = __popc(m);
      if (c == k) rank = __popc(m & lt_mask);
    }
    __syncthreads();
    if (threadIdx.x < kCsrClasses) {
      int tot = 0;
      for (int w = 0; w < kWarps; ++w) {
        const int v = wpos[w][threadIdx.x];
        wpos[w][threadIdx.x] = tot;
        tot += v;
      }
      bbase[threadIdx.x] =
          tot ? static_cast<long long>(atomicAdd(reinterpret_cast<unsigned long long*>(&counters[6 + threadIdx.x]),
                                                 static_cast<unsigned long long>(tot)))
              : 0;
    }
    __syncthreads();
    if (c >= 0) rows[start[c] + bbase[c] + wpos[warp][c] + rank] = static_cast<int32_t>(i);
    if (c == 4) {
      const int64_t nc = n_chunks_of(len);
      const unsigned long long base =
          atomicAdd(reinterpret_cast<unsigned long long*>(&counters[11]), static_cast<unsigned long long>(nc));
      if (static_cast<int64_t>(base) + nc > max_chunks) {  // offsets disagree with the declared nnz
        atomicExch(err, 2);
      } else {
        for (int64_t k = 0; k < nc; ++k) {
          chunk_row[base + k] = static_cast<int32_t>(i);
          chunk_idx[base + k] = static_cast<int32_t>(k);
          chunk_cnt[base + k] = static_cast<int32_t>(nc);
        }
      }
    }
    __syncthreads();  // wpos / bbase are reused by the next tile
  }
}

struct CsrArgs {
  const int64_t* off;
  const int32_t* col;
  const float* val;
  const float* x;
  float* y;
  long long* hist;      // fused histogram (global), or nullptr
  int32_t* err;         // device error word: 2 = offsets or columns outside the declared sizes
  int64_t nnz;
  int64_t n_cols;
  int shift;
  int64_t n_bins;
  int smem_bins;        // bins counted in shared memory (0: count straight into global memory)
};

__device__ __forceinline__ void hist_add(const CsrArgs& a, int* sh, int32_t c) {
  const int64_t b = static_cast<int64_t>(c) >> a.shift;
  if (b < a.n_bins) {
    if (a.smem_bins) atomicAdd(&sh[b], 1);
    else atomicAdd(reinterpret_cast<unsigned long long*>(&a.hist[b]), 1ull);
  }
}

// fold entries s + t, s + t + L, ... < e into 4 accumulators (entry k goes to acc[(k / L) % 4])
template <class Op, bool HIST>
__device__ __forceinline__ void csr_fold(const CsrArgs& a, int* sh, int64_t s, int64_t e, int t, int L,
                                         typename Op::Acc (&acc)[4]) {
  if (s < 0 || e > a.nnz || s > e) {  // offsets outside [0, nnz]: flag, fold nothing
    if (t == 0) atomicExch(a.err, 2);
    return;
  }
  for (int64_t b = s + t; b < e; b += 4 * static_cast<int64_t>(L)) {
    int32_t c[4];
    float v[4];
    bool ok[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t idx = b + static_cast<int64_t>(u) * L;
      ok[u] = idx < e;
      c[u] = ok[u] ? __ldcs(a.col + idx) : 0;
      v[u] = ok[u] ? __ldcs(a.val + idx) : 0.0f;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (ok[u]) {
        if (static_cast<uint32_t>(c[u]) < static_cast<uint64_t>(a.n_cols)) {
          Op::add_prod(acc[u], v[u], __ldcg(a.x + c[u]));
          if constexpr (HIST) hist_add(a, sh, c[u]);
        } else {
          atomicExch(a.err, 2);
        }
      }
    }
  }
}

template <class Op, bool HIST>
__device__ __forceinline__ void csr_fold_one(const CsrArgs& a, int* sh, int64_t idx, typename Op::Acc& acc) {
  const int32_t c = __ldcs(a.col + idx);
  const float v = __ldcs(a.val + idx);
  if (static_cast<uint32_t>(c) < static_cast<uint64_t>(a.n_cols)) {
    Op::add_prod(acc, v, __ldcg(a.x + c));
    if constexpr (HIST) hist_add(a, sh, c);
  } else {
    atomicExch(a.err, 2);
  }
}

template <class Op, bool HIST>
__device__ __forceinline__ void csr_fold_group(const CsrArgs& a, int* sh, const int4& c, const float4& v,
                                               typename Op::Acc (&acc)[4]) {
  const int32_t cc[4] = {c.x, c.y, c.z, c.w};
  const float vv[4] = {v.x, v.y, v.z, v.w};
  float xv[4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
    xv[u] = (static_cast<uint32_t>(cc[u]) < static_cast<uint64_t>(a.n_cols)) ? __ldcg(a.x + cc[u]) : 0.0f;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    if (static_cast<uint32_t>(cc[u]) < static_cast<uint64_t>(a.n_cols)) {
      Op::add_prod(acc[u], vv[u], xv[u]);
      if constexpr (HIST) hist_add(a, sh, cc[u]);
    } else {
      atomicExch(a.err, 2);
    }
  }
}

// Entries [s, e) for wide teams: the 16-byte-aligned middle is read as 128-bit
// groups of col and val (lane t takes groups g0 + t, g0 + t + L, ...,
// HP_CSR_GROUPS at a time so that 4 x HP_CSR_GROUPS gathers of x are in
// flight; the fold order does not depend on it), the unaligned head and tail
// (< 4 entries each) by lanes 0..3 into their first and second accumulators.
// The tree depends only on (s, e), so a row's result is reproducible.
template <class Op, bool HIST>
__device__ __forceinline__ void csr_fold_vec(const CsrArgs& a, int* sh, int64_t s, int64_t e, int t, int L,
                                             typename Op::Acc (&acc)[4]) {
  if (s < 0 || e > a.nnz || s > e) {
    if (t == 0) atomicExch(a.err, 2);
    return;
  }
  const int64_t g0 = (s + 3) >> 2, g1 = e >> 2;
  if (g0 >= g1) {
    csr_fold<Op, HIST>(a, sh, s, e, t, L, acc);
    return;
  }
  if (t < 4 * g0 - s) csr_fold_one<Op, HIST>(a, sh, s + t, acc[0]);
  if (t < e - 4 * g1) csr_fold_one<Op, HIST>(a, sh, 4 * g1 + t, acc[1]);
  const int4* col4 = reinterpret_cast<const int4*>(a.col);
  const float4* val4 = reinterpret_cast<const float4*>(a.val);
  constexpr int K = HP_CSR_GROUPS;
  for (int64_t g = g0 + t; g < g1; g += K * static_cast<int64_t>(L)) {
    int4 c[K];
    float4 v[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      c[k] = make_int4(0, 0, 0, 0);
      v[k] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (g + k * static_cast<int64_t>(L) < g1) {
        c[k] = __ldcs(col4 + g + k * static_cast<int64_t>(L));
        v[k] = __ldcs(val4 + g + k * static_cast<int64_t>(L));
      }
    }
#pragma unroll
    for (int k = 0; k < K; ++k)
      if (g + k * static_cast<int64_t>(L) < g1) csr_fold_group<Op, HIST>(a, sh, c[k], v[k], acc);
  }
}

template <class Op>
__device__ __forceinline__ typename Op::Acc fold4(const typename Op::Acc (&acc)[4]) {
  return Op::combine(Op::combine(acc[0], acc[1]), Op::combine(acc[2], acc[3]));
}

template <class Op>
__device__ __forceinline__ typename Op::Acc team_reduce(typename Op::Acc a, int width) {
  for (int m = width >> 1; m >= 1; m >>= 1) a = Op::combine(a, Op::shfl_xor(a, m, width));
  return a;
}

__device__ __forceinline__ void hist_init(int* sh, int bins) {
  for (int i = threadIdx.x; i < bins; i += blockDim.x) sh[i] = 0;
  __syncthreads();
}

__device__ __forceinline__ void hist_flush(const CsrArgs& a, int* sh) {
  __syncthreads();
  for (int i = threadIdx.x; i < a.smem_bins; i += blockDim.x)
    if (sh[i]) atomicAdd(reinterpret_cast<unsigned long long*>(&a.hist[i]), static_cast<unsigned long long>(sh[i]));
}

// classes 0..2: a team of L lanes (1, 8 or 32) per row; persistent over the class list
template <class Op, int L, bool HIST>
__global__ void __launch_bounds__(256, HP_CSR_MIN_BLOCKS) csr_rows_kernel(CsrArgs a, const int32_t* __restrict__ rows, const int64_t* counters,
                                                       int cls) {
  extern __shared__ int sh_hist[];
  if constexpr (HIST) {
    if (a.smem_bins) hist_init(sh_hist, a.smem_bins);
  }
  int64_t start = 0;
  for (int c = 0; c < cls; ++c) start += counters[c];
  const int64_t count = counters[cls];
  const int lane = threadIdx.x & 31;
  const int lt = lane % L;
  const int64_t team = (blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x) / L;
  const int64_t n_teams = static_cast<int64_t>(gridDim.x) * blockDim.x / L;
  const int64_t warp_first_team = (blockIdx.x * static_cast<int64_t>(blockDim.x) + (threadIdx.x & ~31)) / L;
  // every lane of a warp runs the same number of rounds (shuffles need the whole warp);
  // the row id two rounds ahead and the offsets one round ahead are loaded
  // before the current round's fold, so that their dependent loads overlap it
  const int64_t dk = team - warp_first_team;
  int64_t r0 = warp_first_team;
  int32_t row = r0 + dk < count ? rows[start + r0 + dk] : 0;
  int32_t row1 = r0 + n_teams + dk < count ? rows[start + r0 + n_teams + dk] : 0;
  int64_t s0 = r0 + dk < count ? a.off[row] : 0, e0 = r0 + dk < count ? a.off[row + 1] : 0;
  for (; r0 < count; r0 += n_teams) {
    const int64_t k = r0 + dk;
    const bool valid = k < count;
    const int32_t row2 = k + 2 * n_teams < count ? rows[start + k + 2 * n_teams] : 0;
    const int64_t s1 = k + n_teams < count ? a.off[row1] : 0;
    const int64_t e1 = k + n_teams < count ? a.off[row1 + 1] : 0;
    typename Op::Acc acc[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) acc[u] = Op::ident();
    if (valid) {
      if constexpr (L == 32) csr_fold_vec<Op, HIST>(a, sh_hist, s0, e0, lt, L, acc);
      else csr_fold<Op, HIST>(a, sh_hist, s0, e0, lt, L, acc);
    }
    typename Op::Acc r = fold4<Op>(acc);
    if constexpr (L > 1) r = team_reduce<Op>(r, L);
    if (valid && lt == 0) a.y[row] = Op::finish(r);
    row = row1;
    row1 = row2;
    s0 = s1;
    e0 = e1;
  }
  if constexpr (HIST) {
    if (a.smem_bins) hist_flush(a, sh_hist);
  }
}

// CTA-wide fold of one entry range; the result is valid in thread 0.  One
// barrier: callers alternate between the two halves of their warp-partial
// buffer, so that the next range's partials never overwrite the ones thread 0
// may still be reading.
template <class Op, bool HIST>
__device__ __forceinline__ typename Op::Acc cta_fold(const CsrArgs& a, int* sh, int64_t s, int64_t e,
                                                     typename Op::Acc* wsh) {
  typename Op::Acc acc[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) acc[u] = Op::ident();
  csr_fold_vec<Op, HIST>(a, sh, s, e, threadIdx.x, blockDim.x, acc);
  typename Op::Acc r = team_reduce<Op>(fold4<Op>(acc), 32);
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if ((threadIdx.x & 31) == 0) wsh[warp] = r;
  __syncthreads();
  if (threadIdx.x == 0) {
    r = wsh[0];
    for (int w = 1; w < nw; ++w) r = Op::combine(r, wsh[w]);
  }
  return r;
}

// class 3: a CTA per row
template <class Op, bool HIST>
__global__ void __launch_bounds__(kCsrRowCtaThreads, HP_CSR_MIN_BLOCKS * kCsrCtaThreads / kCsrRowCtaThreads)
    csr_cta_kernel(CsrArgs a, const int32_t* __restrict__ rows,
                                                                 const int64_t* counters) {
  extern __shared__ int sh_hist[];
  __shared__ typename Op::Acc wsh[2][kCsrRowCtaThreads / 32];
  if constexpr (HIST) {
    if (a.smem_bins) hist_init(sh_hist, a.smem_bins);
  }
  int64_t start = 0;
  for (int c = 0; c < 3; ++c) start += counters[c];
  const int64_t count = counters[3];
  int buf = 0;
  for (int64_t k = blockIdx.x; k < count; k += gridDim.x, buf ^= 1) {
    const int32_t row = rows[start + k];
    const typename Op::Acc r = cta_fold<Op, HIST>(a, sh_hist, a.off[row], a.off[row + 1], wsh[buf]);
    if (threadIdx.x == 0) a.y[row] = Op::finish(r);
  }
  if constexpr (HIST) {
    if (a.smem_bins) hist_flush(a, sh_hist);
  }
}

// class 4: a CTA per chunk of a long row; each chunk's partial goes to its
// slot, and csr_split_combine_kernel folds a row's slots after this kernel
template <class Op, bool HIST>
__global__ void __launch_bounds__(kCsrCtaThreads, HP_CSR_MIN_BLOCKS) csr_split_kernel(CsrArgs a, const int64_t* counters,
                                                                   const int32_t* __restrict__ chunk_row,
                                                                   const int32_t* __restrict__ chunk_idx,
                                                                   typename Op::Acc* part, int64_t max_chunks) {
  extern __shared__ int sh_hist[];
  __shared__ typename Op::Acc wsh[2][kCsrCtaThreads / 32];
  if constexpr (HIST) {
    if (a.smem_bins) hist_init(sh_hist, a.smem_bins);
  }
  const int64_t n_slots = counters[11] < max_chunks ? counters[11] : max_chunks;
  int buf = 0;
  for (int64_t k = blockIdx.x; k < n_slots; k += gridDim.x, buf ^= 1) {
    const int32_t row = chunk_row[k];
    const int64_t c = chunk_idx[k];
    const int64_t s = a.off[row] + c * kCsrChunk;
    const int64_t e0 = a.off[row + 1];
    const int64_t e = (s + kCsrChunk < e0) ? s + kCsrChunk : e0;
    const typename Op::Acc r = cta_fold<Op, HIST>(a, sh_hist, s, e, wsh[buf]);
    if (threadIdx.x == 0) part[k] = r;
  }
  if constexpr (HIST) {
    if (a.smem_bins) hist_flush(a, sh_hist);
  }
}

// the second pass of long rows (Sec. 2's recursive reduction at grid level):
// the thread of a row's first slot folds the row's chunk partials in chunk
// order with the grid-part combine (combine_parts), a fixed tree per row
template <class Op>
__global__ void csr_split_combine_kernel(float* __restrict__ y, const int64_t* counters,
                                         const int32_t* __restrict__ chunk_row, const int32_t* __restrict__ chunk_idx,
                                         const int32_t* __restrict__ chunk_cnt, const typename Op::Acc* __restrict__ part,
                                         int64_t max_chunks) {
  const int64_t n_slots = counters[11] < max_chunks ? counters[11] : max_chunks;
  for (int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; k < n_slots;
       k += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    if (chunk_idx[k] != 0) continue;
    const int n = chunk_cnt[k];
    if (n < 1 || k + n > n_slots) continue;   // a row the binning could not place whole (flagged there)
    y[chunk_row[k]] = combine_parts<Op>(part + k, n, nullptr);
  }
}

// standalone count histogram over all entries
__global__ void __launch_bounds__(256) csr_hist_kernel(const int32_t* __restrict__ col, int64_t nnz, int shift,
                                                       int64_t n_bins, int smem_bins, long long* hist) {
  extern __shared__ int sh_hist[];
  if (smem_bins) hist_init(sh_hist, smem_bins);
  CsrArgs a{};
  a.hist = hist;
  a.shift = shift;
  a.n_cols = 0;
  a.n_bins = n_bins;
  a.smem_bins = smem_bins;
  const int64_t n4 = nnz / 4;
  const int4* col4 = reinterpret_cast<const int4*>(col);
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n4;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int4 c = __ldcs(col4 + i);
    hist_add(a, sh_hist, c.x);
    hist_add(a, sh_hist, c.y);
    hist_add(a, sh_hist, c.z);
    hist_add(a, sh_hist, c.w);
  }
  for (int64_t i = n4 * 4 + blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < nnz;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    hist_add(a, sh_hist, __ldcs(col + i));
  if (smem_bins) hist_flush(a, sh_hist);
}

inline hp_status cuda_fail(cudaError_t e, const char* what) {
  return fail(HP_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// the attribute belongs to the kernel (shared by every nest): always the
// largest histogram any nest counts in shared memory
template <class K>
hp_status set_smem(K kernel, size_t dyn) {
  if (dyn == 0) return HP_OK;
  const cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(kCsrHistSmemMax * sizeof(int)));
  return e == cudaSuccess ? HP_OK : cuda_fail(e, "CSR kernel shared memory");
}

template <class Op, bool HIST>
hp_status launch_classes(hp_nest* n, const CsrArgs& a, cudaStream_t st) {
  CsrState& cs = *n->cs;
  const size_t dyn = HIST ? static_cast<size_t>(a.smem_bins) * sizeof(int) : 0;
  hp_status s;
  if ((s = set_smem(csr_rows_kernel<Op, 1, HIST>, dyn)) != HP_OK) return s;
  if ((s = set_smem(csr_rows_kernel<Op, 8, HIST>, dyn)) != HP_OK) return s;
  if ((s = set_smem(csr_rows_kernel<Op, 32, HIST>, dyn)) != HP_OK) return s;
  if ((s = set_smem(csr_cta_kernel<Op, HIST>, dyn)) != HP_OK) return s;
  if ((s = set_smem(csr_split_kernel<Op, HIST>, dyn)) != HP_OK) return s;
  const int fixed = n->csr.fixed_class;
  if (fixed < 0 || fixed == 0) csr_rows_kernel<Op, 1, HIST><<<cs.grid_rows, 256, dyn, st>>>(a, cs.rows, cs.counters, 0);
  if (fixed < 0 || fixed == 1) csr_rows_kernel<Op, 8, HIST><<<cs.grid_rows, 256, dyn, st>>>(a, cs.rows, cs.counters, 1);
  if (fixed < 0 || fixed == 2) csr_rows_kernel<Op, 32, HIST><<<cs.grid_rows, 256, dyn, st>>>(a, cs.rows, cs.counters, 2);
  if (fixed < 0 || fixed == 3)
    csr_cta_kernel<Op, HIST><<<cs.grid_row_cta, kCsrRowCtaThreads, dyn, st>>>(a, cs.rows, cs.counters);
  if (fixed < 0 || fixed == 4) {
    csr_split_kernel<Op, HIST><<<cs.grid_cta, kCsrCtaThreads, dyn, st>>>(
        a, cs.counters, cs.chunk_row, cs.chunk_idx, static_cast<typename Op::Acc*>(cs.part), cs.max_chunks);
    const int cgrid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>((cs.max_chunks + 255) / 256, 4 * n->sms)));
    csr_split_combine_kernel<Op><<<cgrid, 256, 0, st>>>(a.y, cs.counters, cs.chunk_row, cs.chunk_idx, cs.chunk_cnt,
                                                        static_cast<const typename Op::Acc*>(cs.part), cs.max_chunks);
  }
  const cudaError_t e = cudaPeekAtLastError();
  return e == cudaSuccess ? HP_OK : cuda_fail(e, "CSR class kernel launch");
}

template <class Op>
hp_status launch_op(hp_nest* n, const CsrArgs& a, cudaStream_t st) {
  return a.hist ? launch_classes<Op, true>(n, a, st) : launch_classes<Op, false>(n, a, st);
}

int smem_bins_for(int64_t n_bins) { return n_bins <= kCsrHistSmemMax ? static_cast<int>(n_bins) : 0; }

}  // namespace

// ---------------------------------------------------------------- host side
hp_status csr_prepare(hp_nest* n) {
  const CsrPlan& p = n->csr;
  CsrState* cs = new (std::nothrow) CsrState();
  if (!cs) return fail(HP_ENOMEM, "host allocation failed");
  n->cs = cs;
  cudaError_t e;
  e = cudaMalloc(&cs->counters, 16 * sizeof(int64_t));
  if (e != cudaSuccess) return fail(HP_ENOMEM, "cudaMalloc (CSR counters)");
  if (p.op == HP_RED_HIST_COUNT) return HP_OK;
  const int64_t rows = std::max<int64_t>(p.n_rows, 1);
  // long rows have > kCsrChunk entries, so chunk slots <= 2 * nnz / kCsrChunk + 1
  cs->max_chunks = 2 * (p.nnz / kCsrChunk) + 2;
  if (p.fixed_class == 4) cs->max_chunks = p.nnz / kCsrChunk + p.n_rows + 2;
  e = cudaMalloc(&cs->rows, rows * sizeof(int32_t));
  if (e != cudaSuccess) return fail(HP_ENOMEM, "cudaMalloc (CSR row lists)");
  const size_t mc = static_cast<size_t>(cs->max_chunks);
  if (cudaMalloc(&cs->chunk_row, mc * sizeof(int32_t)) != cudaSuccess ||
      cudaMalloc(&cs->chunk_idx, mc * sizeof(int32_t)) != cudaSuccess ||
      cudaMalloc(&cs->chunk_cnt, mc * sizeof(int32_t)) != cudaSuccess ||
      cudaMalloc(&cs->part, mc * sizeof(f2)) != cudaSuccess)
    return fail(HP_ENOMEM, "cudaMalloc (CSR chunk tables)");
  // every slot starts as a valid (row 0, chunk 0) entry, so a slot the binning
  // could not fill (offsets beyond the declared nnz, flagged) reads in bounds
  for (int32_t* t : {cs->chunk_row, cs->chunk_idx, cs->chunk_cnt}) {
    e = cudaMemset(t, 0, mc * sizeof(int32_t));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemset (chunk tables)");
  }
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, csr_rows_kernel<OpF32Comp, 32, true>, 256,
                                                smem_bins_for(p.n_bins) * sizeof(int));
  cs->grid_rows = std::max(1, per_sm) * n->sms;
  per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, csr_split_kernel<OpF32Comp, true>, kCsrCtaThreads,
                                                smem_bins_for(p.n_bins) * sizeof(int));
  cs->grid_cta = std::max(1, per_sm) * n->sms;
  per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, csr_cta_kernel<OpF32Comp, true>, kCsrRowCtaThreads,
                                                smem_bins_for(p.n_bins) * sizeof(int));
  cs->grid_row_cta = std::max(1, per_sm) * n->sms;
  return HP_OK;
}

hp_status run_csr(hp_nest* n, const void* const* in_dev, void* out_dev, cudaStream_t st) {
  const CsrPlan& p = n->csr;
  CsrState& cs = *n->cs;
  if (!in_dev) return fail(HP_EINVAL, "in_dev is NULL");
  if (!out_dev) return fail(HP_EINVAL, "out_dev is NULL");
  if (p.op == HP_RED_HIST_COUNT) {
    const int32_t* col = static_cast<const int32_t*>(in_dev[1]);
    if (!col && p.nnz > 0) return fail(HP_EINVAL, "missing col");
    if (reinterpret_cast<uintptr_t>(col) & 15u) return fail(HP_EINVAL, "col must be 16-byte aligned");
    long long* hist = static_cast<long long*>(out_dev);
    csr_zero_kernel<<<std::max<int64_t>(1, std::min<int64_t>((p.n_bins + 255) / 256, 4 * n->sms)), 256, 0, st>>>(
        cs.counters, 0, hist, p.n_bins);
    const int sb = smem_bins_for(p.n_bins);
    const size_t dyn = static_cast<size_t>(sb) * sizeof(int);
    hp_status s = set_smem(csr_hist_kernel, dyn);
    if (s != HP_OK) return s;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, csr_hist_kernel, 256, dyn);
    const int64_t want = (p.nnz / 4 + 255) / 256;
    const int grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(want, std::max(1, per_sm) * n->sms)));
    csr_hist_kernel<<<grid, 256, dyn, st>>>(col, p.nnz, p.hist_shift, p.n_bins, sb, hist);
    const cudaError_t e = cudaPeekAtLastError();
    return e == cudaSuccess ? HP_OK : cuda_fail(e, "CSR histogram launch");
  }
  for (int i = 0; i < 4; ++i)
    if (!in_dev[i]) return fail(HP_EINVAL, "missing CSR input " + std::to_string(i));
  if ((reinterpret_cast<uintptr_t>(in_dev[1]) | reinterpret_cast<uintptr_t>(in_dev[2])) & 15u)
    return fail(HP_EINVAL, "CSR col and val must be 16-byte aligned (128-bit loads)");
  CsrArgs a{};
  a.off = static_cast<const int64_t*>(in_dev[0]);
  a.col = static_cast<const int32_t*>(in_dev[1]);
  a.val = static_cast<const float*>(in_dev[2]);
  a.x = static_cast<const float*>(in_dev[3]);
  a.y = static_cast<float*>(out_dev);
  a.hist = nullptr;
  a.err = n->err;
  a.nnz = p.nnz;
  a.n_cols = p.n_cols;
  if (p.fuse_hist) {
    a.hist = static_cast<long long*>(const_cast<void*>(in_dev[4]));
    if (!a.hist) return fail(HP_EINVAL, "fuse_hist needs the histogram output in in_dev[4]");
    a.shift = p.hist_shift;
    a.n_bins = p.n_bins;
    a.smem_bins = smem_bins_for(p.n_bins);
  }
  if (p.n_rows == 0) return HP_OK;
  const int zgrid = static_cast<int>(
      std::max<int64_t>(1, std::min<int64_t>((std::max<int64_t>(p.fuse_hist ? p.n_bins : 0, 16) + 255) / 256, 4 * n->sms)));
  csr_zero_kernel<<<zgrid, 256, 0, st>>>(cs.counters, 16, a.hist, p.fuse_hist ? p.n_bins : 0);
  const int bgrid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>((p.n_rows + kCsrBinThreads - 1) / kCsrBinThreads,
                                                                           8 * n->sms)));
  csr_bin_count_kernel<<<bgrid, kCsrBinThreads, 0, st>>>(a.off, p.n_rows, p.fixed_class, cs.counters);
  csr_bin_scatter_kernel<<<bgrid, kCsrBinThreads, 0, st>>>(a.off, p.n_rows, p.fixed_class, cs.counters, cs.rows,
                                                          cs.chunk_row, cs.chunk_idx, cs.chunk_cnt,
                                                          cs.max_chunks, n->err);
  cudaError_t e = cudaPeekAtLastError();
  if (e != cudaSuccess) return cuda_fail(e, "CSR binning launch");
  switch (p.op) {
    case HP_RED_SUM:
      return p.prec == HP_F32_COMP ? launch_op<OpF32Comp>(n, a, st) : launch_op<OpF32Sum>(n, a, st);
    case HP_RED_MAX:
      return launch_op<OpF32Max>(n, a, st);
    case HP_RED_MIN:
      return launch_op<OpF32Min>(n, a, st);
    default:
      return fail(HP_EINVAL, "bad CSR op");
  }
}

// ---------------------------------------------------------------- gather-rate probe
namespace {

// counter hash (murmur3's 32-bit finalizer over index ^ seed): uniform indices
__device__ __forceinline__ uint32_t probe_hash(uint64_t i, uint32_t seed) {
  uint32_t h = static_cast<uint32_t>(i) ^ static_cast<uint32_t>(i >> 32) * 0x9e3779b9u ^ seed;
  h ^= h >> 16;
  h *= 0x85ebca6bu;
  h ^= h >> 13;
  h *= 0xc2b2ae35u;
  h ^= h >> 16;
  return h;
}

// n random 4-byte reads of x through the CSR executor's x-gather path (__ldcg:
// cached in L2 only), 8 independent reads in flight per thread per round;
// each block adds its sum to *out so that no read is dead code
__global__ void __launch_bounds__(256) gather_probe_kernel(const float* __restrict__ x, uint32_t n_x, int64_t n,
                                                           uint32_t seed, float* out) {
  __shared__ float wsum[8];
  float acc = 0.0f;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  for (; i + 7 * stride < n; i += 8 * stride) {
    float v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const uint32_t h = probe_hash(static_cast<uint64_t>(i + u * stride), seed);
      v[u] = __ldcg(x + static_cast<uint32_t>((static_cast<uint64_t>(h) * n_x) >> 32));
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) acc += v[u];
  }
  for (; i < n; i += stride) {
    const uint32_t h = probe_hash(static_cast<uint64_t>(i), seed);
    acc += __ldcg(x + static_cast<uint32_t>((static_cast<uint64_t>(h) * n_x) >> 32));
  }
  for (int m = 16; m >= 1; m >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, m);
  if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.0f;
    for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) t += wsum[w];
    atomicAdd(out, t);
  }
}

}  // namespace

size_t csr_out_bytes(const hp_nest* n) {
  return n->csr.op == HP_RED_HIST_COUNT ? static_cast<size_t>(n->csr.n_bins) * 8
                                        : static_cast<size_t>(n->csr.n_rows) * 4;
}

void csr_release(hp_nest* n) {
  CsrState* cs = n->cs;
  if (!cs) return;
  cudaFree(cs->counters);
  cudaFree(cs->rows);
  cudaFree(cs->chunk_row);
  cudaFree(cs->chunk_idx);
  cudaFree(cs->chunk_cnt);
  cudaFree(cs->part);
  delete cs;
  n->cs = nullptr;
}

}  // namespace hp

extern "C" hp_status hp_probe_gather(const float* x_dev, int64_t n_x, int64_t n_gathers, uint32_t seed, float* sum_dev,
                                     void* stream) {
  using namespace hp;
  if (!x_dev || !sum_dev) return fail(HP_EINVAL, "x_dev and sum_dev must be device pointers");
  if (n_x < 1 || n_x > (int64_t(1) << 32) - 1) return fail(HP_EINVAL, "n_x must be in [1, 2^32)");
  if (n_gathers < 0) return fail(HP_EINVAL, "n_gathers must be >= 0");
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gather_probe_kernel, 256, 0);
  if (e != cudaSuccess) return cuda_fail(e, "gather probe set-up");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  e = cudaMemsetAsync(sum_dev, 0, sizeof(float), st);
  if (e != cudaSuccess) return cuda_fail(e, "gather probe memset");
  if (n_gathers == 0) return HP_OK;
  const int64_t want = (n_gathers + 255) / 256;
  const int grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(want, static_cast<int64_t>(std::max(1, per_sm)) * sms)));
  gather_probe_kernel<<<grid, 256, 0, st>>>(x_dev, static_cast<uint32_t>(n_x), n_gathers, seed, sum_dev);
  e = cudaPeekAtLastError();
  return e == cudaSuccess ? HP_OK : cuda_fail(e, "gather probe launch");
}
