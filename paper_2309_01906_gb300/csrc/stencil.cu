// stencil.cu — stencil nests with ghost zones (include/hp.h, hp_stencil_*).
//
// Sec. 2: a stencil can be tiled to any level that has local memory, choosing
// a region whose input region fits it; Sec. 4: each unit of a level maps an
// array section, the `to` sections overlapping by a ghost surface and the
// `from` sections partitioning the array.
//
// Levels here: GRID-level sections (groups of whole tiles, processed section
// after section so that neighbouring tiles share their ghost rows through L2)
// and CTA-level tiles.  A CTA maps its tile plus a ghost border of h = r*T
// points (x: rounded up to 4, the 16-byte rule of tensor copies) into shared
// memory with one 2-D tensor copy (cp.async.bulk.tensor; points outside the
// array read as 0: the zero ghost surface of the array edge), runs all T steps
// there (two buffers, each step's region one radius narrower, points outside
// the array forced to 0), and stores only its tile.  Every point of every step
// is one FP32 FMA chain over the window in row-major order from 0, so a run of
// T steps equals T runs of one step bit for bit.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <new>
#include <sstream>
#include <string>
#include <vector>

#include "hp_internal.h"

namespace hp {

constexpr int kStencilThreads = 256;
constexpr int kStencilMaxR = 4;
constexpr int kStencilMaxSteps = 8;
constexpr int kStencilBox = 256;                 // largest tensor-copy box side (points)
constexpr size_t kStencilSmem = 226 * 1024;      // dynamic shared memory of one CTA (opt-in maximum less static use)

struct StencilPlan {
  int64_t ny = 0, nx = 0;
  int r = 0, T = 1;
  int TY = 0, TX = 0;            // CTA tile
  int h = 0, hx = 0;             // ghost border (rows, columns; hx = h rounded up to 4)
  int boxH = 0, boxW = 0;        // tensor box = tile + 2 * ghost
  int nbuf = 1;                  // shared buffers (2 when steps > 1)
  int buf_floats = 0;            // one buffer, rounded up to 128 bytes
  int64_t SY = 0, SX = 0;        // GRID-level sections
  int64_t tiles_y = 0, tiles_x = 0;
  std::vector<int32_t> order;    // tiles (ty, tx) pairs, section after section
  float c[(2 * kStencilMaxR + 1) * (2 * kStencilMaxR + 1)] = {};
  size_t smem() const { return static_cast<size_t>(nbuf) * buf_floats * sizeof(float); }
};

namespace {

inline int round_up(int v, int m) { return (v + m - 1) / m * m; }

hp_status plan_stencil(int64_t ny, int64_t nx, int radius, const float* coeffs, int steps, const hp_stencil_map* map,
                       StencilPlan* out, std::string* why) {
  auto bad = [&](const std::string& m) {
    *why = m;
    return HP_EINVAL;
  };
  if (ny < 0 || nx < 0) return bad("ny and nx must be >= 0");
  if (ny > (int64_t(1) << 31) || nx > (int64_t(1) << 31) || ny * nx > (int64_t(1) << 40))
    return bad("array too large (ny, nx <= 2^31, ny * nx <= 2^40)");
  if (radius < 0 || radius > kStencilMaxR) return bad("radius must be in [0, 4]");
  if (steps < 1 || steps > kStencilMaxSteps) return bad("steps must be in [1, 8]");
  if (!coeffs) return bad("coeffs is NULL");
  StencilPlan p;
  p.ny = ny;
  p.nx = nx;
  p.r = radius;
  p.T = steps;
  const int K = (2 * radius + 1) * (2 * radius + 1);
  std::memcpy(p.c, coeffs, sizeof(float) * K);
  p.h = radius * steps;
  p.hx = round_up(p.h, 4);
  p.nbuf = steps > 1 ? 2 : 1;
  auto box_smem = [&](int ty, int tx) {
    const int bw = tx + 2 * p.hx, bh = ty + 2 * p.h;
    return static_cast<size_t>(p.nbuf) * round_up(bw * bh, 32) * sizeof(float);
  };
  int TY = map ? map->tile_y : 0, TX = map ? map->tile_x : 0;
  // narrow ghost borders: 64-column tiles, 128 rows for one step and 96 for
  // fused steps (measured at 16384^2, radius 1: 0.347 ms against 0.362 for
  // 64 x 128 with one step, 1.027 ms against 1.143 with four)
  if (TX == 0) TX = p.h <= 4 ? 64 : 128;
  if (TY == 0) {
    // about two CTAs per SM; taller tiles when the ghost border is wide, and
    // one CTA per SM rather than tiles shorter than the border (redundant work)
    auto pick = [&](size_t budget) {
      int ty = p.h <= 4 ? (p.T == 1 ? 128 : 96) : 128;
      while (ty > 1 && (box_smem(ty, TX) > budget || ty + 2 * p.h > kStencilBox)) ty /= 2;
      return ty;
    };
    TY = pick(110 * 1024);
    if (TY < 2 * p.h) TY = std::max(TY, pick(kStencilSmem));
  }
  if (TX < 4 || TX % 4 != 0) return bad("tile_x must be a positive multiple of 4");
  if (TY < 1) return bad("tile_y must be >= 1");
  if (TX + 2 * p.hx > kStencilBox || TY + 2 * p.h > kStencilBox)
    return bad("tile plus ghost border exceeds one tensor copy (256 x 256 points)");
  if (box_smem(TY, TX) > kStencilSmem) return bad("tile plus ghost border does not fit one CTA's shared memory");
  p.TY = TY;
  p.TX = TX;
  p.boxW = TX + 2 * p.hx;
  p.boxH = TY + 2 * p.h;
  p.buf_floats = round_up(p.boxW * p.boxH, 32);
  p.tiles_y = (ny + TY - 1) / TY;
  p.tiles_x = (nx + TX - 1) / TX;
  p.SY = map && map->section_y ? map->section_y : std::max<int64_t>(TY, p.tiles_y * TY);
  p.SX = map && map->section_x ? map->section_x : std::max<int64_t>(TX, p.tiles_x * TX);
  if (p.SY < 0 || p.SX < 0 || p.SY % TY != 0 || p.SX % TX != 0)
    return bad("sections must be positive multiples of the tile");
  // tile order: section after section (row-major), tiles row-major inside a section
  const int64_t sty = p.SY / TY, stx = p.SX / TX;
  if (p.tiles_y * p.tiles_x > (int64_t(1) << 26)) return bad("too many tiles");
  p.order.reserve(static_cast<size_t>(2 * p.tiles_y * p.tiles_x));
  for (int64_t sy = 0; sy < p.tiles_y; sy += sty)
    for (int64_t sx = 0; sx < p.tiles_x; sx += stx)
      for (int64_t ty = sy; ty < std::min(p.tiles_y, sy + sty); ++ty)
        for (int64_t tx = sx; tx < std::min(p.tiles_x, sx + stx); ++tx) {
          p.order.push_back(static_cast<int32_t>(ty));
          p.order.push_back(static_cast<int32_t>(tx));
        }
  *out = std::move(p);
  return HP_OK;
}

std::string describe_stencil(const StencilPlan& p) {
  std::ostringstream s;
  s << "{\"kind\":\"stencil\",\"ny\":" << p.ny << ",\"nx\":" << p.nx << ",\"radius\":" << p.r << ",\"steps\":" << p.T
    << ",\"tile\":[" << p.TY << "," << p.TX << "],\"ghost\":[" << p.h << "," << p.hx << "],\"box\":[" << p.boxH << ","
    << p.boxW << "],\"buffers\":" << p.nbuf << ",\"smem\":" << p.smem() << ",\"tiles\":" << p.order.size() / 2
    << ",\"section\":[" << p.SY << "," << p.SX << "]";
  const int64_t secs_y = (p.ny + p.SY - 1) / std::max<int64_t>(p.SY, 1), secs_x = (p.nx + p.SX - 1) / std::max<int64_t>(p.SX, 1);
  if (p.ny > 0 && p.nx > 0 && secs_y * secs_x <= 64) {
    // the GRID level's map sections: `to` = section + ghost border (clipped), `from` = section (clipped)
    s << ",\"sections\":[";
    bool first = true;
    for (int64_t a = 0; a < secs_y; ++a)
      for (int64_t b = 0; b < secs_x; ++b) {
        const int64_t y0 = a * p.SY, x0 = b * p.SX, y1 = std::min(p.ny, y0 + p.SY), x1 = std::min(p.nx, x0 + p.SX);
        s << (first ? "" : ",") << "{\"to\":[[" << std::max<int64_t>(0, y0 - p.h) << "," << std::min(p.ny, y1 + p.h)
          << "],[" << std::max<int64_t>(0, x0 - p.h) << "," << std::min(p.nx, x1 + p.h) << "]],\"from\":[[" << y0 << ","
          << y1 << "],[" << x0 << "," << x1 << "]]}";
        first = false;
      }
    s << "]";
  }
  s << "}";
  return s.str();
}

}  // namespace
}  // namespace hp

namespace hp {
namespace {

struct StencilArgs {
  const float* in;
  float* out;
  const int32_t* order;     // tile (ty, tx) pairs
  int32_t* err;
  int64_t ny, nx;
  int32_t n_tiles, T, TY, TX, h, hx, boxW, boxH, buf_floats, use_tma;
  float c[(2 * kStencilMaxR + 1) * (2 * kStencilMaxR + 1)];
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ bool bar_test(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait (1 s of the global timer); false when it ran out
__device__ __noinline__ bool bar_wait(uint32_t bar, uint32_t parity) {
  unsigned long long t0, t;
  asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t0));
  for (uint32_t i = 0;; ++i) {
    if (bar_test(bar, parity)) return true;
    if ((i & 31u) == 31u) {
      asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
      if (t - t0 > 1000000000ull) return false;
    }
  }
}

// N rows from j0 of buffer column i, inside the array: no per-point checks.
// The strip's N + 2R input rows are loaded once each into a fully unrolled
// register array and indexed (nothing is shifted).
template <int R, int N>
__device__ __forceinline__ void fast_strip(const float* __restrict__ src, float* __restrict__ dst,
                                           const StencilArgs& a, int i, int j0, bool final, int64_t gy, int64_t gx) {
  constexpr int D = 2 * R + 1;
  const int P = a.boxW;
  const float* sp = src + (j0 - R) * P + (i - R);
  float v[N + 2 * R][D];
#pragma unroll
  for (int y = 0; y < N + 2 * R; ++y)
#pragma unroll
    for (int dx = 0; dx < D; ++dx) v[y][dx] = sp[y * P + dx];
  float* dp = dst + j0 * P + i;
  float* gp = a.out + (gy * a.nx + gx);
#pragma unroll
  for (int k = 0; k < N; ++k) {
    float acc = 0.0f;
#pragma unroll
    for (int dy = 0; dy < D; ++dy)
#pragma unroll
      for (int dx = 0; dx < D; ++dx) acc = __fmaf_rn(a.c[dy * D + dx], v[k + dy][dx], acc);
    if (final) {
      *gp = acc;
      gp += a.nx;
    } else {
      *dp = acc;
      dp += P;
    }
  }
}

// rows [j0, j0 + n) of buffer column i, any position: a sliding window of
// 2R+1 rows x 2R+1 columns in registers and per-point array checks (points
// outside the array: not stored in the last step, 0 in the others)
template <int R, int S>
__device__ __forceinline__ void checked_strip(const float* __restrict__ src, float* __restrict__ dst,
                                              const StencilArgs& a, int i, int j0, int n, bool final, int64_t gy,
                                              int64_t gx) {
  constexpr int D = 2 * R + 1;
  const int P = a.boxW;
  const float* sp = src + (j0 - R) * P + (i - R);
  float w[D][D];
#pragma unroll
  for (int dy = 1; dy < D; ++dy)
#pragma unroll
    for (int dx = 0; dx < D; ++dx) w[dy][dx] = sp[(dy - 1) * P + dx];
  sp += (D - 1) * P;
  const bool col_in = gx >= 0 && gx < a.nx;
  float* dp = dst + j0 * P + i;
  for (int k = 0; k < n; ++k) {
#pragma unroll
    for (int dy = 0; dy < D - 1; ++dy)
#pragma unroll
      for (int dx = 0; dx < D; ++dx) w[dy][dx] = w[dy + 1][dx];
#pragma unroll
    for (int dx = 0; dx < D; ++dx) w[D - 1][dx] = sp[dx];
    sp += P;
    float acc = 0.0f;
#pragma unroll
    for (int dy = 0; dy < D; ++dy)
#pragma unroll
      for (int dx = 0; dx < D; ++dx) acc = __fmaf_rn(a.c[dy * D + dx], w[dy][dx], acc);
    const bool in = col_in && gy + k >= 0 && gy + k < a.ny;
    if (final) {
      if (in) a.out[(gy + k) * a.nx + gx] = acc;
    } else {
      dp[k * P] = in ? acc : 0.0f;   // the zero ghost surface stays zero at every step
    }
  }
}

// one strip: rows [j0, j0 + n), n <= S; whole strips inside the array take
// the check-free path
template <int R, int S>
__device__ __forceinline__ void strip(const float* __restrict__ src, float* __restrict__ dst, const StencilArgs& a,
                                      int i, int j0, int n, bool final, int64_t gy0, int64_t gx0) {
  const int64_t gx = gx0 + i, gy = gy0 + j0;
  if (n == S && gx >= 0 && gx < a.nx && gy >= 0 && gy + S <= a.ny)
    fast_strip<R, S>(src, dst, a, i, j0, final, gy, gx);
  else
    checked_strip<R, S>(src, dst, a, i, j0, n, final, gy, gx);
}

// FUSED: more than one step per launch (two buffers: 2 CTAs per SM at most,
// so registers are spent on instruction-level parallelism); one step: radius
// <= 1 keeps 4 CTAs per SM resident for memory-level parallelism
#ifndef HP_STENCIL_STEP1_BLOCKS
#define HP_STENCIL_STEP1_BLOCKS 3   // resident CTAs per SM the one-step kernels' registers are sized for (measured best)
#endif
template <int R, bool FUSED>
__global__ void __launch_bounds__(kStencilThreads, R >= 4 ? 1 : ((R >= 2 || FUSED) ? 2 : HP_STENCIL_STEP1_BLOCKS))
    stencil_kernel(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ StencilArgs a) {
  extern __shared__ __align__(128) float sbuf[];
  __shared__ __align__(8) unsigned long long bar_word;
  __shared__ int ok_flag;
  const int tid = threadIdx.x;
  const uint32_t bar = smem_addr(&bar_word);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  uint32_t parity = 0;
  float* buf0 = sbuf;
  float* buf1 = sbuf + a.buf_floats;
  for (int k = blockIdx.x; k < a.n_tiles; k += gridDim.x) {
    const int64_t y0 = static_cast<int64_t>(a.order[2 * k]) * a.TY;
    const int64_t x0 = static_cast<int64_t>(a.order[2 * k + 1]) * a.TX;
    const int64_t gy0 = y0 - a.h, gx0 = x0 - a.hx;   // global coordinates of buffer (0, 0)
    // ---- the `to` section: tile + ghost border into buf0
    if (a.use_tma) {
      if (tid == 0) {
        int ok = 1;
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");   // earlier reads of buf0 before the copy
        asm volatile(
            "{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(bar),
            "r"(static_cast<uint32_t>(a.boxW * a.boxH * 4))
            : "memory");
        asm volatile(
            "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::
                "r"(smem_addr(buf0)),
            "l"(reinterpret_cast<uint64_t>(&tmap)), "r"(static_cast<int32_t>(gx0)), "r"(static_cast<int32_t>(gy0)),
            "r"(bar)
            : "memory");
        if (!bar_wait(bar, parity)) {
          ok = 0;
          atomicExch(a.err, 1);
          bar_wait(bar, parity);   // give the copy in flight another second before leaving
        }
        ok_flag = ok;
      }
      parity ^= 1u;
      __syncthreads();
      if (!ok_flag) return;   // every thread reads the same flag after the barrier
    } else {
      const int n = a.boxW * a.boxH;
      for (int q = tid; q < n; q += kStencilThreads) {
        const int j = q / a.boxW, i = q - j * a.boxW;
        const int64_t gy = gy0 + j, gx = gx0 + i;
        buf0[q] = (gy >= 0 && gy < a.ny && gx >= 0 && gx < a.nx) ? a.in[gy * a.nx + gx] : 0.0f;
      }
      __syncthreads();
    }
    // ---- T steps; step s computes the tile widened by e = h - R s (the last one: the tile)
    for (int s = 1; s <= a.T; ++s) {
      const float* src = (s & 1) ? buf0 : buf1;
      float* dst = (s & 1) ? buf1 : buf0;
      const int e = a.h - R * s;
      const int jl = a.h - e, jh = a.h + a.TY + e;
      const int il = a.hx - e, ih = a.hx + a.TX + e;
      // (column, strip) items, columns fastest: every lane busy, neighbouring lanes on
      // neighbouring columns; strips of S rows, the last one shorter
      constexpr int S = R <= 1 ? 16 : (R == 2 ? 8 : 4);   // S + 2R rows of 2R+1 registers
      const int H = jh - jl, W = ih - il, n_rs = (H + S - 1) / S;
      const bool final = s == a.T;
      for (int q = tid; q < W * n_rs; q += kStencilThreads) {
        const int rs = q / W, i = il + (q - rs * W);
        const int j0 = jl + rs * S, n = min(S, jh - j0);
        strip<R, S>(src, dst, a, i, j0, n, final, gy0, gx0);
      }
      __syncthreads();
    }
  }
}

}  // namespace
}  // namespace hp

struct hp_stencil {
  hp::StencilPlan plan;
  int device = -1;
  int sms = 0;
  int32_t* d_order = nullptr;
  int32_t* err = nullptr;
  std::mutex mu;                 // guards the cached tensor map
  CUtensorMap tmap;
  const float* tmap_ptr = nullptr;
};

namespace hp {
namespace {

hp_status stencil_cuda_fail(cudaError_t e, const char* what) {
  return fail(HP_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

template <int R, bool FUSED>
cudaError_t stencil_prepare_kernel() {
  static const cudaError_t e = cudaFuncSetAttribute(
      stencil_kernel<R, FUSED>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(kStencilSmem));
  return e;
}

template <int R, bool FUSED>
cudaError_t stencil_launch_as(const CUtensorMap& tmap, const StencilArgs& a, size_t smem, int sms, cudaStream_t st) {
  cudaError_t e = stencil_prepare_kernel<R, FUSED>();
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, stencil_kernel<R, FUSED>, kStencilThreads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int grid = static_cast<int>(std::min<int64_t>(a.n_tiles, static_cast<int64_t>(per_sm) * sms));
  stencil_kernel<R, FUSED><<<grid, kStencilThreads, smem, st>>>(tmap, a);
  return cudaPeekAtLastError();
}

template <int R>
cudaError_t stencil_launch(const CUtensorMap& tmap, const StencilArgs& a, size_t smem, int sms, cudaStream_t st) {
  return a.T > 1 ? stencil_launch_as<R, true>(tmap, a, smem, sms, st)
                 : stencil_launch_as<R, false>(tmap, a, smem, sms, st);
}

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encoder() {
  static EncodeTiled fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    return reinterpret_cast<EncodeTiled>(p);
  }();
  return fn;
}

// tensor map of the input: 2-D FP32 (nx, ny), box (boxW, boxH), zero fill outside
bool encode_input(hp_stencil* s, const float* in) {
  const StencilPlan& p = s->plan;
  EncodeTiled fn = encoder();
  if (!fn) return false;
  const cuuint64_t dims[2] = {static_cast<cuuint64_t>(p.nx), static_cast<cuuint64_t>(p.ny)};
  const cuuint64_t strides[1] = {static_cast<cuuint64_t>(p.nx) * sizeof(float)};
  const cuuint32_t box[2] = {static_cast<cuuint32_t>(p.boxW), static_cast<cuuint32_t>(p.boxH)};
  const cuuint32_t estr[2] = {1, 1};
  return fn(&s->tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(in), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

hp_status stencil_ensure_device(hp_stencil* s) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return stencil_cuda_fail(e, "no CUDA device");
  if (s->device >= 0) return dev == s->device ? HP_OK : fail(HP_EINVAL, "stencil was first run on another device");
  if ((e = cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return stencil_cuda_fail(e, "device query");
  const size_t ob = std::max<size_t>(s->plan.order.size(), 2) * sizeof(int32_t);
  if ((e = cudaMalloc(&s->d_order, ob)) != cudaSuccess) return fail(HP_ENOMEM, "cudaMalloc (tile order)");
  if (!s->plan.order.empty() &&
      (e = cudaMemcpy(s->d_order, s->plan.order.data(), s->plan.order.size() * sizeof(int32_t),
                      cudaMemcpyHostToDevice)) != cudaSuccess)
    return stencil_cuda_fail(e, "upload tile order");
  if ((e = cudaMalloc(&s->err, sizeof(int32_t))) != cudaSuccess) return fail(HP_ENOMEM, "cudaMalloc (error word)");
  if ((e = cudaMemset(s->err, 0, sizeof(int32_t))) != cudaSuccess) return stencil_cuda_fail(e, "cudaMemset");
  s->device = dev;
  return HP_OK;
}

}  // namespace
}  // namespace hp

using namespace hp;

extern "C" hp_status hp_stencil_create(int64_t ny, int64_t nx, int radius, const float* coeffs, int steps,
                                       const hp_stencil_map* map, hp_stencil** out) {
  if (!out) return fail(HP_EINVAL, "out is NULL");
  *out = nullptr;
  StencilPlan p;
  std::string why;
  const hp_status st = plan_stencil(ny, nx, radius, coeffs, steps, map, &p, &why);
  if (st != HP_OK) return fail(st, why);
  hp_stencil* s = new (std::nothrow) hp_stencil;
  if (!s) return fail(HP_ENOMEM, "out of host memory");
  s->plan = std::move(p);
  *out = s;
  set_error("");
  return HP_OK;
}

extern "C" hp_status hp_stencil_run(hp_stencil* s, const float* in_dev, float* out_dev, void* stream) {
  if (!s) return fail(HP_EINVAL, "stencil is NULL");
  const StencilPlan& p = s->plan;
  if (p.order.empty()) return HP_OK;   // empty array
  if (!in_dev || !out_dev) return fail(HP_EINVAL, "NULL buffer");
  const size_t bytes = static_cast<size_t>(p.ny * p.nx) * sizeof(float);
  const char *a = reinterpret_cast<const char*>(in_dev), *b = reinterpret_cast<const char*>(out_dev);
  if (a < b + bytes && b < a + bytes) return fail(HP_EINVAL, "in and out overlap (the stencil runs out of place)");
  hp_status st = stencil_ensure_device(s);
  if (st != HP_OK) return st;
  StencilArgs args;
  args.in = in_dev;
  args.out = out_dev;
  args.order = s->d_order;
  args.err = s->err;
  args.ny = p.ny;
  args.nx = p.nx;
  args.n_tiles = static_cast<int32_t>(p.order.size() / 2);
  args.T = p.T;
  args.TY = p.TY;
  args.TX = p.TX;
  args.h = p.h;
  args.hx = p.hx;
  args.boxW = p.boxW;
  args.boxH = p.boxH;
  args.buf_floats = p.buf_floats;
  std::memcpy(args.c, p.c, sizeof(args.c));
  CUtensorMap tmap;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    // tensor copies need 16-byte rows and base; otherwise plain loads (same values)
    args.use_tma = (p.nx % 4 == 0) && (reinterpret_cast<uintptr_t>(in_dev) % 16 == 0);
    if (args.use_tma && s->tmap_ptr != in_dev) {
      if (encode_input(s, in_dev)) s->tmap_ptr = in_dev;
      else args.use_tma = 0;
    }
    if (args.use_tma) tmap = s->tmap;
    else std::memset(&tmap, 0, sizeof(tmap));
  }
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  switch (p.r) {
    case 0: e = stencil_launch<0>(tmap, args, p.smem(), s->sms, cs); break;
    case 1: e = stencil_launch<1>(tmap, args, p.smem(), s->sms, cs); break;
    case 2: e = stencil_launch<2>(tmap, args, p.smem(), s->sms, cs); break;
    case 3: e = stencil_launch<3>(tmap, args, p.smem(), s->sms, cs); break;
    default: e = stencil_launch<4>(tmap, args, p.smem(), s->sms, cs); break;
  }
  if (e != cudaSuccess) return stencil_cuda_fail(e, "stencil launch");
  return HP_OK;
}

extern "C" hp_status hp_stencil_describe(const hp_stencil* s, char* buf, size_t len) {
  if (!s || !buf || len == 0) return fail(HP_EINVAL, "NULL argument");
  const std::string d = describe_stencil(s->plan);
  std::strncpy(buf, d.c_str(), len - 1);
  buf[len - 1] = '\0';
  return HP_OK;
}

extern "C" hp_status hp_stencil_check(hp_stencil* s, void* stream, int32_t* device_error) {
  if (!s) return fail(HP_EINVAL, "stencil is NULL");
  if (device_error) *device_error = 0;
  if (s->device < 0 || !s->err) return HP_OK;
  cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return stencil_cuda_fail(e, "stream synchronize");
  int32_t v = 0;
  if ((e = cudaMemcpy(&v, s->err, sizeof(v), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return stencil_cuda_fail(e, "read error word");
  if (device_error) *device_error = v;
  if (v != 0) return fail(HP_ETIMEOUT, "device error word set (code " + std::to_string(v) + ": a tensor-copy wait ran out)");
  return HP_OK;
}

extern "C" void hp_stencil_destroy(hp_stencil* s) {
  if (!s) return;
  if (s->device >= 0) {
    if (s->d_order) cudaFree(s->d_order);
    if (s->err) cudaFree(s->err);
  }
  delete s;
}
