// rect_launch.cuh — host-side launch of the rectangular executor for one
// accumulation policy.  Each rect_*.cu translation unit instantiates it for
// its policies so that the kernels compile in parallel.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "hp_internal.h"
#include "rect_kernels.cuh"

namespace hp {

struct RectArgs {
  const void* const* in;   // device inputs
  void* out;               // device outputs
  void* part;              // grid-part partials (G > 1)
  const float* geo;        // GEOMETRIC table (device)
  cudaStream_t stream;
  float* comp = nullptr;   // compensated sums: residual output (hp_nest_run_comp), or null
};

inline hp_status cuda_fail(cudaError_t e, const char* what) {
  return fail(HP_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

template <class Op, int V, class Body>
hp_status launch_team(const NestPlan& np, RectPlan rp, LaunchCfg& cfg, const Body& body, const RectArgs& a) {
  using Out = typename Op::Out;
  using Acc = typename Op::Acc;
  cudaError_t e;
  rp.comp = a.comp;
  if (rp.team == TEAM_MAP) {
    auto k = rect_map_kernel<Op, Body>;
    if (!cfg.ready) {
      cfg.threads = 256;
      const int64_t blocks = (rp.O + 255) / 256;
      cfg.grid = static_cast<int>(blocks < 8LL * cfg.sms ? (blocks > 0 ? blocks : 1) : 8LL * cfg.sms);
      cfg.ready = true;
    }
    if (rp.O == 0) return HP_OK;
    k<<<cfg.grid, cfg.threads, 0, a.stream>>>(rp, body, static_cast<Out*>(a.out));
    e = cudaPeekAtLastError();
    return e == cudaSuccess ? HP_OK : cuda_fail(e, "rect_map_kernel launch");
  }
  const bool block = rp.team == TEAM_BLOCK;
  constexpr bool kPipeable = Body::kPipeable && V == 4;
  const bool pipe = kPipeable && block && rp.pipe;
  auto kb = rect_block_kernel<Op, V, Body>;
  auto kl = rect_lanes_kernel<Op, V, Body>;
  const bool deep = rp.groups <= 4;
  auto kp = deep ? rect_block_pipe_kernel<Op, Body::kDot, pipe_depth(4)> : rect_block_pipe_kernel<Op, Body::kDot, pipe_depth(8)>;
  const void* kfn = pipe ? reinterpret_cast<const void*>(kp)
                         : block ? reinterpret_cast<const void*>(kb) : reinterpret_cast<const void*>(kl);
  const size_t dyn =
      pipe ? static_cast<size_t>(32 * rp.W) *
                 std::max<size_t>(pipe_depth(rp.groups) * rp.groups * 16, kPatMax * sizeof(int32_t))
           : 0;
  if (!cfg.ready) {
    cfg.threads = 32 * rp.W;
    cfg.cluster = block ? rp.C : 1;
    if (pipe) {
      // the attribute belongs to the kernel, not to this nest: always the
      // largest size any plan of this kernel uses (static + dynamic may
      // exceed the 48 KiB default)
      e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(kPipeDynMax));
      if (e != cudaSuccess) return cuda_fail(e, "dynamic shared memory size");
    }
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, cfg.threads, dyn);
    if (e != cudaSuccess) return cuda_fail(e, "occupancy query");
    if (per_sm < 1) return fail(HP_EUNSUPPORTED, "kernel does not fit on an SM with this CTA size");
    int64_t max_teams;
    if (block && rp.C > 1) {
      if (rp.C > 8) {
        e = cudaFuncSetAttribute(kfn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return cuda_fail(e, "non-portable cluster size");
      }
      cudaLaunchConfig_t lc = {};
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = rp.C;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      lc.gridDim = dim3(rp.C * cfg.sms);
      lc.blockDim = dim3(cfg.threads);
      lc.dynamicSmemBytes = dyn;
      lc.attrs = at;
      lc.numAttrs = 1;
      int n_clusters = 0;
      e = cudaOccupancyMaxActiveClusters(&n_clusters, kfn, &lc);
      if (e != cudaSuccess) return cuda_fail(e, "cluster occupancy query");
      if (n_clusters < 1) return fail(HP_EUNSUPPORTED, "a cluster of this size does not fit on the GPU");
      max_teams = n_clusters;
    } else if (block) {
      max_teams = static_cast<int64_t>(per_sm) * cfg.sms;
    } else {
      max_teams = static_cast<int64_t>(per_sm) * cfg.sms * rp.W * (32 / rp.L);
    }
    if (block) {
      int64_t teams = rp.items < max_teams ? rp.items : max_teams;
      if (teams < 1) teams = 1;
      int64_t M = (rp.items + teams - 1) / teams;
      cfg.M = static_cast<int>(M < 1 ? 1 : (M > kMaxM ? kMaxM : M));
      cfg.grid = static_cast<int>(teams * cfg.cluster);
    } else {
      const int64_t teams_per_cta = static_cast<int64_t>(rp.W) * (32 / rp.L);
      int64_t blocks = (rp.items + teams_per_cta - 1) / teams_per_cta;
      const int64_t max_blocks = static_cast<int64_t>(per_sm) * cfg.sms;
      if (blocks > max_blocks) blocks = max_blocks;
      cfg.grid = static_cast<int>(blocks < 1 ? 1 : blocks);
    }
    const int64_t cb = (rp.O + kCombineWarps - 1) / kCombineWarps;   // a warp per output
    cfg.combine_grid = static_cast<int>(cb < 4LL * cfg.sms ? (cb > 0 ? cb : 1) : 4LL * cfg.sms);
    cfg.ready = true;
  }
  if (rp.items == 0) return HP_OK;
  rp.M = cfg.M;
  Out* out = static_cast<Out*>(a.out);
  Acc* part = static_cast<Acc*>(a.part);
  if (block) {
    cudaLaunchConfig_t lc = {};
    cudaLaunchAttribute at[1];
    lc.gridDim = dim3(cfg.grid);
    lc.blockDim = dim3(cfg.threads);
    lc.stream = a.stream;
    if (cfg.cluster > 1) {
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = cfg.cluster;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      lc.attrs = at;
      lc.numAttrs = 1;
    }
    if constexpr (kPipeable) {
      if (pipe) {
        lc.dynamicSmemBytes = dyn;
        e = cudaLaunchKernelEx(&lc, kp, rp, body.A, body.wptr(), out, part);
        if (e != cudaSuccess) return cuda_fail(e, "rect_block_pipe_kernel launch");
      } else {
        e = cudaLaunchKernelEx(&lc, kb, rp, body, out, part);
        if (e != cudaSuccess) return cuda_fail(e, "rect_block_kernel launch");
      }
    } else {
      e = cudaLaunchKernelEx(&lc, kb, rp, body, out, part);
      if (e != cudaSuccess) return cuda_fail(e, "rect_block_kernel launch");
    }
  } else {
    kl<<<cfg.grid, cfg.threads, 0, a.stream>>>(rp, body, out, part);
    e = cudaPeekAtLastError();
    if (e != cudaSuccess) return cuda_fail(e, "rect_lanes_kernel launch");
  }
  if (rp.G > 1) {
    rect_combine_kernel<Op><<<cfg.combine_grid, 32 * kCombineWarps, 0, a.stream>>>(rp.O, rp.G, part, out, a.comp);
    e = cudaPeekAtLastError();
    if (e != cudaSuccess) return cuda_fail(e, "rect_combine_kernel launch");
  }
  (void)np;
  return HP_OK;
}

template <class Op, class Body>
hp_status launch_v(const NestPlan& np, const RectPlan& rp, LaunchCfg& cfg, const Body& body, const RectArgs& a) {
  if (rp.V == 4) return launch_team<Op, 4>(np, rp, cfg, body, a);
  return launch_team<Op, 1>(np, rp, cfg, body, a);
}

// Entry for one accumulation policy: pick the body.
template <class Op>
hp_status launch_rect(const NestPlan& np, LaunchCfg& cfg, const RectArgs& a) {
  const RectPlan& rp = np.rp;
  using In = typename Op::In;
  switch (np.body) {
    case HP_BODY_LOAD: {
      BodyLoad<Op> b{static_cast<const In*>(a.in[0])};
      return launch_v<Op>(np, rp, cfg, b, a);
    }
    case HP_BODY_DOT_BCAST: {
      BodyDot<Op> b{static_cast<const In*>(a.in[0]), static_cast<const In*>(a.in[1])};
      return launch_v<Op>(np, rp, cfg, b, a);
    }
    case HP_BODY_AFFINE: {
      BodyAffine<Op> b;
      b.a = rp.aff_a;
      b.b = rp.aff_b;
      b.m = rp.aff_m;
      return launch_v<Op>(np, rp, cfg, b, a);
    }
    case HP_BODY_GEOMETRIC: {
      if constexpr (Op::kFp && sizeof(typename Op::Out) == 4) {
        BodyGeo<Op> b;
        b.table = a.geo;
        b.m = rp.geo_m;
        return launch_v<Op>(np, rp, cfg, b, a);
      }
      return fail(HP_EUNSUPPORTED, "GEOMETRIC body needs an FP precision");
    }
    default:
      return fail(HP_EUNSUPPORTED, "body not supported by the rectangular executor");
  }
}

// explicit instantiations live in rect_f32.cu, rect_f32mm.cu, rect_i32.cu, rect_i64.cu
hp_status launch_rect_f32_sum(const NestPlan&, LaunchCfg&, const RectArgs&);
hp_status launch_rect_f32_comp(const NestPlan&, LaunchCfg&, const RectArgs&);
hp_status launch_rect_f32_max(const NestPlan&, LaunchCfg&, const RectArgs&);
hp_status launch_rect_f32_min(const NestPlan&, LaunchCfg&, const RectArgs&);
hp_status launch_rect_i32_sum(const NestPlan&, LaunchCfg&, const RectArgs&);
hp_status launch_rect_i32_max(const NestPlan&, LaunchCfg&, const RectArgs&);
hp_status launch_rect_i32_min(const NestPlan&, LaunchCfg&, const RectArgs&);
hp_status launch_rect_i64_sum(const NestPlan&, LaunchCfg&, const RectArgs&);
hp_status launch_rect_i64_max(const NestPlan&, LaunchCfg&, const RectArgs&);
hp_status launch_rect_i64_min(const NestPlan&, LaunchCfg&, const RectArgs&);

// size in bytes of one grid-part partial for a precision / op
inline size_t partial_bytes(hp_prec prec, hp_red_op op) {
  if (prec == HP_F32_COMP && op == HP_RED_SUM) return 8;
  if (prec == HP_I64) return 8;
  return 4;
}

}  // namespace hp
