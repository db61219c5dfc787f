// plan.cpp — validation of nest descriptors and level -> hardware maps, and
// lowering of a map onto the executor's team / slot / grid-part structure.
// Pure host code: creating a nest never touches the GPU.
//
// Lowering (Sec. 3.1 level clause with collapse; Sec. 3.3 reserve: outer nest
// levels take the coarser hardware levels, inner ones the finer; Sec. 3.4
// strip-mining of the iterations left over; Sec. 3.8 sub-warp partitions):
//   * consecutive nest levels bound to the same hardware level collapse into
//     one virtual level; a virtual level covers its hardware level and every
//     finer one down to the next virtual level's;
//   * the first reduced level's hardware level decides the team that combines
//     one output: a cluster or CTA (TEAM_BLOCK), a warp, a sub-warp group or a
//     single thread (TEAM_LANES);
//   * within a virtual level, iteration x goes to slot x mod P (finest hardware
//     coordinate fastest, so neighbouring lanes read neighbouring elements) and
//     step x div P; a reduced level bound to GRID is cut into G contiguous
//     parts that are combined by a second, fixed-order pass.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <functional>
#include <map>
#include <mutex>
#include <sstream>
#include <tuple>

#include <cuda_runtime.h>

#include "hp_internal.h"

namespace hp {

namespace {
thread_local std::string g_last_error;

const char* hw_name(int hw) {
  static const char* names[] = {"grid", "cluster", "cta", "warp", "subwarp", "lane", "seq", "auto"};
  return (hw >= 0 && hw <= 7) ? names[hw] : "?";
}

const char* team_name(int t) {
  return t == TEAM_BLOCK ? "block" : t == TEAM_LANES ? "lanes" : "map";
}

bool is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }

// Auto-map heuristics assume a full GB300 (152 SMs); the grid itself is sized
// from the real device at the first run.
constexpr int64_t kAssumedSMs = 152;
constexpr int64_t kMinPart = 16384;   // smallest grid part the planner picks by itself
#ifndef HP_PLAN_TEAMS_PER_SM
#define HP_PLAN_TEAMS_PER_SM 4          // block teams per SM a grid split aims at
#endif
}  // namespace

Options& options() {
  static Options o;
  return o;
}

void set_error(const std::string& msg) { g_last_error = msg; }
hp_status fail(hp_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}
const std::string& last_error_string() { return g_last_error; }

namespace {
std::mutex g_tune_mu;
std::map<TuneKey, TuneChoice> g_tune;

int32_t ceil_log2(int64_t v) {
  int32_t b = 0;
  while ((int64_t(1) << b) < v && b < 62) ++b;
  return b;
}
}  // namespace

bool TuneKey::operator<(const TuneKey& o) const {
  return std::tie(lo, lr, vec, body, prec, op, req) < std::tie(o.lo, o.lr, o.vec, o.body, o.prec, o.op, o.req);
}

// shape class: log2 buckets of outputs and reduced size, whether the reduced
// block is a whole number of 128-bit groups, body, precision, operator
TuneKey tune_key(const NestPlan& p) {
  int64_t O = 1, R = 1;
  for (int l = 0; l < p.red_level; ++l) O *= p.ext[l];
  for (int l = p.red_level; l < p.depth; ++l) R *= p.ext[l];
  return TuneKey{ceil_log2(O), ceil_log2(R), (R % 4 == 0) ? 1 : 0, static_cast<int32_t>(p.body),
                 static_cast<int32_t>(p.prec), static_cast<int32_t>(p.op)};
}

bool tune_lookup(const TuneKey& k, TuneChoice* c) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  auto it = g_tune.find(k);
  if (it == g_tune.end()) return false;
  *c = it->second;
  return true;
}

void tune_store(const TuneKey& k, const TuneChoice& c) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune[k] = c;
}

size_t tune_cache_size() {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  return g_tune.size();
}

static void auto_map(const NestPlan& p, hp_level_map* m);

// outputs over the grid; every reduced level on the chosen hardware level
// (HP_HW_AUTO: the planner's own map)
// A choice is structural (the hardware of the first reduced level and of the
// inner ones), so that a shape class's choice applies to every nest of the
// class whatever its depth; only explicit maps are tied to one depth.
void tune_apply(const NestPlan& p, const TuneChoice& c, hp_level_map* m) {
  if (c.n_map > 0) {
    if (c.n_map == p.depth) {
      for (int l = 0; l < p.depth; ++l) m[l] = c.map[l];
    } else {
      auto_map(p, m);
    }
    return;
  }
  if (c.red_hw == HP_HW_AUTO) {
    auto_map(p, m);
    return;
  }
  const int d = p.depth, r = p.red_level;
  int64_t R = 1;
  for (int l = r; l < d; ++l) R *= p.ext[l];
  for (int l = 0; l < d; ++l) m[l] = {HP_HW_GRID, 0, 0};
  if (r == d) return;
  const bool mixed = c.inner_hw != HP_HW_AUTO;
  if (c.split_parts > 0 && !mixed) {
    const int64_t tile = std::max<int64_t>(1, (R + c.split_parts - 1) / c.split_parts);
    for (int l = r; l < d; ++l) m[l] = {HP_HW_GRID, 0, l == r ? tile : 0};
    return;
  }
  if (c.split_parts > 0) {   // the first reduced level split over grid parts, the inner ones on inner_hw
    m[r] = {HP_HW_GRID, 0, std::max<int64_t>(1, (p.ext[r] + c.split_parts - 1) / c.split_parts)};
  } else {
    m[r] = {c.red_hw, c.sub, 0};
  }
  for (int l = r + 1; l < d; ++l)
    m[l] = mixed ? hp_level_map{c.inner_hw, c.inner_sub, 0} : hp_level_map{c.red_hw, c.sub, 0};
}

static void auto_map(const NestPlan& p, hp_level_map* m) {
  const int d = p.depth, r = p.red_level;
  for (int l = 0; l < d; ++l) m[l] = {HP_HW_GRID, 0, 0};
  if (r == d) return;
  int64_t O = 1, R = 1;
  for (int l = 0; l < r; ++l) O *= p.ext[l];
  for (int l = r; l < d; ++l) R *= p.ext[l];
  // Teams are sized so that every lane folds at least ~16 iterations of an
  // output: below that, the team's reduction tree and per-output bookkeeping
  // cost as much as the folds themselves.
  int red_hw;
  int sub = 0;
  if (R >= 4096) {
    red_hw = (O < 2 * kAssumedSMs && R >= 65536) ? HP_HW_GRID : HP_HW_CTA;
  } else if (R >= 512) {
    red_hw = HP_HW_WARP;
  } else if (R >= 32) {
    red_hw = HP_HW_SUBWARP;
    sub = 2;
    while (sub < 16 && sub * 2 * 16 <= R) sub *= 2;
  } else if (R % 4 == 0) {
    red_hw = HP_HW_LANE;   // one thread per output, 4 vector slots (128-bit loads)
    sub = 4;
  } else {
    red_hw = HP_HW_SEQ;
  }
  // all reduced levels collapse into one contiguous virtual level
  for (int l = r; l < d; ++l) m[l] = {red_hw, red_hw == HP_HW_SUBWARP || red_hw == HP_HW_LANE ? sub : 0, 0};
  if (r == 0 && red_hw == HP_HW_SUBWARP) {
    // a single output: one sub-warp group would leave the rest of the warp idle
    for (int l = r; l < d; ++l) m[l] = {HP_HW_WARP, 0, 0};
  }
}

hp_status plan_rect(int depth, const int64_t* extents, const hp_level_map* map, hp_red_op op, int red_level,
                    hp_prec prec, hp_body body, const void* body_params, NestPlan* out, std::string* why) {
  auto bad = [&](const std::string& s) {
    *why = s;
    return HP_EINVAL;
  };
  if (depth < 1 || depth > HP_MAX_DEPTH) return bad("depth must be in [1, 5]");
  if (!extents) return bad("extents is NULL");
  if (red_level < 0 || red_level > depth) return bad("red_level must be in [0, depth]");
  if (op != HP_RED_SUM && op != HP_RED_MAX && op != HP_RED_MIN)
    return bad("rectangular nests reduce with SUM, MAX or MIN (HIST_COUNT is for CSR nests)");
  if (prec < HP_F32 || prec > HP_I64) return bad("unknown precision");
  if (body != HP_BODY_LOAD && body != HP_BODY_DOT_BCAST && body != HP_BODY_AFFINE && body != HP_BODY_GEOMETRIC)
    return bad("rectangular nests take the LOAD, DOT_BCAST, AFFINE or GEOMETRIC body");
  NestPlan p;
  p.depth = depth;
  p.red_level = red_level;
  p.op = op;
  p.prec = prec;
  p.body = body;
  int64_t total = 1;
  for (int l = 0; l < depth; ++l) {
    if (extents[l] < 0) return bad("extents must be >= 0");
    p.ext[l] = extents[l];
    int64_t t;
    if (__builtin_mul_overflow(total, extents[l], &t) || t > (int64_t(1) << 62))
      return bad("iteration space exceeds 2^62");
    total = t;
  }
  p.total = total;
  RectPlan& rp = p.rp;
  std::memset(&rp, 0, sizeof(rp));
  rp.body = body;
  if (body == HP_BODY_AFFINE) {
    if (!body_params) return bad("AFFINE body needs hp_affine_params");
    auto* a = static_cast<const hp_affine_params*>(body_params);
    if (a->m < 1) return bad("AFFINE: m must be >= 1");
    rp.aff_a = a->a;
    rp.aff_b = a->b;
    rp.aff_m = a->m;
  } else if (body == HP_BODY_GEOMETRIC) {
    if (prec != HP_F32 && prec != HP_F32_COMP) return bad("GEOMETRIC body is an FP body");
    if (op != HP_RED_SUM) return bad("GEOMETRIC body is for sums");
    if (!body_params) return bad("GEOMETRIC body needs hp_geometric_params");
    auto* g = static_cast<const hp_geometric_params*>(body_params);
    if (g->m < 1 || g->m > kGeoMax) return bad("GEOMETRIC: m must be in [1, 1024]");
    if (!std::isfinite(g->q)) return bad("GEOMETRIC: q must be finite");
    rp.geo_m = static_cast<int32_t>(g->m);
    p.geo_table.resize(g->m);
    double v = 1.0;
    for (int64_t k = 0; k < g->m; ++k) {
      p.geo_table[k] = static_cast<float>(v);
      v *= g->q;
    }
  }
  p.n_inputs = body == HP_BODY_LOAD ? 1 : body == HP_BODY_DOT_BCAST ? 2 : 0;
  const bool int_prec = prec == HP_I32 || prec == HP_I64;
  p.in_elem_bytes = 4;
  p.out_elem_bytes = prec == HP_I64 ? 8 : 4;
  (void)int_prec;

  // ---- the level map
  bool all_auto = (map == nullptr);
  if (map) {
    all_auto = true;
    bool any_auto = false;
    for (int l = 0; l < depth; ++l) {
      if (map[l].hw == HP_HW_AUTO) any_auto = true;
      else all_auto = false;
    }
    if (any_auto && !all_auto) return bad("HP_HW_AUTO must be given for every level or for none");
  }
  p.auto_map = all_auto;
  if (all_auto) {
    TuneChoice tc;
    if (red_level < depth && tune_lookup(tune_key(p), &tc)) {
      // the shape class's tuned binding, if it is legal for this nest's own
      // levels (a class spans several depths); else the planner's map
      hp_level_map tm[HP_MAX_DEPTH];
      tune_apply(p, tc, tm);
      NestPlan tp;
      std::string twhy;
      if (plan_rect(depth, extents, tm, op, red_level, prec, body, body_params, &tp, &twhy) == HP_OK) {
        tp.auto_map = true;
        tp.tuned = true;
        *out = tp;
        return HP_OK;
      }
    }
    auto_map(p, p.map);
  }
  else
    for (int l = 0; l < depth; ++l) p.map[l] = map[l];

  const hp_level_map* m = p.map;
  for (int l = 0; l < depth; ++l) {
    if (m[l].hw < HP_HW_GRID || m[l].hw > HP_HW_SEQ) return bad("level " + std::to_string(l) + ": unknown hardware level");
    if (l > 0 && m[l].hw < m[l - 1].hw)
      return bad("level " + std::to_string(l) + " is bound to a coarser hardware level than level " +
                 std::to_string(l - 1) + " (inner levels take finer hardware, Sec. 3.3 reserve)");
    if (m[l].tile < 0) return bad("tile must be >= 0");
  }
  // widths
  int C = 1, W = 8, grp_lanes = 32, Vreq = 4;
  bool has_cluster = false, has_cta = false, has_sub = false, has_lane_map = false;
  for (int l = 0; l < depth; ++l) {
    const int hw = m[l].hw, sw = m[l].sub_width;
    if (hw == HP_HW_CLUSTER && !has_cluster) {
      has_cluster = true;
      C = sw ? sw : 8;
      if (C < 1 || C > 16) return bad("CLUSTER sub_width (CTAs per cluster) must be in [1, 16]");
    } else if (hw == HP_HW_CLUSTER && sw && sw != C) {
      return bad("all levels bound to CLUSTER must give the same cluster size");
    }
    if (hw == HP_HW_CTA && !has_cta) {
      has_cta = true;
      W = sw ? sw : 8;
      if (W < 1 || W > kMaxWarps) return bad("CTA sub_width (warps per CTA) must be in [1, 32]");
    } else if (hw == HP_HW_CTA && sw && sw != W) {
      return bad("all levels bound to CTA must give the same warp count");
    }
    if (hw == HP_HW_SUBWARP) {
      if (!is_pow2(sw) || sw > 32) return bad("SUBWARP sub_width must be 1, 2, 4, 8, 16 or 32");
      if (has_sub && sw != grp_lanes) return bad("all levels bound to SUBWARP must give the same width");
      has_sub = true;
      grp_lanes = sw;
    }
    if (hw == HP_HW_LANE && !has_lane_map) {
      has_lane_map = true;
      Vreq = sw ? sw : 4;
      if (Vreq != 1 && Vreq != 4) return bad("LANE sub_width (vector slots) must be 1 or 4");
    }
  }
  const int d = depth, r = red_level;
  int64_t O = 1, R = 1;
  for (int l = 0; l < r; ++l) O *= p.ext[l];
  for (int l = r; l < d; ++l) R *= p.ext[l];
  rp.O = O;
  rp.R = R;
  rp.W = W;
  rp.C = 1;
  rp.grp_lanes = grp_lanes;
  rp.V = 1;
  rp.G = 1;
  rp.L = 32;
  rp.M = 1;
  p.in_elems[0] = total;
  p.in_elems[1] = body == HP_BODY_DOT_BCAST ? R : 0;

  if (r == d) {
    rp.team = TEAM_MAP;
    rp.items = O;
    rp.nv = 0;
    rp.V = (body == HP_BODY_LOAD || body == HP_BODY_DOT_BCAST) ? 4 : 1;
    p.kernel = "rect_map";
    *out = p;
    return HP_OK;
  }

  // ---- team
  const int T = m[r].hw;
  for (int l = 0; l < r; ++l) {
    if (m[l].hw == T && T != HP_HW_GRID)
      return bad("output level " + std::to_string(l) + " and the first reduced level are both bound to " +
                 hw_name(T) + ": a reduction must sit below the output levels it serves (only GRID may split one)");
  }
  if (T <= HP_HW_CTA) {
    rp.team = TEAM_BLOCK;
    // the cluster is the team when a reduced level covers the cluster scope
    bool red_covers_cluster = false;
    for (int l = r; l < d; ++l) {
      const int lo = m[l].hw;
      const int hi = (l + 1 < d) ? m[l + 1].hw : HP_HW_SEQ + 1;
      if (lo <= HP_HW_CLUSTER && HP_HW_CLUSTER < hi) red_covers_cluster = true;
    }
    rp.C = (red_covers_cluster && has_cluster) ? C : 1;
    rp.L = 32;
  } else {
    rp.team = TEAM_LANES;
    rp.L = (T == HP_HW_WARP) ? 32 : (T == HP_HW_SUBWARP) ? grp_lanes : 1;
    rp.C = 1;
  }
  if (rp.team == TEAM_LANES && T == HP_HW_SUBWARP) {
    // the sub-warp group is the team; no finer groups inside
  }

  // ---- reduced virtual levels
  struct VL {
    int hw;
    int64_t n;
    int64_t stride;
    int first, last;
  };
  std::vector<VL> vls;
  for (int l = r; l < d; ++l) {
    if (!vls.empty() && vls.back().hw == m[l].hw) {
      vls.back().n *= p.ext[l];
      vls.back().last = l;
    } else {
      vls.push_back({m[l].hw, p.ext[l], 1, l, l});
    }
  }
  {
    int64_t s = 1;
    for (int v = static_cast<int>(vls.size()) - 1; v >= 0; --v) {
      vls[v].stride = s;
      s *= vls[v].n;
    }
  }
  const int nv = static_cast<int>(vls.size());
  if (nv > kMaxV) return bad("too many reduced levels");
  rp.nv = nv;

  // which virtual level covers the LANE scope, and does it get vector slots?
  int lane_level = -1;
  for (int v = 0; v < nv; ++v) {
    const int lo = vls[v].hw;
    const int hi = (v + 1 < nv) ? vls[v + 1].hw : HP_HW_SEQ + 1;
    if (lo <= HP_HW_LANE && HP_HW_LANE < hi) lane_level = v;
  }
  int V = 1;
  if (lane_level == nv - 1) {
    V = Vreq;
    // vector slots fold V consecutive iterations at once: the innermost run
    // must be a whole number of vectors (for memory bodies: 128-bit loads)
    if ((vls[nv - 1].n % V) != 0) V = 1;
  }
  rp.V = V;

  // split over the grid
  rp.split = 0;
  rp.G = 1;
  rp.tile = 0;
  if (vls[0].hw == HP_HW_GRID) {
    rp.split = 1;
    const int64_t n0 = vls[0].n;
    int64_t tile = 0;
    for (int l = vls[0].first; l <= vls[0].last; ++l)
      if (m[l].tile > 0) tile = m[l].tile;
    if (tile <= 0) {
      // aim at about four block teams per SM over all outputs (two left a
      // 1 GiB single-output sum at 3.7 TB/s, four reach 5.7), with parts of
      // at least kMinPart iterations (a part's reduction tree and its ticket
      // cost about as much as folding a few thousand iterations)
      const int64_t teams = HP_PLAN_TEAMS_PER_SM * kAssumedSMs;
      int64_t want_parts = std::max<int64_t>(1, (teams + O - 1) / std::max<int64_t>(O, 1));
      want_parts = std::min<int64_t>(want_parts, std::max<int64_t>(1, n0 / kMinPart));
      tile = (n0 + want_parts - 1) / std::max<int64_t>(want_parts, 1);
    }
    if (nv == 1 && V > 1) tile = (tile + V - 1) / V * V;
    if (tile < 1) tile = 1;
    int64_t G = n0 > 0 ? (n0 + tile - 1) / tile : 1;
    if (G > (int64_t(1) << 30)) return bad("too many grid parts");
    rp.G = static_cast<int32_t>(G);
    rp.tile = tile;
  }

  // slot coefficients (finest scope fastest)
  const bool team_block = rp.team == TEAM_BLOCK;
  for (int v = 0; v < nv; ++v) {
    const int lo = vls[v].hw;
    const int hi = (v + 1 < nv) ? vls[v + 1].hw : HP_HW_SEQ + 1;
    int64_t mult = (v == nv - 1) ? V : 1;  // vector slots are the finest coordinate of the innermost level
    rp.cr[v] = rp.cw[v] = rp.cg[v] = rp.cl[v] = 0;
    for (int s = std::min(hi - 1, static_cast<int>(HP_HW_LANE)); s >= lo; --s) {
      switch (s) {
        case HP_HW_LANE:
          break;  // handled by V on the innermost level; 1 slot elsewhere
        case HP_HW_SUBWARP:
          if (has_sub && (team_block || T <= HP_HW_SUBWARP)) {
            rp.cl[v] = static_cast<int32_t>(mult);
            mult *= grp_lanes;
          }
          break;
        case HP_HW_WARP:
          if (team_block || T <= HP_HW_WARP) {
            if (has_sub) {
              rp.cg[v] = static_cast<int32_t>(mult);
              mult *= 32 / grp_lanes;
            } else {
              rp.cl[v] = static_cast<int32_t>(mult);
              mult *= 32;
            }
          }
          break;
        case HP_HW_CTA:
          if (team_block) {
            rp.cw[v] = static_cast<int32_t>(mult);
            mult *= W;
          }
          break;
        case HP_HW_CLUSTER:
          if (team_block && rp.C > 1) {
            rp.cr[v] = static_cast<int32_t>(mult);
            mult *= rp.C;
          }
          break;
        default:
          break;
      }
    }
    if (mult > (int64_t(1) << 30)) return bad("too many parallel slots on one level");
    rp.vP[v] = static_cast<int32_t>(mult);
    rp.vn[v] = vls[v].n;
    rp.vstride[v] = vls[v].stride;
  }
  // team lanes: the number of lanes inside one team
  if (rp.team == TEAM_LANES) {
    if (T == HP_HW_SUBWARP) rp.grp_lanes = rp.L;     // no finer groups inside a sub-warp team
    if (T >= HP_HW_LANE) rp.grp_lanes = 1;
  }
  int64_t items;
  if (__builtin_mul_overflow(O, static_cast<int64_t>(rp.G), &items)) return bad("too many work items");
  rp.items = items;
  rp.M = 1;
  // element groups per thread per item: the thread with slot 0 on every level has the most
  int64_t groups = 1;
  for (int v = 0; v < nv; ++v) {
    const int64_t n = (rp.split && v == 0) ? rp.tile : rp.vn[v];
    groups *= (n + rp.vP[v] - 1) / rp.vP[v];
    if (groups > (int64_t(1) << 30)) groups = int64_t(1) << 30;
  }
  rp.groups = static_cast<int32_t>(groups);
  const bool mem_body = body == HP_BODY_LOAD || body == HP_BODY_DOT_BCAST;
  rp.pipe = (options().pipeline != 0 && team_block && rp.V == 4 && mem_body && rp.G == 1 && rp.W <= 8 &&
             R < (int64_t(1) << 31) && groups <= kPipeGroupsMax)
                ? 1
                : 0;
  p.kernel = team_block ? (rp.pipe ? (rp.C > 1 ? "rect_block_pipe_cluster" : "rect_block_pipe")
                                   : (rp.C > 1 ? "rect_block_cluster" : "rect_block"))
                        : "rect_lanes";
  *out = p;
  return HP_OK;
}

std::string describe_plan(const NestPlan& p) {
  std::ostringstream s;
  const RectPlan& rp = p.rp;
  s << "{\"kind\":\"rect\",\"depth\":" << p.depth << ",\"red_level\":" << p.red_level << ",\"extents\":[";
  for (int l = 0; l < p.depth; ++l) s << (l ? "," : "") << p.ext[l];
  s << "],\"map\":[";
  for (int l = 0; l < p.depth; ++l)
    s << (l ? "," : "") << "{\"hw\":\"" << hw_name(p.map[l].hw) << "\",\"sub_width\":" << p.map[l].sub_width
      << ",\"tile\":" << p.map[l].tile << "}";
  s << "],\"auto_map\":" << (p.auto_map ? "true" : "false") << ",\"tuned\":" << (p.tuned ? "true" : "false")
    << ",\"team\":\"" << team_name(rp.team)
    << "\",\"outputs\":" << rp.O << ",\"reduced\":" << rp.R << ",\"items\":" << rp.items
    << ",\"cluster\":" << rp.C << ",\"warps\":" << rp.W << ",\"team_lanes\":" << rp.L
    << ",\"group_lanes\":" << rp.grp_lanes << ",\"vec\":" << rp.V << ",\"grid_parts\":" << rp.G
    << ",\"tile\":" << rp.tile << ",\"groups\":" << rp.groups << ",\"pipe\":" << rp.pipe << ",\"levels\":[";
  for (int v = 0; v < rp.nv; ++v)
    s << (v ? "," : "") << "{\"n\":" << rp.vn[v] << ",\"stride\":" << rp.vstride[v] << ",\"slots\":" << rp.vP[v]
      << ",\"c_rank\":" << rp.cr[v] << ",\"c_warp\":" << rp.cw[v] << ",\"c_group\":" << rp.cg[v]
      << ",\"c_lane\":" << rp.cl[v] << "}";
  s << "],\"kernel\":\"" << p.kernel << "\"}";
  return s.str();
}

}  // namespace hp

namespace hp {

// Normwise a-priori bound: |got - exact| <= bound * sum|t|.
//   plain FP32: gamma_k with k = the longest chain of roundings one term goes
//   through (its thread's sequential share, the vector fold, the lane
//   butterfly, the warp / rank / grid-part folds);
//   compensated FP32 (Dot2): u + gamma_k^2, plus, with G > 1 grid parts, the
//   double-float part combine's gamma_2G (gamma_G + 2 gamma_k).
double error_bound_rect(const NestPlan& p) {
  const RectPlan& rp = p.rp;
  if (p.prec == HP_I32 || p.prec == HP_I64 || p.op != HP_RED_SUM || rp.team == TEAM_MAP) return 0.0;
  const double u = std::ldexp(1.0, -24);
  int64_t seq = 1;
  for (int v = 0; v < rp.nv; ++v) {
    int64_t n = rp.vn[v];
    if (rp.split && v == 0) n = rp.tile;
    seq *= (n + rp.vP[v] - 1) / std::max<int64_t>(rp.vP[v], 1);
  }
  int64_t k = seq + 2 /*vector*/ + 5 /*butterfly*/;
  if (rp.team == TEAM_BLOCK) k += rp.W + rp.C;
  if (p.prec == HP_F32) k += rp.G;
  const double g = (k * u) / (1.0 - k * u);
  if (p.prec == HP_F32) return g;
  double combine = 0.0;
  if (rp.G > 1) {
    const auto gamma = [&](double n) { return (n * u) / (1.0 - n * u); };
    combine = gamma(2.0 * rp.G) * (gamma(static_cast<double>(rp.G)) + 2.0 * g);
  }
  return u + g * g + combine;
}

}  // namespace hp

// ---------------------------------------------------------------- level selection by property
// Sec. 3.2 (sync clause, the table of level properties) and Sec. 3.3 (reserve).
namespace hp {
namespace {

struct LevelCaps {
  hp_hw hw;
  uint32_t props;
};

// GB300 as this executor uses it, coarsest first.  GRID: CTAs are time-shared
// (not all resident), have no barrier and no forward-progress guarantee among
// each other, reach L2 and global memory, and take work from atomic queues.
// CLUSTER: co-scheduled CTAs with a hardware barrier and distributed shared
// memory.  CTA: warps with __syncthreads, shared memory and L1.  WARP: lanes
// with __syncwarp and shuffles, independent thread scheduling, registers per
// lane.  LANE: the vector slots of one thread, advancing in lockstep.  SEQ: a
// thread's sequential loop.
constexpr uint32_t P(hp_prop p) { return static_cast<uint32_t>(p); }
const LevelCaps kCaps[] = {
    {HP_HW_GRID, P(HP_PROP_ATOMIC) | P(HP_PROP_OVERSUB) | P(HP_PROP_DYNAMIC) | P(HP_PROP_GLOBALMEM) | P(HP_PROP_CACHE)},
    {HP_HW_CLUSTER, P(HP_PROP_BARRIER) | P(HP_PROP_CRITICAL) | P(HP_PROP_ATOMIC) | P(HP_PROP_PROGRESS) |
                        P(HP_PROP_GLOBALMEM) | P(HP_PROP_LOCALMEM)},
    {HP_HW_CTA, P(HP_PROP_BARRIER) | P(HP_PROP_CRITICAL) | P(HP_PROP_ATOMIC) | P(HP_PROP_PROGRESS) |
                    P(HP_PROP_GLOBALMEM) | P(HP_PROP_LOCALMEM) | P(HP_PROP_CACHE)},
    {HP_HW_WARP, P(HP_PROP_BARRIER) | P(HP_PROP_CRITICAL) | P(HP_PROP_ATOMIC) | P(HP_PROP_SHUFFLE) |
                     P(HP_PROP_PROGRESS) | P(HP_PROP_GLOBALMEM) | P(HP_PROP_GROUPMEM)},
    {HP_HW_LANE, P(HP_PROP_LOCKSTEP) | P(HP_PROP_GLOBALMEM) | P(HP_PROP_GROUPMEM)},
    {HP_HW_SEQ, P(HP_PROP_LOCKSTEP) | P(HP_PROP_GLOBALMEM) | P(HP_PROP_GROUPMEM)},
};
constexpr int kNumCaps = sizeof(kCaps) / sizeof(kCaps[0]);

int device_sms() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
      sms > 0)
    return sms;
  cudaGetLastError();   // no device: GB300's count
  return static_cast<int>(kAssumedSMs);
}

int64_t level_num(hp_hw hw, int sub) {
  switch (hw) {
    case HP_HW_GRID: return static_cast<int64_t>(device_sms()) * 8;   // CTAs of 256 threads resident
    case HP_HW_CLUSTER: return 8;                                      // portable cluster size (16 opt-in)
    case HP_HW_CTA: return 32;                                         // warps
    case HP_HW_WARP: return 32;                                        // lanes
    case HP_HW_SUBWARP: return sub > 0 ? sub : 16;
    case HP_HW_LANE: return 4;                                         // 128-bit vector slots
    default: return 1;
  }
}

uint32_t level_props(hp_hw hw) {
  if (hw == HP_HW_SUBWARP) return kCaps[3].props;   // a partition of the warp keeps its properties (Sec. 3.8)
  for (const LevelCaps& c : kCaps)
    if (c.hw == hw) return c.props;
  return 0;
}

// coarse-to-fine position of a hardware level; a sub-warp partition sits
// between the warp and the vector slots
int level_rank(int hw) {
  switch (hw) {
    case HP_HW_GRID: return 0;
    case HP_HW_CLUSTER: return 2;
    case HP_HW_CTA: return 4;
    case HP_HW_WARP: return 6;
    case HP_HW_SUBWARP: return 7;
    case HP_HW_LANE: return 8;
    case HP_HW_SEQ: return 10;
    default: return -1;
  }
}

}  // namespace

bool map_meets(int depth, const hp_level_req* req, const hp_level_map* map, std::string* why) {
  for (int l = 0; l < depth; ++l) {
    const hp_level_req& r = req[l];
    const int hw = map[l].hw;
    const int rank = level_rank(hw);
    auto no = [&](const std::string& m) {
      *why = "level " + std::to_string(l) + ": " + m;
      return false;
    };
    if (rank < 0) return no("not a hardware level (AUTO maps are checked after planning)");
    if (l > 0) {
      const int prev = level_rank(map[l - 1].hw);
      if (rank < prev) return no("coarser than its enclosing level");
      if (req[l - 1].reserve && rank == prev) return no("on the level its enclosing level reserves parallelism below");
      if (hw == HP_HW_SUBWARP && map[l - 1].hw == HP_HW_SUBWARP && map[l].sub_width > map[l - 1].sub_width)
        return no("a sub-warp partition wider than its enclosing one");
    }
    const uint32_t props = level_props(static_cast<hp_hw>(hw));
    if ((props & r.sync) != r.sync) return no("its hardware level lacks a required sync property");
    // tasks of the level: the team's size where the map fixes one (CTA warps,
    // sub-warp width, vector slots), else the level's capacity
    const int sub = map[l].sub_width;
    const int64_t num = (sub > 0 && (hw == HP_HW_CTA || hw == HP_HW_SUBWARP || hw == HP_HW_LANE))
                            ? sub : level_num(static_cast<hp_hw>(hw), 0);
    if (r.min_num > 0 && num < r.min_num) return no("fewer parallel tasks than min_num");
    if (r.reserve) {
      if ((props & r.reserve) == r.reserve) return no("its hardware level has the properties it reserves");
      bool left = false;
      for (const LevelCaps& c : kCaps) left = left || (level_rank(c.hw) > rank && (c.props & r.reserve) == r.reserve);
      if (!left) return no("no finer hardware level has the reserved properties");
    }
  }
  return true;
}

}  // namespace hp

using namespace hp;

extern "C" hp_status hp_level_properties(hp_hw hw, uint32_t* props, int64_t* num) {
  if (!props || !num) return fail(HP_EINVAL, "NULL argument");
  if (hw < HP_HW_GRID || hw > HP_HW_SEQ) return fail(HP_EINVAL, "hw must be a hardware level (not AUTO)");
  *props = level_props(hw);
  *num = level_num(hw, 0);
  return HP_OK;
}

extern "C" hp_status hp_level_check(int depth, const hp_level_req* req, const hp_level_map* map) {
  if (depth < 1 || depth > HP_MAX_DEPTH) return fail(HP_EINVAL, "depth must be in [1, HP_MAX_DEPTH]");
  if (!req || !map) return fail(HP_EINVAL, "NULL argument");
  std::string why;
  if (!map_meets(depth, req, map, &why)) return fail(HP_EINVAL, why);
  set_error("");
  return HP_OK;
}

extern "C" hp_status hp_level_select(int depth, const hp_level_req* req, hp_level_map* map_out) {
  if (depth < 1 || depth > HP_MAX_DEPTH) return fail(HP_EINVAL, "depth must be in [1, HP_MAX_DEPTH]");
  if (!req || !map_out) return fail(HP_EINVAL, "NULL argument");
  // wcap: the lanes a level at the warp's index may use (32, or the width of
  // the enclosing sub-warp partition it collapses onto); w: the lanes it takes
  auto fits = [&](int l, int h, int w) {
    const hp_level_req& r = req[l];
    if ((kCaps[h].props & r.sync) != r.sync) return false;
    const int64_t num = kCaps[h].hw == HP_HW_WARP ? w : level_num(kCaps[h].hw, 0);
    if (r.min_num > 0 && num < r.min_num) return false;
    if (r.reserve) {
      // Sec. 3.3: the level uses every hardware level except those with the
      // reserved properties, which a strictly finer level must still offer
      if ((kCaps[h].props & r.reserve) == r.reserve) return false;
      bool left = false;
      for (int f = h + 1; f < kNumCaps && !left; ++f) left = (kCaps[f].props & r.reserve) == r.reserve;
      if (!left) return false;
    }
    return true;
  };
  // the partitions a level may take at index h, in order of preference: at the
  // warp's index the narrowest power-of-two sub-warp with min_num lanes first
  // (Sec. 3.8), wider ones up to the whole warp if its inner levels need them,
  // or only the enclosing partition it collapses onto
  auto widths = [&](int l, int h, int wcap) {
    std::vector<int> ws;
    if (kCaps[h].hw != HP_HW_WARP) {
      ws.push_back(32);
    } else if (wcap < 32) {
      ws.push_back(wcap);
    } else {
      const int64_t mn = req[l].min_num;
      int w = 32;
      if (mn > 0 && mn < 32) {
        w = 2;
        while (w < mn) w *= 2;
      }
      for (; w <= 32; w *= 2) ws.push_back(w);
    }
    return ws;
  };
  // inner levels start at the same hardware level (collapse, keeping a
  // sub-warp partition) or, below a level that reserves parallelism, strictly
  // below it
  auto next_lo = [&](int l, int h) { return req[l].reserve ? h + 1 : h; };
  auto next_w = [&](int l, int h, int w) { return (req[l].reserve || kCaps[h].hw != HP_HW_WARP) ? 32 : w; };
  std::function<bool(int, int, int)> feasible = [&](int l, int lo, int wcap) -> bool {
    if (l == depth) return true;
    for (int h = lo; h < kNumCaps; ++h)
      for (int w : widths(l, h, wcap))
        if (fits(l, h, w) && feasible(l + 1, next_lo(l, h), next_w(l, h, w))) return true;
    return false;
  };
  int prev = 0, wcap = 32;
  for (int l = 0; l < depth; ++l) {
    int pick = -1, pw = 32;
    for (int h = prev; h < kNumCaps && pick < 0; ++h)
      for (int w : widths(l, h, wcap))
        if (pick < 0 && fits(l, h, w) && feasible(l + 1, next_lo(l, h), next_w(l, h, w))) {
          pick = h;
          pw = w;
        }
    if (pick < 0)
      return fail(HP_EINVAL, "no hardware level has the properties level " + std::to_string(l) +
                                 " needs (sync, reserve, min_num) below the levels chosen for the enclosing ones");
    map_out[l] = pw < 32 ? hp_level_map{HP_HW_SUBWARP, pw, 0} : hp_level_map{kCaps[pick].hw, 0, 0};
    prev = next_lo(l, pick);
    wcap = next_w(l, pick, pw);
  }
  set_error("");
  return HP_OK;
}
