// hp_internal.h — plan structures shared by the library's translation units.
//
// The planner (plan.cpp) turns a nest descriptor and its level -> hardware map
// into a RectPlan / CsrPlan; the kernels read the plan by value.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "hp.h"

namespace hp {

constexpr int kMaxV = HP_MAX_DEPTH;  // reduced virtual levels
constexpr int kMaxM = 32;            // items per synchronisation round of a block team
constexpr int kMaxWarps = 32;
constexpr int kGeoMax = 1024;        // GEOMETRIC table entries
constexpr int kPipeGroupsMax = 8;    // element groups per thread per item of the pipelined kernel

// Hardware scopes, coarse to fine (same order and values as hp_hw).
enum Scope : int32_t { S_GRID = 0, S_CLUSTER = 1, S_CTA = 2, S_WARP = 3, S_SUB = 4, S_LANE = 5, S_SEQ = 6 };

// Who cooperates on one output.
enum Team : int32_t {
  TEAM_BLOCK = 0,  // a cluster of C CTAs (C = 1: one CTA): reduction via shuffle, smem, DSMEM
  TEAM_LANES = 1,  // a group of L lanes of one warp (L = 32: a warp; L = 1: a thread)
  TEAM_MAP = 2,    // no reduction (red_level == depth): one output per iteration
};

// Everything the rectangular executor needs; passed by value to the kernels.
struct RectPlan {
  int64_t O;               // number of outputs
  int64_t R;               // reduced elements per output
  int64_t items;           // work items = O * G
  int64_t tile;            // iterations of virtual level 0 per grid part (split only)
  int64_t vn[kMaxV];       // extent of each reduced virtual level
  int64_t vstride[kMaxV];  // element stride of each reduced virtual level
  int32_t vP[kMaxV];       // parallel slots of each reduced virtual level
  // slot of level v = rank*cr + warp*cw + grp*cg + lig*cl (+ vec for the vector level)
  int32_t cr[kMaxV], cw[kMaxV], cg[kMaxV], cl[kMaxV];
  int32_t nv;              // number of reduced virtual levels (0 when R == 1 via no levels)
  int32_t split;           // 1: virtual level 0 is split over G grid parts
  int32_t team;            // Team
  int32_t C;               // CTAs per cluster (TEAM_BLOCK)
  int32_t W;               // warps per CTA
  int32_t L;               // lanes per team (TEAM_LANES)
  int32_t grp_lanes;       // lanes per sub-warp group inside the team (32: none)
  int32_t V;               // vector slots per thread on the innermost level (1 or 4)
  int32_t G;               // grid parts per output
  int32_t M;               // items per round (TEAM_BLOCK)
  int32_t body;            // hp_body
  int32_t pipe;            // 1: TEAM_BLOCK runs the cp.async-pipelined kernel
  int32_t groups;          // element groups per thread per item (max over threads)
  int32_t geo_m;
  int64_t aff_a, aff_b, aff_m;
  float* comp;             // compensated FP32 sums: optional residual output (out + comp = s + c), or null
};

// Host-side description of one rectangular nest's plan.
struct NestPlan {
  int depth = 0;
  int red_level = 0;
  int64_t ext[HP_MAX_DEPTH] = {0};
  hp_level_map map[HP_MAX_DEPTH] = {};
  bool auto_map = false;
  hp_red_op op = HP_RED_SUM;
  hp_prec prec = HP_F32;
  hp_body body = HP_BODY_LOAD;
  RectPlan rp = {};
  int64_t total = 0;                 // iterations
  int n_inputs = 0;                  // device inputs the body reads
  int64_t in_elems[2] = {0, 0};      // elements of each input
  size_t in_elem_bytes = 4;
  size_t out_elem_bytes = 4;
  std::vector<float> geo_table;      // GEOMETRIC body values fl32(q^k), k < m
  std::string kernel;                // name of the kernel family the plan runs
  bool tuned = false;                // map taken from the tuning cache
};

// CSR plan (ragged 2-level nests).
struct CsrPlan {
  int64_t n_rows = 0, nnz = 0, n_cols = 0, n_bins = 0;
  int32_t hist_shift = 0;
  int32_t fuse_hist = 0;
  int32_t fixed_class = -1;   // -1: rows binned by length; else every row in this class
  hp_red_op op = HP_RED_SUM;
  hp_prec prec = HP_F32;
};

// Launch geometry, fixed at the first run on a device.
struct LaunchCfg {
  bool ready = false;
  int device = -1;
  int sms = 0;
  int grid = 0;        // CTAs
  int threads = 0;     // per CTA
  int cluster = 1;     // CTAs per cluster
  int combine_grid = 0;
  int M = 1;           // items per round of a block team
};

// Plan of a nest with an ordered (non-commutative) reduction: outputs over the
// grid, each output's reduced range [0, R) (contiguous) cut into G parts of
// `part` iterations, a part folded by a team of `threads` threads, each thread
// a contiguous block of `chunk` iterations.
struct OrderedPlan {
  int depth = 0, red_level = 0;
  int64_t ext[HP_MAX_DEPTH] = {0};
  hp_level_map map[HP_MAX_DEPTH] = {};
  bool auto_map = false;
  int64_t O = 0, R = 0;       // outputs, iterations per output
  int32_t team = 0;           // 0: a warp per output; 1: a CTA of W warps per part
  int32_t W = 8;              // warps per CTA team
  int64_t G = 1, part = 0;    // grid parts per output, iterations per part
  int64_t chunk = 0;          // iterations per warp (a multiple of piece)
  int64_t piece = 8;          // a lane's iterations per round (rounds of 32 pieces per warp)
  int32_t V = 1;              // load width: 8 = 256-bit, 4 = 128-bit, 1 = scalar (R and part whole loads)
  int32_t k = 0;              // longest chain of folds and combines of one iteration
  int32_t op = HP_RED_AFFINE_COMPOSE;   // AFFINE_COMPOSE, MAT2_PRODUCT or LAST_VALID
  int32_t ib = 4;             // bytes of one iteration in each input array (16: a 2x2 matrix)
};

// Plan of a nest on 8- or 16-bit integers (SIMD sub-lanes in 32-bit
// registers): outputs over the grid, each output's reduced range [0, R)
// (contiguous) cut into G parts, a part folded by a team of `threads` threads
// taking 16-byte pieces cyclically (integer results do not depend on the order).
struct NarrowPlan {
  int depth = 0, red_level = 0;
  int64_t ext[HP_MAX_DEPTH] = {0};
  hp_level_map map[HP_MAX_DEPTH] = {};
  bool auto_map = false;
  hp_red_op op = HP_RED_SUM;
  hp_prec prec = HP_I8;
  hp_body body = HP_BODY_LOAD;
  int32_t esize = 1;          // bytes per element
  int64_t O = 0, R = 0;
  int32_t team = 0;           // 0: a warp per output; 1: a CTA of W warps per part
  int32_t W = 8;
  int64_t G = 1, part = 0;
};

// A tuned binding for a shape class (all reduced levels collapsed onto one
// hardware level, outputs over the grid).
struct TuneChoice {
  int32_t red_hw = HP_HW_AUTO;  // hardware level of the reduced levels (AUTO: the planner's map)
  int32_t sub = 0;              // SUBWARP width, LANE vector slots, CTA warps or cluster CTAs
  int64_t split_parts = 0;      // > 0: reduced levels split over this many grid parts
  int32_t inner_hw = HP_HW_AUTO;  // reduced levels after the first: their own level (AUTO: as the first)
  int32_t inner_sub = 0;
  int32_t n_map = 0;            // > 0: this explicit map instead (the map chosen from level requirements)
  hp_level_map map[HP_MAX_DEPTH] = {};
};
struct TuneKey {
  int32_t lo, lr, vec, body, prec, op;
  uint64_t req = 0;             // hash of the level requirements the choice was made under (0: none)
  bool operator<(const TuneKey& o) const;
};
TuneKey tune_key(const NestPlan& p);
bool tune_lookup(const TuneKey& k, TuneChoice* c);
void tune_store(const TuneKey& k, const TuneChoice& c);
void tune_apply(const NestPlan& p, const TuneChoice& c, hp_level_map* m);
// does the map meet the per-level requirements (the rules of hp_level_select)?
bool map_meets(int depth, const hp_level_req* req, const hp_level_map* map, std::string* why);
size_t tune_cache_size();

// Validate a rectangular nest and build its plan.  Returns HP_OK or an error
// with a message in *why.
hp_status plan_rect(int depth, const int64_t* extents, const hp_level_map* map, hp_red_op op, int red_level,
                    hp_prec prec, hp_body body, const void* body_params, NestPlan* out, std::string* why);

std::string describe_plan(const NestPlan& p);

// A-priori bound on |got - exact| / sum|t| for one FP result of the plan.
double error_bound_rect(const NestPlan& p);

// Process-wide options read when a nest is planned (hp_set_option).
struct Options {
  int64_t pipeline = 1;    // allow the cp.async-pipelined block kernel
  int64_t serve_batching = 1;  // servers created now pack admitted requests into batched steps
  int64_t tune_log = 0;    // the tuner writes each candidate's map and time to stderr
  int64_t host_zero_copy = 1;  // hp_nest_run_host reads a mapped page-locked streamed input in place
};
Options& options();

// Thread-local last-error message.
void set_error(const std::string& msg);
hp_status fail(hp_status st, const std::string& msg);

}  // namespace hp
