// api_internal.h — the nest object behind the opaque hp_nest handle.
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "hp_internal.h"

namespace hp {
enum NestKind : int { NEST_RECT = 0, NEST_CSR = 1, NEST_ORDERED = 2, NEST_NARROW = 3 };
struct CsrState;
}  // namespace hp

struct hp_nest {
  int kind = hp::NEST_RECT;
  hp::NestPlan plan;          // rectangular nests
  hp::CsrPlan csr;            // CSR nests
  hp::OrderedPlan ord;        // nests with an ordered (non-commutative) reduction
  hp::NarrowPlan nar;         // nests on 8- / 16-bit integers
  int32_t* tickets = nullptr; // per output, ordered nests split over grid parts
  hp::LaunchCfg cfg;
  int device = -1;            // device of the first run; -1 before it
  int sms = 0;
  void* part = nullptr;       // grid-part partials
  size_t part_bytes = 0;
  float* geo = nullptr;       // GEOMETRIC body table
  int32_t* err = nullptr;     // device error word (bounded waits)
  void* stage_in[2] = {nullptr, nullptr};   // hp_nest_run_host staging
  size_t stage_in_bytes[2] = {0, 0};
  void* stage_out = nullptr;
  size_t stage_out_bytes = 0;
  hp::CsrState* cs = nullptr; // CSR device state
  uint64_t plan_id = 0;       // process-unique id of the current plan (new at create and when tuning replaces it)
};

namespace hp {
uint64_t next_plan_id();
void batch_forget(const hp_nest* n);   // drop cached batch contexts that contain n
hp_status ensure_device(hp_nest* n);
hp_status run_rect(hp_nest* n, const void* const* in_dev, void* out_dev, cudaStream_t st);
hp_status run_rect_with(hp_nest* n, const void* const* in_dev, void* out_dev, void* part, cudaStream_t st,
                        float* comp = nullptr);
size_t out_bytes(const hp_nest* n);
double error_bound(const hp_nest* n);

// CSR nests (csr.cu)
hp_status plan_csr(int depth, int64_t n_rows, const hp_level_map* map, hp_red_op op, int red_level, hp_prec prec,
                   hp_body body, const void* body_params, CsrPlan* out, std::string* why);
std::string describe_csr(const CsrPlan& p);
hp_status csr_prepare(hp_nest* n);
hp_status run_csr(hp_nest* n, const void* const* in_dev, void* out_dev, cudaStream_t st);
size_t csr_out_bytes(const hp_nest* n);
void csr_release(hp_nest* n);

// ordered reductions (ordered.cu)
hp_status plan_ordered(int depth, const int64_t* extents, const hp_level_map* map, hp_red_op op, int red_level,
                       hp_prec prec, hp_body body, OrderedPlan* out, std::string* why);
std::string describe_ordered(const OrderedPlan& p);
hp_status ordered_prepare(hp_nest* n);
hp_status run_ordered(hp_nest* n, const void* const* in_dev, void* out_dev, cudaStream_t st);
size_t ordered_out_bytes(const OrderedPlan& p);

// nests on 8- / 16-bit integers (narrow.cu)
hp_status plan_narrow(int depth, const int64_t* extents, const hp_level_map* map, hp_red_op op, int red_level,
                      hp_prec prec, hp_body body, NarrowPlan* out, std::string* why);
std::string describe_narrow(const NarrowPlan& p);
hp_status narrow_prepare(hp_nest* n);
hp_status run_narrow(hp_nest* n, const void* const* in_dev, void* out_dev, cudaStream_t st);
}  // namespace hp
