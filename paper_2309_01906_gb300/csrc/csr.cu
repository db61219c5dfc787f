// csr.cu — ragged (CSR) nests: planning and execution.
#include <cuda_runtime.h>

#include <sstream>
#include <string>

#include "api_internal.h"

namespace hp {

struct CsrState {
  int dummy = 0;
};

hp_status plan_csr(int depth, int64_t n_rows, const hp_level_map* map, hp_red_op op, int red_level, hp_prec prec,
                   hp_body body, const void* body_params, CsrPlan* out, std::string* why) {
  (void)map;
  if (depth != 2) {
    *why = "CSR nests have depth 2 (rows, entries)";
    return HP_EINVAL;
  }
  if (n_rows < 0) {
    *why = "n_rows must be >= 0";
    return HP_EINVAL;
  }
  if (!body_params) {
    *why = "CSR nests need hp_csr_params";
    return HP_EINVAL;
  }
  const hp_csr_params* cp = static_cast<const hp_csr_params*>(body_params);
  CsrPlan p;
  p.n_rows = n_rows;
  p.nnz = cp->nnz;
  p.n_cols = cp->n_cols;
  p.hist_shift = cp->hist_shift;
  p.fuse_hist = cp->fuse_hist;
  p.n_bins = cp->n_bins;
  p.op = op;
  p.prec = prec;
  (void)red_level;
  (void)body;
  *out = p;
  return HP_OK;
}

std::string describe_csr(const CsrPlan& p) {
  std::ostringstream s;
  s << "{\"kind\":\"csr\",\"rows\":" << p.n_rows << ",\"nnz\":" << p.nnz << "}";
  return s.str();
}

hp_status csr_prepare(hp_nest* n) {
  (void)n;
  return HP_OK;
}

hp_status run_csr(hp_nest* n, const void* const* in_dev, void* out_dev, cudaStream_t st) {
  (void)n;
  (void)in_dev;
  (void)out_dev;
  (void)st;
  return fail(HP_EUNSUPPORTED, "CSR execution is not built yet");
}

size_t csr_out_bytes(const hp_nest* n) { return static_cast<size_t>(n->csr.n_rows) * 4; }

void csr_release(hp_nest* n) {
  delete n->cs;
  n->cs = nullptr;
}

}  // namespace hp
