// batch_int.cu — the persistent batched kernel for the int32 arithmetics, and
// the dispatch over all arithmetics.
#include "batch_kernels.cuh"

namespace hp {
cudaError_t launch_batch_fp(int combo, const BatchLaunch& b, cudaStream_t st);
int batch_fp_blocks_per_sm(int combo);
cudaError_t launch_batch_i64(int combo, const BatchLaunch& b, cudaStream_t st);
int batch_i64_blocks_per_sm(int combo);

cudaError_t launch_batch_combo(int combo, const BatchLaunch& b, cudaStream_t st) {
  switch (combo) {
    case 4: return launch_batch_op<OpI32Sum>(b, st);
    case 5: return launch_batch_op<OpI32Max>(b, st);
    case 6: return launch_batch_op<OpI32Min>(b, st);
    case 7:
    case 8:
    case 9: return launch_batch_i64(combo, b, st);
    default: return launch_batch_fp(combo, b, st);
  }
}

int batch_combo_blocks_per_sm(int combo) {
  switch (combo) {
    case 4: return batch_blocks_per_sm<OpI32Sum>();
    case 5: return batch_blocks_per_sm<OpI32Max>();
    case 6: return batch_blocks_per_sm<OpI32Min>();
    case 7:
    case 8:
    case 9: return batch_i64_blocks_per_sm(combo);
    default: return batch_fp_blocks_per_sm(combo);
  }
}
}  // namespace hp
