// batch_i64.cu — the persistent batched kernel for the int64 arithmetics.
#include "batch_kernels.cuh"

namespace hp {
cudaError_t launch_batch_i64(int combo, const BatchLaunch& b, cudaStream_t st) {
  switch (combo) {
    case 7: return launch_batch_op<OpI64Sum>(b, st);
    case 8: return launch_batch_op<OpI64Max>(b, st);
    default: return launch_batch_op<OpI64Min>(b, st);
  }
}
int batch_i64_blocks_per_sm(int combo) {
  switch (combo) {
    case 7: return batch_blocks_per_sm<OpI64Sum>();
    case 8: return batch_blocks_per_sm<OpI64Max>();
    default: return batch_blocks_per_sm<OpI64Min>();
  }
}
}  // namespace hp
