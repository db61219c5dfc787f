// batch_f32.cu — the persistent batched kernel for the FP32 arithmetics.
#include "batch_kernels.cuh"

namespace hp {
cudaError_t launch_batch_fp(int combo, const BatchLaunch& b, cudaStream_t st) {
  switch (combo) {
    case 0: return launch_batch_op<OpF32Sum>(b, st);
    case 1: return launch_batch_op<OpF32Comp>(b, st);
    case 2: return launch_batch_op<OpF32Max>(b, st);
    default: return launch_batch_op<OpF32Min>(b, st);
  }
}
int batch_fp_blocks_per_sm(int combo) {
  switch (combo) {
    case 0: return batch_blocks_per_sm<OpF32Sum>();
    case 1: return batch_blocks_per_sm<OpF32Comp>();
    case 2: return batch_blocks_per_sm<OpF32Max>();
    default: return batch_blocks_per_sm<OpF32Min>();
  }
}
}  // namespace hp
