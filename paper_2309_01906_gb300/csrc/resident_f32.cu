// resident_f32.cu — the resident serving kernel for the FP32 arithmetics.
#include "resident_kernels.cuh"

namespace hp {
cudaError_t launch_resident_fp(int combo, const ResidentSource& src, int grid, cudaStream_t st) {
  switch (combo) {
    case 0: return launch_resident_op<OpF32Sum>(src, grid, st);
    case 1: return launch_resident_op<OpF32Comp>(src, grid, st);
    case 2: return launch_resident_op<OpF32Max>(src, grid, st);
    default: return launch_resident_op<OpF32Min>(src, grid, st);
  }
}
int resident_fp_blocks_per_sm(int combo) {
  switch (combo) {
    case 0: return resident_blocks_per_sm<OpF32Sum>();
    case 1: return resident_blocks_per_sm<OpF32Comp>();
    case 2: return resident_blocks_per_sm<OpF32Max>();
    default: return resident_blocks_per_sm<OpF32Min>();
  }
}
}  // namespace hp
