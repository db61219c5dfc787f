// resident_i32.cu — the resident serving kernel for the int32 arithmetics.
#include "resident_kernels.cuh"

namespace hp {
cudaError_t launch_resident_fp(int combo, const ResidentSource& src, int grid, cudaStream_t st);
int resident_fp_blocks_per_sm(int combo);

cudaError_t launch_resident_combo(int combo, const ResidentSource& src, int grid, cudaStream_t st) {
  switch (combo) {
    case 4: return launch_resident_op<OpI32Sum>(src, grid, st);
    case 5: return launch_resident_op<OpI32Max>(src, grid, st);
    case 6: return launch_resident_op<OpI32Min>(src, grid, st);
    default: return combo >= 0 && combo < 4 ? launch_resident_fp(combo, src, grid, st) : cudaErrorInvalidValue;
  }
}

int resident_combo_blocks_per_sm(int combo) {
  switch (combo) {
    case 4: return resident_blocks_per_sm<OpI32Sum>();
    case 5: return resident_blocks_per_sm<OpI32Max>();
    case 6: return resident_blocks_per_sm<OpI32Min>();
    default: return resident_fp_blocks_per_sm(combo);
  }
}
}  // namespace hp
