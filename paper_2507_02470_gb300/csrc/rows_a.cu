// Instantiations of the row kernels for K_A1, K_APPLY_A, K_POWER_A (one translation unit per
// operator, so that the variants compile in parallel).
#include "kernels.cuh"

namespace hprqp {

RowKernel row_kernel_a(int kind, int var, int G) {
  switch (kind) {
    case K_A1: return pick_row<K_A1>(var, G);
    case K_APPLY_A: return pick_row<K_APPLY_A>(var, G);
    case K_POWER_A: return pick_row<K_POWER_A>(var, G);
    default: return nullptr;
  }
}

}  // namespace hprqp
