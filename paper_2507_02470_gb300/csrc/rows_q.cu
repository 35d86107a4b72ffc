// Instantiations of the row kernels for K_Q1, K_Q2, K_APPLY_Q, K_POWER_Q, K_Q2H (one translation unit per
// operator, so that the variants compile in parallel).
#include "kernels.cuh"

namespace hprqp {

RowKernel row_kernel_q(int kind, int var, int G) {
  switch (kind) {
    case K_Q1: return pick_row<K_Q1>(var, G);
    case K_Q2: return pick_row<K_Q2>(var, G);
    case K_APPLY_Q: return pick_row<K_APPLY_Q>(var, G);
    case K_POWER_Q: return pick_row<K_POWER_Q>(var, G);
    case K_Q2H: return pick_row<K_Q2H>(var, G);
    default: return nullptr;
  }
}

}  // namespace hprqp
