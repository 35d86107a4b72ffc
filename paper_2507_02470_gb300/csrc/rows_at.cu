// Instantiations of the row kernels for K_AT, K_APPLY_AT, K_APPLY_AT_P, K_ATH (one translation unit per
// operator, so that the variants compile in parallel).
#include "kernels.cuh"

namespace hprqp {

RowKernel row_kernel_at(int kind, int var, int G) {
  switch (kind) {
    case K_AT: return pick_row<K_AT>(var, G);
    case K_APPLY_AT: return pick_row<K_APPLY_AT>(var, G);
    case K_APPLY_AT_P: return pick_row<K_APPLY_AT_P>(var, G);
    case K_ATH: return pick_row<K_ATH>(var, G);
    default: return nullptr;
  }
}

}  // namespace hprqp
