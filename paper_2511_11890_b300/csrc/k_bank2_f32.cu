// Four-plane filter-bank kernel for float32 input.
#include "k_bank.cuh"

namespace hp {
const void* bank2_kernel_f32(int minb) {
  return minb == 2 ? reinterpret_cast<const void*>(&b2::k_bank2<float, 2>)
                   : reinterpret_cast<const void*>(&b2::k_bank2<float, 1>);
}
}  // namespace hp
