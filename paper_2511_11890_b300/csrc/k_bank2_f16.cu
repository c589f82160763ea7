// Four-plane filter-bank kernel for float16 input.
#include "k_bank.cuh"

namespace hp {
const void* bank2_kernel_f16(int minb) {
  return minb == 2 ? reinterpret_cast<const void*>(&b2::k_bank2<__half, 2>)
                   : reinterpret_cast<const void*>(&b2::k_bank2<__half, 1>);
}
}  // namespace hp
