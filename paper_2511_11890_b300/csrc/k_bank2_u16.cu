// Four-plane filter-bank kernel for uint16 input (the other input types have
// their own translation units so that the instantiations compile in
// parallel).
#include "k_bank.cuh"

namespace hp {
const void* bank2_kernel_u16(int minb) {
  return minb == 2 ? reinterpret_cast<const void*>(&b2::k_bank2<uint16_t, 2>)
                   : reinterpret_cast<const void*>(&b2::k_bank2<uint16_t, 1>);
}
}  // namespace hp
