// Register z-march Gaussian kernels for uint16_t input, radii 1..12.
#include "k_gauss_zr.cuh"

namespace hp {
namespace zr {

cudaError_t dispatch_u16(int r, const ZrParams& P, const Job& job, cudaStream_t s) {
  return dispatch_zr_t<uint16_t>(r, P, job, s);
}

}  // namespace zr
}  // namespace hp
