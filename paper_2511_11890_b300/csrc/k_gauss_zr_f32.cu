// Register z-march Gaussian kernels for float input, radii 1..12.
#include "k_gauss_zr.cuh"

namespace hp {
namespace zr {

cudaError_t dispatch_f32(int r, const ZrParams& P, const Job& job, cudaStream_t s) {
  return dispatch_zr_t<float>(r, P, job, s);
}

}  // namespace zr
}  // namespace hp
