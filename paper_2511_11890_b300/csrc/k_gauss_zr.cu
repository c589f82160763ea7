// Host entry of the register z-march Gaussian (kernel and geometry in
// k_gauss_zr.cuh; one instantiation set per input type in
// k_gauss_zr_<type>.cu so that they compile in parallel).
#include "k_gauss_zr.cuh"

namespace hp {

using zr::u64;

// Register z-march Gaussian. Returns cudaErrorNotSupported (nothing
// enqueued) when the job does not fit it: radius outside 1..12, volumes
// narrower than the radius, uint8 input (its 8-column groups are not
// 16-byte aligned), output not f32/f16, or an input layout TMA cannot
// address (16-byte aligned base and rows, tile origins on 16-byte
// boundaries).
cudaError_t launch_gauss_zr(const Job& job, const Taps& taps, cudaStream_t s) {
  const int r = taps.r;
  if (r < 1 || r > kMaxR || job.gdims[2] < r || job.gdims[1] < r) return cudaErrorNotSupported;
  if (job.out.dtype != HP_F32 && job.out.dtype != HP_F16) return cudaErrorNotSupported;
  const int64_t cx = job.core_hi[2] - job.core_lo[2];
  const int64_t cy = job.core_hi[1] - job.core_lo[1];
  const int64_t cz = job.core_hi[0] - job.core_lo[0];
  if (cx <= 0 || cy <= 0 || cz <= 0) return cudaErrorNotSupported;
  if (job.in.dtype != HP_U16 && job.in.dtype != HP_F16 && job.in.dtype != HP_F32)
    return cudaErrorNotSupported;
  const int es = (int)dtype_size(job.in.dtype);
  const int al = 16 / es;
  if ((uintptr_t)job.in.ptr % 16 || (job.in.dims[2] * es) % 16 ||
      (job.core_lo[2] - job.in.lo[2]) % al)
    return cudaErrorNotSupported;
  zr::ZrParams P;
  memset(&P, 0, sizeof(P));
  P.job = job;
  for (int a = 0; a < 3; ++a)
    for (int k = 0; k <= 2 * kMaxR; ++k) {
      const uint32_t bits = k <= 2 * r ? zr::f32_bits(taps.w[a][k]) : 0u;
      P.w2[a][k] = ((u64)bits << 32) | bits;
    }
  P.err = device_error_word();
  switch (job.in.dtype) {
    case HP_U16: return zr::dispatch_u16(r, P, job, s);
    case HP_F16: return zr::dispatch_f16(r, P, job, s);
    case HP_F32: return zr::dispatch_f32(r, P, job, s);
    default: return cudaErrorNotSupported;
  }
}

}  // namespace hp
