// Texture features and local thresholds (Harpia Sec. III-C): the per-voxel
// eigenvalues of the Gaussian Hessian, and box-window local statistics for
// the mean, Niblack and Sauvola threshold algorithms.
//
// Hessian eigenvalues: the six distinct second derivatives come from the
// Gaussian derivative kernels (launch_gauss with orders summing to 2); the
// epilogue here solves the symmetric 3x3 eigenproblem per voxel in FP32 in
// closed form (the trigonometric solution of the characteristic cubic):
// with q = tr(H)/3, p = sqrt(tr((H - qI)^2) / 6) and r = det(H - qI)/(2p^3),
// the eigenvalues are q + 2p cos(acos(r)/3 + 2 pi j / 3), j = 0, 1, 2.
//
// Box statistics: the window sums S1 = sum f and S2 = sum f^2 over the
// (2w+1)^3 cube with reflect boundaries are formed separably, x then y then
// z. Integer inputs (u8, u16) sum in 32/64-bit integers, exactly, as running
// sums along each line; floating-point inputs sum each 1D window in
// increasing source coordinate in FP64 with explicitly rounded operations.
// The decision epilogue evaluates
//   m = S1/N, v = max(S2/N - m*m, 0), s = sqrt(v),
//   T = m - c (mean) | m + k s (Niblack) | m (1 + k (s/c - 1)) (Sauvola)
// in FP64, one IEEE-rounded operation at a time (no contraction), and
// writes f > T; for integer inputs an FP32 evaluation with a proven error
// margin settles every voxel whose f is clear of T, and the FP64 sequence
// the rest.
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <type_traits>

#include "hp_device.cuh"
#include "hp_internal.h"

namespace hp {

namespace {

constexpr int kBlk = 256;

__device__ __forceinline__ void store_f(void* base, int dt, int64_t i, float v) {
  if (dt == HP_F32) static_cast<float*>(base)[i] = v;
  else static_cast<__half*>(base)[i] = __float2half_rn(v);
}

// Eigenvalues of [[a, d, e], [d, b, f], [e, f, c]], ascending.
__device__ __forceinline__ void sym3_eig(float a, float b, float c, float d, float e, float f,
                                         float& l1, float& l2, float& l3) {
  const float p1 = fmaf(d, d, fmaf(e, e, f * f));
  const float q = (a + b + c) * (1.0f / 3.0f);
  if (p1 == 0.0f) {
    l1 = fminf(a, fminf(b, c));
    l3 = fmaxf(a, fmaxf(b, c));
    l2 = (a + b + c) - l1 - l3;
    return;
  }
  const float aa = a - q, bb = b - q, cc = c - q;
  const float p2 = fmaf(aa, aa, fmaf(bb, bb, fmaf(cc, cc, 2.0f * p1)));
  const float p = sqrtf(p2 * (1.0f / 6.0f));
  if (!(p > 0.0f)) {
    l1 = l2 = l3 = q;
    return;
  }
  const float ip = 1.0f / p;
  const float ba = aa * ip, bbb = bb * ip, bc = cc * ip, bd = d * ip, be = e * ip, bf = f * ip;
  // det(B) / 2 for B = (H - qI) / p
  const float det = ba * (bbb * bc - bf * bf) - bd * (bd * bc - bf * be) + be * (bd * bf - bbb * be);
  const float r = fminf(1.0f, fmaxf(-1.0f, 0.5f * det));
  const float phi = acosf(r) * (1.0f / 3.0f);
  l3 = q + 2.0f * p * cosf(phi);
  l1 = q + 2.0f * p * cosf(phi + 2.0943951023931957f);
  l2 = 3.0f * q - l1 - l3;
  // order l1 <= l2 <= l3 against rounding near repeated eigenvalues
  if (l2 < l1) { const float t = l1; l1 = l2; l2 = t; }
  if (l3 < l2) { const float t = l2; l2 = l3; l3 = t; }
  if (l2 < l1) { const float t = l1; l1 = l2; l2 = t; }
}

// comps: six dense FP32 volumes of n voxels (Dzz, Dyy, Dxx, Dzy, Dzx, Dyx),
// one after another; outs: three volumes of out_dtype.
// A thread takes kEigU voxels a grid stride apart per round and issues
// their 6 x kEigU loads before solving any of them.
constexpr int kEigU = 4;

__global__ void k_hessian_eig(const float* __restrict__ comps, int64_t n, void* o1, void* o2,
                              void* o3, int dt) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i0 < n; i0 += kEigU * stride) {
    float h[kEigU][6];
#pragma unroll
    for (int u = 0; u < kEigU; ++u) {
      const int64_t i = i0 + u * stride;
#pragma unroll
      for (int c = 0; c < 6; ++c) h[u][c] = i < n ? comps[c * n + i] : 0.0f;
    }
#pragma unroll
    for (int u = 0; u < kEigU; ++u) {
      const int64_t i = i0 + u * stride;
      if (i >= n) break;
      float l1, l2, l3;
      sym3_eig(h[u][0], h[u][1], h[u][2], h[u][3], h[u][4], h[u][5], l1, l2, l3);
      store_f(o1, dt, i, l1);
      store_f(o2, dt, i, l2);
      store_f(o3, dt, i, l3);
    }
  }
}

// ----------------------------------------------------------- box statistics

// Floating-point sums: FP64.
struct FSum {
  double* s1;
  double* s2;
};

// Floating-point inputs: direct window sums in FP64, each 1D window summed in
// increasing source coordinate with explicitly rounded additions. x pass over
// the region [off, off + n) of the global volume (input: a dense box).
template <typename TIN>
__global__ void k_box_x_fp(const TIN* __restrict__ in, DevBox B, FSum dst, int64_t n0, int64_t n1,
                           int64_t n2, int64_t off0, int64_t off1, int64_t off2, int64_t Gx, int w) {
  const int64_t total = n0 * n1 * n2;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t x = q % n2, y = (q / n2) % n1, z = q / (n1 * n2);
    const int64_t row = ((off0 + z - B.lo[0]) * B.dims[1] + (off1 + y - B.lo[1])) * B.dims[2];
    double t1 = 0.0, t2 = 0.0;
    for (int k = -w; k <= w; ++k) {
      const double v = (double)to_f32<TIN>(in[row + reflect(off2 + x + k, Gx) - B.lo[2]]);
      t1 = __dadd_rn(t1, v);
      t2 = __dadd_rn(t2, __dmul_rn(v, v));
    }
    dst.s1[q] = t1;
    dst.s2[q] = t2;
  }
}

// y (axis 1) or z (axis 0) pass from a dense source region (lo, dims) to
// the region [off, off + n): window sums along the axis.
struct Reg {
  int64_t lo[3], dims[3];
};

__device__ __forceinline__ int64_t reg_index(const Reg& R, int64_t z, int64_t y, int64_t x) {
  return ((z - R.lo[0]) * R.dims[1] + (y - R.lo[1])) * R.dims[2] + (x - R.lo[2]);
}

// Exact decision f > T, T from the FP64 sequence of the oracle (one IEEE
// rounding per operation). Out of line: the integer path reaches it only for
// voxels next to their threshold.
__device__ __noinline__ bool decide_fp64(double s1, double s2, double nw, double f, int method,
                                            double k, double c) {
  const double m = __ddiv_rn(s1, nw);
  double v = __dsub_rn(__ddiv_rn(s2, nw), __dmul_rn(m, m));
  if (v < 0.0) v = 0.0;
  const double sd = __dsqrt_rn(v);
  double t;
  if (method == HP_LOCAL_MEAN) t = __dsub_rn(m, c);
  else if (method == HP_LOCAL_NIBLACK) t = __dadd_rn(m, __dmul_rn(k, sd));
  else t = __dmul_rn(m, __dadd_rn(1.0, __dmul_rn(k, __dsub_rn(__ddiv_rn(sd, c), 1.0))));
  return f > t;
}

// Floating-point inputs: y (axis 1) or z (axis 0) window sums from a dense
// source region, each window summed in increasing source coordinate.
__device__ __forceinline__ void axis_sum_fp(const double* s1, const double* s2, const Reg& R,
                                            int axis, int64_t c0, int64_t c1, int64_t c2,
                                            int64_t Gn, int w, double& t1, double& t2) {
  t1 = 0.0;
  t2 = 0.0;
  for (int k = -w; k <= w; ++k) {
    int64_t c[3] = {c0, c1, c2};
    c[axis] = reflect(c[axis] + k, Gn);
    const int64_t i = reg_index(R, c[0], c[1], c[2]);
    t1 = __dadd_rn(t1, s1[i]);
    t2 = __dadd_rn(t2, s2[i]);
  }
}

__global__ void k_box_y_fp(const double* __restrict__ a1, const double* __restrict__ a2, Reg src,
                           double* b1, double* b2, int64_t n0, int64_t n1, int64_t n2, int64_t off0,
                           int64_t off1, int64_t off2, int64_t Gy, int w) {
  const int64_t total = n0 * n1 * n2;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t x = q % n2, y = (q / n2) % n1, z = q / (n1 * n2);
    double t1, t2;
    axis_sum_fp(a1, a2, src, 1, off0 + z, off1 + y, off2 + x, Gy, w, t1, t2);
    b1[q] = t1;
    b2[q] = t2;
  }
}

// z pass and decision: out (u8, the job's output box) = f > T.
template <typename TIN>
__global__ void k_box_z_decide_fp(const double* __restrict__ b1, const double* __restrict__ b2,
                                  Reg src, const TIN* __restrict__ in, DevBox B, DevOut O,
                                  int64_t n0, int64_t n1, int64_t n2, int64_t off0, int64_t off1,
                                  int64_t off2, int64_t Gz, int w, int method, double k, double c) {
  const int64_t total = n0 * n1 * n2;
  const double nw = (double)(2 * w + 1) * (double)(2 * w + 1) * (double)(2 * w + 1);
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t x = off2 + q % n2, y = off1 + (q / n2) % n1, z = off0 + q / (n1 * n2);
    double t1, t2;
    axis_sum_fp(b1, b2, src, 0, z, y, x, Gz, w, t1, t2);
    const double f = (double)to_f32<TIN>(
        in[((z - B.lo[0]) * B.dims[1] + (y - B.lo[1])) * B.dims[2] + (x - B.lo[2])]);
    static_cast<uint8_t*>(O.ptr)[((z - O.lo[0]) * O.dims[1] + (y - O.lo[1])) * O.dims[2] +
                                 (x - O.lo[2])] = decide_fp64(t1, t2, nw, f, method, k, c) ? 1 : 0;
  }
}

// Integer inputs (u8, u16): window sums are exact integers, so each line
// forms them as a running sum (S(j) = S(j-1) + entering - leaving sample),
// one thread per line, O(1) per output; the result is the same sum in any
// order. The x pass takes rows (one thread each); the y and z passes take
// lines of consecutive x, so their loads and stores are coalesced.
// Eight 16-bit samples starting at sample p (0..7) of the 16 held by the
// 16-byte words A, B, as four 32-bit words (two samples each).
__device__ __forceinline__ void take8(const uint4& A, const uint4& B, int p, uint32_t (&o)[4]) {
  const uint32_t w[8] = {A.x, A.y, A.z, A.w, B.x, B.y, B.z, B.w};
  switch (p) {
#define HP_T8(P)                                                                          \
  case P:                                                                                 \
    _Pragma("unroll") for (int m = 0; m < 4; ++m) o[m] =                                  \
        (P % 2 == 0) ? w[m + P / 2] : __byte_perm(w[m + P / 2], w[m + P / 2 + 1], 0x5432); \
    break;
    HP_T8(0) HP_T8(1) HP_T8(2) HP_T8(3) HP_T8(4) HP_T8(5) HP_T8(6) HP_T8(7)
#undef HP_T8
  }
}

template <typename TIN>
__global__ void k_boxi_x(const TIN* __restrict__ in, DevBox B, int32_t* __restrict__ s1,
                         int64_t* __restrict__ s2, Reg R, int64_t Gx, int w, int vec) {
  const int64_t nrows = R.dims[0] * R.dims[1];
  const int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (l >= nrows) return;
  const int64_t z = R.lo[0] + l / R.dims[1], y = R.lo[1] + l % R.dims[1];
  const TIN* row = in + ((z - B.lo[0]) * B.dims[1] + (y - B.lo[1])) * B.dims[2] - B.lo[2];
  const int n = (int)R.dims[2];
  const int64_t x0 = R.lo[2] - w;  // global x of sample 0
  const bool inner = x0 >= 0 && x0 + n + 2 * w <= Gx;
  auto ld = [&](int i) -> int32_t { return (int32_t)row[inner ? x0 + i : reflect(x0 + i, Gx)]; };
  int32_t a = 0;
  int64_t b = 0;
  for (int i = 0; i <= 2 * w; ++i) {
    const int32_t v = ld(i);
    a += v;
    b += (int64_t)v * v;
  }
  int32_t* o1 = s1 + l * n;
  int64_t* o2 = s2 + l * n;
  // lanes walk different rows: each writes whole 32-byte sectors (chunks of
  // 16 or 8 outputs as 16-byte S1 and S2 stores), so that no sector reaches
  // DRAM partly written; the 2 x 16 loads of a 16-output chunk are in flight
  // together (rows of n % 8 != 0 outputs store one output at a time)
  int j = 0;
  auto run = [&](auto CH) {
    constexpr int C = decltype(CH)::value;  // outputs per chunk: C/8 whole sectors of S1
    for (; j < n; j += C) {
      int32_t v1[C];
      int64_t v2[C];
#pragma unroll
      for (int u = 0; u < C; ++u) {
        if (j + u > 0) {
          const int32_t vi = ld(j + u + 2 * w), vo = ld(j + u - 1);
          a += vi - vo;
          b += (int64_t)vi * vi - (int64_t)vo * vo;
        }
        v1[u] = a;
        v2[u] = b;
      }
#pragma unroll
      for (int u = 0; u < C / 4; ++u)
        reinterpret_cast<int4*>(o1 + j)[u] = make_int4(v1[4 * u], v1[4 * u + 1], v1[4 * u + 2], v1[4 * u + 3]);
#pragma unroll
      for (int u = 0; u < C / 2; ++u)
        reinterpret_cast<longlong2*>(o2 + j)[u] = make_longlong2(v2[2 * u], v2[2 * u + 1]);
    }
  };
  // 16-bit rows that start on 16-byte boundaries (vec, uniform): a chunk of
  // 8 outputs whose entering samples j + 2w + u and leaving samples j - 1 + u
  // all lie inside the volume reads them as two aligned 16-byte words per
  // stream (4 loads per lane and 8 outputs instead of 16 element loads); the
  // windows start at the same sample phase in every row. Chunks at the
  // volume faces take element loads with reflection.
  if (sizeof(TIN) == 2 && vec && n % 8 == 0) {
    const uint16_t* r16 = reinterpret_cast<const uint16_t*>(row);
    for (j = 0; j < n; j += 8) {
      const int64_t e0 = x0 + j + 2 * w, l0 = x0 + j - 1;  // first entering / leaving sample (global x)
      int32_t vi8[8], vo8[8];
      if (j > 0 && l0 >= 0 && e0 + 7 <= Gx - 1) {
        const int64_t fe = e0 & ~(int64_t)7, fl = l0 & ~(int64_t)7;
        const int pe = (int)(e0 - fe), pl = (int)(l0 - fl);
        const uint4 E0 = *reinterpret_cast<const uint4*>(r16 + fe);
        const uint4 E1 = pe ? *reinterpret_cast<const uint4*>(r16 + fe + 8) : E0;
        const uint4 L0 = *reinterpret_cast<const uint4*>(r16 + fl);
        const uint4 L1 = pl ? *reinterpret_cast<const uint4*>(r16 + fl + 8) : L0;
        uint32_t ev[4], lv[4];
        take8(E0, E1, pe, ev);
        take8(L0, L1, pl, lv);
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          vi8[u] = (int32_t)((ev[u >> 1] >> (16 * (u & 1))) & 0xFFFFu);
          vo8[u] = (int32_t)((lv[u >> 1] >> (16 * (u & 1))) & 0xFFFFu);
        }
      } else {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          vi8[u] = j + u > 0 ? ld(j + u + 2 * w) : 0;
          vo8[u] = j + u > 0 ? ld(j + u - 1) : 0;
        }
      }
      int32_t v1[8];
      int64_t v2[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        a += vi8[u] - vo8[u];
        b += (int64_t)vi8[u] * vi8[u] - (int64_t)vo8[u] * vo8[u];
        v1[u] = a;
        v2[u] = b;
      }
      reinterpret_cast<int4*>(o1 + j)[0] = make_int4(v1[0], v1[1], v1[2], v1[3]);
      reinterpret_cast<int4*>(o1 + j)[1] = make_int4(v1[4], v1[5], v1[6], v1[7]);
#pragma unroll
      for (int u = 0; u < 4; ++u)
        reinterpret_cast<longlong2*>(o2 + j)[u] = make_longlong2(v2[2 * u], v2[2 * u + 1]);
    }
    return;
  }
  if (n % 16 == 0) {
    run(std::integral_constant<int, 16>());
    return;
  }
  if (n % 8 == 0) {
    run(std::integral_constant<int, 8>());
    return;
  }
  o1[0] = a;
  o2[0] = b;
#pragma unroll 4
  for (j = 1; j < n; ++j) {
    const int32_t vi = ld(j + 2 * w), vo = ld(j - 1);
    a += vi - vo;
    b += (int64_t)vi * vi - (int64_t)vo * vo;
    o1[j] = a;
    o2[j] = b;
  }
}

// y (AXIS 1) or z (AXIS 0) running sums of the source region S into the
// region D (lines of D enumerate its other two axes, x fastest); with
// DECIDE (z pass) the sums feed the threshold decision of the output box.
struct BoxDecide {
  const void* in;  // the job's input, element type of the kernel
  DevBox B;
  DevOut O;
  int method;
  double k, c;
};

// The same decision from exact integer sums, settled in FP32 where the
// threshold is clear of f and in FP64 (decide_fp64) otherwise. With
// u = 2^-24, the FP32 threshold t32 takes at most 14 roundings over terms of
// size at most |m| + |c| + |k| (sd + |m|)(1 + r), r = |m|/c for Sauvola and
// 0 otherwise: m = S1 * (1/N) three, sd = sqrt(N S2 - S1^2) * (1/N) (the
// numerator exact in int64, converted in two halves) five relative to sd,
// k, c and 1/c one each, the formulas at most five; 14 u < 8.4e-7. The
// oracle's FP64 threshold differs from the exact t through its cancellation
// in S2/N - m^2: at most 4 ulp of S2/N <= top^2 (top: the dtype's largest
// value), so its sd moves by at most 2.2e-8 top, reaching t times
// |k| (1 + r). E takes 1.2e-6 for the first, twice the second and 1e-6;
// where |f - t32| > E, f > t32 and f > T agree.
struct DecideConst {
  float inv_nw, kf, cf, inv_c, top;
};

__device__ __forceinline__ bool decide_int(int32_t S1, int64_t S2, int nwi, int32_t f, int method,
                                           double k, double c, const DecideConst& Q) {
  const int64_t vn = (int64_t)nwi * S2 - (int64_t)S1 * S1;  // exact, >= 0
  const float m = (float)S1 * Q.inv_nw;
  const int64_t v0 = max(vn, (int64_t)0);
  const float vnf = fmaf((float)(int32_t)(v0 >> 31), 2147483648.0f, (float)(int32_t)(v0 & 0x7FFFFFFF));
  const float sd = sqrtf(vnf) * Q.inv_nw;
  float t, r = 0.0f;
  if (method == HP_LOCAL_MEAN) {
    t = m - Q.cf;
  } else if (method == HP_LOCAL_NIBLACK) {
    t = fmaf(Q.kf, sd, m);
  } else {
    r = fabsf(m) * Q.inv_c;
    t = m * (1.0f + Q.kf * fmaf(sd, Q.inv_c, -1.0f));
  }
  const float ak = fabsf(Q.kf) * (1.0f + r);
  const float E = 1.2e-6f * (fabsf(m) + fabsf(Q.cf) + ak * (sd + fabsf(m))) + 4.5e-8f * ak * Q.top + 1e-6f;
  const float d = (float)f - t;
  if (d > E) return true;
  if (d < -E) return false;
  return decide_fp64((double)S1, (double)S2, (double)nwi, (double)f, method, k, c);
}

template <int AXIS, bool DECIDE, typename TIN>
__global__ void k_boxi_line(const int32_t* __restrict__ a1, const int64_t* __restrict__ a2, Reg S,
                            int32_t* __restrict__ b1, int64_t* __restrict__ b2, Reg D, int64_t Gn,
                            int w, BoxDecide P) {
  constexpr int a1x = AXIS == 0 ? 1 : 0;  // the other axes: a1x slow, x fast
  const int64_t nlines = D.dims[a1x] * D.dims[2];
  const int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (l >= nlines) return;
  int64_t c3[3];
  c3[2] = D.lo[2] + l % D.dims[2];
  c3[a1x] = D.lo[a1x] + l / D.dims[2];
  c3[AXIS] = S.lo[AXIS];
  const int64_t sstr = AXIS == 1 ? S.dims[2] : S.dims[1] * S.dims[2];
  const int64_t sb = ((c3[0] - S.lo[0]) * S.dims[1] + (c3[1] - S.lo[1])) * S.dims[2] + (c3[2] - S.lo[2]) -
                     S.lo[AXIS] * sstr;
  const int n = (int)D.dims[AXIS];
  const int64_t p0 = D.lo[AXIS] - w;  // global coordinate of sample 0
  const bool inner = p0 >= 0 && p0 + n + 2 * w <= Gn;
  auto at = [&](int i) -> int64_t { return sb + (inner ? p0 + i : reflect(p0 + i, Gn)) * sstr; };
  int32_t a = 0;
  int64_t b = 0;
  for (int i = 0; i <= 2 * w; ++i) {
    const int64_t q = at(i);
    a += a1[q];
    b += a2[q];
  }
  // output j of this line (global coordinate D.lo[AXIS] + j)
  const int nwi = (2 * w + 1) * (2 * w + 1) * (2 * w + 1);
  DecideConst Q;
  Q.inv_nw = 1.0f / (float)nwi;
  Q.kf = (float)P.k;
  Q.cf = (float)P.c;
  Q.inv_c = P.method == HP_LOCAL_SAUVOLA ? 1.0f / Q.cf : 0.0f;
  Q.top = sizeof(TIN) == 1 ? 255.0f : 65535.0f;
  int64_t ob = 0, ib = 0, dstr = 0, istr = 0;
  if constexpr (DECIDE) {
    c3[AXIS] = D.lo[AXIS];
    ob = ((c3[0] - P.O.lo[0]) * P.O.dims[1] + (c3[1] - P.O.lo[1])) * P.O.dims[2] + (c3[2] - P.O.lo[2]);
    ib = ((c3[0] - P.B.lo[0]) * P.B.dims[1] + (c3[1] - P.B.lo[1])) * P.B.dims[2] + (c3[2] - P.B.lo[2]);
    dstr = AXIS == 1 ? P.O.dims[2] : P.O.dims[1] * P.O.dims[2];
    istr = AXIS == 1 ? P.B.dims[2] : P.B.dims[1] * P.B.dims[2];
  } else {
    c3[AXIS] = D.lo[AXIS];
    ob = ((c3[0] - D.lo[0]) * D.dims[1] + (c3[1] - D.lo[1])) * D.dims[2] + (c3[2] - D.lo[2]);
    dstr = AXIS == 1 ? D.dims[2] : D.dims[1] * D.dims[2];
  }
  auto emit = [&](int j) {
    if constexpr (DECIDE) {
      const int32_t f = (int32_t) static_cast<const TIN*>(P.in)[ib + j * istr];
      static_cast<uint8_t*>(P.O.ptr)[ob + j * dstr] = decide_int(a, b, nwi, f, P.method, P.k, P.c, Q) ? 1 : 0;
    } else {
      b1[ob + j * dstr] = a;
      b2[ob + j * dstr] = b;
    }
  };
  emit(0);
#pragma unroll (DECIDE ? 1 : 4)
  for (int j = 1; j < n; ++j) {
    const int64_t qi = at(j + 2 * w), qo = at(j - 1);
    a += a1[qi] - a1[qo];
    b += a2[qi] - a2[qo];
    emit(j);
  }
}

unsigned grid_for(int64_t t) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((t + kBlk - 1) / kBlk, (int64_t)num_sms() * 32));
}

template <typename TIN, typename S1, typename S2, bool FP>
cudaError_t box_launch(const Job& job, int method, int w, double k, double c, cudaStream_t s) {
  const SepRegions g = sep_regions(job, w);
  const int64_t cz = job.core_hi[0] - job.core_lo[0], cy = job.core_hi[1] - job.core_lo[1],
                cx = job.core_hi[2] - job.core_lo[2];
  const int64_t vx = g.n_x[0] * g.n_x[1] * g.n_x[2], vy = g.n_y[0] * g.n_y[1] * g.n_y[2];
  const size_t need = (sizeof(S1) + sizeof(S2)) * (size_t)(vx + vy) + 64;
  if (!job.scratch || job.scratch_bytes < need) return cudaErrorInvalidValue;
  // scratch: x-pass S2 | y-pass S2 | x-pass S1 | y-pass S1 (8-byte items first)
  char* p = static_cast<char*>(job.scratch);
  S2* a2 = reinterpret_cast<S2*>(p);
  S2* b2 = a2 + vx;
  S1* a1 = reinterpret_cast<S1*>(b2 + vy);
  S1* b1 = a1 + vx;
  const TIN* in = static_cast<const TIN*>(job.in.ptr);
  const Reg rx{{g.rlo[0], g.rlo[1], job.core_lo[2]}, {g.n_x[0], g.n_x[1], g.n_x[2]}};
  const Reg ry{{g.rlo[0], job.core_lo[1], job.core_lo[2]}, {g.n_y[0], g.n_y[1], g.n_y[2]}};
  if constexpr (!FP) {
    // integer inputs: running sums along lines (k_boxi_*)
    const Reg core{{job.core_lo[0], job.core_lo[1], job.core_lo[2]}, {cz, cy, cx}};
    const BoxDecide P{job.in.ptr, job.in, job.out, method, k, c};
    const int64_t rows = g.n_x[0] * g.n_x[1];
    // rows on 16-byte boundaries: every row of the input box is a whole number
    // of 16-byte words from an aligned base
    const int vec = (reinterpret_cast<uintptr_t>(in) % 16 == 0 &&
                     (job.in.dims[2] * (int64_t)sizeof(TIN)) % 16 == 0 && (job.in.lo[2] % 8) == 0);
    k_boxi_x<TIN><<<(unsigned)((rows + kBlk - 1) / kBlk), kBlk, 0, s>>>(in, job.in, a1, a2, rx,
                                                                       job.gdims[2], w, vec);
    const int64_t ly = g.n_y[0] * g.n_y[2];
    k_boxi_line<1, false, TIN><<<(unsigned)((ly + kBlk - 1) / kBlk), kBlk, 0, s>>>(
        a1, a2, rx, b1, b2, ry, job.gdims[1], w, P);
    const int64_t lz = cy * cx;
    k_boxi_line<0, true, TIN><<<(unsigned)((lz + kBlk - 1) / kBlk), kBlk, 0, s>>>(
        b1, b2, ry, nullptr, nullptr, core, job.gdims[0], w, P);
  } else {
    k_box_x_fp<TIN><<<grid_for(vx), kBlk, 0, s>>>(in, job.in, FSum{a1, a2}, g.n_x[0], g.n_x[1],
                                                  g.n_x[2], g.rlo[0], g.rlo[1], job.core_lo[2],
                                                  job.gdims[2], w);
    k_box_y_fp<<<grid_for(vy), kBlk, 0, s>>>(a1, a2, rx, b1, b2, g.n_y[0], g.n_y[1], g.n_y[2],
                                             g.rlo[0], job.core_lo[1], job.core_lo[2], job.gdims[1], w);
    k_box_z_decide_fp<TIN><<<grid_for(cz * cy * cx), kBlk, 0, s>>>(
        b1, b2, ry, in, job.in, job.out, cz, cy, cx, job.core_lo[0], job.core_lo[1], job.core_lo[2],
        job.gdims[0], w, method, k, c);
  }
  return cudaGetLastError();
}

}  // namespace

size_t hessian_eig_scratch(int64_t core_voxels) { return 6 * sizeof(float) * (size_t)core_voxels; }

cudaError_t launch_hessian_eig(const float* comps, int64_t n, void* const* outs, int out_dtype,
                               cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_hessian_eig<<<grid_for(n), kBlk, 0, s>>>(comps, n, outs[0], outs[1], outs[2], out_dtype);
  return cudaGetLastError();
}

size_t box_scratch_bytes(const Job& job, int w) {
  const SepRegions g = sep_regions(job, w);
  const int64_t vx = g.n_x[0] * g.n_x[1] * g.n_x[2], vy = g.n_y[0] * g.n_y[1] * g.n_y[2];
  const bool fp = job.in.dtype == HP_F16 || job.in.dtype == HP_F32;
  const size_t per = fp ? 16 : 12;
  return per * (size_t)(vx + vy) + 64;
}

cudaError_t launch_threshold_box(const Job& job, int method, int w, double k, double c,
                                 cudaStream_t s) {
  if (job.core_hi[0] <= job.core_lo[0] || job.core_hi[1] <= job.core_lo[1] ||
      job.core_hi[2] <= job.core_lo[2])
    return cudaSuccess;
  switch (job.in.dtype) {
    case HP_U8: return box_launch<uint8_t, int32_t, int64_t, false>(job, method, w, k, c, s);
    case HP_U16: return box_launch<uint16_t, int32_t, int64_t, false>(job, method, w, k, c, s);
    case HP_F16: return box_launch<__half, double, double, true>(job, method, w, k, c, s);
    case HP_F32: return box_launch<float, double, double, true>(job, method, w, k, c, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace hp
