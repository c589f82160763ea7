// Separable Gaussian / derivative-of-Gaussian filtering (Harpia Sec. III-C:
// Gaussian smoothing and derivative features) over a core box of a volume,
// with reflect boundaries on global coordinates so that halo-padded bricks
// (Sec. III-D) reproduce the whole-volume result bit for bit.
//
// Tiled z-march kernel (radius r <= 12): a CTA owns a TX x TY column of the
// core and marches along z. Per input plane it
//   1. receives the (TY+2r) x (TX+2r) input patch by one TMA tile load
//      (4-stage mbarrier pipeline; a cooperative-load variant covers layouts
//      TMA cannot address),
//   2. converts it to FP32 in shared memory, resolving reflections at the
//      volume faces,
//   3. runs the x pass (8 outputs per thread, register window) and the y
//      pass (4 outputs per thread) into a ring of XY planes,
// and after every BZ planes runs the z pass over the ring (BZ outputs per
// thread, register window) and stores the results.
//
// Every output is accumulated in FP32 with fmaf, starting from 0, over taps
// in increasing input coordinate. That order does not depend on the tile,
// brick or launch shape, which is what makes chunked == unchunked exact.
// The generic path (any r <= 32, any extents) runs three single-axis passes
// through device scratch with the same per-output order.
#include <cuda_fp16.h>

#include <stdio.h>
#include <string.h>

#include <algorithm>

#include "hp_device.cuh"
#include "hp_internal.h"

namespace hp {

namespace {

constexpr int kTX = 32;
constexpr int kTY = 32;
constexpr int kBZ = 8;
constexpr int kNS = 4;
constexpr int kThreads = 256;
constexpr int kXS = kTX + 4;  // X row stride: 4 mod 8 floats keeps 16-byte stores conflict-free

struct GaussParams {
  Job job;
  float wz[kMaxTaps];
  float wy[kMaxTaps];
  float wx[kMaxTaps];
  int r;
  int zchunk;
  int tiles_x;
  int use_tma;
  int* err;
};

__host__ __device__ constexpr int round_up(int a, int b) { return (a + b - 1) / b * b; }

// Smallest row stride >= n floats that is 4 mod 8: two rows read by one
// 8-thread phase of 16-byte loads then land in disjoint bank groups.
__host__ __device__ constexpr int patch_stride(int n) {
  int f = n;
  while (f % 8 != 4) ++f;
  return f;
}

// Geometry of the z-march kernel for radius R.
//   F  (FP32 patch, double-buffered): col c <-> x = cx0 - R4 + c, rows
//      <-> y = cy0 - R + row. R4 = R rounded up to 4 keeps the x-pass
//      window loads 16-byte aligned.
//   X  (x-pass output, double-buffered): [BH][kXS].
//   ring: kBZ + 2R planes of y-pass output [TY][TX].
template <int R>
struct ZmGeom {
  static constexpr int R4 = round_up(R, 4);
  static constexpr int WL = round_up(R4 + R + 8, 4);  // x window (floats) for 8 outputs
  static constexpr int FWN = (kTX - 8) + WL;           // F columns read
  static constexpr int FW = patch_stride(FWN);
  static constexpr int BH = kTY + 2 * R;
  static constexpr int NC = (FWN + 31) / 32;           // F columns per lane
  static constexpr int NRING = kBZ + 2 * R;
  static constexpr int FSZ = BH * FW;
  static constexpr int XSZ = BH * kXS;
  // bytes after the TMA stages
  static constexpr int TAIL = (2 * FSZ + 2 * XSZ + NRING * kTY * kTX) * 4 + BH * 4;
  static_assert(FW >= FWN && FW % 8 == 4, "FP32 patch row stride must be 4 mod 8 floats");
  static_assert(FWN % 4 == 0, "patch width must be a multiple of 4");
};

// Per-dtype TMA box geometry: left halo ra (R rounded up to 16 bytes) and
// width bw (elements); raw col c <-> x = cx0 - ra + c.
__host__ __device__ inline void box_geom(int r, int es, int* ra, int* bw) {
  const int al = 16 / es;
  *ra = round_up(r, al);
  *bw = round_up(kTX + *ra + r, al);
}

__host__ __device__ inline int stage_bytes(int r, int es) {
  int ra, bw;
  box_geom(r, es, &ra, &bw);
  return round_up(bw * (kTY + 2 * r) * es, 128);
}

template <int R>
__host__ __device__ inline int zm_smem_bytes(int es) {
  return 128 + kNS * stage_bytes(R, es) + ZmGeom<R>::TAIL;
}

// One plane of input -> FP32 patch F. Sources are looked up in per-CTA
// tables that already resolve the reflect boundary: srow[row] is the raw
// stage row (TMA) or box row (global loads), scol[k] the column of lane
// column lane + 32k; -1 marks taps no stored output uses.
template <typename TIN, int R>
__device__ __forceinline__ void stage_from_tma(float* Fb, const unsigned char* rawb, int bw,
                                               const int* srow, const int (&scol)[ZmGeom<R>::NC],
                                               int warp, int lane) {
  using G = ZmGeom<R>;
  const TIN* raw = reinterpret_cast<const TIN*>(rawb);
  for (int row = warp; row < G::BH; row += kThreads / 32) {
    const int sr = srow[row];
#pragma unroll
    for (int k = 0; k < G::NC; ++k) {
      const int col = lane + 32 * k;
      if (col < G::FWN) {
        const int sc = scol[k];
        Fb[row * G::FW + col] = (sr >= 0 && sc >= 0) ? to_f32<TIN>(raw[sr * bw + sc]) : 0.0f;
      }
    }
  }
}

// Interior tiles: no reflection, F col c <-> raw col c + (ra - R4); four
// columns per item with one vector load (16-, 8- or 4-byte aligned since
// ra - R4 is a multiple of 4 elements) and one 16-byte store.
template <typename TIN, int R>
__device__ __forceinline__ void stage_from_tma_interior(float* Fb, const unsigned char* rawb,
                                                        int ra, int bw, int tid) {
  using G = ZmGeom<R>;
  constexpr int Q = G::FWN / 4;
  const TIN* raw = reinterpret_cast<const TIN*>(rawb) + (ra - G::R4);
  for (int it = tid; it < G::BH * Q; it += kThreads) {
    const int row = it / Q, q = it - row * Q;
    *reinterpret_cast<float4*>(Fb + row * G::FW + 4 * q) = load4_f32<TIN>(raw + row * bw + 4 * q);
  }
}

template <typename TIN, int R>
__device__ __forceinline__ void stage_from_global(float* Fb, const Job& J, int64_t sz,
                                                  const int* srow,
                                                  const int (&scol)[ZmGeom<R>::NC], int warp,
                                                  int lane) {
  using G = ZmGeom<R>;
  const TIN* in = static_cast<const TIN*>(J.in.ptr);
  const bool zok = sz >= 0 && sz < J.in.dims[0];
  const TIN* plane = in + sz * J.in.dims[1] * J.in.dims[2];
  for (int row = warp; row < G::BH; row += kThreads / 32) {
    const int sr = srow[row];
#pragma unroll
    for (int k = 0; k < G::NC; ++k) {
      const int col = lane + 32 * k;
      if (col < G::FWN) {
        const int sc = scol[k];
        Fb[row * G::FW + col] = (zok && sr >= 0 && sc >= 0)
                                    ? to_f32<TIN>(plane[(int64_t)sr * J.in.dims[2] + sc])
                                    : 0.0f;
      }
    }
  }
}

template <int R>
__global__ void __launch_bounds__(kThreads, 1)
    k_gauss_zm(const __grid_constant__ GaussParams P, const __grid_constant__ CUtensorMap tmap) {
  using G = ZmGeom<R>;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ int s_abort;

  const Job& J = P.job;
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const int tx = blockIdx.x % P.tiles_x, ty = blockIdx.x / P.tiles_x;
  const int64_t cx0 = J.core_lo[2] + (int64_t)tx * kTX;
  const int64_t cy0 = J.core_lo[1] + (int64_t)ty * kTY;
  const int64_t cz0 = J.core_lo[0] + (int64_t)blockIdx.y * P.zchunk;
  const int64_t cz1 = min(cz0 + (int64_t)P.zchunk, J.core_hi[0]);
  if (cz0 >= cz1) return;
  const int nout = (int)(cz1 - cz0);
  const int total = nout + 2 * R;  // input planes cz0-R .. cz1+R-1
  const int64_t Gz = J.gdims[0], Gy = J.gdims[1], Gx = J.gdims[2];
  const int dt = J.in.dtype;
  const int es = dt == HP_U8 ? 1 : (dt == HP_F32 ? 4 : 2);
  int ra, bw;
  box_geom(R, es, &ra, &bw);
  const int sbytes = stage_bytes(R, es);
  const bool tma = P.use_tma != 0;
  // tiles whose halo stays inside the volume need no reflection
  const bool face = (cx0 - R < 0) || (cx0 + kTX + R > Gx) || (cy0 - R < 0) || (cy0 + kTY + R > Gy);

  uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
  unsigned char* stages = smem + 128;
  float* F = reinterpret_cast<float*>(stages + kNS * sbytes);
  float* X = F + 2 * G::FSZ;
  float* ring = X + 2 * G::XSZ;
  int* srow = reinterpret_cast<int*>(ring + G::NRING * kTY * kTX);

  // source tables (reflection resolved once per CTA)
  for (int row = tid; row < G::BH; row += kThreads) {
    const int64_t sy = reflect(cy0 - R + row, Gy);
    int v;
    if (tma) {
      const int64_t s = sy - (cy0 - R);
      v = (s >= 0 && s < G::BH) ? (int)s : -1;
    } else {
      const int64_t s = sy - J.in.lo[1];
      v = (s >= 0 && s < J.in.dims[1]) ? (int)s : -1;
    }
    srow[row] = v;
  }
  int scol[G::NC];
#pragma unroll
  for (int k = 0; k < G::NC; ++k) {
    const int col = lane + 32 * k;
    const int64_t sx = reflect(cx0 - G::R4 + col, Gx);
    int v = -1;
    if (tma) {
      const int64_t s = sx - (cx0 - ra);
      if (s >= 0 && s < bw) v = (int)s;
    } else {
      const int64_t s = sx - J.in.lo[2];
      if (s >= 0 && s < J.in.dims[2]) v = (int)s;
    }
    scol[k] = col < G::FWN ? v : -1;
  }
  if (tid == 0) {
    s_abort = 0;
    if (tma) {
      prefetch_tmap(&tmap);
      for (int s = 0; s < kNS; ++s) mbar_init(&bars[s], 1);
      fence_mbar_init();
    }
  }
  __syncthreads();

  auto issue = [&](int n) {  // TMA load of input plane n into stage n % kNS
    const int zl = (int)(reflect(cz0 - R + n, Gz) - J.in.lo[0]);
    const int xl = (int)(cx0 - ra - J.in.lo[2]);
    const int yl = (int)(cy0 - R - J.in.lo[1]);
    uint64_t* bar = &bars[n % kNS];
    mbar_arrive_expect_tx(bar, bw * G::BH * es);
    tma_load_3d(stages + (n % kNS) * sbytes, &tmap, xl, yl, zl, bar);
  };
  if (tma && tid == 0) {
    fence_proxy_async();
    for (int n = 0; n < min(kNS, total); ++n) issue(n);
  }

  const int xrow = tid / (kTX / 8), xg = (tid % (kTX / 8)) * 8;  // x pass
  const int yp = tid % (kTX / 2), yb2 = (tid / (kTX / 2)) * 2;     // y pass
  const int zy = tid / (kTX / 4), zx4 = (tid % (kTX / 4)) * 4;    // z pass

  // ---- one pipeline phase p: stage plane p, x pass of plane p-1, y pass
  // of plane p-2 (double-buffered F and X), then one barrier.
  int zb = 0;
  int p = 0;
  for (; p < total + 2; ++p) {
    if (p < total) {
      float* Fb = F + (p & 1) * G::FSZ;
      if (tma) {
        if (!mbar_wait(&bars[p % kNS], (p / kNS) & 1)) atomicOr(&s_abort, 1);
        const unsigned char* rawb = stages + (p % kNS) * sbytes;
        if (!face) {
          switch (dt) {
            case HP_U8: stage_from_tma_interior<uint8_t, R>(Fb, rawb, ra, bw, tid); break;
            case HP_U16: stage_from_tma_interior<uint16_t, R>(Fb, rawb, ra, bw, tid); break;
            case HP_F16: stage_from_tma_interior<__half, R>(Fb, rawb, ra, bw, tid); break;
            default: stage_from_tma_interior<float, R>(Fb, rawb, ra, bw, tid); break;
          }
        } else {
          switch (dt) {
            case HP_U8: stage_from_tma<uint8_t, R>(Fb, rawb, bw, srow, scol, warp, lane); break;
            case HP_U16: stage_from_tma<uint16_t, R>(Fb, rawb, bw, srow, scol, warp, lane); break;
            case HP_F16: stage_from_tma<__half, R>(Fb, rawb, bw, srow, scol, warp, lane); break;
            default: stage_from_tma<float, R>(Fb, rawb, bw, srow, scol, warp, lane); break;
          }
        }
      } else {
        const int64_t sz = reflect(cz0 - R + p, Gz) - J.in.lo[0];
        switch (dt) {
          case HP_U8: stage_from_global<uint8_t, R>(Fb, J, sz, srow, scol, warp, lane); break;
          case HP_U16: stage_from_global<uint16_t, R>(Fb, J, sz, srow, scol, warp, lane); break;
          case HP_F16: stage_from_global<__half, R>(Fb, J, sz, srow, scol, warp, lane); break;
          default: stage_from_global<float, R>(Fb, J, sz, srow, scol, warp, lane); break;
        }
      }
    }
    if (p >= 1 && p - 1 < total && xrow < G::BH) {
      // x pass: 8 outputs of row xrow from a 16-byte aligned window of F
      const float* Fb = F + ((p - 1) & 1) * G::FSZ;
      float w[G::WL];
      const float4* src = reinterpret_cast<const float4*>(Fb + xrow * G::FW + xg);
#pragma unroll
      for (int j = 0; j < G::WL / 4; ++j) {
        const float4 v = src[j];
        w[4 * j] = v.x;
        w[4 * j + 1] = v.y;
        w[4 * j + 2] = v.z;
        w[4 * j + 3] = v.w;
      }
      float o[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        float acc = 0.0f;
        // window index j <-> x = cx0 + xg - R4 + j; tap k = i + R4 - j
#pragma unroll
        for (int j = i + G::R4 - R; j <= i + G::R4 + R; ++j)
          acc = fmaf(P.wx[i + G::R4 - j + R], w[j], acc);
        o[i] = acc;
      }
      float4* dst = reinterpret_cast<float4*>(X + ((p - 1) & 1) * G::XSZ + xrow * kXS + xg);
      dst[0] = make_float4(o[0], o[1], o[2], o[3]);
      dst[1] = make_float4(o[4], o[5], o[6], o[7]);
    }
    if (p >= 2) {
      // y pass of plane p-2 into its ring slot: one x pair, two rows per
      // thread, packed fmas over the pair
      const float* Xb = X + ((p - 2) & 1) * G::XSZ;
      unsigned long long a0 = 0ull, a1 = 0ull;
#pragma unroll
      for (int j = 0; j < 2 + 2 * R; ++j) {
        const unsigned long long v = pack2(*reinterpret_cast<const float2*>(Xb + (yb2 + j) * kXS + 2 * yp));
        if (j <= 2 * R) a0 = ffma2(splat2(P.wy[2 * R - j]), v, a0);
        if (j >= 1) a1 = ffma2(splat2(P.wy[2 * R + 1 - j]), v, a1);
      }
      float* slot = ring + ((p - 2) % G::NRING) * (kTY * kTX);
      *reinterpret_cast<float2*>(slot + yb2 * kTX + 2 * yp) = unpack2(a0);
      *reinterpret_cast<float2*>(slot + (yb2 + 1) * kTX + 2 * yp) = unpack2(a1);
    }
    __syncthreads();
    if (s_abort) break;
    if (tma && tid == 0 && p + kNS < total) {
      fence_proxy_async();
      issue(p + kNS);
    }
    // z pass for every block whose ring planes are all present
    const int done = min(p - 1, total);  // planes 0 .. done-1 are in the ring
    while (zb < nout && done >= min(zb + kBZ + 2 * R, total)) {
      unsigned long long acc0[kBZ], acc1[kBZ];  // x pairs (0,1) and (2,3)
#pragma unroll
      for (int j = 0; j < kBZ; ++j) acc0[j] = acc1[j] = 0ull;
      int slot = zb % G::NRING;
#pragma unroll
      for (int m = 0; m < kBZ + 2 * R; ++m) {
        const float4 v =
            *reinterpret_cast<const float4*>(ring + slot * (kTY * kTX) + zy * kTX + zx4);
        slot = slot + 1 == G::NRING ? 0 : slot + 1;
        const unsigned long long v0 = pack2(make_float2(v.x, v.y)), v1 = pack2(make_float2(v.z, v.w));
#pragma unroll
        for (int j = 0; j < kBZ; ++j) {
          if (m >= j && m <= j + 2 * R) {
            const unsigned long long g = splat2(P.wz[j - m + 2 * R]);
            acc0[j] = ffma2(g, v0, acc0[j]);
            acc1[j] = ffma2(g, v1, acc1[j]);
          }
        }
      }
      float4 acc[kBZ];
#pragma unroll
      for (int j = 0; j < kBZ; ++j) {
        const float2 lo = unpack2(acc0[j]), hi = unpack2(acc1[j]);
        acc[j] = make_float4(lo.x, lo.y, hi.x, hi.y);
      }
      const int64_t gy = cy0 + zy, gx = cx0 + zx4;
      if (gy < J.core_hi[1]) {
        const DevOut& O = J.out;
        const int64_t pstride = O.dims[1] * O.dims[2];
        int64_t idx = ((cz0 + zb - O.lo[0]) * O.dims[1] + (gy - O.lo[1])) * O.dims[2] + (gx - O.lo[2]);
        const bool full4 = gx + 3 < J.core_hi[2];
        const bool vec = O.dtype == HP_F32 && full4 &&
                         ((reinterpret_cast<uintptr_t>(static_cast<float*>(O.ptr) + idx) |
                           (uintptr_t)(pstride * 4)) & 15) == 0;
#pragma unroll
        for (int j = 0; j < kBZ; ++j, idx += pstride) {
          if (zb + j >= nout) break;
          if (vec) {
            *reinterpret_cast<float4*>(static_cast<float*>(O.ptr) + idx) = acc[j];
          } else {
            const float vv[4] = {acc[j].x, acc[j].y, acc[j].z, acc[j].w};
#pragma unroll
            for (int e = 0; e < 4; ++e)
              if (gx + e < J.core_hi[2]) {
                if (O.dtype == HP_F32)
                  static_cast<float*>(O.ptr)[idx + e] = vv[e];
                else
                  static_cast<__half*>(O.ptr)[idx + e] = __float2half_rn(vv[e]);
              }
          }
        }
      }
      zb += kBZ;
      __syncthreads();  // ring slots of this block are rewritten next
    }
  }
  if (s_abort) {
    set_device_error(P.err, kErrTimeout);
    // drain TMA loads still in flight into this CTA's shared memory
    if (tma && tid == 0)
      for (int n = p; n < min(p + kNS, total); ++n) (void)mbar_wait(&bars[n % kNS], (n / kNS) & 1);
    __syncthreads();
  }
}

// --------------------------------------------------------------------------
// Generic single-axis pass: dst = conv_axis(src) over the global volume
// (dense, whole volume in device memory), y[i] = sum_k g(k) x[R(i-k)].
// src may be the job's input (any dtype, box) for the first pass.
template <typename TIN>
__global__ void k_axis_pass(const TIN* src, const int64_t* src_lo, const int64_t* src_dims,
                            float* dst, int64_t n0, int64_t n1, int64_t n2, int axis,
                            const float* __restrict__ w, int r, int64_t G0, int64_t G1,
                            int64_t G2, int64_t off0, int64_t off1, int64_t off2) {
  // dst covers region [off, off + n) of the global volume, densely.
  const int64_t total = n0 * n1 * n2;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t x = q % n2, y = (q / n2) % n1, z = q / (n1 * n2);
    int64_t c[3] = {off0 + z, off1 + y, off2 + x};
    const int64_t Gs[3] = {G0, G1, G2};
    float acc = 0.0f;
    for (int j = 0; j <= 2 * r; ++j) {  // input coordinate increasing: k = r - j
      int64_t s[3] = {c[0], c[1], c[2]};
      s[axis] = reflect(c[axis] - (r - j), Gs[axis]);
      const int64_t l0 = s[0] - src_lo[0], l1 = s[1] - src_lo[1], l2 = s[2] - src_lo[2];
      float v = 0.0f;
      if (l0 >= 0 && l0 < src_dims[0] && l1 >= 0 && l1 < src_dims[1] && l2 >= 0 && l2 < src_dims[2])
        v = to_f32<TIN>(src[(l0 * src_dims[1] + l1) * src_dims[2] + l2]);
      acc = fmaf(w[2 * r - j], v, acc);
    }
    dst[q] = acc;
  }
}

__global__ void k_copy_out(const float* src, int64_t n0, int64_t n1, int64_t n2, DevOut O,
                           int64_t off0, int64_t off1, int64_t off2) {
  const int64_t total = n0 * n1 * n2;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t x = q % n2, y = (q / n2) % n1, z = q / (n1 * n2);
    const int64_t idx =
        ((off0 + z - O.lo[0]) * O.dims[1] + (off1 + y - O.lo[1])) * O.dims[2] + (off2 + x - O.lo[2]);
    if (O.dtype == HP_F32)
      static_cast<float*>(O.ptr)[idx] = src[q];
    else
      static_cast<__half*>(O.ptr)[idx] = __float2half_rn(src[q]);
  }
}

template <int R>
cudaError_t launch_zm_t(const GaussParams& P, const CUtensorMap& map, dim3 grid, cudaStream_t s) {
  static bool attr_set = false;  // per instantiation; set once per process
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_gauss_zm<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         zm_smem_bytes<R>(4));
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const int es = (int)dtype_size(P.job.in.dtype);
  k_gauss_zm<R><<<grid, kThreads, zm_smem_bytes<R>(es), s>>>(P, map);
  return cudaGetLastError();
}

cudaError_t dispatch_zm(int r, const GaussParams& P, const CUtensorMap& map, dim3 grid,
                        cudaStream_t s) {
  switch (r) {
#define HP_CASE(RR) \
  case RR: return launch_zm_t<RR>(P, map, grid, s);
    HP_CASE(1) HP_CASE(2) HP_CASE(3) HP_CASE(4) HP_CASE(5) HP_CASE(6)
    HP_CASE(7) HP_CASE(8) HP_CASE(9) HP_CASE(10) HP_CASE(11) HP_CASE(12)
#undef HP_CASE
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_generic(const Job& job, const Taps& taps, cudaStream_t s) {
  // Three passes x -> y -> z through two FP32 scratch volumes covering the
  // regions each pass needs (core grown by r along the later axes, clipped
  // to the source hull). Scratch is stream-ordered.
  const int r = taps.r;
  int64_t lo[3], hi[3];
  for (int a = 0; a < 3; ++a) {
    lo[a] = job.core_lo[a];
    hi[a] = job.core_hi[a];
  }
  // region after x pass: z and y grown to the hull of their reflected
  // sources, x = core
  int64_t rlo[3], rhi[3];
  for (int a = 0; a < 2; ++a) {
    const int64_t n = job.gdims[a];
    int64_t mn = n, mx = -1;
    if (hi[a] - lo[a] + 2 * r >= 2 * n) {
      mn = 0;
      mx = n - 1;
    } else {
      for (int64_t c = lo[a] - r; c < hi[a] + r; ++c) {
        const int64_t sidx = reflect(c, n);
        mn = std::min(mn, sidx);
        mx = std::max(mx, sidx);
      }
    }
    rlo[a] = mn;
    rhi[a] = mx + 1;
  }
  const int64_t n_x[3] = {rhi[0] - rlo[0], rhi[1] - rlo[1], hi[2] - lo[2]};
  const int64_t n_y[3] = {rhi[0] - rlo[0], hi[1] - lo[1], hi[2] - lo[2]};
  const int64_t n_z[3] = {hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2]};
  size_t b1 = sizeof(float) * n_x[0] * n_x[1] * n_x[2];
  size_t b2 = sizeof(float) * n_y[0] * n_y[1] * n_y[2];
  size_t bz = sizeof(float) * n_z[0] * n_z[1] * n_z[2];
  float *t1 = nullptr, *t2 = nullptr, *t3 = nullptr;
  float* dw = nullptr;
  int64_t* dmeta = nullptr;
  cudaError_t e;
  if ((e = cudaMallocAsync(&t1, b1, s)) != cudaSuccess) return e;
  if ((e = cudaMallocAsync(&t2, b2, s)) != cudaSuccess) return e;
  if ((e = cudaMallocAsync(&t3, bz, s)) != cudaSuccess) return e;
  if ((e = cudaMallocAsync(&dw, sizeof(float) * 3 * kMaxTaps, s)) != cudaSuccess) return e;
  if ((e = cudaMallocAsync(&dmeta, sizeof(int64_t) * 18, s)) != cudaSuccess) return e;
  int64_t meta[18] = {job.in.lo[0], job.in.lo[1], job.in.lo[2], job.in.dims[0], job.in.dims[1],
                      job.in.dims[2],
                      rlo[0], rlo[1], lo[2], n_x[0], n_x[1], n_x[2],
                      rlo[0], lo[1], lo[2], n_y[0], n_y[1], n_y[2]};
  e = cudaMemcpyAsync(dmeta, meta, sizeof(meta), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dw, taps.w, sizeof(float) * 3 * kMaxTaps, cudaMemcpyHostToDevice, s);
  // cudaMemcpyAsync from pageable memory is staged synchronously, so the
  // host arrays above may go out of scope after return.
  if (e == cudaSuccess) {
    const int blk = 256;
    auto grid_for = [&](const int64_t* n) {
      int64_t t = n[0] * n[1] * n[2];
      return (unsigned)std::min<int64_t>((t + blk - 1) / blk, 148 * 32);
    };
    const float* wz = dw;
    const float* wy = dw + kMaxTaps;
    const float* wx = dw + 2 * kMaxTaps;
    switch (job.in.dtype) {
#define HP_PASS1(T)                                                                            \
  k_axis_pass<T><<<grid_for(n_x), blk, 0, s>>>(static_cast<const T*>(job.in.ptr), dmeta,     \
                                               dmeta + 3, t1, n_x[0], n_x[1], n_x[2], 2, wx, r, \
                                               job.gdims[0], job.gdims[1], job.gdims[2],        \
                                               rlo[0], rlo[1], lo[2]);                         \
  break;
      case HP_U8: HP_PASS1(uint8_t)
      case HP_U16: HP_PASS1(uint16_t)
      case HP_F16: HP_PASS1(__half)
      case HP_F32: HP_PASS1(float)
#undef HP_PASS1
    }
    k_axis_pass<float><<<grid_for(n_y), blk, 0, s>>>(t1, dmeta + 6, dmeta + 9, t2, n_y[0], n_y[1],
                                                     n_y[2], 1, wy, r, job.gdims[0], job.gdims[1],
                                                     job.gdims[2], rlo[0], lo[1], lo[2]);
    k_axis_pass<float><<<grid_for(n_z), blk, 0, s>>>(t2, dmeta + 12, dmeta + 15, t3, n_z[0],
                                                     n_z[1], n_z[2], 0, wz, r, job.gdims[0],
                                                     job.gdims[1], job.gdims[2], lo[0], lo[1],
                                                     lo[2]);
    k_copy_out<<<grid_for(n_z), blk, 0, s>>>(t3, n_z[0], n_z[1], n_z[2], job.out, lo[0], lo[1],
                                            lo[2]);
    e = cudaGetLastError();
  }
  cudaFreeAsync(t1, s);
  cudaFreeAsync(t2, s);
  cudaFreeAsync(t3, s);
  cudaFreeAsync(dw, s);
  cudaFreeAsync(dmeta, s);
  return e;
}

}  // namespace

cudaError_t launch_gauss(const Job& job, const Taps& taps, cudaStream_t s) {
  const int r = taps.r;
  bool tiled = r >= 1 && r <= kMaxR && job.gdims[2] >= r && job.gdims[1] >= r;
  if (!tiled) return launch_generic(job, taps, s);

  GaussParams P;
  P.job = job;
  for (int k = 0; k < kMaxTaps; ++k) {
    P.wz[k] = taps.w[0][k];
    P.wy[k] = taps.w[1][k];
    P.wx[k] = taps.w[2][k];
  }
  P.r = r;
  P.err = device_error_word();
  const int64_t cx = job.core_hi[2] - job.core_lo[2];
  const int64_t cy = job.core_hi[1] - job.core_lo[1];
  const int64_t cz = job.core_hi[0] - job.core_lo[0];
  if (cx <= 0 || cy <= 0 || cz <= 0) return cudaSuccess;
  P.tiles_x = (int)((cx + kTX - 1) / kTX);
  const int64_t tiles = (int64_t)P.tiles_x * ((cy + kTY - 1) / kTY);
  // z chunk: aim for >= 8 CTAs per SM in total, chunks of at least 4*BZ
  // planes so that the 2r halo planes stay a small fraction.
  const int64_t want = (int64_t)num_sms() * 8;
  int64_t nchunks = std::max<int64_t>(1, (want + tiles - 1) / tiles);
  int64_t zc = (cz + nchunks - 1) / nchunks;
  zc = std::max<int64_t>(zc, std::min<int64_t>(cz, 4 * kBZ));
  zc = (zc + kBZ - 1) / kBZ * kBZ;
  P.zchunk = (int)zc;
  dim3 grid((unsigned)tiles, (unsigned)((cz + zc - 1) / zc));

  // TMA needs 16-byte aligned rows and tile origins.
  CUtensorMap map;
  memset(&map, 0, sizeof(map));
  const size_t es = dtype_size(job.in.dtype);
  const int al = 16 / (int)es;
  bool use_tma = ((uintptr_t)job.in.ptr % 16 == 0) && ((job.in.dims[2] * (int64_t)es) % 16 == 0) &&
                 ((job.core_lo[2] - job.in.lo[2]) % al == 0);
  if (use_tma) {
    int ra = 0, bw = 0;
    box_geom(r, (int)es, &ra, &bw);
    const int64_t dims[3] = {job.in.dims[2], job.in.dims[1], job.in.dims[0]};
    use_tma = make_tmap_3d(&map, job.in.ptr, job.in.dtype, dims, bw, kTY + 2 * r);
  }
  P.use_tma = use_tma ? 1 : 0;
  if (log_level() > 0)
    fprintf(stderr, "[hp] gauss z-march r=%d tma=%d grid=%ux%u zchunk=%d smem=%d\n", r,
            P.use_tma, grid.x, grid.y, P.zchunk, 0);
  return dispatch_zm(r, P, map, grid, s);
}

}  // namespace hp
