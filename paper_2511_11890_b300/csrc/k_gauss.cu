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

// Shared-memory layout of the z-march kernel for radius R. The TMA box
// width depends on the element size (its x origin must be 16-byte aligned),
// so the stage buffers are sized for the widest element (4 bytes).
template <int R>
struct ZmGeom {
  static constexpr int BH = kTY + 2 * R;                  // TMA box height
  static constexpr int FWN = kTX + 2 * R;                 // needed FP32 patch width
  static constexpr int FW = patch_stride(FWN);
  static constexpr int NRING = kBZ + 2 * R;
  static constexpr int STAGE_BYTES = round_up(round_up(kTX + round_up(R, 4) + R, 4) * BH * 4, 128);
  static constexpr int OFF_STAGE = 128;
  static constexpr int OFF_F = OFF_STAGE + kNS * STAGE_BYTES;
  static constexpr int OFF_X = OFF_F + round_up(BH * FW * 4, 128);
  static constexpr int OFF_RING = OFF_X + round_up(BH * kXS * 4, 128);
  static constexpr int SMEM = OFF_RING + NRING * kTY * kTX * 4;
  static_assert(FW >= FWN && FW % 8 == 4, "FP32 patch row stride must be 4 mod 8 floats");
};

// Per-dtype TMA box geometry: left halo ra rounded up to 16 bytes, width bw.
__host__ __device__ inline void box_geom(int r, int es, int* ra, int* bw) {
  const int al = 16 / es;
  *ra = round_up(r, al);
  *bw = round_up(kTX + *ra + r, al);
}

// Convert rows of the raw TMA stage into the FP32 patch, resolving
// reflections at the volume faces (raw col c <-> x = cx0 - ra + c).
template <typename TIN, int R>
__device__ __forceinline__ void convert_patch(float* F, const unsigned char* rawb, int ra, int bw,
                                              bool face, int64_t cx0, int64_t cy0, int64_t Gx,
                                              int64_t Gy, int warp, int lane) {
  using G = ZmGeom<R>;
  const TIN* raw = reinterpret_cast<const TIN*>(rawb);
  for (int row = warp; row < G::BH; row += kThreads / 32) {
    int srow = row;
    if (face) srow = (int)(reflect(cy0 - R + row, Gy) - (cy0 - R));
    for (int col = lane; col < G::FWN; col += 32) {
      int scol = col + (ra - R);
      bool ok = true;
      if (face) {
        scol = (int)(reflect(cx0 - R + col, Gx) - (cx0 - ra));
        ok = scol >= 0 && scol < bw && srow >= 0 && srow < G::BH;
      }
      F[row * G::FW + col] = ok ? to_f32<TIN>(raw[srow * bw + scol]) : 0.0f;
    }
  }
}

// Cooperative load of one plane straight from global memory (layouts TMA
// cannot address), with reflection on global coordinates.
template <typename TIN, int R>
__device__ __forceinline__ void load_patch(float* F, const Job& J, int64_t iz, int64_t cx0,
                                           int64_t cy0, int warp, int lane) {
  using G = ZmGeom<R>;
  const TIN* in = static_cast<const TIN*>(J.in.ptr);
  const int64_t sz = reflect(iz, J.gdims[0]) - J.in.lo[0];
  for (int row = warp; row < G::BH; row += kThreads / 32) {
    const int64_t sy = reflect(cy0 - R + row, J.gdims[1]) - J.in.lo[1];
    for (int col = lane; col < G::FWN; col += 32) {
      const int64_t sx = reflect(cx0 - R + col, J.gdims[2]) - J.in.lo[2];
      float v = 0.0f;
      if (sz >= 0 && sz < J.in.dims[0] && sy >= 0 && sy < J.in.dims[1] && sx >= 0 &&
          sx < J.in.dims[2])
        v = to_f32<TIN>(in[(sz * J.in.dims[1] + sy) * J.in.dims[2] + sx]);
      F[row * G::FW + col] = v;
    }
  }
}

template <typename T>
__device__ __forceinline__ void store_out(void* base, int dt, int64_t idx, float v) {
  if (dt == HP_F32)
    static_cast<float*>(base)[idx] = v;
  else
    static_cast<__half*>(base)[idx] = __float2half_rn(v);
}

template <int R>
__global__ void __launch_bounds__(kThreads, 1)
    k_gauss_zm(const __grid_constant__ GaussParams P, const __grid_constant__ CUtensorMap tmap) {
  using G = ZmGeom<R>;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
  float* F = reinterpret_cast<float*>(smem + G::OFF_F);
  float* X = reinterpret_cast<float*>(smem + G::OFF_X);
  float* ring = reinterpret_cast<float*>(smem + G::OFF_RING);
  __shared__ int s_abort;

  const Job& J = P.job;
  const int tid = threadIdx.x;
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
  const bool face = (cx0 - R < 0) || (cx0 + kTX + R > Gx) || (cy0 - R < 0) || (cy0 + kTY + R > Gy);
  const bool tma = P.use_tma != 0;

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
    const int64_t iz = cz0 - R + n;
    const int zl = (int)(reflect(iz, Gz) - J.in.lo[0]);
    const int xl = (int)(cx0 - ra - J.in.lo[2]);
    const int yl = (int)(cy0 - R - J.in.lo[1]);
    uint64_t* bar = &bars[n % kNS];
    mbar_arrive_expect_tx(bar, bw * G::BH * es);
    tma_load_3d(smem + G::OFF_STAGE + (n % kNS) * G::STAGE_BYTES, &tmap, xl, yl, zl, bar);
  };
  if (tma && tid == 0) {
    fence_proxy_async();
    for (int n = 0; n < min(kNS, total); ++n) issue(n);
  }

  // thread roles
  const int xrow = tid / (kTX / 8), xg = (tid % (kTX / 8)) * 8;       // x pass
  const int yx = tid % kTX, yb = (tid / kTX) * 4;                      // y pass
  const int zy = tid / (kTX / 4), zx4 = (tid % (kTX / 4)) * 4;         // z pass
  const int warp = tid / 32, lane = tid % 32;

  int produced = 0;
  for (int zb = 0; zb < nout; zb += kBZ) {
    const int need = min(zb + kBZ + 2 * R, total);
    for (; produced < need; ++produced) {
      const int n = produced;
      const int64_t iz = cz0 - R + n;
      // ---- 1. stage the FP32 patch F[BH][FW] (cols <-> x = cx0-R .. cx0+TX+R-1)
      if (tma) {
        if (!mbar_wait(&bars[n % kNS], (n / kNS) & 1)) atomicOr(&s_abort, 1);
        const unsigned char* rawb = smem + G::OFF_STAGE + (n % kNS) * G::STAGE_BYTES;
        switch (dt) {
          case HP_U8: convert_patch<uint8_t, R>(F, rawb, ra, bw, face, cx0, cy0, Gx, Gy, warp, lane); break;
          case HP_U16: convert_patch<uint16_t, R>(F, rawb, ra, bw, face, cx0, cy0, Gx, Gy, warp, lane); break;
          case HP_F16: convert_patch<__half, R>(F, rawb, ra, bw, face, cx0, cy0, Gx, Gy, warp, lane); break;
          default: convert_patch<float, R>(F, rawb, ra, bw, face, cx0, cy0, Gx, Gy, warp, lane); break;
        }
      } else {
        switch (dt) {
          case HP_U8: load_patch<uint8_t, R>(F, J, iz, cx0, cy0, warp, lane); break;
          case HP_U16: load_patch<uint16_t, R>(F, J, iz, cx0, cy0, warp, lane); break;
          case HP_F16: load_patch<__half, R>(F, J, iz, cx0, cy0, warp, lane); break;
          default: load_patch<float, R>(F, J, iz, cx0, cy0, warp, lane); break;
        }
      }
      __syncthreads();
      if (s_abort) break;
      if (tma && tid == 0 && n + kNS < total) {
        fence_proxy_async();
        issue(n + kNS);
      }
      // ---- 2. x pass: X[row][x] for BH rows, TX columns
      if (xrow < G::BH) {
        constexpr int WN = 8 + 2 * R;
        float w[round_up(WN, 4)];
        const float4* src = reinterpret_cast<const float4*>(F + xrow * G::FW + xg);
#pragma unroll
        for (int j = 0; j < round_up(WN, 4) / 4; ++j) {
          float4 v = src[j];
          w[4 * j] = v.x;
          w[4 * j + 1] = v.y;
          w[4 * j + 2] = v.z;
          w[4 * j + 3] = v.w;
        }
        float o[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          float acc = 0.0f;
#pragma unroll
          for (int j = i; j <= i + 2 * R; ++j) acc = fmaf(P.wx[i - j + 2 * R], w[j], acc);
          o[i] = acc;
        }
        float4* dst = reinterpret_cast<float4*>(X + xrow * kXS + xg);
        dst[0] = make_float4(o[0], o[1], o[2], o[3]);
        dst[1] = make_float4(o[4], o[5], o[6], o[7]);
      }
      __syncthreads();
      // ---- 3. y pass into the ring slot of plane n
      {
        float w[4 + 2 * R];
#pragma unroll
        for (int j = 0; j < 4 + 2 * R; ++j) w[j] = X[(yb + j) * kXS + yx];
        float* slot = ring + (n % G::NRING) * (kTY * kTX);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          float acc = 0.0f;
#pragma unroll
          for (int j = i; j <= i + 2 * R; ++j) acc = fmaf(P.wy[i - j + 2 * R], w[j], acc);
          slot[(yb + i) * kTX + yx] = acc;
        }
      }
      __syncthreads();
    }
    if (s_abort) break;
    // ---- 4. z pass: outputs zb .. zb+BZ-1 from ring planes zb .. zb+BZ+2R-1
    {
      float4 acc[kBZ];
#pragma unroll
      for (int j = 0; j < kBZ; ++j) acc[j] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int m = 0; m < kBZ + 2 * R; ++m) {
        const float4 v = *reinterpret_cast<const float4*>(
            ring + ((zb + m) % G::NRING) * (kTY * kTX) + zy * kTX + zx4);
#pragma unroll
        for (int j = 0; j < kBZ; ++j) {
          if (m >= j && m <= j + 2 * R) {
            const float g = P.wz[j - m + 2 * R];
            acc[j].x = fmaf(g, v.x, acc[j].x);
            acc[j].y = fmaf(g, v.y, acc[j].y);
            acc[j].z = fmaf(g, v.z, acc[j].z);
            acc[j].w = fmaf(g, v.w, acc[j].w);
          }
        }
      }
      const int64_t gy = cy0 + zy, gx = cx0 + zx4;
      if (gy < J.core_hi[1]) {
        const DevOut& O = J.out;
        const int64_t od1 = O.dims[1], od2 = O.dims[2];
        const bool full4 = gx + 3 < J.core_hi[2];
#pragma unroll
        for (int j = 0; j < kBZ; ++j) {
          const int64_t gz = cz0 + zb + j;
          if (gz >= cz1) break;
          const int64_t idx = ((gz - O.lo[0]) * od1 + (gy - O.lo[1])) * od2 + (gx - O.lo[2]);
          const float vv[4] = {acc[j].x, acc[j].y, acc[j].z, acc[j].w};
          if (O.dtype == HP_F32 && full4 &&
              (reinterpret_cast<uintptr_t>(static_cast<float*>(O.ptr) + idx) & 15) == 0) {
            *reinterpret_cast<float4*>(static_cast<float*>(O.ptr) + idx) = acc[j];
          } else {
#pragma unroll
            for (int e = 0; e < 4; ++e)
              if (full4 || gx + e < J.core_hi[2]) store_out<float>(O.ptr, O.dtype, idx + e, vv[e]);
          }
        }
      }
    }
    __syncthreads();  // ring slots are overwritten by the next block
  }
  if (s_abort) {
    set_device_error(P.err, kErrTimeout);
    // drain TMA loads still in flight into this CTA's shared memory
    if (tma && tid == 0)
      for (int n = max(0, produced); n < min(produced + kNS, total); ++n)
        (void)mbar_wait(&bars[n % kNS], (n / kNS) & 1);
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
  using G = ZmGeom<R>;
  static bool attr_set = false;  // per instantiation; set once per process
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_gauss_zm<R>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  k_gauss_zm<R><<<grid, kThreads, G::SMEM, s>>>(P, map);
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
