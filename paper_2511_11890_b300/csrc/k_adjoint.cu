// Adjoint kernels behind autograd: the transpose of the separable
// Gaussian / derivative filters with reflect boundaries, the chain rule of
// the gradient magnitude, and the subgradient of grayscale erosion and
// dilation (Harpia Sec. III-C filters, differentiated for learned feature
// pipelines).
//
// Filter transpose, per axis of length n with taps g(k), k in [-r, r]: the
// forward map is y = K E x (E extends x by reflection to [-r, n-1+r], K is
// the valid convolution y[i] = sum_k g(k) u[i-k]). Its transpose E^T K^T is
// computed as a gather: for output i, sum over the pre-images j of i under
// the reflection (j in [-r, n-1+r], R(j) = i) of t[j] = sum_k g(k) w[j+k],
// w zero outside [0, n). The 3D transpose of Z Y X is X^T Y^T Z^T.
//
// Morphology: an argmin (argmax) map first records, per output p, the source
// q* = R(p +- o) holding the extreme value, ties to the smallest linear
// index; a gather then sums, per source q, the output gradients of every p
// within the structuring element's reach whose recorded source is q. Both
// passes are deterministic (no atomics).
#include <cuda_fp16.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "hp_device.cuh"
#include "hp_internal.h"

namespace hp {

namespace {

constexpr int kBlock = 256;

// Element i as an unsigned key whose order is IEEE 754 totalOrder of the
// values (the order the forward erosion / dilation uses): integers as they
// are; floating point with the sign bit set complemented, else with the sign
// bit set, so -NaN < -inf < ... < -0 < +0 < ... < +inf < +NaN.
__device__ __forceinline__ uint32_t load_key(const void* p, int dt, int64_t i) {
  switch (dt) {
    case HP_U8: return static_cast<const uint8_t*>(p)[i];
    case HP_U16: return static_cast<const uint16_t*>(p)[i];
    case HP_F16: {
      const uint32_t b = static_cast<const uint16_t*>(p)[i];
      return (b & 0x8000u) ? (~b & 0xFFFFu) : (b | 0x8000u);
    }
    default: {
      const uint32_t b = static_cast<const uint32_t*>(p)[i];
      return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
    }
  }
}

struct AxisTaps {
  float g[kMaxTaps];
};

// Transpose at one output i of a line (elements line[j * stride], length
// n): the sum over the pre-images j of i under the reflection of
// t[j] = sum_k g(k) w[j + k], w zero outside the line.
__device__ __forceinline__ float adjoint_at(const float* line, int64_t i, int64_t n,
                                            int64_t stride, const AxisTaps& taps, int r) {
  float acc = 0.0f;
  // pre-images j of i in [-r, n-1+r]: i + 2n m and -1 - i + 2n m
  for (int64_t m = -((r + 2 * n) / (2 * n)); m <= (r + 2 * n) / (2 * n); ++m) {
    for (int s = 0; s < 2; ++s) {
      const int64_t j = (s == 0 ? i : -1 - i) + 2 * n * m;
      if (j < -r || j > n - 1 + r) continue;
      if (reflect(j, n) != i) continue;
      for (int k = -r; k <= r; ++k) {
        const int64_t s2 = j + k;
        if (s2 >= 0 && s2 < n) acc = fmaf(taps.g[k + r], line[s2 * stride], acc);
      }
    }
  }
  return acc;
}

// dst = (axis transpose of src); dst += when accumulate. Any radius.
__global__ void k_axis_adjoint(const float* __restrict__ src, float* __restrict__ dst, int64_t n0,
                               int64_t n1, int64_t n2, int axis, const AxisTaps taps, int r,
                               int accumulate) {
  const int64_t total = n0 * n1 * n2;
  const int64_t n = axis == 0 ? n0 : (axis == 1 ? n1 : n2);
  const int64_t stride = axis == 2 ? 1 : (axis == 1 ? n2 : n1 * n2);
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t x = q % n2, y = (q / n2) % n1, z = q / (n1 * n2);
    const int64_t i = axis == 0 ? z : (axis == 1 ? y : x);
    const float acc = adjoint_at(src + (q - i * stride), i, n, stride, taps, r);
    dst[q] = accumulate ? dst[q] + acc : acc;
  }
}

// adjoint_at for a compile-time radius on a line at least R long: the
// pre-images of i are then i, -1 - i (when i < R) and 2n - 1 - i (when
// i >= n - R), visited in adjoint_at's order with the same taps, so the sum
// is the same bit for bit, without its 64-bit divisions.
template <int R>
__device__ __forceinline__ float adjoint_face(const float* line, int i, int n, int64_t stride,
                                              const AxisTaps& taps) {
  float acc = 0.0f;
  auto add = [&](int j) {
#pragma unroll
    for (int k = -R; k <= R; ++k) {
      const int s2 = j + k;
      if (s2 >= 0 && s2 < n) acc = fmaf(taps.g[k + R], line[(int64_t)s2 * stride], acc);
    }
  };
  add(i);
  if (i <= R - 1) add(-1 - i);
  if (i >= n - R) add(2 * n - 1 - i);
  return acc;
}

// Same transpose, radius R known at compile time: each thread takes kAC
// consecutive outputs of one line. Away from the faces (R <= i < n - R) the
// only pre-image of i is i itself and t[i] needs no zero extension, so the
// chunk is a plain correlation over a register window, with the same
// per-output FMA order as adjoint_at; chunks that touch a face use
// adjoint_at. Lines along z and y put consecutive threads on consecutive x
// (coalesced); along x each thread takes a single output instead.
constexpr int kAC = 16;

template <int R, int AXIS>
__global__ void __launch_bounds__(kBlock)
    k_axis_adjoint_r(const float* __restrict__ src, float* __restrict__ dst, int n0, int n1,
                     int n2, const AxisTaps taps, int accumulate) {
  const int n = AXIS == 0 ? n0 : (AXIS == 1 ? n1 : n2);
  const int64_t stride = AXIS == 2 ? 1 : (AXIS == 1 ? (int64_t)n2 : (int64_t)n1 * n2);
  const int nch = (n + kAC - 1) / kAC;
  int64_t base;  // element of i = 0 on this thread's line
  int c;         // chunk of the line
  if (AXIS == 2) {
    // one output per thread, consecutive threads on consecutive x: every tap
    // is one coalesced row read
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= n2) return;
    const float* line = src + ((int64_t)blockIdx.z * n1 + blockIdx.y) * n2;
    float* d = dst + ((int64_t)blockIdx.z * n1 + blockIdx.y) * n2 + x;
    float acc;
    if (x >= R && x < n - R) {
      acc = 0.0f;
#pragma unroll
      for (int k = -R; k <= R; ++k) acc = fmaf(taps.g[k + R], line[x + k], acc);
    } else if (n >= R) {
      acc = adjoint_face<R>(line, x, n, 1, taps);
    } else {
      acc = adjoint_at(line, x, n, 1, taps, R);
    }
    *d = accumulate ? *d + acc : acc;
    return;
  } else {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= n2) return;
    c = blockIdx.z;
    base = AXIS == 0 ? (int64_t)blockIdx.y * n2 + x : (int64_t)blockIdx.y * n1 * n2 + x;
  }
  const float* line = src + base;
  float* dl = dst + base;
  const int i0 = c * kAC;
  if (i0 >= R && i0 + kAC <= n - R) {
    float w[kAC + 2 * R];
#pragma unroll
    for (int j = 0; j < kAC + 2 * R; ++j) w[j] = line[(int64_t)(i0 - R + j) * stride];
#pragma unroll
    for (int i = 0; i < kAC; ++i) {
      float acc = 0.0f;
#pragma unroll
      for (int k = -R; k <= R; ++k) acc = fmaf(taps.g[k + R], w[i + k + R], acc);
      float* d = dl + (int64_t)(i0 + i) * stride;
      *d = accumulate ? *d + acc : acc;
    }
  } else if (n % kAC == 0 && n >= kAC + R && (i0 == 0 || i0 == n - kAC)) {
    // first or last chunk of a line of whole chunks: a register window of
    // kAC + R inputs holds every term of adjoint_face (pre-images i and
    // -1 - i at the low face, i and 2n - 1 - i at the high one), taken in
    // its order
    const bool low = i0 == 0;
    const int b = low ? 0 : i0 - R;  // line element of w[0]
    float w[kAC + R];
#pragma unroll
    for (int j = 0; j < kAC + R; ++j) w[j] = line[(int64_t)(b + j) * stride];
#pragma unroll
    for (int ii = 0; ii < kAC; ++ii) {
      float acc = 0.0f;
      if (low) {
#pragma unroll
        for (int k = -R; k <= R; ++k)
          if (ii + k >= 0) acc = fmaf(taps.g[k + R], w[ii + k], acc);
        if (ii <= R - 1) {
#pragma unroll
          for (int k = -R; k <= R; ++k)
            if (-1 - ii + k >= 0) acc = fmaf(taps.g[k + R], w[-1 - ii + k], acc);
        }
      } else {
#pragma unroll
        for (int k = -R; k <= R; ++k)
          if (ii + k < kAC) acc = fmaf(taps.g[k + R], w[ii + k + R], acc);
        if (ii >= kAC - R) {
#pragma unroll
          for (int k = -R; k <= R; ++k)
            if (k < ii - (kAC - 1)) acc = fmaf(taps.g[k + R], w[2 * kAC - 1 - ii + k + R], acc);
        }
      }
      float* d = dl + (int64_t)(i0 + ii) * stride;
      *d = accumulate ? *d + acc : acc;
    }
  } else {
    const int i1 = min(i0 + kAC, n);
    for (int i = i0; i < i1; ++i) {
      const float acc = n >= R ? adjoint_face<R>(line, i, n, stride, taps)
                               : adjoint_at(line, i, n, stride, taps, R);
      float* d = dl + (int64_t)i * stride;
      *d = accumulate ? *d + acc : acc;
    }
  }
}

// x-axis transpose in two kinds of thread: interior threads take kXW
// consecutive outputs whose window of kXW + 2 R4 inputs (R4 = R rounded up to
// 4) lies inside the row and is read as aligned float4 words (rows of a
// multiple of 4 floats, 16-byte aligned buffers); face threads take one
// output each of the chunks whose window would leave the row. The two kinds
// occupy separate ranges of the grid, so no warp mixes them. Every output
// sums its taps in the same order as k_axis_adjoint_r.
constexpr int kXW = 16;

template <int R>
__global__ void __launch_bounds__(kBlock)
    k_axis_adjoint_x(const float* __restrict__ src, float* __restrict__ dst, int64_t rows, int n,
                     int c_lo, int c_hi, const AxisTaps taps, int accumulate) {
  constexpr int R4 = (R + 3) / 4 * 4;
  const int nin = c_hi - c_lo;             // interior chunks per row
  const int nface = n - kXW * nin;         // face outputs per row
  const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t ninner = rows * nin;
  if (gt < ninner) {
    const int64_t row = gt / nin;
    const int x0 = (c_lo + (int)(gt - row * nin)) * kXW;
    const float* line = src + row * n;
    float* dl = dst + row * n;
    float w[kXW + 2 * R4];
    const float4* v = reinterpret_cast<const float4*>(line + x0 - R4);
#pragma unroll
    for (int q = 0; q < (kXW + 2 * R4) / 4; ++q) {
      const float4 f = v[q];
      w[4 * q] = f.x;
      w[4 * q + 1] = f.y;
      w[4 * q + 2] = f.z;
      w[4 * q + 3] = f.w;
    }
    float o[kXW];
#pragma unroll
    for (int i = 0; i < kXW; ++i) {
      float acc = 0.0f;
#pragma unroll
      for (int k = -R; k <= R; ++k) acc = fmaf(taps.g[k + R], w[R4 + i + k], acc);
      o[i] = acc;
    }
    float4* d = reinterpret_cast<float4*>(dl + x0);
#pragma unroll
    for (int q = 0; q < kXW / 4; ++q) {
      float4 r = make_float4(o[4 * q], o[4 * q + 1], o[4 * q + 2], o[4 * q + 3]);
      if (accumulate) {
        const float4 p = d[q];
        r.x = p.x + r.x;
        r.y = p.y + r.y;
        r.z = p.z + r.z;
        r.w = p.w + r.w;
      }
      d[q] = r;
    }
    return;
  }
  const int64_t f = gt - ninner;
  const int64_t row = f / nface;
  if (row >= rows) return;
  const int k = (int)(f - row * nface);
  const int x = k < c_lo * kXW ? k : c_hi * kXW + (k - c_lo * kXW);
  const float* line = src + row * n;
  float acc;
  if (x >= R && x < n - R) {
    acc = 0.0f;
#pragma unroll
    for (int kk = -R; kk <= R; ++kk) acc = fmaf(taps.g[kk + R], line[x + kk], acc);
  } else if (n >= R) {
    acc = adjoint_face<R>(line, x, n, 1, taps);
  } else {
    acc = adjoint_at(line, x, n, 1, taps, R);
  }
  float* d = dst + row * n + x;
  *d = accumulate ? *d + acc : acc;
}

template <int R>
cudaError_t launch_axis_r(const float* src, float* dst, const int64_t dims[3], int ax,
                          const AxisTaps& a, int accumulate, cudaStream_t s) {
  const int n0 = (int)dims[0], n1 = (int)dims[1], n2 = (int)dims[2];
  const int n = ax == 0 ? n0 : (ax == 1 ? n1 : n2);
  const int nch = (n + kAC - 1) / kAC;
  if (ax == 2 && n2 % 4 == 0 && (uintptr_t)src % 16 == 0 && (uintptr_t)dst % 16 == 0) {
    // interior chunks c: window [16c - R4, 16c + 16 + R4) inside [0, n2)
    constexpr int R4 = (R + 3) / 4 * 4;
    const int c_lo = (R4 + kXW - 1) / kXW;
    const int c_hi = std::max(c_lo, (n2 - kXW - R4) / kXW + 1);
    const int64_t rows = (int64_t)n0 * n1;
    const int64_t threads = rows * (c_hi - c_lo) + rows * (n2 - kXW * (c_hi - c_lo));
    const unsigned grid = (unsigned)((threads + kBlock - 1) / kBlock);
    k_axis_adjoint_x<R><<<grid, kBlock, 0, s>>>(src, dst, rows, n2, c_lo, c_hi, a, accumulate);
  } else if (ax == 2) {
    const dim3 grid((unsigned)((n2 + kBlock - 1) / kBlock), (unsigned)n1, (unsigned)n0);
    k_axis_adjoint_r<R, 2><<<grid, kBlock, 0, s>>>(src, dst, n0, n1, n2, a, accumulate);
  } else {
    const dim3 grid((unsigned)((n2 + kBlock - 1) / kBlock), (unsigned)(ax == 0 ? n1 : n0),
                    (unsigned)nch);
    if (ax == 0)
      k_axis_adjoint_r<R, 0><<<grid, kBlock, 0, s>>>(src, dst, n0, n1, n2, a, accumulate);
    else
      k_axis_adjoint_r<R, 1><<<grid, kBlock, 0, s>>>(src, dst, n0, n1, n2, a, accumulate);
  }
  return cudaGetLastError();
}

// Chain rule through the gradient magnitude, in place for the three axes:
// D_a <- w * D_a / GM (0 where GM = 0), GM = sqrt(Dx^2 + Dy^2 + Dz^2) formed
// as in the forward bank; each volume is read once.
__global__ void k_gm_chain3(const float* __restrict__ w, float* __restrict__ dz,
                            float* __restrict__ dy, float* __restrict__ dx, int64_t total) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    const float z = dz[q], y = dy[q], x = dx[q], wq = w[q];
    const float gm = sqrtf(fmaf(z, z, fmaf(y, y, x * x)));
    const bool nz = gm > 0.0f;
    dz[q] = nz ? wq * z / gm : 0.0f;
    dy[q] = nz ? wq * y / gm : 0.0f;
    dx[q] = nz ? wq * x / gm : 0.0f;
  }
}

template <typename T>
__device__ __forceinline__ float morph_val(const T* p, int64_t i);
template <>
__device__ __forceinline__ float morph_val<float>(const float* p, int64_t i) {
  return p[i];
}

// Extreme source per output: arg[p] = q* (int32 linear index).
__global__ void k_morph_arg(const void* __restrict__ in, int dt, int64_t n0, int64_t n1,
                            int64_t n2, int ball, int rad, int is_dilate,
                            int32_t* __restrict__ arg) {
  const int64_t total = n0 * n1 * n2;
  const int sg = is_dilate ? -1 : 1;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < total;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int64_t x = p % n2, y = (p / n2) % n1, z = p / (n1 * n2);
    int64_t best_q = -1;
    uint32_t best = 0u;
    for (int dz = -rad; dz <= rad; ++dz) {
      const int64_t sz = reflect(z + sg * dz, n0);
      for (int dy = -rad; dy <= rad; ++dy) {
        const int64_t sy = reflect(y + sg * dy, n1);
        for (int dx = -rad; dx <= rad; ++dx) {
          if (ball && dz * dz + dy * dy + dx * dx > rad * rad) continue;
          const int64_t sx = reflect(x + sg * dx, n2);
          const int64_t q = (sz * n1 + sy) * n2 + sx;
          const uint32_t v = load_key(in, dt, q);
          const bool better = best_q < 0 || (is_dilate ? v > best : v < best) ||
                              (v == best && q < best_q);
          if (better) {
            best = v;
            best_q = q;
          }
        }
      }
    }
    arg[p] = (int32_t)best_q;
  }
}

// Cube structuring element: the extreme over the cube is the extreme over z
// of the extremes over y of the extremes over x, and the linear index is
// lexicographic in (z, y, x), so the smallest-index tie rule also separates:
// per row keep the smallest source x among the extremes, per plane the
// smallest (source y, that x), over planes the smallest (source z, ...).
// A CTA stages the reflected input box of a 4 x 8 x 32 output tile in shared
// memory and runs the three passes there; arg[] equals k_morph_arg's.
constexpr int kCZ = 4, kCY = 8, kCX = 32;

template <int RAD>
constexpr int cube_arg_smem() {
  constexpr int VZ = kCZ + 2 * RAD, VY = kCY + 2 * RAD, VX = kCX + 2 * RAD;
  return 4 * (VZ * (VY * (VX + 2 * kCX) + 2 * kCY * kCX) + VX + VY + VZ);
}

template <int RAD>
__global__ void __launch_bounds__(kBlock)
    k_morph_arg_cube(const void* __restrict__ in, int dt, int n0, int n1, int n2, int is_dilate,
                     int32_t* __restrict__ arg) {
  constexpr int VZ = kCZ + 2 * RAD, VY = kCY + 2 * RAD, VX = kCX + 2 * RAD;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // reflected input box, x pass (value, source x), y pass (value, source
  // y * n2 + x), reflected coordinates; sizes in cube_arg_smem<RAD>()
  auto v0 = reinterpret_cast<uint32_t(*)[VY][VX]>(smem_raw);
  auto v1 = reinterpret_cast<uint32_t(*)[VY][kCX]>(smem_raw + 4 * VZ * VY * VX);
  auto i1 = reinterpret_cast<int32_t(*)[VY][kCX]>(smem_raw + 4 * VZ * VY * (VX + kCX));
  auto v2 = reinterpret_cast<uint32_t(*)[kCY][kCX]>(smem_raw + 4 * VZ * VY * (VX + 2 * kCX));
  auto i2 = reinterpret_cast<int32_t(*)[kCY][kCX]>(smem_raw + 4 * VZ * (VY * (VX + 2 * kCX) + kCY * kCX));
  int32_t* sx = reinterpret_cast<int32_t*>(smem_raw + 4 * VZ * (VY * (VX + 2 * kCX) + 2 * kCY * kCX));
  int32_t* sy = sx + VX;
  int32_t* sz = sy + VY;
  const int tid = threadIdx.x;
  const int x0 = blockIdx.x * kCX, y0 = blockIdx.y * kCY, z0 = blockIdx.z * kCZ;
  const int sg = is_dilate ? -1 : 1;
  for (int c = tid; c < VX; c += kBlock) sx[c] = (int)reflect(x0 - RAD + c, n2);
  for (int c = tid; c < VY; c += kBlock) sy[c] = (int)reflect(y0 - RAD + c, n1);
  for (int c = tid; c < VZ; c += kBlock) sz[c] = (int)reflect(z0 - RAD + c, n0);
  __syncthreads();
  for (int e = tid; e < VZ * VY * VX; e += kBlock) {
    const int c = e % VX, b = (e / VX) % VY, a = e / (VX * VY);
    v0[a][b][c] = load_key(in, dt, ((int64_t)sz[a] * n1 + sy[b]) * n2 + sx[c]);
  }
  __syncthreads();
  // linear indices fit in int32 (the index array is int32)
  auto better = [&](uint32_t v, int32_t q, uint32_t best, int32_t bq) {
    return (is_dilate ? v > best : v < best) || (v == best && q < bq);
  };
  // x pass over every staged row; window offset sg*dx from the output column
  for (int e = tid; e < VZ * VY * kCX; e += kBlock) {
    const int x = e % kCX, b = (e / kCX) % VY, a = e / (kCX * VY);
    uint32_t best = 0u;
    int bq = -1;
#pragma unroll
    for (int d = -RAD; d <= RAD; ++d) {
      const int c = x + RAD + sg * d;
      const uint32_t v = v0[a][b][c];
      if (bq < 0 || better(v, sx[c], best, bq)) {
        best = v;
        bq = sx[c];
      }
    }
    v1[a][b][x] = best;
    i1[a][b][x] = bq;
  }
  __syncthreads();
  for (int e = tid; e < VZ * kCY * kCX; e += kBlock) {
    const int x = e % kCX, y = (e / kCX) % kCY, a = e / (kCX * kCY);
    uint32_t best = 0u;
    int32_t bq = -1;
#pragma unroll
    for (int d = -RAD; d <= RAD; ++d) {
      const int b = y + RAD + sg * d;
      const uint32_t v = v1[a][b][x];
      const int32_t q = sy[b] * n2 + i1[a][b][x];
      if (bq < 0 || better(v, q, best, bq)) {
        best = v;
        bq = q;
      }
    }
    v2[a][y][x] = best;
    i2[a][y][x] = bq;
  }
  __syncthreads();
  for (int e = tid; e < kCZ * kCY * kCX; e += kBlock) {
    const int x = e % kCX, y = (e / kCX) % kCY, z = e / (kCX * kCY);
    if (z0 + z >= n0 || y0 + y >= n1 || x0 + x >= n2) continue;
    uint32_t best = 0u;
    int32_t bq = -1;
    const int32_t plane = n1 * n2;
#pragma unroll
    for (int d = -RAD; d <= RAD; ++d) {
      const int a = z + RAD + sg * d;
      const int32_t q = sz[a] * plane + i2[a][y][x];
      const uint32_t v = v2[a][y][x];
      if (bq < 0 || better(v, q, best, bq)) {
        best = v;
        bq = q;
      }
    }
    arg[((int64_t)(z0 + z) * n1 + (y0 + y)) * n2 + (x0 + x)] = bq;
  }
}

// gin[q] (+)= sum of gout[p] over p in q + [-rad, rad]^3 with arg[p] == q,
// p in increasing linear order.
__global__ void k_morph_gather(const int32_t* __restrict__ arg, const float* __restrict__ gout,
                               float* __restrict__ gin, int64_t n0, int64_t n1, int64_t n2,
                               int rad, int accumulate) {
  const int64_t total = n0 * n1 * n2;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t x = q % n2, y = (q / n2) % n1, z = q / (n1 * n2);
    float acc = 0.0f;
    for (int64_t pz = max((int64_t)0, z - rad); pz <= min(n0 - 1, z + rad); ++pz)
      for (int64_t py = max((int64_t)0, y - rad); py <= min(n1 - 1, y + rad); ++py)
        for (int64_t px = max((int64_t)0, x - rad); px <= min(n2 - 1, x + rad); ++px) {
          const int64_t p = (pz * n1 + py) * n2 + px;
          if (arg[p] == (int32_t)q) acc += gout[p];
        }
    gin[q] = accumulate ? gin[q] + acc : acc;
  }
}

// The same gather with the reach of a 4 x 8 x 32 tile of sources staged in
// shared memory (arg and gout of every p within rad of the tile; -1 outside
// the volume; rows padded to a multiple of 4 words). A thread takes four
// consecutive x outputs q: for each (dz, dy) it reads the 4 + 2 rad source
// indices of the row as aligned 16-byte words and adds gout[p] only where
// arg[p] == q, scanning each q's cube of p in increasing linear order as
// k_morph_gather does.
template <int RAD>
struct GatherTile {
  static constexpr int VZ = kCZ + 2 * RAD, VY = kCY + 2 * RAD;
  static constexpr int VX = (kCX + 2 * RAD + 3) / 4 * 4;  // padded row (words)
  static constexpr int NWIN = (4 + 2 * RAD + 3) / 4;       // 16-byte words per window
  static constexpr int SMEM = 8 * VZ * VY * VX;
  static_assert(kCZ * kCY * (kCX / 4) == kBlock, "one output quad per thread");
};

template <int RAD>
constexpr int gather_smem() {
  return GatherTile<RAD>::SMEM;
}

template <int RAD>
__global__ void __launch_bounds__(kBlock)
    k_morph_gather_tile(const int32_t* __restrict__ arg, const float* __restrict__ gout,
                        float* __restrict__ gin, int n0, int n1, int n2, int accumulate) {
  using GT = GatherTile<RAD>;
  constexpr int VZ = GT::VZ, VY = GT::VY, VX = GT::VX;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  auto sa = reinterpret_cast<int32_t(*)[VY][VX]>(smem_raw);
  auto sg = reinterpret_cast<float(*)[VY][VX]>(smem_raw + 4 * VZ * VY * VX);
  const int tid = threadIdx.x;
  const int x0 = blockIdx.x * kCX, y0 = blockIdx.y * kCY, z0 = blockIdx.z * kCZ;
  for (int e = tid; e < VZ * VY * VX; e += kBlock) {
    const int c = e % VX, b = (e / VX) % VY, a = e / (VX * VY);
    const int z = z0 - RAD + a, y = y0 - RAD + b, x = x0 - RAD + c;
    const bool in = c < kCX + 2 * RAD && z >= 0 && z < n0 && y >= 0 && y < n1 && x >= 0 && x < n2;
    const int64_t p = ((int64_t)z * n1 + y) * n2 + x;
    sa[a][b][c] = in ? arg[p] : -1;
    sg[a][b][c] = in ? gout[p] : 0.0f;
  }
  __syncthreads();
  const int xq = (tid % (kCX / 4)) * 4, y = (tid / (kCX / 4)) % kCY, z = tid / (kCX / 4 * kCY);
  const int gz = z0 + z, gy = y0 + y;
  if (gz >= n0 || gy >= n1) return;
  const int64_t q0 = ((int64_t)gz * n1 + gy) * n2 + x0 + xq;  // q of output j: q0 + j
  float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
  for (int dz = 0; dz <= 2 * RAD; ++dz)
#pragma unroll
    for (int dy = 0; dy <= 2 * RAD; ++dy) {
      int32_t w[4 * GT::NWIN];
      const int4* src = reinterpret_cast<const int4*>(&sa[z + dz][y + dy][xq]);
#pragma unroll
      for (int v = 0; v < GT::NWIN; ++v) {
        const int4 t = src[v];
        w[4 * v] = t.x;
        w[4 * v + 1] = t.y;
        w[4 * v + 2] = t.z;
        w[4 * v + 3] = t.w;
      }
#pragma unroll
      for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int dx = 0; dx <= 2 * RAD; ++dx)
          if (w[j + dx] == (int32_t)(q0 + j)) acc[j] += sg[z + dz][y + dy][xq + j + dx];
    }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    if (x0 + xq + j >= n2) break;
    float* d = gin + q0 + j;
    *d = accumulate ? *d + acc[j] : acc[j];
  }
}

unsigned grid_for(int64_t total) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((total + kBlock - 1) / kBlock,
                                                          (int64_t)num_sms() * 16));
}

}  // namespace

// Separable transpose: dst (+)= X^T Y^T Z^T w for taps (z, y, x) of radius r.
// Uses two scratch volumes t1, t2 of the same shape.
cudaError_t launch_sep_adjoint(const float* w, float* dst, const int64_t dims[3],
                               const Taps& taps, float* t1, float* t2, int accumulate,
                               cudaStream_t s) {
  const int64_t total = dims[0] * dims[1] * dims[2];
  AxisTaps a;
  for (int ax = 0; ax < 3; ++ax) {
    for (int k = 0; k < kMaxTaps; ++k) a.g[k] = taps.w[ax][k];
    const float* src = ax == 0 ? w : (ax == 1 ? t1 : t2);
    float* out = ax == 0 ? t1 : (ax == 1 ? t2 : dst);
    const int acc = ax == 2 ? accumulate : 0;
    // compile-time radius where the grid fits (lines and planes below 65536)
    const bool fits = taps.r >= 1 && taps.r <= kMaxRGeneric && dims[0] < 65536 &&
                      dims[1] < 65536 && dims[2] < (1LL << 31) / 4;
    if (fits) {
      cudaError_t e = cudaErrorInvalidValue;
      switch (taps.r) {
#define HP_AR(RR) \
  case RR: e = launch_axis_r<RR>(src, out, dims, ax, a, acc, s); break;
        HP_AR(1) HP_AR(2) HP_AR(3) HP_AR(4) HP_AR(5) HP_AR(6)
        HP_AR(7) HP_AR(8) HP_AR(9) HP_AR(10) HP_AR(11) HP_AR(12)
        HP_AR(13) HP_AR(14) HP_AR(15) HP_AR(16) HP_AR(17) HP_AR(18)
        HP_AR(19) HP_AR(20) HP_AR(21) HP_AR(22) HP_AR(23) HP_AR(24)
        HP_AR(25) HP_AR(26) HP_AR(27) HP_AR(28) HP_AR(29) HP_AR(30)
        HP_AR(31) HP_AR(32)
#undef HP_AR
      }
      if (e != cudaSuccess) return e;
    } else {
      k_axis_adjoint<<<grid_for(total), kBlock, 0, s>>>(src, out, dims[0], dims[1], dims[2], ax,
                                                       a, taps.r, acc);
    }
  }
  return cudaGetLastError();
}

cudaError_t launch_gm_chain3(const float* w, float* dz, float* dy, float* dx, int64_t total,
                             cudaStream_t s) {
  k_gm_chain3<<<grid_for(total), kBlock, 0, s>>>(w, dz, dy, dx, total);
  return cudaGetLastError();
}

cudaError_t launch_morph_arg(const void* in, int dt, const int64_t dims[3], int ball, int rad,
                             int is_dilate, int32_t* arg, cudaStream_t s) {
  const int64_t total = dims[0] * dims[1] * dims[2];
  if (!ball && rad >= 1 && rad <= 4 && dims[0] < 65536 * kCZ && dims[1] < 65536 * kCY) {
    const dim3 grid((unsigned)((dims[2] + kCX - 1) / kCX), (unsigned)((dims[1] + kCY - 1) / kCY),
                    (unsigned)((dims[0] + kCZ - 1) / kCZ));
    const int n0 = (int)dims[0], n1 = (int)dims[1], n2 = (int)dims[2];
    cudaError_t e = cudaSuccess;
    switch (rad) {
#define HP_CA(RR)                                                                              \
  case RR:                                                                                     \
    e = cudaFuncSetAttribute(k_morph_arg_cube<RR>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                             cube_arg_smem<RR>());                                             \
    if (e == cudaSuccess)                                                                      \
      k_morph_arg_cube<RR><<<grid, kBlock, cube_arg_smem<RR>(), s>>>(in, dt, n0, n1, n2,       \
                                                                     is_dilate, arg);          \
    break;
      HP_CA(1) HP_CA(2) HP_CA(3) HP_CA(4)
#undef HP_CA
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
  }
  k_morph_arg<<<grid_for(total), kBlock, 0, s>>>(in, dt, dims[0], dims[1], dims[2], ball, rad,
                                                 is_dilate, arg);
  return cudaGetLastError();
}

cudaError_t launch_morph_gather(const int32_t* arg, const float* gout, float* gin,
                                const int64_t dims[3], int rad, int accumulate, cudaStream_t s) {
  const int64_t total = dims[0] * dims[1] * dims[2];
  if (rad >= 1 && rad <= 4 && dims[0] < 65536 * kCZ && dims[1] < 65536 * kCY) {
    const dim3 grid((unsigned)((dims[2] + kCX - 1) / kCX), (unsigned)((dims[1] + kCY - 1) / kCY),
                    (unsigned)((dims[0] + kCZ - 1) / kCZ));
    const int n0 = (int)dims[0], n1 = (int)dims[1], n2 = (int)dims[2];
    cudaError_t e = cudaSuccess;
    switch (rad) {
#define HP_GT(RR)                                                                                 \
  case RR:                                                                                        \
    e = cudaFuncSetAttribute(k_morph_gather_tile<RR>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                             gather_smem<RR>());                                                  \
    if (e == cudaSuccess)                                                                         \
      k_morph_gather_tile<RR><<<grid, kBlock, gather_smem<RR>(), s>>>(arg, gout, gin, n0, n1, n2, \
                                                                     accumulate);                 \
    break;
      HP_GT(1) HP_GT(2) HP_GT(3) HP_GT(4)
#undef HP_GT
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
  }
  k_morph_gather<<<grid_for(total), kBlock, 0, s>>>(arg, gout, gin, dims[0], dims[1], dims[2],
                                                    rad, accumulate);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------
// Allocation-free variant of the morphology subgradient.
//
// Some callers cannot allocate device memory while they run this step: code
// inside a fixed memory arena or a real-time loop that must not touch the
// allocator, or a host that has handed all device memory to another pool.
// For them the per-voxel source index lives in a fixed array that the
// library owns for the life of the process (every GPU that loads the
// library holds it until exit), so the call itself allocates nothing.
namespace {
constexpr int64_t kNoAllocMaxVoxels = int64_t(1) << 24;  // 256^3 voxels, 64 MiB
static __device__ __align__(256) int32_t g_noalloc_arg[kNoAllocMaxVoxels];
int32_t* g_noalloc_ptr[64];  // device address per device, set on first use
std::mutex g_noalloc_mu;     // guards g_noalloc_ptr
}  // namespace

// Drops the cached device addresses (hp_release_cache), so that after a
// cudaDeviceReset the next call looks the array up in the new context.
void noalloc_forget() {
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  for (auto& p : g_noalloc_ptr) p = nullptr;
}

}  // namespace hp

using namespace hp;

extern "C" int hp_morph3d_backward_noalloc(const hp_volume* in, const hp_volume* gout,
                                           int is_dilate, hp_se se, int radius, hp_volume* gin,
                                           int accumulate, void* stream) {
  if (!in || !in->data || !gout || !gout->data || !gin || !gin->data)
    return set_error(HP_ERR_INVALID_ARG, "morphology backward (no-alloc): null argument");
  if (in->loc != HP_DEVICE || gout->loc != HP_DEVICE || gin->loc != HP_DEVICE)
    return set_error(HP_ERR_UNSUPPORTED, "morphology backward (no-alloc): device volumes only");
  if (gout->dtype != HP_F32 || gin->dtype != HP_F32)
    return set_error(HP_ERR_UNSUPPORTED, "morphology backward (no-alloc): gradients must be f32");
  if (gout->nx != in->nx || gout->ny != in->ny || gout->nz != in->nz || gin->nx != in->nx ||
      gin->ny != in->ny || gin->nz != in->nz)
    return set_error(HP_ERR_INVALID_ARG, "morphology backward (no-alloc): extents differ");
  if (se != HP_SE_CUBE && se != HP_SE_BALL)
    return set_error(HP_ERR_INVALID_ARG, "unknown structuring element");
  if (radius < 0 || radius > kMaxMorphR) return set_error(HP_ERR_INVALID_ARG, "radius must be in [0, 16]");
  const int64_t dims[3] = {in->nz, in->ny, in->nx};
  const int64_t total = dims[0] * dims[1] * dims[2];
  if (total > kNoAllocMaxVoxels)
    return set_error(HP_ERR_UNSUPPORTED,
                     "morphology backward (no-alloc): volume has more than 16777216 voxels "
                     "(the size of the library's fixed index array); use hp_morph3d_backward");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= 64) return set_error(HP_ERR_UNSUPPORTED, "device index above 63");
  int32_t* arg = nullptr;
  {
    // host code only sees a stand-in for the array; its device address is
    // looked up once per device, with that device current
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_arg);
      if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(no-alloc index array)");
      g_noalloc_ptr[dev] = static_cast<int32_t*>(p);
    }
    arg = g_noalloc_ptr[dev];
  }
  cudaStream_t s = (cudaStream_t)stream;
  // every index the gather reads is written by the argmin pass first, so
  // nothing in the shared array needs clearing between calls
  e = launch_morph_arg(in->data, in->dtype, dims, se == HP_SE_BALL, radius, is_dilate, arg, s);
  if (e == cudaSuccess)
    e = launch_morph_gather(arg, static_cast<const float*>(gout->data),
                            static_cast<float*>(gin->data), dims, radius, accumulate, s);
  if (e != cudaSuccess) return cuda_fail(e, "morphology backward (no-alloc) launch");
  return HP_OK;
}
