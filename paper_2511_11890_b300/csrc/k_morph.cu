// Grayscale erosion / dilation (Harpia Sec. III-C, morphological label
// editing) with cube and ball structuring elements, reflect boundaries on
// global coordinates, exact results.
//
// Values are mapped to order-preserving unsigned keys (u8/u16 as is; f16/f32
// sign-magnitude flipped), so min/max are integer operations and exact.
// Dilation is erosion of the complemented keys (complement reverses order).
//
// Tiled z-march kernel (radius 1..6): a CTA owns a 32 x 32 column of the
// core and marches along z. Per input plane it stages the halo-padded patch
// (TMA tile load into a 4-stage mbarrier pipeline, or cooperative loads),
// then
//   x: running minima M_L over x-lines of half-length L = 0..r (for the
//      cube only L = r is kept);
//   y: the ball is the union of x-lines {|dx| <= L(dy,dz)}, with
//      L(dy,dz) = floor(sqrt(r^2 - dy^2 - dz^2)), so each plane's disk
//      minima D_|dz| = min over dy of M_L(dy,dz)(y + dy) (cube: D = min over
//      |dy| <= r of M_r) are formed per thread from a register window;
//   z: D_|dz| of plane z' is pushed into the accumulators of outputs
//      z' -+ dz held in a register ring of 2r+1 slots; an output is complete
//      r planes after its own plane and is stored then.
// Min is associative and exact, so the result does not depend on tiling.
#include <cuda_fp16.h>

#include <float.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>

#include <type_traits>

#include "hp_device.cuh"
#include "hp_internal.h"

namespace hp {

namespace {

constexpr int kTX = 32;
constexpr int kTY = 32;
constexpr int kYB = 4;
constexpr int kNS = 4;
constexpr int kThreads = 256;
constexpr int kMaxTiledR = 6;      // cube (larger cubes: van Herk / Gil-Werman passes)
constexpr int kMaxTiledBallR = kMaxMorphR;  // ball: every accepted radius
// Balls above this radius take 16-row tiles with two output rows per thread
// (so that the z ring of 2r + 1 slots stays in registers) and a single
// line-minimum buffer (the r + 1 levels of the tile's rows fill ~108 KB at
// r = 16), with a second barrier per phase.
constexpr int kMaxDblR = 10;

struct MorphParams {
  Job job;
  int zchunk;
  int tiles_x;
  int use_tma;
  int is_dilate;
  int* err;
};

__host__ __device__ constexpr int round_up(int a, int b) { return (a + b - 1) / b * b; }
__host__ __device__ constexpr int isqrt(int v) {
  int s = 0;
  while ((s + 1) * (s + 1) <= v) ++s;
  return s;
}
// Ball decomposition, fixed at compile time: the x-line at (dy, dz) has
// half-length L = floor(sqrt(R^2 - dy^2 - dz^2)); template recursion over dy
// keeps every L and every shared-memory offset a compile-time constant.
// (Cube: one line of half-length R for every dy.)
template <int R, int BALL, int BH, int DZ, int DY>
__device__ __forceinline__ void disk_min(uint32_t& d, const uint32_t* Mb) {
  if constexpr (DY <= R) {
    if constexpr (!BALL || DZ * DZ + DY * DY <= R * R) {
      constexpr int L = BALL ? isqrt(R * R - DZ * DZ - DY * DY) : 0;
      d = min(d, Mb[(L * BH + DY + R) * (32 + 1)]);
    }
    disk_min<R, BALL, BH, DZ, DY + 1>(d, Mb);
  }
}

// Ball of radius 3: the disks share one 3-row minimum A of M2:
//   D1 = min(M2[y-2..y+2]) = min(A, M2[y-2], M2[y+2])      (|dz| = 1)
//   D0 = min(D1, M3[y], M0[y-3], M0[y+3])                  (|dz| = 0; M2[y] >= M3[y])
//   D2 = min(A, M1[y-2], M1[y+2])                          (|dz| = 2)
//   D3 = M0[y]                                             (|dz| = 3)
// (half-lengths floor(sqrt(9 - dy^2 - dz^2)); 9 min operations per row
// instead of 18).
template <int BH, int YB>
__device__ __forceinline__ void disk_rows_ball3(uint32_t (&D)[4][YB], const uint32_t* Mb) {
  constexpr int S = 32 + 1;
  auto m = [&](int L, int dy, int i) { return Mb[(L * BH + dy + 3) * S + i * S]; };
#pragma unroll
  for (int i = 0; i < YB; ++i) {
    const uint32_t a = min(min(m(2, -1, i), m(2, 0, i)), m(2, 1, i));
    const uint32_t d1 = min(a, min(m(2, -2, i), m(2, 2, i)));
    D[1][i] = d1;
    D[0][i] = min(min(d1, m(3, 0, i)), min(m(0, -3, i), m(0, 3, i)));
    D[2][i] = min(a, min(m(1, -2, i), m(1, 2, i)));
    D[3][i] = m(0, 0, i);
  }
}

template <int R, int BALL, int BH, int DZ, int YB>
__device__ __forceinline__ void disk_rows(uint32_t (&D)[BALL ? R + 1 : 1][YB], const uint32_t* Mb) {
  if constexpr (DZ <= (BALL ? R : 0)) {
#pragma unroll
    for (int i = 0; i < YB; ++i) {
      uint32_t d = 0xFFFFFFFFu;
      disk_min<R, BALL, BH, DZ, -R>(d, Mb + i * (32 + 1));
      D[DZ][i] = d;
    }
    disk_rows<R, BALL, BH, DZ + 1, YB>(D, Mb);
  }
}

// Odd row strides (in 32-bit words) spread the 8 rows x 4 column groups a
// warp touches over all 32 banks.
__host__ __device__ constexpr int key_stride(int n) { return n | 1; }
constexpr int kMS = kTX + 1;  // row stride of the line-minimum arrays

// Order-preserving keys.
template <typename T>
__device__ __forceinline__ uint32_t to_key(T v);
template <>
__device__ __forceinline__ uint32_t to_key<uint8_t>(uint8_t v) {
  return v;
}
template <>
__device__ __forceinline__ uint32_t to_key<uint16_t>(uint16_t v) {
  return v;
}
template <>
__device__ __forceinline__ uint32_t to_key<__half>(__half v) {
  uint32_t b = __half_as_ushort(v);
  return (b & 0x8000u) ? (~b & 0xFFFFu) : (b | 0x8000u);
}
template <>
__device__ __forceinline__ uint32_t to_key<float>(float v) {
  uint32_t b = __float_as_uint(v);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
template <typename T>
__device__ __forceinline__ T from_key(uint32_t k);
template <>
__device__ __forceinline__ uint8_t from_key<uint8_t>(uint32_t k) {
  return (uint8_t)k;
}
template <>
__device__ __forceinline__ uint16_t from_key<uint16_t>(uint32_t k) {
  return (uint16_t)k;
}
template <>
__device__ __forceinline__ __half from_key<__half>(uint32_t k) {
  uint32_t b = (k & 0x8000u) ? (k & 0x7FFFu) : (~k & 0xFFFFu);
  return __ushort_as_half((unsigned short)b);
}
template <>
__device__ __forceinline__ float from_key<float>(uint32_t k) {
  uint32_t b = (k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k;
  return __uint_as_float(b);
}
// Keys of narrow types occupy the low bits; complementing within the type's
// width keeps them comparable.
template <typename T>
struct KeyMask {
  static constexpr uint32_t value = sizeof(T) == 4 ? 0xFFFFFFFFu : (sizeof(T) == 2 ? 0xFFFFu : 0xFFu);
};

// Geometry for radius R: K (keys, double-buffered) col c <-> x = cx0 - R + c,
// row <-> y = cy0 - R + row; M (x-line minima, double-buffered) [NL][BH][kMS].
template <int R, int BALL>
struct MGeom {
  static constexpr bool BIG = BALL && R > kMaxDblR;
  static constexpr int TY = BIG ? 16 : kTY;   // tile rows
  static constexpr int YB = BIG ? 2 : kYB;    // output rows per thread (disks, z ring)
  static constexpr int NMB = BIG ? 1 : 2;     // line-minimum buffers
  static constexpr int BH = TY + 2 * R;
  static constexpr int KWN = kTX + 2 * R;
  static constexpr int KW = key_stride(KWN);
  static constexpr int NC = (KWN + 31) / 32;
  static constexpr int NL = BALL ? R + 1 : 1;  // stored x-line minima
  static constexpr int NR = 2 * R + 1;         // z accumulator ring
  static constexpr int KSZ = BH * KW;
  static constexpr int MSZ = NL * BH * kMS;
  static constexpr int TAIL = (2 * KSZ + NMB * MSZ) * 4 + BH * 4;
  static_assert(kThreads == kTX * TY / YB && BH <= kThreads / (kTX / 8), "thread map");
};

__host__ __device__ inline void mbox_geom(int r, int es, int* ra, int* bw) {
  const int al = 16 / es;
  *ra = round_up(r, al);
  *bw = round_up(kTX + *ra + r, al);
}

__host__ __device__ inline int mstage_bytes(int r, int es, int ty) {
  int ra, bw;
  mbox_geom(r, es, &ra, &bw);
  return round_up(bw * (ty + 2 * r) * es, 128);
}

template <int R, int BALL>
__host__ __device__ inline int mzm_smem_bytes(int es) {
  return 128 + kNS * mstage_bytes(R, es, MGeom<R, BALL>::TY) + MGeom<R, BALL>::TAIL;
}

template <typename TIN, int R, int BALL>
__device__ __forceinline__ void keys_from_tma(uint32_t* Kb, const unsigned char* rawb, int bw,
                                              const int* srow,
                                              const int (&scol)[MGeom<R, BALL>::NC],
                                              uint32_t flip, int warp, int lane) {
  using G = MGeom<R, BALL>;
  const TIN* raw = reinterpret_cast<const TIN*>(rawb);
  for (int row = warp; row < G::BH; row += kThreads / 32) {
    const int sr = srow[row];
#pragma unroll
    for (int k = 0; k < G::NC; ++k) {
      const int col = lane + 32 * k;
      if (col < G::KWN) {
        const int sc = scol[k];
        Kb[row * G::KW + col] = (sr >= 0 && sc >= 0) ? (to_key<TIN>(raw[sr * bw + sc]) ^ flip) : 0u;
      }
    }
  }
}

// Interior tiles: K col c <-> raw col c + (ra - R), four keys per item.
template <typename TIN, int R, int BALL>
__device__ __forceinline__ void keys_from_tma_interior(uint32_t* Kb, const unsigned char* rawb,
                                                       int ra, int bw, uint32_t flip, int tid) {
  using G = MGeom<R, BALL>;
  constexpr int Q = (G::KWN + 3) / 4;
  const TIN* raw = reinterpret_cast<const TIN*>(rawb) + (ra - R);
  for (int it = tid; it < G::BH * Q; it += kThreads) {
    const int row = it / Q, q = it - row * Q;
    const TIN* src = raw + row * bw + 4 * q;
    uint32_t* dst = Kb + row * G::KW + 4 * q;
#pragma unroll
    for (int e = 0; e < 4; ++e)
      if (4 * q + e < G::KWN) dst[e] = to_key<TIN>(src[e]) ^ flip;
  }
}

template <typename TIN, int R, int BALL>
__device__ __forceinline__ void keys_from_global(uint32_t* Kb, const Job& J, int64_t sz,
                                                 const int* srow,
                                                 const int (&scol)[MGeom<R, BALL>::NC],
                                                 uint32_t flip, int warp, int lane) {
  using G = MGeom<R, BALL>;
  const TIN* in = static_cast<const TIN*>(J.in.ptr);
  const bool zok = sz >= 0 && sz < J.in.dims[0];
  const TIN* plane = in + sz * J.in.dims[1] * J.in.dims[2];
  for (int row = warp; row < G::BH; row += kThreads / 32) {
    const int sr = srow[row];
#pragma unroll
    for (int k = 0; k < G::NC; ++k) {
      const int col = lane + 32 * k;
      if (col < G::KWN) {
        const int sc = scol[k];
        Kb[row * G::KW + col] = (zok && sr >= 0 && sc >= 0)
                                    ? (to_key<TIN>(plane[(int64_t)sr * J.in.dims[2] + sc]) ^ flip)
                                    : 0u;
      }
    }
  }
}

__device__ __forceinline__ uint32_t key_mask(int dt) {
  return dt == HP_F32 ? 0xFFFFFFFFu : (dt == HP_U8 ? 0xFFu : 0xFFFFu);
}

__device__ __forceinline__ void store_key(void* base, int dt, int64_t idx, uint32_t k) {
  switch (dt) {
    case HP_U8: static_cast<uint8_t*>(base)[idx] = from_key<uint8_t>(k); break;
    case HP_U16: static_cast<uint16_t*>(base)[idx] = from_key<uint16_t>(k); break;
    case HP_F16: static_cast<__half*>(base)[idx] = from_key<__half>(k); break;
    default: static_cast<float*>(base)[idx] = from_key<float>(k); break;
  }
}

// Push one plane's disk minima D[|dz|] into the z ring with the ring
// rotation U (compile time, so the ring stays in registers), then hand out
// the output that became complete and recycle its slot.
template <int R, int BALL, int U>
__device__ __forceinline__ void push_rot(uint32_t (&acc)[2 * R + 1][kYB],
                                         const uint32_t (&D)[BALL ? R + 1 : 1][kYB],
                                         uint32_t (&done)[kYB]) {
  constexpr int NR = 2 * R + 1;
#pragma unroll
  for (int i = 0; i < kYB; ++i) {
    if (BALL) {
#pragma unroll
      for (int dz = 0; dz <= R; ++dz) {
        acc[(U + dz) % NR][i] = min(acc[(U + dz) % NR][i], D[BALL ? dz : 0][i]);
        if (dz > 0) acc[(U - dz + NR) % NR][i] = min(acc[(U - dz + NR) % NR][i], D[BALL ? dz : 0][i]);
      }
    } else {
#pragma unroll
      for (int e = -R; e <= R; ++e) acc[(U + e + NR) % NR][i] = min(acc[(U + e + NR) % NR][i], D[0][i]);
    }
    constexpr int slot = (U - R + NR) % NR;
    done[i] = acc[slot][i];
    acc[slot][i] = 0xFFFFFFFFu;
  }
}

template <int R, int BALL, int U = 0>
__device__ __forceinline__ void push_dispatch(int u, uint32_t (&acc)[2 * R + 1][kYB],
                                              const uint32_t (&D)[BALL ? R + 1 : 1][kYB],
                                              uint32_t (&done)[kYB]) {
  if constexpr (U < 2 * R + 1) {
    if (u == U)
      push_rot<R, BALL, U>(acc, D, done);
    else
      push_dispatch<R, BALL, U + 1>(u, acc, D, done);
  }
}

template <int R, int BALL>
__global__ void __launch_bounds__(kThreads, 1)
    k_morph_zm(const __grid_constant__ MorphParams P, const __grid_constant__ CUtensorMap tmap) {
  using G = MGeom<R, BALL>;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ int s_abort;

  const Job& J = P.job;
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const int tx = blockIdx.x % P.tiles_x, ty = blockIdx.x / P.tiles_x;
  const int64_t cx0 = J.core_lo[2] + (int64_t)tx * kTX;
  const int64_t cy0 = J.core_lo[1] + (int64_t)ty * G::TY;
  const int64_t cz0 = J.core_lo[0] + (int64_t)blockIdx.y * P.zchunk;
  const int64_t cz1 = min(cz0 + (int64_t)P.zchunk, J.core_hi[0]);
  if (cz0 >= cz1) return;
  const int nout = (int)(cz1 - cz0);
  const int total = nout + 2 * R;
  const int64_t Gz = J.gdims[0], Gy = J.gdims[1], Gx = J.gdims[2];
  const int dt = J.in.dtype;
  const int es = dt == HP_U8 ? 1 : (dt == HP_F32 ? 4 : 2);
  int ra, bw;
  mbox_geom(R, es, &ra, &bw);
  const int sbytes = mstage_bytes(R, es, G::TY);
  const bool tma = P.use_tma != 0;
  const uint32_t flip = P.is_dilate ? key_mask(dt) : 0u;
  const bool face = (cx0 - R < 0) || (cx0 + kTX + R > Gx) || (cy0 - R < 0) || (cy0 + G::TY + R > Gy);

  uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
  unsigned char* stages = smem + 128;
  uint32_t* K = reinterpret_cast<uint32_t*>(stages + kNS * sbytes);
  uint32_t* M = K + 2 * G::KSZ;
  int* srow = reinterpret_cast<int*>(M + G::NMB * G::MSZ);

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
    const int64_t sx = reflect(cx0 - R + col, Gx);
    int v = -1;
    if (tma) {
      const int64_t s = sx - (cx0 - ra);
      if (s >= 0 && s < bw) v = (int)s;
    } else {
      const int64_t s = sx - J.in.lo[2];
      if (s >= 0 && s < J.in.dims[2]) v = (int)s;
    }
    scol[k] = col < G::KWN ? v : -1;
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

  auto issue = [&](int n) {
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

  const int xrow = tid / (kTX / 8), xg = (tid % (kTX / 8)) * 8;
  constexpr int YB = G::YB;
  const int yx = tid % kTX, yb = (tid / kTX) * YB;

  uint32_t acc[G::NR][YB];
#pragma unroll
  for (int s = 0; s < G::NR; ++s)
#pragma unroll
    for (int i = 0; i < YB; ++i) acc[s][i] = 0xFFFFFFFFu;

  // phase p: stage keys of plane p, x-line minima of plane p-1, disk minima
  // and z push of plane p-2; one barrier per phase. With one line-minimum
  // buffer (large balls) the disks of plane p-2 come first, then a barrier,
  // then the x-line minima of plane p-1 overwrite the buffer.
  int p = 0;
  for (; p < total + 2; ++p) {
    if (p < total) {
      uint32_t* Kb = K + (p & 1) * G::KSZ;
      if (tma) {
        if (!mbar_wait(&bars[p % kNS], (p / kNS) & 1)) atomicOr(&s_abort, 1);
        const unsigned char* rawb = stages + (p % kNS) * sbytes;
        if (!face) {
          switch (dt) {
            case HP_U8: keys_from_tma_interior<uint8_t, R, BALL>(Kb, rawb, ra, bw, flip, tid); break;
            case HP_U16: keys_from_tma_interior<uint16_t, R, BALL>(Kb, rawb, ra, bw, flip, tid); break;
            case HP_F16: keys_from_tma_interior<__half, R, BALL>(Kb, rawb, ra, bw, flip, tid); break;
            default: keys_from_tma_interior<float, R, BALL>(Kb, rawb, ra, bw, flip, tid); break;
          }
        } else {
          switch (dt) {
            case HP_U8: keys_from_tma<uint8_t, R, BALL>(Kb, rawb, bw, srow, scol, flip, warp, lane); break;
            case HP_U16: keys_from_tma<uint16_t, R, BALL>(Kb, rawb, bw, srow, scol, flip, warp, lane); break;
            case HP_F16: keys_from_tma<__half, R, BALL>(Kb, rawb, bw, srow, scol, flip, warp, lane); break;
            default: keys_from_tma<float, R, BALL>(Kb, rawb, bw, srow, scol, flip, warp, lane); break;
          }
        }
      } else {
        const int64_t sz = reflect(cz0 - R + p, Gz) - J.in.lo[0];
        switch (dt) {
          case HP_U8: keys_from_global<uint8_t, R, BALL>(Kb, J, sz, srow, scol, flip, warp, lane); break;
          case HP_U16: keys_from_global<uint16_t, R, BALL>(Kb, J, sz, srow, scol, flip, warp, lane); break;
          case HP_F16: keys_from_global<__half, R, BALL>(Kb, J, sz, srow, scol, flip, warp, lane); break;
          default: keys_from_global<float, R, BALL>(Kb, J, sz, srow, scol, flip, warp, lane); break;
        }
      }
    }
    auto xline_part = [&]() {
      if (p >= 1 && p - 1 < total && xrow < G::BH) {
        const uint32_t* Kb = K + ((p - 1) & 1) * G::KSZ;
        uint32_t* Mb = M + (G::BIG ? 0 : ((p - 1) & 1) * G::MSZ);
        uint32_t w[8 + 2 * R];
#pragma unroll
        for (int j = 0; j < 8 + 2 * R; ++j) w[j] = Kb[xrow * G::KW + xg + j];
        // window index j <-> x = cx0 + xg - R + j. Line minima of growing
        // half-length: M1 = min of 3, then M_L[j] = min(M_{L-1}[j-1], M_{L-1}[j+1])
        // (the two windows of half-length L-1 cover the one of half-length L).
        uint32_t m[8 + 2 * R];
#pragma unroll
        for (int j = 0; j < 8 + 2 * R; ++j) m[j] = w[j];
#pragma unroll
        for (int i = 0; i < 8; ++i)
          if (BALL) Mb[(0 * G::BH + xrow) * kMS + xg + i] = w[i + R];
#pragma unroll
        for (int L = 1; L <= R; ++L) {
          uint32_t t[8 + 2 * R];
#pragma unroll
          for (int j = L; j < 8 + 2 * R - L; ++j)
            t[j] = L == 1 ? min(min(m[j - 1], m[j]), m[j + 1]) : min(m[j - 1], m[j + 1]);
#pragma unroll
          for (int j = L; j < 8 + 2 * R - L; ++j) m[j] = t[j];
          if (BALL || L == R) {
#pragma unroll
            for (int i = 0; i < 8; ++i)
              Mb[((BALL ? L : 0) * G::BH + xrow) * kMS + xg + i] = m[i + R];
          }
        }
      }
    };
    auto disk_part = [&]() {
      if (p >= 2) {
        const int n = p - 2;
        const uint32_t* Mb = M + (G::BIG ? 0 : (n & 1) * G::MSZ);
        uint32_t D[BALL ? R + 1 : 1][YB];
        static_assert(kMS == 32 + 1, "disk_min assumes the line-minimum row stride");
        if constexpr (BALL && R == 3)
          disk_rows_ball3<G::BH, YB>(D, Mb + yb * kMS + yx);
        else
          disk_rows<R, BALL, G::BH, 0, YB>(D, Mb + yb * kMS + yx);
        uint32_t done[YB];
        if constexpr (G::BIG) {
          // shift ring: acc[s] holds the output centred on plane n - R + s;
          // plane n adds its disk at |s - R|, the output of slot 0 is complete
#pragma unroll
          for (int i = 0; i < YB; ++i) {
            done[i] = min(acc[0][i], D[R][i]);
#pragma unroll
            for (int s2 = 1; s2 <= 2 * R; ++s2) acc[s2 - 1][i] = min(acc[s2][i], D[s2 > R ? s2 - R : R - s2][i]);
            acc[2 * R][i] = 0xFFFFFFFFu;
          }
        } else {
          push_dispatch<R, BALL>(n % G::NR, acc, D, done);
        }
        const int64_t gz = cz0 - R + n - R, gx = cx0 + yx;  // plane n's input z minus R
        if (gz >= cz0 && gz < cz1 && gx < J.core_hi[2]) {
          const DevOut& O = J.out;
#pragma unroll
          for (int i = 0; i < YB; ++i) {
            const int64_t gy = cy0 + yb + i;
            if (gy < J.core_hi[1]) {
              const int64_t idx =
                  ((gz - O.lo[0]) * O.dims[1] + (gy - O.lo[1])) * O.dims[2] + (gx - O.lo[2]);
              store_key(O.ptr, dt, idx, done[i] ^ flip);
            }
          }
        }
      }
    };
    if constexpr (G::BIG) {
      disk_part();
      __syncthreads();
      xline_part();
    } else {
      xline_part();
      disk_part();
    }
    __syncthreads();
    if (s_abort) break;
    if (tma && tid == 0 && p + kNS < total) {
      fence_proxy_async();
      issue(p + kNS);
    }
  }
  if (s_abort) {
    set_device_error(P.err, kErrTimeout);
    if (tma && tid == 0)
      for (int m = p; m < min(p + kNS, total); ++m) (void)mbar_wait(&bars[m % kNS], (m / kNS) & 1);
    __syncthreads();
  }
}

// Generic brute force over the structuring element (any radius <= 16, any
// extents): one thread per output voxel.
template <typename TIN>
__global__ void k_morph_generic(const Job J, int ball, int rad, int is_dilate) {
  const int64_t n0 = J.core_hi[0] - J.core_lo[0], n1 = J.core_hi[1] - J.core_lo[1],
                n2 = J.core_hi[2] - J.core_lo[2];
  const int64_t total = n0 * n1 * n2;
  const uint32_t flip = is_dilate ? KeyMask<TIN>::value : 0u;
  const TIN* in = static_cast<const TIN*>(J.in.ptr);
  const int sg = is_dilate ? -1 : 1;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t x = J.core_lo[2] + q % n2, y = J.core_lo[1] + (q / n2) % n1,
                  z = J.core_lo[0] + q / (n1 * n2);
    uint32_t m = 0xFFFFFFFFu;
    for (int dz = -rad; dz <= rad; ++dz)
      for (int dy = -rad; dy <= rad; ++dy)
        for (int dx = -rad; dx <= rad; ++dx) {
          if (ball && dz * dz + dy * dy + dx * dx > rad * rad) continue;
          const int64_t sz = reflect(z + sg * dz, J.gdims[0]) - J.in.lo[0];
          const int64_t sy = reflect(y + sg * dy, J.gdims[1]) - J.in.lo[1];
          const int64_t sx = reflect(x + sg * dx, J.gdims[2]) - J.in.lo[2];
          if (sz < 0 || sz >= J.in.dims[0] || sy < 0 || sy >= J.in.dims[1] || sx < 0 ||
              sx >= J.in.dims[2])
            continue;
          m = min(m, to_key<TIN>(in[(sz * J.in.dims[1] + sy) * J.in.dims[2] + sx]) ^ flip);
        }
    const DevOut& O = J.out;
    const int64_t idx = ((z - O.lo[0]) * O.dims[1] + (y - O.lo[1])) * O.dims[2] + (x - O.lo[2]);
    static_cast<TIN*>(O.ptr)[idx] = from_key<TIN>(m ^ flip);
  }
}

template <int R, int BALL>
cudaError_t launch_mzm(const MorphParams& P, const CUtensorMap& map, dim3 grid, cudaStream_t s) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_morph_zm<R, BALL>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         mzm_smem_bytes<R, BALL>(4));
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const int es = (int)dtype_size(P.job.in.dtype);
  k_morph_zm<R, BALL><<<grid, kThreads, mzm_smem_bytes<R, BALL>(es), s>>>(P, map);
  return cudaGetLastError();
}

template <int BALL>
cudaError_t dispatch_r(int r, const MorphParams& P, const CUtensorMap& map, dim3 grid,
                       cudaStream_t s) {
  switch (r) {
    case 1: return launch_mzm<1, BALL>(P, map, grid, s);
    case 2: return launch_mzm<2, BALL>(P, map, grid, s);
    case 3: return launch_mzm<3, BALL>(P, map, grid, s);
    case 4: return launch_mzm<4, BALL>(P, map, grid, s);
    case 5: return launch_mzm<5, BALL>(P, map, grid, s);
    case 6: return launch_mzm<6, BALL>(P, map, grid, s);
  }
  if constexpr (BALL) {
    switch (r) {
      case 7: return launch_mzm<7, BALL>(P, map, grid, s);
      case 8: return launch_mzm<8, BALL>(P, map, grid, s);
      case 9: return launch_mzm<9, BALL>(P, map, grid, s);
      case 10: return launch_mzm<10, BALL>(P, map, grid, s);
      case 11: return launch_mzm<11, BALL>(P, map, grid, s);
      case 12: return launch_mzm<12, BALL>(P, map, grid, s);
      case 13: return launch_mzm<13, BALL>(P, map, grid, s);
      case 14: return launch_mzm<14, BALL>(P, map, grid, s);
      case 15: return launch_mzm<15, BALL>(P, map, grid, s);
      case 16: return launch_mzm<16, BALL>(P, map, grid, s);
    }
  }
  return cudaErrorInvalidValue;
}

}  // namespace

template <typename T>
__global__ void k_difference(const T* __restrict__ in, T* __restrict__ out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float d = to_f32<T>(in[i]) - to_f32<T>(out[i]);
    if constexpr (std::is_same<T, __half>::value)
      out[i] = __float2half_rn(d);
    else if constexpr (std::is_same<T, float>::value)
      out[i] = d;
    else
      out[i] = (T)d;  // integers: in >= opening, the difference is exact
  }
}

// Same difference over 16-byte words (16 / sizeof(T) elements per word) of
// 16-byte aligned buffers whose length is a whole number of words.
template <typename T>
__global__ void k_difference_v(const uint4* __restrict__ in, uint4* __restrict__ out, int64_t nw) {
  constexpr int V = 16 / sizeof(T);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nw;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint4 a = in[i], b = out[i];
    const T* pa = reinterpret_cast<const T*>(&a);
    T* pb = reinterpret_cast<T*>(&b);
#pragma unroll
    for (int k = 0; k < V; ++k) {
      const float d = to_f32<T>(pa[k]) - to_f32<T>(pb[k]);
      if constexpr (std::is_same<T, __half>::value)
        pb[k] = __float2half_rn(d);
      else if constexpr (std::is_same<T, float>::value)
        pb[k] = d;
      else
        pb[k] = (T)d;
    }
    out[i] = b;
  }
}

// Rows of `rows` x `n` elements of type T (dense, source) into rows of
// `pitch` elements (destination, 16-byte aligned, pitch a whole number of
// 16-byte words): one thread per destination word, elements past n zero.
template <typename T>
__global__ void k_pad_rows(const T* __restrict__ src, uint4* __restrict__ dst, int64_t n,
                           int64_t pitch, int64_t rows) {
  constexpr int V = 16 / sizeof(T);
  const int64_t wpr = pitch / V;  // words per destination row
  const int64_t total = rows * wpr;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = q / wpr, c0 = (q - r * wpr) * V;
    const T* sr = src + r * n;
    uint4 w;
    T* e = reinterpret_cast<T*>(&w);
#pragma unroll
    for (int k = 0; k < V; ++k) e[k] = c0 + k < n ? sr[c0 + k] : T(0);
    dst[q] = w;
  }
}

cudaError_t launch_pad_rows(const void* src, void* dst, int dtype, int64_t n, int64_t pitch,
                            int64_t rows, cudaStream_t s) {
  const size_t es = dtype_size(dtype);
  if (es == 0 || (pitch * (int64_t)es) % 16 != 0 || (uintptr_t)dst % 16 != 0 || pitch < n)
    return cudaErrorInvalidValue;
  const int64_t words = rows * pitch * (int64_t)es / 16;
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((words + 255) / 256, (int64_t)num_sms() * 32));
  uint4* d = static_cast<uint4*>(dst);
  switch (es) {
    case 1: k_pad_rows<uint8_t><<<grid, 256, 0, s>>>(static_cast<const uint8_t*>(src), d, n, pitch, rows); break;
    case 2: k_pad_rows<uint16_t><<<grid, 256, 0, s>>>(static_cast<const uint16_t*>(src), d, n, pitch, rows); break;
    default: k_pad_rows<uint32_t><<<grid, 256, 0, s>>>(static_cast<const uint32_t*>(src), d, n, pitch, rows); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_difference(const void* in, void* out, int dtype, int64_t n, cudaStream_t s) {
  const int64_t es = (int64_t)dtype_size(dtype);
  if (es > 0 && (uintptr_t)in % 16 == 0 && (uintptr_t)out % 16 == 0 && (n * es) % 16 == 0) {
    const int64_t nw = n * es / 16;
    const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>((nw + 255) / 256, (int64_t)num_sms() * 32));
    const uint4* a = static_cast<const uint4*>(in);
    uint4* b = static_cast<uint4*>(out);
    switch (dtype) {
      case HP_U8: k_difference_v<uint8_t><<<g, 256, 0, s>>>(a, b, nw); break;
      case HP_U16: k_difference_v<uint16_t><<<g, 256, 0, s>>>(a, b, nw); break;
      case HP_F16: k_difference_v<__half><<<g, 256, 0, s>>>(a, b, nw); break;
      case HP_F32: k_difference_v<float><<<g, 256, 0, s>>>(a, b, nw); break;
      default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
  }
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)num_sms() * 32));
  switch (dtype) {
    case HP_U8: k_difference<uint8_t><<<grid, 256, 0, s>>>(static_cast<const uint8_t*>(in), static_cast<uint8_t*>(out), n); break;
    case HP_U16: k_difference<uint16_t><<<grid, 256, 0, s>>>(static_cast<const uint16_t*>(in), static_cast<uint16_t*>(out), n); break;
    case HP_F16: k_difference<__half><<<grid, 256, 0, s>>>(static_cast<const __half*>(in), static_cast<__half*>(out), n); break;
    case HP_F32: k_difference<float><<<grid, 256, 0, s>>>(static_cast<const float*>(in), static_cast<float*>(out), n); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename T>
__global__ void k_unsharp(const T* __restrict__ f, float* __restrict__ g, float amount, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float v = to_f32<T>(f[i]);
    g[i] = fmaf(amount, v - g[i], v);
  }
}

cudaError_t launch_unsharp(const void* f, int dtype, float* g, float amount, int64_t n, cudaStream_t s) {
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)num_sms() * 32));
  switch (dtype) {
    case HP_U8: k_unsharp<uint8_t><<<grid, 256, 0, s>>>(static_cast<const uint8_t*>(f), g, amount, n); break;
    case HP_U16: k_unsharp<uint16_t><<<grid, 256, 0, s>>>(static_cast<const uint16_t*>(f), g, amount, n); break;
    case HP_F16: k_unsharp<__half><<<grid, 256, 0, s>>>(static_cast<const __half*>(f), g, amount, n); break;
    case HP_F32: k_unsharp<float><<<grid, 256, 0, s>>>(static_cast<const float*>(f), g, amount, n); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename T>
__global__ void k_local_threshold(const T* __restrict__ f, const float* __restrict__ m, float offset,
                                  uint8_t* __restrict__ out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = to_f32<T>(f[i]) > m[i] - offset ? 1 : 0;
}

cudaError_t launch_local_threshold(const void* f, int dtype, const float* m, float offset,
                                   uint8_t* out, int64_t n, cudaStream_t s) {
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)num_sms() * 32));
  switch (dtype) {
    case HP_U8: k_local_threshold<uint8_t><<<grid, 256, 0, s>>>(static_cast<const uint8_t*>(f), m, offset, out, n); break;
    case HP_U16: k_local_threshold<uint16_t><<<grid, 256, 0, s>>>(static_cast<const uint16_t*>(f), m, offset, out, n); break;
    case HP_F16: k_local_threshold<__half><<<grid, 256, 0, s>>>(static_cast<const __half*>(f), m, offset, out, n); break;
    case HP_F32: k_local_threshold<float><<<grid, 256, 0, s>>>(static_cast<const float*>(f), m, offset, out, n); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// ------------------------------------------------- van Herk / Gil-Werman
// Cube erosion / dilation as three line passes (x, y, z), each a running
// min of keys over windows of 2L + 1 reflected samples by the van Herk /
// Gil-Werman scheme: the extended line is cut into blocks of 2L + 1, and
// per block the prefix minima G and suffix minima H are formed; the window
// starting at j is then min(H[j], G[j + 2L]) (it spans at most two adjacent
// blocks). Three comparisons per sample and axis, whatever L.
//
// Each line streams through registers in blocks of 2L + 1 (k_vhgw_col for
// z and y lines, one thread per line with coalesced rows; k_vhgw_rows for x
// lines, staged through shared memory). The x and y passes write keys to
// scratch regions (sep_regions); the z pass writes the output dtype.
namespace {
struct VBox {
  int64_t lo[3], dims[3];  // dense box of the global volume
};

// Running min along z or y, one thread per line: consecutive threads take
// consecutive x, so every load and store of a warp is one coalesced row. A thread streams its line's samples (a segment of kVC
// outputs plus 2L on each side) in blocks of K = 2L + 1 kept in registers:
// the suffix minima h of the current block and the next block's samples c;
// the output at block offset t is h[0] for t = 0, else min(h[t], c[0..t-1]).
// No shared memory; the K loads of a block are issued before they are used.
constexpr int kVC = 256;  // outputs per line segment
constexpr int kVCT = 128; // threads per CTA

template <typename TIN, bool RAW, int AXIS, int L>
__global__ void __launch_bounds__(kVCT) k_vhgw_col(const TIN* __restrict__ src, VBox S,
                                                   void* __restrict__ dst, VBox D, int dst_dtype,
                                                   int64_t Gn, uint32_t flip, int64_t nlines,
                                                   int64_t nseg) {
  constexpr int K = 2 * L + 1;
  constexpr int a1 = AXIS == 0 ? 1 : 0, a2 = AXIS == 2 ? 1 : 2;  // the other axes, slow then fast
  const int64_t l = (int64_t)blockIdx.x * kVCT + threadIdx.x;
  if (l >= nlines) return;
  const int64_t s0 = (int64_t)blockIdx.y * kVC;  // first output of the segment (region index)
  const int n = (int)min((int64_t)kVC, nseg - s0);
  int64_t c3[3];
  c3[a2] = D.lo[a2] + l % D.dims[a2];
  c3[a1] = D.lo[a1] + l / D.dims[a2];
  c3[AXIS] = S.lo[AXIS];
  const int64_t sb = ((c3[0] - S.lo[0]) * S.dims[1] + (c3[1] - S.lo[1])) * S.dims[2] + (c3[2] - S.lo[2]);
  c3[AXIS] = D.lo[AXIS];
  const int64_t db = ((c3[0] - D.lo[0]) * D.dims[1] + (c3[1] - D.lo[1])) * D.dims[2] + (c3[2] - D.lo[2]);
  const int64_t sstr = AXIS == 2 ? 1 : (AXIS == 1 ? S.dims[2] : S.dims[1] * S.dims[2]);
  const int64_t dstr = AXIS == 2 ? 1 : (AXIS == 1 ? D.dims[2] : D.dims[1] * D.dims[2]);
  const int64_t p0 = D.lo[AXIS] + s0 - L;  // global axis coordinate of sample 0
  const int ns = n + 2 * L;                // samples of the segment
  const bool inner = p0 >= 0 && p0 + ns <= Gn;  // the same for the whole CTA
  const TIN* sp = src + sb - S.lo[AXIS] * sstr;
  auto load = [&](int i) -> uint32_t {
    const int64_t g = inner ? p0 + i : reflect(p0 + i, Gn);
    if constexpr (RAW) return to_key<TIN>(sp[g * sstr]) ^ flip;
    else return (uint32_t)sp[g * sstr];
  };
  auto put = [&](int j, uint32_t m) {
    const int64_t q = db + (s0 + j) * dstr;
    switch (dst_dtype) {
      case -1: static_cast<uint32_t*>(dst)[q] = m; break;  // keys (scratch)
      case HP_U8: static_cast<uint8_t*>(dst)[q] = from_key<uint8_t>(m ^ flip); break;
      case HP_U16: static_cast<uint16_t*>(dst)[q] = from_key<uint16_t>(m ^ flip); break;
      case HP_F16: static_cast<__half*>(dst)[q] = from_key<__half>(m ^ flip); break;
      default: static_cast<float*>(dst)[q] = from_key<float>(m ^ flip); break;
    }
  };
  uint32_t h[K];
#pragma unroll
  for (int t = 0; t < K; ++t) h[t] = load(t);  // ns >= K: a segment has n >= 1
#pragma unroll
  for (int t = K - 2; t >= 0; --t) h[t] = min(h[t], h[t + 1]);
  for (int b0 = 0; b0 < n; b0 += K) {
    uint32_t c[K];
#pragma unroll
    for (int t = 0; t < K; ++t) c[t] = b0 + K + t < ns ? load(b0 + K + t) : 0xFFFFFFFFu;
    put(b0, h[0]);
    uint32_t g = 0xFFFFFFFFu;
#pragma unroll
    for (int t = 1; t < K; ++t) {
      g = min(g, c[t - 1]);
      if (b0 + t < n) put(b0 + t, min(h[t], g));
    }
#pragma unroll
    for (int t = K - 1; t >= 0; --t) h[t] = t == K - 1 ? c[t] : min(c[t], h[t + 1]);
  }
}

template <typename TIN, bool RAW, int AXIS, int L>
cudaError_t vhgw_col_launch_l(const TIN* src, const VBox& S, void* dst, const VBox& D,
                              int dst_dtype, int64_t Gn, uint32_t flip, cudaStream_t s) {
  constexpr int a1 = AXIS == 0 ? 1 : 0, a2 = AXIS == 2 ? 1 : 2;
  const int64_t nlines = D.dims[a1] * D.dims[a2], nseg = D.dims[AXIS];
  if (nlines <= 0 || nseg <= 0) return cudaSuccess;
  const dim3 grid((unsigned)((nlines + kVCT - 1) / kVCT), (unsigned)((nseg + kVC - 1) / kVC));
  k_vhgw_col<TIN, RAW, AXIS, L><<<grid, kVCT, 0, s>>>(src, S, dst, D, dst_dtype, Gn, flip, nlines,
                                                      nseg);
  return cudaGetLastError();
}

template <typename TIN, bool RAW, int AXIS>
cudaError_t vhgw_col_launch(const TIN* src, const VBox& S, void* dst, const VBox& D,
                            int dst_dtype, int L, int64_t Gn, uint32_t flip, cudaStream_t s) {
  switch (L) {
#define HP_VC(LL) \
  case LL: return vhgw_col_launch_l<TIN, RAW, AXIS, LL>(src, S, dst, D, dst_dtype, Gn, flip, s);
    HP_VC(1) HP_VC(2) HP_VC(3) HP_VC(4) HP_VC(5) HP_VC(6) HP_VC(7) HP_VC(8)
    HP_VC(9) HP_VC(10) HP_VC(11) HP_VC(12) HP_VC(13) HP_VC(14) HP_VC(15) HP_VC(16)
#undef HP_VC
  }
  return cudaErrorInvalidValue;
}

// The x pass of the same recurrence: a CTA stages kVR rows x (kVX + 2L)
// samples as keys in shared memory with coalesced loads, one thread then
// streams each row through the register recurrence (threads of a warp read
// one column of 32 rows: an odd row stride puts them in distinct banks) and
// writes its outputs over the samples it has consumed, and the CTA stores
// the outputs with coalesced writes.
constexpr int kVR = 128;  // rows per CTA, one thread each
constexpr int kVX = 64;   // outputs per row per CTA

template <int L>
constexpr int vhgw_rows_ws() { return (kVX + 2 * L) | 1; }

template <typename TIN, int L>
__global__ void __launch_bounds__(kVR) k_vhgw_rows(const TIN* __restrict__ src, VBox S,
                                                   uint32_t* __restrict__ dst, VBox D, int64_t Gn,
                                                   uint32_t flip, int64_t nlines, int64_t nseg,
                                                   int vec_rows) {
  constexpr int K = 2 * L + 1, W = kVX + 2 * L, WS = vhgw_rows_ws<L>();
  constexpr int EPV = 16 / (int)sizeof(TIN);  // elements per 16-byte word
  extern __shared__ uint32_t Er[];
  __shared__ int64_t s_sb[kVR], s_db[kVR];
  const int tid = threadIdx.x;
  // segments are the fast grid index: CTAs that run together take adjacent
  // segments of the same rows and share their halo lines in L2; row groups
  // beyond the grid's y extent are taken in further rounds
  const int64_t s0 = (int64_t)blockIdx.x * kVX;  // first output of the segment (region index)
  for (int64_t line0 = (int64_t)blockIdx.y * kVR; line0 < nlines; line0 += (int64_t)gridDim.y * kVR) {
    const int nlin = (int)min((int64_t)kVR, nlines - line0);
    const int n = (int)min((int64_t)kVX, nseg - s0);
    const int ns = n + 2 * L;
    {
      // this thread's row: lines enumerate (z, y) of D, y fastest
      const int64_t l = min(line0 + tid, nlines - 1);
      const int64_t z = D.lo[0] + l / D.dims[1], y = D.lo[1] + l % D.dims[1];
      s_sb[tid] = ((z - S.lo[0]) * S.dims[1] + (y - S.lo[1])) * S.dims[2] - S.lo[2];
      s_db[tid] = ((z - D.lo[0]) * D.dims[1] + (y - D.lo[1])) * D.dims[2];
    }
    const int64_t p0 = D.lo[2] + s0 - L;  // global x of sample 0
    const bool inner = p0 >= 0 && p0 + ns <= Gn;
    __syncthreads();
    if (inner && vec_rows) {
      // rows start on 16-byte boundaries (vec_rows): stage whole aligned
      // 16-byte words covering samples [0, ns) of each row; a word never
      // crosses the end of its row (row lengths are whole words)
      const int64_t off0 = p0 - S.lo[2];               // element offset of sample 0 in its row
      const int64_t w0 = off0 & ~(int64_t)(EPV - 1);   // first word's element offset
      const int nw = (int)((off0 + ns - w0 + EPV - 1) / EPV);
      constexpr int kU = 4;  // 16-byte loads in flight per thread
      for (int i0 = tid; i0 < nlin * nw; i0 += kVR * kU) {
        uint4 v[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
          const int i = i0 + u * kVR;
          if (i < nlin * nw) {
            const int r = i / nw, k = i - r * nw;
            v[u] = *reinterpret_cast<const uint4*>(src + s_sb[r] + S.lo[2] + w0 + (int64_t)k * EPV);
          }
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) {
          const int i = i0 + u * kVR;
          if (i < nlin * nw) {
            const int r = i / nw, k = i - r * nw;
            const TIN* el = reinterpret_cast<const TIN*>(&v[u]);
            const int pos0 = (int)(w0 - off0) + k * EPV;
#pragma unroll
            for (int q = 0; q < EPV; ++q)
              if (pos0 + q >= 0 && pos0 + q < ns) Er[r * WS + pos0 + q] = to_key<TIN>(el[q]) ^ flip;
          }
        }
      }
      // rows past the last line and samples past ns keep the identity
      for (int i = tid; i < kVR * W; i += kVR) {
        const int r = i / W, pos = i - r * W;
        if (r >= nlin || pos >= ns) Er[r * WS + pos] = 0xFFFFFFFFu;
      }
    } else {
      constexpr int kU = 8;  // loads in flight per thread
      for (int i0 = tid; i0 < kVR * W; i0 += kVR * kU) {
        uint32_t key[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
          const int i = i0 + u * kVR, r = i / W, pos = i - r * W;
          key[u] = 0xFFFFFFFFu;
          if (i < kVR * W && r < nlin && pos < ns) {
            const int64_t g = inner ? p0 + pos : reflect(p0 + pos, Gn);
            key[u] = to_key<TIN>(src[s_sb[r] + g]) ^ flip;
          }
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) {
          const int i = i0 + u * kVR;
          if (i < kVR * W) Er[(i / W) * WS + (i % W)] = key[u];
        }
      }
    }
    __syncthreads();
    {
      uint32_t* e = Er + tid * WS;
      uint32_t h[K];
#pragma unroll
      for (int t = 0; t < K; ++t) h[t] = e[t];
#pragma unroll
      for (int t = K - 2; t >= 0; --t) h[t] = min(h[t], h[t + 1]);
      for (int b0 = 0; b0 < n; b0 += K) {
        uint32_t c[K];
#pragma unroll
        for (int t = 0; t < K; ++t) c[t] = b0 + K + t < ns ? e[b0 + K + t] : 0xFFFFFFFFu;
        // outputs b0 .. b0 + K - 1 overwrite samples this thread has consumed
        e[b0] = h[0];
        uint32_t g = 0xFFFFFFFFu;
#pragma unroll
        for (int t = 1; t < K; ++t) {
          g = min(g, c[t - 1]);
          if (b0 + t < n) e[b0 + t] = min(h[t], g);
        }
#pragma unroll
        for (int t = K - 1; t >= 0; --t) h[t] = t == K - 1 ? c[t] : min(c[t], h[t + 1]);
      }
    }
    __syncthreads();
    for (int i = tid; i < kVR * kVX; i += kVR) {
      const int r = i / kVX, o = i - r * kVX;
      if (r < nlin && o < n) dst[s_db[r] + s0 + o] = Er[r * WS + o];
    }
    __syncthreads();  // the next round restages Er and the row offsets
  }
}

template <typename TIN, int L>
cudaError_t vhgw_rows_launch_l(const TIN* src, const VBox& S, uint32_t* dst, const VBox& D,
                               int64_t Gn, uint32_t flip, cudaStream_t s) {
  const int64_t nlines = D.dims[0] * D.dims[1], nseg = D.dims[2];
  if (nlines <= 0 || nseg <= 0) return cudaSuccess;
  const int smem = kVR * vhgw_rows_ws<L>() * 4;
  static bool attr = false;  // per instantiation
  if (!attr) {
    const cudaError_t e =
        cudaFuncSetAttribute(k_vhgw_rows<TIN, L>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const dim3 grid((unsigned)((nseg + kVX - 1) / kVX),
                  (unsigned)std::min<int64_t>((nlines + kVR - 1) / kVR, 65535));
  // 16-byte staging where every row of the source box starts on a 16-byte boundary
  const int vec_rows = (reinterpret_cast<uintptr_t>(src) % 16 == 0 && (S.dims[2] * (int64_t)sizeof(TIN)) % 16 == 0);
  k_vhgw_rows<TIN, L><<<grid, kVR, smem, s>>>(src, S, dst, D, Gn, flip, nlines, nseg, vec_rows);
  return cudaGetLastError();
}

template <typename TIN>
cudaError_t vhgw_rows_launch(const TIN* src, const VBox& S, uint32_t* dst, const VBox& D, int L,
                             int64_t Gn, uint32_t flip, cudaStream_t s) {
  switch (L) {
#define HP_VR(LL) \
  case LL: return vhgw_rows_launch_l<TIN, LL>(src, S, dst, D, Gn, flip, s);
    HP_VR(1) HP_VR(2) HP_VR(3) HP_VR(4) HP_VR(5) HP_VR(6) HP_VR(7) HP_VR(8)
    HP_VR(9) HP_VR(10) HP_VR(11) HP_VR(12) HP_VR(13) HP_VR(14) HP_VR(15) HP_VR(16)
#undef HP_VR
  }
  return cudaErrorInvalidValue;
}

template <typename TIN>
cudaError_t vhgw_cube(const Job& job, int rad, int is_dilate, cudaStream_t s) {
  const SepRegions g = sep_regions(job, rad);
  const int64_t vx = g.n_x[0] * g.n_x[1] * g.n_x[2], vy = g.n_y[0] * g.n_y[1] * g.n_y[2];
  if (!job.scratch || job.scratch_bytes < 4 * (size_t)(vx + vy)) return cudaErrorInvalidValue;
  uint32_t* k1 = static_cast<uint32_t*>(job.scratch);
  uint32_t* k2 = k1 + vx;
  const uint32_t flip = is_dilate ? KeyMask<TIN>::value : 0u;
  const VBox in{{job.in.lo[0], job.in.lo[1], job.in.lo[2]}, {job.in.dims[0], job.in.dims[1], job.in.dims[2]}};
  const VBox rx{{g.rlo[0], g.rlo[1], job.core_lo[2]}, {g.n_x[0], g.n_x[1], g.n_x[2]}};
  const VBox ry{{g.rlo[0], job.core_lo[1], job.core_lo[2]}, {g.n_y[0], g.n_y[1], g.n_y[2]}};
  const VBox out{{job.out.lo[0], job.out.lo[1], job.out.lo[2]},
                 {job.out.dims[0], job.out.dims[1], job.out.dims[2]}};
  const VBox core{{job.core_lo[0], job.core_lo[1], job.core_lo[2]},
                  {job.core_hi[0] - job.core_lo[0], job.core_hi[1] - job.core_lo[1],
                   job.core_hi[2] - job.core_lo[2]}};
  cudaError_t e = vhgw_rows_launch<TIN>(static_cast<const TIN*>(job.in.ptr), in, k1, rx, rad,
                                        job.gdims[2], flip, s);
  if (e == cudaSuccess)
    e = vhgw_col_launch<uint32_t, false, 1>(k1, rx, k2, ry, -1, rad, job.gdims[1], 0u, s);
  if (e != cudaSuccess) return e;
  // z pass: region = core, written into the output box (which contains it)
  if (core.lo[0] == out.lo[0] && core.lo[1] == out.lo[1] && core.lo[2] == out.lo[2] &&
      core.dims[0] == out.dims[0] && core.dims[1] == out.dims[1] && core.dims[2] == out.dims[2])
    return vhgw_col_launch<uint32_t, false, 0>(k2, ry, job.out.ptr, out, job.out.dtype, rad,
                                               job.gdims[0], flip, s);
  return cudaErrorInvalidValue;  // output boxes equal the core on every path that gets here
}
}  // namespace

bool morph_uses_vhgw(const Job& job, int se, int rad) {
  return se == HP_SE_CUBE && rad >= 1 &&
         !(rad <= kMaxTiledR && job.gdims[2] >= rad && job.gdims[1] >= rad);
}

size_t morph_scratch_bytes(const Job& job, int se, int rad) {
  if (!morph_uses_vhgw(job, se, rad)) return 0;
  const SepRegions g = sep_regions(job, rad);
  return 4 * (size_t)(g.n_x[0] * g.n_x[1] * g.n_x[2] + g.n_y[0] * g.n_y[1] * g.n_y[2]);
}

cudaError_t launch_morph(const Job& job, int se, int rad, int is_dilate, cudaStream_t s) {
  const int64_t cx = job.core_hi[2] - job.core_lo[2];
  const int64_t cy = job.core_hi[1] - job.core_lo[1];
  const int64_t cz = job.core_hi[0] - job.core_lo[0];
  if (cx <= 0 || cy <= 0 || cz <= 0) return cudaSuccess;
  // 16-bit data: packed-key kernel (k_morph16.cu) where its layout rules hold
  const cudaError_t e16 = launch_morph16(job, se, rad, is_dilate, s);
  if (e16 != cudaErrorNotSupported) return e16;
  const int ball = se == HP_SE_BALL;
  const bool tiled = rad >= 1 && rad <= (ball ? kMaxTiledBallR : kMaxTiledR) &&
                     job.gdims[2] >= rad && job.gdims[1] >= rad;
  if (!tiled && morph_uses_vhgw(job, se, rad)) {
    switch (job.in.dtype) {
      case HP_U8: return vhgw_cube<uint8_t>(job, rad, is_dilate, s);
      case HP_U16: return vhgw_cube<uint16_t>(job, rad, is_dilate, s);
      case HP_F16: return vhgw_cube<__half>(job, rad, is_dilate, s);
      case HP_F32: return vhgw_cube<float>(job, rad, is_dilate, s);
      default: return cudaErrorInvalidValue;
    }
  }
  if (!tiled) {
    const int64_t total = cx * cy * cz;
    const unsigned grid = (unsigned)std::min<int64_t>((total + 255) / 256, (int64_t)num_sms() * 32);
    switch (job.in.dtype) {
      case HP_U8: k_morph_generic<uint8_t><<<grid, 256, 0, s>>>(job, ball, rad, is_dilate); break;
      case HP_U16: k_morph_generic<uint16_t><<<grid, 256, 0, s>>>(job, ball, rad, is_dilate); break;
      case HP_F16: k_morph_generic<__half><<<grid, 256, 0, s>>>(job, ball, rad, is_dilate); break;
      case HP_F32: k_morph_generic<float><<<grid, 256, 0, s>>>(job, ball, rad, is_dilate); break;
      default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
  }
  MorphParams P;
  P.job = job;
  P.is_dilate = is_dilate;
  P.err = device_error_word();
  const int ty_rows = (ball && rad > kMaxDblR) ? 16 : kTY;  // MGeom<rad, ball>::TY
  P.tiles_x = (int)((cx + kTX - 1) / kTX);
  const int64_t tiles = (int64_t)P.tiles_x * ((cy + ty_rows - 1) / ty_rows);
  const int64_t want = (int64_t)num_sms() * 8;
  int64_t nchunks = std::max<int64_t>(1, (want + tiles - 1) / tiles);
  int64_t zc = (cz + nchunks - 1) / nchunks;
  zc = std::max<int64_t>(zc, std::min<int64_t>(cz, 32));
  P.zchunk = (int)zc;
  dim3 grid((unsigned)tiles, (unsigned)((cz + zc - 1) / zc));

  CUtensorMap map;
  memset(&map, 0, sizeof(map));
  const size_t es = dtype_size(job.in.dtype);
  const int al = 16 / (int)es;
  bool use_tma = ((uintptr_t)job.in.ptr % 16 == 0) && ((job.in.dims[2] * (int64_t)es) % 16 == 0) &&
                 ((job.core_lo[2] - job.in.lo[2]) % al == 0);
  if (use_tma) {
    int ra = 0, bw = 0;
    mbox_geom(rad, (int)es, &ra, &bw);
    const int64_t dims[3] = {job.in.dims[2], job.in.dims[1], job.in.dims[0]};
    use_tma = make_tmap_3d(&map, job.in.ptr, job.in.dtype, dims, bw, ty_rows + 2 * rad);
  }
  P.use_tma = use_tma ? 1 : 0;
  if (log_level() > 0)
    fprintf(stderr, "[hp] morph z-march r=%d ball=%d tma=%d grid=%ux%u zchunk=%d\n", rad, ball,
            P.use_tma, grid.x, grid.y, P.zchunk);
  return ball ? dispatch_r<1>(rad, P, map, grid, s) : dispatch_r<0>(rad, P, map, grid, s);
}

// ------------------------------------------------------------ threshold
namespace {
template <typename TIN>
__global__ void k_threshold(const Job J, float t) {
  const int64_t n0 = J.core_hi[0] - J.core_lo[0], n1 = J.core_hi[1] - J.core_lo[1],
                n2 = J.core_hi[2] - J.core_lo[2];
  const int64_t total = n0 * n1 * n2;
  const TIN* in = static_cast<const TIN*>(J.in.ptr);
  uint8_t* out = static_cast<uint8_t*>(J.out.ptr);
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t x = J.core_lo[2] + q % n2, y = J.core_lo[1] + (q / n2) % n1,
                  z = J.core_lo[0] + q / (n1 * n2);
    const int64_t qi = ((z - J.in.lo[0]) * J.in.dims[1] + (y - J.in.lo[1])) * J.in.dims[2] + (x - J.in.lo[2]);
    const int64_t qo = ((z - J.out.lo[0]) * J.out.dims[1] + (y - J.out.lo[1])) * J.out.dims[2] + (x - J.out.lo[2]);
    out[qo] = to_f32<TIN>(in[qi]) > t ? 1 : 0;
  }
}
}  // namespace

// The largest value of the input's type that is <= t (t not NaN), returned
// as a float, which holds it exactly for every input type. For every value
// f of that type, f > t_below(t) exactly when f > t, so the kernel's FP32
// comparison decides f > t without rounding t.
float threshold_below(double t, int dtype) {
  if (dtype == HP_U8 || dtype == HP_U16) {
    const double top = dtype == HP_U8 ? 255.0 : 65535.0;
    return (float)std::min(std::max(std::floor(t), -1.0), top);
  }
  float tf;
  if (t >= (double)FLT_MAX) tf = std::isinf(t) ? INFINITY : FLT_MAX;
  else if (t < -(double)FLT_MAX) tf = -INFINITY;
  else {
    tf = (float)t;  // nearest; step down when it rounded up
    if ((double)tf > t) tf = std::nextafter(tf, -INFINITY);
  }
  if (dtype == HP_F32) return tf;
  // float16: the largest half <= tf (hence <= t)
  if (tf >= 65504.0f) return std::isinf(tf) ? INFINITY : 65504.0f;
  if (tf < -65504.0f) return -INFINITY;
  return __half2float(__float2half_rd(tf));
}

// out = in > t, decided exactly: the kernel compares the input (converted
// to FP32 without rounding) against threshold_below(t).
cudaError_t launch_threshold(const Job& job, double t, cudaStream_t s) {
  const int64_t n = (job.core_hi[0] - job.core_lo[0]) * (job.core_hi[1] - job.core_lo[1]) *
                    (job.core_hi[2] - job.core_lo[2]);
  if (n <= 0) return cudaSuccess;
  const unsigned grid = (unsigned)std::min<int64_t>((n + 255) / 256, (int64_t)num_sms() * 32);
  const float tb = threshold_below(t, job.in.dtype);
  switch (job.in.dtype) {
    case HP_U8: k_threshold<uint8_t><<<grid, 256, 0, s>>>(job, tb); break;
    case HP_U16: k_threshold<uint16_t><<<grid, 256, 0, s>>>(job, tb); break;
    case HP_F16: k_threshold<__half><<<grid, 256, 0, s>>>(job, tb); break;
    case HP_F32: k_threshold<float><<<grid, 256, 0, s>>>(job, tb); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace hp
