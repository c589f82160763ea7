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

constexpr int kBZ = 8;
constexpr int kNS = 4;

typedef unsigned long long u64;

struct GaussParams {
  Job job;
  // taps per axis (z, y, x), each duplicated into an FP32 pair so packed
  // fmas take them as one 64-bit operand
  u64 w2[3][2 * kMaxR + 1];
  int r;
  int zchunk;
  int tiles_x;
  int use_tma;
  int* err;
};

__host__ __device__ constexpr int round_up(int a, int b) { return (a + b - 1) / b * b; }

inline uint32_t __float_as_uint_host(float f) {
  uint32_t u;
  memcpy(&u, &f, 4);
  return u;
}

// Row-pair stride (in FP32 pairs) of the interleaved patch: 2 mod 4 puts the
// 16-byte loads of 8 consecutive row pairs into 8 distinct bank groups.
__host__ __device__ constexpr int pair_stride(int n) {
  int f = n;
  while (f % 4 != 2) ++f;
  return f;
}

// Geometry of the z-march kernel for radius R.
//   F2 (FP32 patch, row pairs interleaved, double-buffered): element
//      (rp, c) is the pair (row 2rp, row 2rp+1) at column c; column c <->
//      x = cx0 - R4 + c, row <-> y = cy0 - R + row. R4 = R rounded up to 4
//      keeps the x-pass window loads 16-byte aligned.
//   X  (x-pass output, double-buffered): [BH][kXS] floats.
//   ring: kBZ + 2R planes of y-pass output [TY][TX].
template <int R, int TX, int TY>
struct ZmGeom {
  static constexpr int NT = TX * TY / 4;                // threads: 4 outputs each per plane
  static constexpr int XS = TX + 4;                     // X row stride (floats)
  static constexpr int R4 = round_up(R, 4);
  static constexpr int WL = round_up(R4 + R + 8, 4);  // x window (columns) for 8 outputs
  static constexpr int FWN = (TX - 8) + WL;            // columns read
  static constexpr int BH = TY + 2 * R;
  static constexpr int RP = BH / 2;                     // row pairs
  static constexpr int FW2 = pair_stride(FWN);
  static constexpr int CP = FWN / 2;                    // column pairs per row pair
  static constexpr int NI = (RP * CP + NT - 1) / NT;   // staging items per thread
  static constexpr int NC = (FWN + 31) / 32;            // columns per lane (face path)
  static constexpr int NRING = kBZ + 2 * R;
  static constexpr int FSZ2 = RP * FW2;                 // in FP32 pairs
  static constexpr int XSZ = BH * XS;
  static constexpr int TAIL = 2 * FSZ2 * 8 + (2 * XSZ + NRING * TY * TX) * 4 + BH * 4;
  static_assert(FWN % 4 == 0 && BH % 2 == 0, "patch shape");
};

// Per-dtype TMA box geometry: left halo ra (R rounded up to 16 bytes) and
// width bw (elements); raw col c <-> x = cx0 - ra + c.
__host__ __device__ constexpr void box_geom(int r, int es, int tx, int* ra, int* bw) {
  const int al = 16 / es;
  *ra = round_up(r, al);
  *bw = round_up(tx + *ra + r, al);
}

__host__ __device__ constexpr int stage_bytes(int r, int es, int tx, int ty) {
  int ra = 0, bw = 0;
  box_geom(r, es, tx, &ra, &bw);
  return round_up(bw * (ty + 2 * r) * es, 128);
}

template <int R, int TX, int TY>
__host__ __device__ constexpr int zm_smem_bytes(int es) {
  return 128 + kNS * stage_bytes(R, es, TX, TY) + ZmGeom<R, TX, TY>::TAIL;
}

// Tile shape per radius. TMA box loads are limited by their row count, so
// small radii use wide, short tiles (22 rows per 1024 outputs at r = 3); large
// radii use square tiles, whose x pass repeats fewer halo rows.
template <int R>
struct ZmTile {
  static constexpr int TX = R <= 6 ? 64 : 32;
  static constexpr int TY = R <= 6 ? 16 : 32;
};

// Two consecutive elements -> two floats. Integers use the exact 2^23 bias:
// a byte permute builds 0x4B00_0000 | v, then one packed subtract.
template <typename T>
__device__ __forceinline__ float2 load2_f32(const T* p);
template <>
__device__ __forceinline__ float2 load2_f32<uint16_t>(const uint16_t* p) {
  const uint32_t w = *reinterpret_cast<const uint32_t*>(p);
  const float a = __uint_as_float(__byte_perm(w, 0x4B000000u, 0x7410));
  const float b = __uint_as_float(__byte_perm(w, 0x4B000000u, 0x7432));
  return make_float2(a - 8388608.0f, b - 8388608.0f);
}
template <>
__device__ __forceinline__ float2 load2_f32<uint8_t>(const uint8_t* p) {
  const uint32_t w = *reinterpret_cast<const uint16_t*>(p);
  const float a = __uint_as_float(__byte_perm(w, 0x4B000000u, 0x7440));
  const float b = __uint_as_float(__byte_perm(w, 0x4B000000u, 0x7441));
  return make_float2(a - 8388608.0f, b - 8388608.0f);
}
template <>
__device__ __forceinline__ float2 load2_f32<__half>(const __half* p) {
  return __half22float2(*reinterpret_cast<const __half2*>(p));
}
template <>
__device__ __forceinline__ float2 load2_f32<float>(const float* p) {
  return *reinterpret_cast<const float2*>(p);
}

// Interior tiles: no reflection. Item k of this thread covers row pair rp,
// columns 2c, 2c+1: two 2-element loads (rows 2rp, 2rp+1), one 16-byte store
// of the interleaved pairs. Offsets were precomputed per CTA.
template <typename TIN, int R, int TX, int TY>
__device__ __forceinline__ void stage_interior(float2* F2, const unsigned char* rawb, int bw,
                                               const int (&roff)[ZmGeom<R, TX, TY>::NI],
                                               const int (&foff)[ZmGeom<R, TX, TY>::NI]) {
  using G = ZmGeom<R, TX, TY>;
  const TIN* raw = reinterpret_cast<const TIN*>(rawb);
#pragma unroll
  for (int k = 0; k < G::NI; ++k) {
    if (foff[k] >= 0) {
      const float2 a = load2_f32<TIN>(raw + roff[k]);
      const float2 b = load2_f32<TIN>(raw + roff[k] + bw);
      *reinterpret_cast<float4*>(F2 + foff[k]) = make_float4(a.x, b.x, a.y, b.y);
    }
  }
}

// Face tiles (and the cooperative-load path): element by element through
// the source tables, which resolve the reflection; srow[row] is the raw
// stage row (TMA) or box row (global loads), scol[k] the column of lane
// column lane + 32k; -1 marks taps no stored output uses.
template <typename TIN, int R, int TX, int TY>
__device__ __forceinline__ void stage_tables(float2* F2, const TIN* plane, int64_t pitch,
                                             bool ok_plane, const int* srow,
                                             const int (&scol)[ZmGeom<R, TX, TY>::NC], int warp,
                                             int lane) {
  using G = ZmGeom<R, TX, TY>;
  float* F = reinterpret_cast<float*>(F2);
  for (int row = warp; row < G::BH; row += G::NT / 32) {
    const int sr = ok_plane ? srow[row] : -1;
    float* dst = F + (row >> 1) * (2 * G::FW2) + (row & 1);
#pragma unroll
    for (int k = 0; k < G::NC; ++k) {
      const int col = lane + 32 * k;
      if (col < G::FWN) {
        const int sc = scol[k];
        dst[2 * col] = (sr >= 0 && sc >= 0) ? to_f32<TIN>(plane[sr * pitch + sc]) : 0.0f;
      }
    }
  }
}

// Face tiles: after the vectorised staging (out-of-volume cells hold the
// TMA zero fill), overwrite the cells outside the volume with their
// reflected sources, which lie inside the volume and inside the patch.
// frow/fcol map patch rows/columns to their source rows/columns (identity
// inside the volume, -1 where no stored output needs the cell); brow/bcol
// list the rows/columns that are outside.
template <int R, int TX, int TY>
__device__ __forceinline__ void fix_faces(float2* F2, const int* frow, const int* fcol,
                                          const int* brow, int nbr, const int* bcol, int nbc,
                                          int tid) {
  using G = ZmGeom<R, TX, TY>;
  float* F = reinterpret_cast<float*>(F2);
  auto cell = [&](int r, int c) -> float& { return F[(r >> 1) * (2 * G::FW2) + 2 * c + (r & 1)]; };
  for (int i = tid; i < nbr * G::FWN; i += G::NT) {
    const int r = brow[i / G::FWN], c = i % G::FWN;
    const int sr = frow[r], sc = fcol[c];
    cell(r, c) = (sr >= 0 && sc >= 0) ? cell(sr, sc) : 0.0f;
  }
  for (int i = tid; i < nbc * G::BH; i += G::NT) {
    const int c = bcol[i / G::BH], r = i % G::BH;
    const int sr = frow[r], sc = fcol[c];
    cell(r, c) = (sr >= 0 && sc >= 0) ? cell(sr, sc) : 0.0f;
  }
}

template <int R, typename TIN, int TX, int TY>
__global__ void __launch_bounds__(TX * TY / 4, 1)
    k_gauss_zm(const __grid_constant__ GaussParams P, const __grid_constant__ CUtensorMap tmap) {
  using G = ZmGeom<R, TX, TY>;
  constexpr int NT = G::NT;
  constexpr int kXS = G::XS;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ int s_abort;
  __shared__ int s_frow[G::BH], s_fcol[G::FWN], s_brow[G::BH], s_bcol[G::FWN];
  __shared__ int s_nbr, s_nbc;

  const Job& J = P.job;
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const int tx = blockIdx.x % P.tiles_x, ty = blockIdx.x / P.tiles_x;
  const int64_t cx0 = J.core_lo[2] + (int64_t)tx * TX;
  const int64_t cy0 = J.core_lo[1] + (int64_t)ty * TY;
  const int64_t cz0 = J.core_lo[0] + (int64_t)blockIdx.y * P.zchunk;
  const int64_t cz1 = min(cz0 + (int64_t)P.zchunk, J.core_hi[0]);
  if (cz0 >= cz1) return;
  const int nout = (int)(cz1 - cz0);
  const int total = nout + 2 * R;  // input planes cz0-R .. cz1+R-1
  const int64_t Gz = J.gdims[0], Gy = J.gdims[1], Gx = J.gdims[2];
  constexpr int es = sizeof(TIN);
  int ra, bw;
  box_geom(R, es, TX, &ra, &bw);
  const int sbytes = stage_bytes(R, es, TX, TY);
  const bool tma = P.use_tma != 0;
  // tiles whose halo stays inside the volume need no reflection
  const bool face = (cx0 - R < 0) || (cx0 + TX + R > Gx) || (cy0 - R < 0) || (cy0 + TY + R > Gy);

  uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
  unsigned char* stages = smem + 128;
  float2* F2 = reinterpret_cast<float2*>(stages + kNS * sbytes);
  float* X = reinterpret_cast<float*>(F2 + 2 * G::FSZ2);
  float* ring = X + 2 * G::XSZ;
  int* srow = reinterpret_cast<int*>(ring + G::NRING * TY * TX);

  // source tables (reflection resolved once per CTA)
  for (int row = tid; row < G::BH; row += NT) {
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
  // interior staging items: raw element offset of (row 2rp, col 2c) and the
  // F2 offset of (rp, 2c); F col c <-> raw col c + ra - R4
  int roff[G::NI], foff[G::NI];
#pragma unroll
  for (int k = 0; k < G::NI; ++k) {
    const int it = tid + k * NT;
    const int rp = it / G::CP, c = it - rp * G::CP;
    const bool ok = it < G::RP * G::CP;
    roff[k] = ok ? (2 * rp) * bw + 2 * c + (ra - G::R4) : 0;
    foff[k] = ok ? rp * G::FW2 + 2 * c : -1;
  }
  if (tma && face) {
    // patch-coordinate reflection maps for the face fix-up
    for (int r = tid; r < G::BH; r += NT) {
      const int64_t s = reflect(cy0 - R + r, Gy) - (cy0 - R);
      s_frow[r] = (s >= 0 && s < G::BH) ? (int)s : -1;
    }
    for (int c = tid; c < G::FWN; c += NT) {
      const int64_t s = reflect(cx0 - G::R4 + c, Gx) - (cx0 - G::R4);
      s_fcol[c] = (s >= 0 && s < G::FWN) ? (int)s : -1;
    }
    __syncthreads();
    if (tid == 0) {
      int nr = 0, nc = 0;
      for (int r = 0; r < G::BH; ++r)
        if (s_frow[r] != r) s_brow[nr++] = r;
      for (int c = 0; c < G::FWN; ++c)
        if (s_fcol[c] != c) s_bcol[nc++] = c;
      s_nbr = nr;
      s_nbc = nc;
    }
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
  const int nbr = (tma && face) ? s_nbr : 0, nbc = (tma && face) ? s_nbc : 0;

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

  // x pass: 8 consecutive row pairs per 8-thread group, 4 column groups
  // x pass: 8 consecutive threads take 8 row pairs of one 8-column group
  const int xrp = (tid % 8) + 8 * (tid / TX), xg = ((tid / 8) % (TX / 8)) * 8;
  const int yp = tid % (TX / 2), yb2 = (tid / (TX / 2)) * 2;     // y pass
  const int zy = tid / (TX / 4), zx4 = (tid % (TX / 4)) * 4;    // z pass

  // ---- one pipeline phase p: stage plane p, x pass of plane p-1, y pass
  // of plane p-2 (double-buffered F2 and X), then one barrier.
  int zb = 0;
  int p = 0;
  for (; p < total + 2; ++p) {
    if (p < total) {
      float2* Fb = F2 + (p & 1) * G::FSZ2;
      if (tma) {
        if (!mbar_wait(&bars[p % kNS], (p / kNS) & 1)) atomicOr(&s_abort, 1);
        const unsigned char* rawb = stages + (p % kNS) * sbytes;
        stage_interior<TIN, R, TX, TY>(Fb, rawb, bw, roff, foff);
        if (face) {
          __syncthreads();  // the fix-up reads cells staged by other threads
          fix_faces<R, TX, TY>(Fb, s_frow, s_fcol, s_brow, nbr, s_bcol, nbc, tid);
        }
      } else {
        const int64_t sz = reflect(cz0 - R + p, Gz) - J.in.lo[0];
        const bool zok = sz >= 0 && sz < J.in.dims[0];
        const int64_t off = (zok ? sz : 0) * J.in.dims[1] * J.in.dims[2];
        const int64_t pitch = J.in.dims[2];
        stage_tables<TIN, R, TX, TY>(Fb, static_cast<const TIN*>(J.in.ptr) + off, pitch, zok, srow, scol,
                             warp, lane);
      }
    }
    if (p >= 1 && p - 1 < total && xrp < G::RP) {
      // x pass on a row pair: 8 outputs of rows 2rp and 2rp+1 with packed
      // fmas over the pair; window column j <-> x = cx0 + xg - R4 + j
      const u64* src = reinterpret_cast<const u64*>(F2 + ((p - 1) & 1) * G::FSZ2 + xrp * G::FW2 + xg);
      u64 w[G::WL];
#pragma unroll
      for (int j = 0; j < G::WL / 2; ++j) {
        const ulonglong2 v = reinterpret_cast<const ulonglong2*>(src)[j];
        w[2 * j] = v.x;
        w[2 * j + 1] = v.y;
      }
      float* X0 = X + ((p - 1) & 1) * G::XSZ + (2 * xrp) * kXS + xg;
      float o0[8], o1[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        u64 acc = 0ull;
#pragma unroll
        for (int j = i + G::R4 - R; j <= i + G::R4 + R; ++j)
          acc = ffma2(P.w2[2][i + G::R4 - j + R], w[j], acc);
        const float2 a = unpack2(acc);
        o0[i] = a.x;
        o1[i] = a.y;
      }
      reinterpret_cast<float4*>(X0)[0] = make_float4(o0[0], o0[1], o0[2], o0[3]);
      reinterpret_cast<float4*>(X0)[1] = make_float4(o0[4], o0[5], o0[6], o0[7]);
      reinterpret_cast<float4*>(X0 + kXS)[0] = make_float4(o1[0], o1[1], o1[2], o1[3]);
      reinterpret_cast<float4*>(X0 + kXS)[1] = make_float4(o1[4], o1[5], o1[6], o1[7]);
    }
    if (p >= 2) {
      // y pass of plane p-2 into its ring slot: one x pair, two rows per
      // thread, packed fmas over the pair
      const float* Xb = X + ((p - 2) & 1) * G::XSZ + yb2 * kXS + 2 * yp;
      u64 a0 = 0ull, a1 = 0ull;
#pragma unroll
      for (int j = 0; j < 2 + 2 * R; ++j) {
        const u64 v = *reinterpret_cast<const u64*>(Xb + j * kXS);
        if (j <= 2 * R) a0 = ffma2(P.w2[1][2 * R - j], v, a0);
        if (j >= 1) a1 = ffma2(P.w2[1][2 * R + 1 - j], v, a1);
      }
      float* slot = ring + ((p - 2) % G::NRING) * (TY * TX) + yb2 * TX + 2 * yp;
      *reinterpret_cast<u64*>(slot) = a0;
      *reinterpret_cast<u64*>(slot + TX) = a1;
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
      u64 acc0[kBZ], acc1[kBZ];  // x pairs (0,1) and (2,3)
#pragma unroll
      for (int j = 0; j < kBZ; ++j) acc0[j] = acc1[j] = 0ull;
      int slot = zb % G::NRING;
#pragma unroll
      for (int m = 0; m < kBZ + 2 * R; ++m) {
        const ulonglong2 v =
            *reinterpret_cast<const ulonglong2*>(ring + slot * (TY * TX) + zy * TX + zx4);
        slot = slot + 1 == G::NRING ? 0 : slot + 1;
#pragma unroll
        for (int j = 0; j < kBZ; ++j) {
          if (m >= j && m <= j + 2 * R) {
            acc0[j] = ffma2(P.w2[0][j - m + 2 * R], v.x, acc0[j]);
            acc1[j] = ffma2(P.w2[0][j - m + 2 * R], v.y, acc1[j]);
          }
        }
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
            *reinterpret_cast<ulonglong2*>(static_cast<float*>(O.ptr) + idx) =
                make_ulonglong2(acc0[j], acc1[j]);
          } else {
            const float2 lo = unpack2(acc0[j]), hi = unpack2(acc1[j]);
            const float vv[4] = {lo.x, lo.y, hi.x, hi.y};
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
// Generic single-axis pass: dst = conv_axis(src), y[i] = sum_k g(k) x[R(i-k)],
// over the region [off, off + n) of the global volume G (dense in dst).
// src is a dense box (lo, dims) of the global volume: the job's input (any
// dtype) for the first pass, a scratch volume after it. The last pass
// stores straight into the job's output (FP32, or rounded once to f16).
struct AxisBox {
  int64_t lo[3], dims[3];
};
struct AxisTaps1 {
  float w[kMaxTaps];
};

__device__ __forceinline__ void store_out(const DevOut& O, int64_t idx, float v) {
  if (O.dtype == HP_F32) static_cast<float*>(O.ptr)[idx] = v;
  else static_cast<__half*>(O.ptr)[idx] = __float2half_rn(v);
}

template <typename TIN, bool TO_OUT>
__global__ void k_axis_pass(const TIN* __restrict__ src, const AxisBox S, float* __restrict__ dst,
                            DevOut O, int64_t n0, int64_t n1, int64_t n2, int axis,
                            const AxisTaps1 w, int r, int64_t G0, int64_t G1, int64_t G2,
                            int64_t off0, int64_t off1, int64_t off2) {
  const int64_t total = n0 * n1 * n2;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t x = q % n2, y = (q / n2) % n1, z = q / (n1 * n2);
    int64_t c[3] = {off0 + z, off1 + y, off2 + x};
    const int64_t Gs[3] = {G0, G1, G2};
    float acc = 0.0f;
    for (int j = 0; j <= 2 * r; ++j) {  // input coordinate increasing: k = r - j
      int64_t sc[3] = {c[0], c[1], c[2]};
      sc[axis] = reflect(c[axis] - (r - j), Gs[axis]);
      const int64_t l0 = sc[0] - S.lo[0], l1 = sc[1] - S.lo[1], l2 = sc[2] - S.lo[2];
      float v = 0.0f;
      if (l0 >= 0 && l0 < S.dims[0] && l1 >= 0 && l1 < S.dims[1] && l2 >= 0 && l2 < S.dims[2])
        v = to_f32<TIN>(src[(l0 * S.dims[1] + l1) * S.dims[2] + l2]);
      acc = fmaf(w.w[2 * r - j], v, acc);
    }
    if (TO_OUT)
      store_out(O, ((c[0] - O.lo[0]) * O.dims[1] + (c[1] - O.lo[1])) * O.dims[2] + (c[2] - O.lo[2]), acc);
    else
      dst[q] = acc;
  }
}

// The same passes for every radius 1 .. kMaxRGeneric (above the z-march
// kernels' 12, and any radius on volumes thinner than it in x or y), with
// every output still one FMA chain from +0 over its taps in increasing
// input coordinate (so the results equal k_axis_pass's bit for bit):
//   z / y (k_gcol): one thread per line of the destination region, lines of
//     consecutive x (every warp access is one coalesced row); the thread
//     marches the line's reflected samples and keeps the 2R + 1 partial
//     outputs in registers as a shift ring: sample i adds tap s to the output
//     in slot s, slot 0 is then complete, and every slot moves down one.
//   x (k_grow): a CTA stages kGR rows x (kGX + 2R) reflected samples as FP32
//     in shared memory with coalesced loads, one thread marches each row the
//     same way (odd row stride: conflict free) and writes its outputs over the
//     samples it has consumed, and the CTA stores them coalesced.
// Taps sit in the kernel parameters at compile-time indices, so each FMA
// takes its weight from the constant bank.
template <int R>
struct GW {
  float w[2 * R + 1];
};

template <int R, int AXIS, bool TO_OUT>
__global__ void __launch_bounds__(128) k_gcol(const float* __restrict__ src, const AxisBox S,
                                              float* __restrict__ dst, const AxisBox D, DevOut O,
                                              const GW<R> W, int64_t Gn) {
  constexpr int L = 2 * R + 1;
  constexpr int a1 = AXIS == 0 ? 1 : 0;  // the other axes: a1 slow, x fast
  const int64_t nlines = D.dims[a1] * D.dims[2];
  const int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (l >= nlines) return;
  int64_t c3[3];
  c3[2] = D.lo[2] + l % D.dims[2];
  c3[a1] = D.lo[a1] + l / D.dims[2];
  c3[AXIS] = S.lo[AXIS];
  const int64_t sstr = AXIS == 1 ? S.dims[2] : S.dims[1] * S.dims[2];
  const float* sp = src + ((c3[0] - S.lo[0]) * S.dims[1] + (c3[1] - S.lo[1])) * S.dims[2] +
                    (c3[2] - S.lo[2]) - S.lo[AXIS] * sstr;
  c3[AXIS] = D.lo[AXIS];
  int64_t ob, ostr;
  if constexpr (TO_OUT) {
    ob = ((c3[0] - O.lo[0]) * O.dims[1] + (c3[1] - O.lo[1])) * O.dims[2] + (c3[2] - O.lo[2]);
    ostr = AXIS == 1 ? O.dims[2] : O.dims[1] * O.dims[2];
  } else {
    ob = ((c3[0] - D.lo[0]) * D.dims[1] + (c3[1] - D.lo[1])) * D.dims[2] + (c3[2] - D.lo[2]);
    ostr = AXIS == 1 ? D.dims[2] : D.dims[1] * D.dims[2];
  }
  const int n = (int)D.dims[AXIS];
  const int64_t p0 = D.lo[AXIS] - R;  // global coordinate of sample 0
  const bool inner = p0 >= 0 && p0 + n + 2 * R <= Gn;
  float acc[L];
#pragma unroll
  for (int k = 0; k < L; ++k) acc[k] = 0.0f;
  // after sample i, output i - 2R is complete. The samples of a chunk of
  // kGQ are loaded into registers before any of its outputs is stored (the
  // stores could alias the source as far as the compiler can tell, which
  // would otherwise keep each load behind the previous sample's store).
  constexpr int kGQ = 16;
  const int ns = n + 2 * R;
  for (int i0 = 0; i0 < ns; i0 += kGQ) {
    float v[kGQ];
#pragma unroll
    for (int u = 0; u < kGQ; ++u)
      v[u] = i0 + u < ns ? sp[(inner ? p0 + i0 + u : reflect(p0 + i0 + u, Gn)) * sstr] : 0.0f;
#pragma unroll
    for (int u = 0; u < kGQ; ++u) {
      const int i = i0 + u;
      if (i >= ns) break;
      const float done = fmaf(W.w[0], v[u], acc[0]);
#pragma unroll
      for (int k = 1; k < L; ++k) acc[k - 1] = fmaf(W.w[k], v[u], acc[k]);
      acc[L - 1] = 0.0f;
      if (i >= 2 * R) {
        const int64_t q = ob + (int64_t)(i - 2 * R) * ostr;
        if constexpr (TO_OUT) store_out(O, q, done);
        else dst[q] = done;
      }
    }
  }
}

constexpr int kGR = 128;  // rows per CTA (one thread each)
constexpr int kGX = 64;   // outputs per row per CTA

template <int R>
constexpr int grow_ws() { return (kGX + 2 * R) | 1; }

template <typename TIN, int R>
__global__ void __launch_bounds__(kGR) k_grow(const TIN* __restrict__ src, const AxisBox S,
                                              float* __restrict__ dst, const AxisBox D,
                                              const GW<R> W, int64_t Gx, int vec_rows) {
  constexpr int L = 2 * R + 1, WS = grow_ws<R>();
  extern __shared__ float Eg[];
  __shared__ int64_t s_sb[kGR], s_db[kGR];
  const int tid = threadIdx.x;
  const int64_t nlines = D.dims[0] * D.dims[1];
  const int64_t s0 = (int64_t)blockIdx.x * kGX;  // first output of the segment (region index)
  const int n = (int)min((int64_t)kGX, D.dims[2] - s0);
  const int ns = n + 2 * R;
  const int64_t p0 = D.lo[2] + s0 - R;           // global x of sample 0
  const bool inner = p0 >= 0 && p0 + ns <= Gx;
  for (int64_t line0 = (int64_t)blockIdx.y * kGR; line0 < nlines; line0 += (int64_t)gridDim.y * kGR) {
    const int nlin = (int)min((int64_t)kGR, nlines - line0);
    {
      const int64_t l = min(line0 + tid, nlines - 1);
      const int64_t z = D.lo[0] + l / D.dims[1], y = D.lo[1] + l % D.dims[1];
      s_sb[tid] = ((z - S.lo[0]) * S.dims[1] + (y - S.lo[1])) * S.dims[2] - S.lo[2];
      s_db[tid] = ((z - D.lo[0]) * D.dims[1] + (y - D.lo[1])) * D.dims[2];
    }
    __syncthreads();
    constexpr int kU = 8;  // loads in flight per thread
    if (inner && vec_rows) {
      // rows start on 16-byte boundaries: stage whole aligned 16-byte words
      // covering samples [0, ns) of each row (a word never crosses the end of
      // its row: row lengths are whole words)
      constexpr int EPV = 16 / (int)sizeof(TIN);
      const int64_t off0 = p0 - S.lo[2];
      const int64_t w0 = off0 & ~(int64_t)(EPV - 1);
      const int nw = (int)((off0 + ns - w0 + EPV - 1) / EPV);
      constexpr int kV = 4;
      for (int i0 = tid; i0 < nlin * nw; i0 += kGR * kV) {
        uint4 q[kV];
#pragma unroll
        for (int u = 0; u < kV; ++u) {
          const int i = i0 + u * kGR;
          if (i < nlin * nw) {
            const int r = i / nw, k = i - r * nw;
            q[u] = *reinterpret_cast<const uint4*>(src + s_sb[r] + S.lo[2] + w0 + (int64_t)k * EPV);
          }
        }
#pragma unroll
        for (int u = 0; u < kV; ++u) {
          const int i = i0 + u * kGR;
          if (i < nlin * nw) {
            const int r = i / nw, k = i - r * nw;
            const TIN* el = reinterpret_cast<const TIN*>(&q[u]);
            const int pos0 = (int)(w0 - off0) + k * EPV;
#pragma unroll
            for (int c = 0; c < EPV; ++c)
              if (pos0 + c >= 0 && pos0 + c < ns) Eg[r * WS + pos0 + c] = to_f32<TIN>(el[c]);
          }
        }
      }
    } else
    for (int i0 = tid; i0 < kGR * ns; i0 += kGR * kU) {
      float v[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int i = i0 + u * kGR, r = i / ns, pos = i - r * ns;
        v[u] = 0.0f;
        if (i < kGR * ns && r < nlin)
          v[u] = to_f32<TIN>(src[s_sb[r] + (inner ? p0 + pos : reflect(p0 + pos, Gx))]);
      }
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int i = i0 + u * kGR;
        if (i < kGR * ns) Eg[(i / ns) * WS + i % ns] = v[u];
      }
    }
    __syncthreads();
    {
      float* e = Eg + tid * WS;
      float acc[L];
#pragma unroll
      for (int k = 0; k < L; ++k) acc[k] = 0.0f;
      // chunks of 8 samples loaded into registers before their outputs are
      // written back (output i - 2R overwrites a sample of this or an earlier
      // chunk, already in registers or consumed)
      for (int i0 = 0; i0 < ns; i0 += 8) {
        float v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = i0 + u < ns ? e[i0 + u] : 0.0f;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int i = i0 + u;
          if (i >= ns) break;
          const float done = fmaf(W.w[0], v[u], acc[0]);
#pragma unroll
          for (int k = 1; k < L; ++k) acc[k - 1] = fmaf(W.w[k], v[u], acc[k]);
          acc[L - 1] = 0.0f;
          if (i >= 2 * R) e[i - 2 * R] = done;
        }
      }
    }
    __syncthreads();
    for (int i = tid; i < kGR * kGX; i += kGR) {
      const int r = i / kGX, o = i - r * kGX;
      if (r < nlin && o < n) dst[s_db[r] + s0 + o] = Eg[r * WS + o];
    }
    __syncthreads();  // the next round restages Eg and the row offsets
  }
}

template <int R, typename TIN>
cudaError_t launch_zm_t(const GaussParams& P, const CUtensorMap& map, dim3 grid, cudaStream_t s) {
  static bool attr_set = false;  // per instantiation; set once per process
  constexpr int TX = ZmTile<R>::TX, TY = ZmTile<R>::TY;
  constexpr int smem = zm_smem_bytes<R, TX, TY>((int)sizeof(TIN));
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_gauss_zm<R, TIN, TX, TY>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  k_gauss_zm<R, TIN, TX, TY><<<grid, TX * TY / 4, smem, s>>>(P, map);
  return cudaGetLastError();
}

template <typename TIN>
cudaError_t dispatch_zm_t(int r, const GaussParams& P, const CUtensorMap& map, dim3 grid,
                          cudaStream_t s) {
  switch (r) {
#define HP_CASE(RR) \
  case RR: return launch_zm_t<RR, TIN>(P, map, grid, s);
    HP_CASE(1) HP_CASE(2) HP_CASE(3) HP_CASE(4) HP_CASE(5) HP_CASE(6)
    HP_CASE(7) HP_CASE(8) HP_CASE(9) HP_CASE(10) HP_CASE(11) HP_CASE(12)
#undef HP_CASE
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t dispatch_zm(int r, const GaussParams& P, const CUtensorMap& map, dim3 grid,
                        cudaStream_t s) {
  switch (P.job.in.dtype) {
    case HP_U8: return dispatch_zm_t<uint8_t>(r, P, map, grid, s);
    case HP_U16: return dispatch_zm_t<uint16_t>(r, P, map, grid, s);
    case HP_F16: return dispatch_zm_t<__half>(r, P, map, grid, s);
    default: return dispatch_zm_t<float>(r, P, map, grid, s);
  }
}

bool needs_generic(const Job& job, int r) {
  return !(r >= 1 && r <= kMaxR && job.gdims[2] >= r && job.gdims[1] >= r);
}

// Generic path for radius R above the z-march kernels: k_grow, then k_gcol
// along y, then along z into the job's output.
template <int R>
cudaError_t launch_generic_r(const Job& job, const Taps& taps, float* t1, float* t2,
                             const SepRegions& g, cudaStream_t s) {
  GW<R> wz, wy, wx;
  for (int k = 0; k < 2 * R + 1; ++k) {
    wz.w[k] = taps.w[0][k];
    wy.w[k] = taps.w[1][k];
    wx.w[k] = taps.w[2][k];
  }
  const AxisBox sin{{job.in.lo[0], job.in.lo[1], job.in.lo[2]},
                    {job.in.dims[0], job.in.dims[1], job.in.dims[2]}};
  const AxisBox s1{{g.rlo[0], g.rlo[1], job.core_lo[2]}, {g.n_x[0], g.n_x[1], g.n_x[2]}};
  const AxisBox s2{{g.rlo[0], job.core_lo[1], job.core_lo[2]}, {g.n_y[0], g.n_y[1], g.n_y[2]}};
  const AxisBox core{{job.core_lo[0], job.core_lo[1], job.core_lo[2]},
                     {job.core_hi[0] - job.core_lo[0], job.core_hi[1] - job.core_lo[1],
                      job.core_hi[2] - job.core_lo[2]}};
  const int smem = kGR * grow_ws<R>() * 4;
  const int64_t rows = s1.dims[0] * s1.dims[1];
  const dim3 gx((unsigned)((s1.dims[2] + kGX - 1) / kGX),
                (unsigned)std::min<int64_t>((rows + kGR - 1) / kGR, 65535));
  cudaError_t e = cudaSuccess;
  switch (job.in.dtype) {
#define HP_GROW(T)                                                                             \
  {                                                                                            \
    static bool attr = false;                                                                  \
    if (!attr) {                                                                               \
      e = cudaFuncSetAttribute(k_grow<T, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem); \
      if (e != cudaSuccess) return e;                                                          \
      attr = true;                                                                             \
    }                                                                                          \
    const int vec = reinterpret_cast<uintptr_t>(job.in.ptr) % 16 == 0 &&                       \
                    (job.in.dims[2] * (int64_t)sizeof(T)) % 16 == 0;                            \
    k_grow<T, R><<<gx, kGR, smem, s>>>(static_cast<const T*>(job.in.ptr), sin, t1, s1, wx,      \
                                       job.gdims[2], vec);                                     \
  } break;
    case HP_U8: HP_GROW(uint8_t)
    case HP_U16: HP_GROW(uint16_t)
    case HP_F16: HP_GROW(__half)
    case HP_F32: HP_GROW(float)
#undef HP_GROW
    default: return cudaErrorInvalidValue;
  }
  const int64_t ly = s2.dims[0] * s2.dims[2], lz = core.dims[1] * core.dims[2];
  k_gcol<R, 1, false><<<(unsigned)((ly + 127) / 128), 128, 0, s>>>(t1, s1, t2, s2, job.out, wy,
                                                                    job.gdims[1]);
  k_gcol<R, 0, true><<<(unsigned)((lz + 127) / 128), 128, 0, s>>>(t2, s2, nullptr, core, job.out,
                                                                   wz, job.gdims[0]);
  return cudaGetLastError();
}

cudaError_t launch_generic(const Job& job, const Taps& taps, cudaStream_t s) {
  // Three passes x -> y -> z; the x and y passes go through two FP32
  // scratch volumes that the caller provides in job.scratch (the z pass
  // stores into the output). The kernels take taps and boxes by value.
  const int r = taps.r;
  const int64_t cz = job.core_hi[0] - job.core_lo[0], cy = job.core_hi[1] - job.core_lo[1],
                cx = job.core_hi[2] - job.core_lo[2];
  if (cz <= 0 || cy <= 0 || cx <= 0) return cudaSuccess;
  const SepRegions g = sep_regions(job, r);
  const size_t b1 = sizeof(float) * (size_t)(g.n_x[0] * g.n_x[1] * g.n_x[2]);
  const size_t b2 = sizeof(float) * (size_t)(g.n_y[0] * g.n_y[1] * g.n_y[2]);
  if (!job.scratch || job.scratch_bytes < b1 + b2) return cudaErrorInvalidValue;
  float* t1 = static_cast<float*>(job.scratch);
  float* t2 = t1 + b1 / sizeof(float);
  switch (r) {
#define HP_GR(RR) \
  case RR: return launch_generic_r<RR>(job, taps, t1, t2, g, s);
    HP_GR(1) HP_GR(2) HP_GR(3) HP_GR(4) HP_GR(5) HP_GR(6) HP_GR(7) HP_GR(8) HP_GR(9) HP_GR(10)
    HP_GR(11) HP_GR(12) HP_GR(13) HP_GR(14) HP_GR(15) HP_GR(16) HP_GR(17) HP_GR(18) HP_GR(19) HP_GR(20)
    HP_GR(21) HP_GR(22) HP_GR(23) HP_GR(24) HP_GR(25) HP_GR(26) HP_GR(27) HP_GR(28)
    HP_GR(29) HP_GR(30) HP_GR(31) HP_GR(32)
#undef HP_GR
    default: break;  // radius 0: per-output passes
  }
  AxisTaps1 wz, wy, wx;
  for (int k = 0; k < kMaxTaps; ++k) {
    wz.w[k] = taps.w[0][k];
    wy.w[k] = taps.w[1][k];
    wx.w[k] = taps.w[2][k];
  }
  const AxisBox sin{{job.in.lo[0], job.in.lo[1], job.in.lo[2]},
                    {job.in.dims[0], job.in.dims[1], job.in.dims[2]}};
  const AxisBox s1{{g.rlo[0], g.rlo[1], job.core_lo[2]}, {g.n_x[0], g.n_x[1], g.n_x[2]}};
  const AxisBox s2{{g.rlo[0], job.core_lo[1], job.core_lo[2]}, {g.n_y[0], g.n_y[1], g.n_y[2]}};
  const int blk = 256;
  auto grid_for = [&](const int64_t* n) {
    const int64_t t = n[0] * n[1] * n[2];
    return (unsigned)std::min<int64_t>((t + blk - 1) / blk, (int64_t)num_sms() * 32);
  };
  const int64_t n_z[3] = {cz, cy, cx};
  const int64_t G0 = job.gdims[0], G1 = job.gdims[1], G2 = job.gdims[2];
  switch (job.in.dtype) {
#define HP_PASS1(T)                                                                             \
  k_axis_pass<T, false><<<grid_for(g.n_x), blk, 0, s>>>(                                       \
      static_cast<const T*>(job.in.ptr), sin, t1, job.out, g.n_x[0], g.n_x[1], g.n_x[2], 2, wx, \
      r, G0, G1, G2, g.rlo[0], g.rlo[1], job.core_lo[2]);                                       \
  break;
    case HP_U8: HP_PASS1(uint8_t)
    case HP_U16: HP_PASS1(uint16_t)
    case HP_F16: HP_PASS1(__half)
    case HP_F32: HP_PASS1(float)
#undef HP_PASS1
    default: return cudaErrorInvalidValue;
  }
  k_axis_pass<float, false><<<grid_for(g.n_y), blk, 0, s>>>(
      t1, s1, t2, job.out, g.n_y[0], g.n_y[1], g.n_y[2], 1, wy, r, G0, G1, G2, g.rlo[0],
      job.core_lo[1], job.core_lo[2]);
  k_axis_pass<float, true><<<grid_for(n_z), blk, 0, s>>>(
      t2, s2, nullptr, job.out, n_z[0], n_z[1], n_z[2], 0, wz, r, G0, G1, G2, job.core_lo[0],
      job.core_lo[1], job.core_lo[2]);
  return cudaGetLastError();
}

}  // namespace

// Regions of a separable three-pass job of radius r: after the x pass, z
// and y grown to the hull of their reflected sources and x = core; after
// the y pass, z grown and y, x = core.
SepRegions sep_regions(const Job& job, int r) {
  SepRegions g;
  int64_t rhi[2];
  for (int a = 0; a < 2; ++a) {
    const int64_t n = job.gdims[a], lo = job.core_lo[a], hi = job.core_hi[a];
    int64_t mn = n, mx = -1;
    if (hi - lo + 2 * r >= 2 * n) {
      mn = 0;
      mx = n - 1;
    } else {
      for (int64_t c = lo - r; c < hi + r; ++c) {
        const int64_t sidx = reflect(c, n);
        mn = std::min(mn, sidx);
        mx = std::max(mx, sidx);
      }
    }
    g.rlo[a] = mn;
    rhi[a] = mx + 1;
  }
  const int64_t cx = job.core_hi[2] - job.core_lo[2], cy = job.core_hi[1] - job.core_lo[1];
  g.n_x[0] = rhi[0] - g.rlo[0];
  g.n_x[1] = rhi[1] - g.rlo[1];
  g.n_x[2] = cx;
  g.n_y[0] = g.n_x[0];
  g.n_y[1] = cy;
  g.n_y[2] = cx;
  return g;
}

size_t gauss_scratch_bytes(const Job& job, int r) {
  if (!needs_generic(job, r)) return 0;
  const SepRegions g = sep_regions(job, r);
  return sizeof(float) * (size_t)(g.n_x[0] * g.n_x[1] * g.n_x[2] + g.n_y[0] * g.n_y[1] * g.n_y[2]);
}

cudaError_t launch_gauss(const Job& job, const Taps& taps, cudaStream_t s) {
  const int r = taps.r;
  // register z-march (k_gauss_zr.cu) wherever its layout rules hold
  const cudaError_t ezr = launch_gauss_zr(job, taps, s);
  if (ezr != cudaErrorNotSupported) return ezr;
  if (needs_generic(job, r)) return launch_generic(job, taps, s);

  GaussParams P;
  P.job = job;
  for (int a = 0; a < 3; ++a)
    for (int k = 0; k <= 2 * kMaxR; ++k) {
      const uint32_t b = k <= 2 * r ? __float_as_uint_host(taps.w[a][k]) : 0u;
      P.w2[a][k] = ((u64)b << 32) | b;
    }
  P.r = r;
  P.err = device_error_word();
  const int64_t cx = job.core_hi[2] - job.core_lo[2];
  const int64_t cy = job.core_hi[1] - job.core_lo[1];
  const int64_t cz = job.core_hi[0] - job.core_lo[0];
  if (cx <= 0 || cy <= 0 || cz <= 0) return cudaSuccess;
  const int tx = r <= 6 ? 64 : 32, ty = r <= 6 ? 16 : 32;  // ZmTile<r>
  P.tiles_x = (int)((cx + tx - 1) / tx);
  const int64_t tiles = (int64_t)P.tiles_x * ((cy + ty - 1) / ty);
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
    box_geom(r, (int)es, tx, &ra, &bw);
    const int64_t dims[3] = {job.in.dims[2], job.in.dims[1], job.in.dims[0]};
    use_tma = make_tmap_3d(&map, job.in.ptr, job.in.dtype, dims, bw, ty + 2 * r);
  }
  P.use_tma = use_tma ? 1 : 0;
  if (log_level() > 0)
    fprintf(stderr, "[hp] gauss z-march r=%d tile=%dx%d tma=%d grid=%ux%u zchunk=%d\n", r, tx, ty,
            P.use_tma, grid.x, grid.y, P.zchunk);
  return dispatch_zm(r, P, map, grid, s);
}

}  // namespace hp
