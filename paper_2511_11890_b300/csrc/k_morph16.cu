// Grayscale erosion / dilation of 16-bit volumes (uint16, float16) with
// packed keys (Harpia Sec. III-C). Exact, reflect boundaries on global
// coordinates, same result as the 32-bit-key kernel in k_morph.cu.
//
// Two x-neighbours share one 32-bit register: the pair (x, x+1) of
// order-preserving 16-bit keys, so every min is one SIMD instruction over
// two voxels (__vminu2 / the three-input __vimin3_u16x2; dilation uses the
// max forms). uint16 keys are the values themselves, float16 keys the
// sign-magnitude flip applied to whole 32-bit words.
//
// Tiled z-march: a CTA owns a 64 x 32 column of the core and marches along
// z through a 4-stage TMA pipeline of halo-padded planes. Phase p:
//   x (plane p-1, read straight from its TMA stage): x-line minima M_L of
//     half-length L = 0..r over 8 outputs per item, with
//       M_1 = min3(v[-1], v[0], v[+1])            (odd shift: one byte permute)
//       M_2 = min3(v[-2], M_1[0], v[+2])           (even shifts: whole words)
//       M_L = min3(M_{L-2}[-2], M_{L-2}[0], M_{L-2}[+2])   (L >= 3)
//     (cube: only M_r is kept);
//   y + z (plane p-2): disk minima D_|dz| = min over dy of M_L(dy,dz)(y+dy),
//     L(dy,dz) = floor(sqrt(r^2 - dy^2 - dz^2)) (cube: D = min over |dy| <= r
//     of M_r), pushed into a shift-register ring of the 2r+1 outputs that
//     plane p-2 contributes to; the oldest output is complete and stored.
// One CTA barrier per phase. Tiles whose halo leaves the volume overwrite
// the out-of-volume cells of the TMA stage with their reflected sources
// before the x pass reads it.
#include <cuda_fp16.h>

#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <type_traits>

#include "hp_device.cuh"
#include "hp_internal.h"

namespace hp {

namespace {

constexpr int kPX = 64;        // tile width (outputs along x)
constexpr int kPY = 32;        // tile height
constexpr int kPT = 256;       // threads per CTA
constexpr int kPB = 4;         // rows per thread in the y and z passes
constexpr int kPS = 4;         // TMA stages
constexpr int kPC = kPX / 2;   // pair columns of the tile
constexpr int kXI = 8;         // outputs per x-pass item (four pairs)
constexpr int kMaxR16 = 6;

struct Morph16Params {
  Job job;
  int zchunk;
  int tiles_x;
  int* err;
};

__host__ __device__ constexpr int rup(int a, int b) { return (a + b - 1) / b * b; }

// floor(sqrt(v)) for 0 <= v < 64 without a loop, so that it folds to a
// constant inside unrolled loops.
__host__ __device__ constexpr int isqrt63(int v) {
  return (v >= 1) + (v >= 4) + (v >= 9) + (v >= 16) + (v >= 25) + (v >= 36) + (v >= 49);
}

// Half-length of the ball's x-line at (dz, dy); -1 outside the ball.
__host__ __device__ constexpr int line_len(int R, int dz, int dy) {
  return dz * dz + dy * dy <= R * R ? isqrt63(R * R - dz * dz - dy * dy) : -1;
}

template <int R, int BALL>
struct PG {
  static constexpr int BH = kPY + 2 * R;            // patch rows (y halo included)
  static constexpr int RA = rup(R, 8);              // left halo of the TMA box (16-byte aligned)
  static constexpr int BW = rup(kPX + RA + R, 8);   // TMA box width, elements
  static constexpr int BWW = BW / 2;                // stage row stride, 32-bit words
  static constexpr int HP = (R + 1) / 2;            // halo pairs per side of an x item
  static constexpr int NW = kXI / 2 + 2 * HP;       // window pairs of an x item
  static constexpr int W0 = RA / 2 - HP;            // stage word of window pair 0 of item 0
  static constexpr int NXI = BH * (kPX / kXI);      // x items per plane
  static constexpr int NL = BALL ? R + 1 : 1;       // stored line-minimum levels
  static constexpr int NDZ = BALL ? R + 1 : 1;      // distinct disks
  static constexpr int MSZ = NL * BH * kPC;         // words per line-minimum buffer
  static constexpr int SB = rup(BW * BH * 2, 128);  // bytes per TMA stage
  static constexpr int SMEM = 128 + kPS * SB + 2 * MSZ * 4;
  static_assert(W0 >= 0 && RA / 2 + kPC + HP <= BWW, "x window inside the TMA box");
  static_assert((BWW * 4) % 16 == 0 &&
                    (W0 - W0 % 4) + 4 * (kPX / kXI - 1) + 4 * ((W0 % 4 + NW + 3) / 4) <= BWW,
                "aligned x windows inside the stage row");
};

// 16-bit keys of a word holding two elements. float16: positive values get
// the sign bit set, negative ones are complemented (order-preserving).
template <int KIND>
__device__ __forceinline__ uint32_t to_keys(uint32_t w) {
  if (KIND == 1) {
    const uint32_t s = (w >> 15) & 0x00010001u;
    w ^= 0x80008000u | (s * 0x7FFFu);
  }
  return w;
}

template <int KIND>
__device__ __forceinline__ uint32_t from_keys(uint32_t k) {
  if (KIND == 1) {
    const uint32_t s = (k >> 15) & 0x00010001u;
    k ^= 0xFFFFFFFFu ^ (s * 0x7FFFu);
  }
  return k;
}

// Erosion takes minima, dilation maxima (of the same keys).
template <int DIL>
struct Op {
  static constexpr uint32_t id = DIL ? 0u : 0xFFFFFFFFu;  // identity element
  static __device__ __forceinline__ uint32_t f2(uint32_t a, uint32_t b) {
    return DIL ? __vmaxu2(a, b) : __vminu2(a, b);
  }
  static __device__ __forceinline__ uint32_t f3(uint32_t a, uint32_t b, uint32_t c) {
    return DIL ? __vimax3_u16x2(a, b, c) : __vimin3_u16x2(a, b, c);
  }
};

// x pass of one item: 8 outputs (pairs HP .. HP+3 of the window) of stage
// row `row`, x group g. Window pair k holds x = cx0 + 8g - 2HP + 2k, +1.
template <int R, int BALL, int KIND, int DIL>
__device__ __forceinline__ void xpass_item(uint32_t* Mb, const uint32_t* S, int row, int g) {
  using G = PG<R, BALL>;
  using O = Op<DIL>;
  constexpr int NW = G::NW;
  // The window is read as whole 16-byte words starting at the aligned word
  // below it: the 8 items of a quarter warp (one row, consecutive groups)
  // then read one contiguous 128-byte line per load, free of bank conflicts.
  constexpr int A0 = G::W0 % 4;
  constexpr int NQ = (A0 + NW + 3) / 4;
  const uint4* src = reinterpret_cast<const uint4*>(S + row * G::BWW + (G::W0 - A0) + 4 * g);
  uint32_t t[4 * NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const uint4 v = src[q];
    t[4 * q] = v.x;
    t[4 * q + 1] = v.y;
    t[4 * q + 2] = v.z;
    t[4 * q + 3] = v.w;
  }
  uint32_t lv[R + 1][NW];
#pragma unroll
  for (int k = 0; k < NW; ++k) lv[0][k] = to_keys<KIND>(t[A0 + k]);
  // q[k] = (v at pair k high half, pair k+1 low half): the odd shift
  uint32_t q[NW - 1];
#pragma unroll
  for (int k = 0; k + 1 < NW; ++k) q[k] = __byte_perm(lv[0][k], lv[0][k + 1], 0x5432);
#pragma unroll
  for (int k = 1; k + 1 < NW; ++k) lv[1][k] = O::f3(q[k - 1], lv[0][k], q[k]);
  if constexpr (R >= 2) {
#pragma unroll
    for (int k = 1; k + 1 < NW; ++k) lv[2][k] = O::f3(lv[0][k - 1], lv[1][k], lv[0][k + 1]);
  }
#pragma unroll
  for (int L = 3; L <= R; ++L) {
    const int c = (L + 1) / 2;
#pragma unroll
    for (int k = c; k < NW - c; ++k) lv[L][k] = O::f3(lv[L - 2][k - 1], lv[L - 2][k], lv[L - 2][k + 1]);
  }
  uint32_t* dst = Mb + row * kPC + 4 * g;
  constexpr int H = G::HP;
  if constexpr (BALL) {
#pragma unroll
    for (int L = 0; L <= R; ++L)
      *reinterpret_cast<uint4*>(dst + L * G::BH * kPC) =
          make_uint4(lv[L][H], lv[L][H + 1], lv[L][H + 2], lv[L][H + 3]);
  } else {
    *reinterpret_cast<uint4*>(dst) = make_uint4(lv[R][H], lv[R][H + 1], lv[R][H + 2], lv[R][H + 3]);
  }
}

// Disk minima of kPB consecutive output rows at one pair column. Mc points
// at level 0, the row of output row 0 (dy = 0).
template <int R, int BALL, int DIL>
__device__ __forceinline__ void disks(uint32_t (&D)[PG<R, BALL>::NDZ][kPB], const uint32_t* Mc) {
  using G = PG<R, BALL>;
  using O = Op<DIL>;
  auto m = [&](int L, int i, int dy) { return Mc[(L * G::BH + i + dy) * kPC]; };
  if constexpr (BALL && R == 3) {
    // shared three-row minimum of M_2 (see the line lengths of the r = 3 ball)
#pragma unroll
    for (int i = 0; i < kPB; ++i) {
      const uint32_t a = O::f3(m(2, i, -1), m(2, i, 0), m(2, i, 1));
      const uint32_t d1 = O::f3(a, m(2, i, -2), m(2, i, 2));
      D[1][i] = d1;
      D[0][i] = O::f3(d1, m(3, i, 0), O::f2(m(0, i, -3), m(0, i, 3)));
      D[2][i] = O::f3(a, m(1, i, -2), m(1, i, 2));
      D[3][i] = m(0, i, 0);
    }
  } else {
#pragma unroll
    for (int dz = 0; dz < G::NDZ; ++dz)
#pragma unroll
      for (int i = 0; i < kPB; ++i) D[dz][i] = O::id;
#pragma unroll
    for (int dz = 0; dz < G::NDZ; ++dz)
#pragma unroll
      for (int dy = -R; dy <= R; ++dy) {
        const int L = BALL ? line_len(R, dz, dy) : 0;
        if (L >= 0) {
#pragma unroll
          for (int i = 0; i < kPB; ++i) D[dz][i] = O::f2(D[dz][i], m(L, i, dy));
        }
      }
  }
}

// Resident CTAs per SM the register budget is sized for: three for radii up
// to 3 (63 KB of shared memory per CTA), two above.
template <int R>
struct MinBlocks {
  static constexpr int value = R <= 3 ? 3 : 2;
};

template <int R, int BALL, int KIND, int DIL>
__global__ void __launch_bounds__(kPT, MinBlocks<R>::value)
    k_morph16(const __grid_constant__ Morph16Params P, const __grid_constant__ CUtensorMap tmap) {
  using G = PG<R, BALL>;
  using O = Op<DIL>;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ int s_abort;
  __shared__ int s_frow[G::BH], s_fcol[G::BW], s_brow[G::BH], s_bcol[G::BW];
  __shared__ int s_nbr, s_nbc;

  const Job& J = P.job;
  const int tid = threadIdx.x;
  const int tx = blockIdx.x % P.tiles_x, ty = blockIdx.x / P.tiles_x;
  const int64_t cx0 = J.core_lo[2] + (int64_t)tx * kPX;
  const int64_t cy0 = J.core_lo[1] + (int64_t)ty * kPY;
  const int64_t cz0 = J.core_lo[0] + (int64_t)blockIdx.y * P.zchunk;
  const int64_t cz1 = min(cz0 + (int64_t)P.zchunk, J.core_hi[0]);
  if (cz0 >= cz1) return;
  const int nout = (int)(cz1 - cz0);
  const int total = nout + 2 * R;  // input planes cz0-R .. cz1+R-1
  const int64_t Gz = J.gdims[0], Gy = J.gdims[1], Gx = J.gdims[2];
  const bool face = (cx0 - R < 0) || (cx0 + kPX + R > Gx) || (cy0 - R < 0) || (cy0 + kPY + R > Gy);

  uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
  unsigned char* stages = smem + 128;
  uint32_t* M = reinterpret_cast<uint32_t*>(stages + kPS * G::SB);

  if (face) {
    // stage row r <-> y = cy0 - R + r, stage col c <-> x = cx0 - RA + c;
    // -1 where the reflected source is outside the box (no stored output
    // reads that cell)
    for (int r = tid; r < G::BH; r += kPT) {
      const int64_t s = reflect(cy0 - R + r, Gy) - (cy0 - R);
      s_frow[r] = (s >= 0 && s < G::BH) ? (int)s : -1;
    }
    for (int c = tid; c < G::BW; c += kPT) {
      const int64_t s = reflect(cx0 - G::RA + c, Gx) - (cx0 - G::RA);
      s_fcol[c] = (s >= 0 && s < G::BW) ? (int)s : -1;
    }
    __syncthreads();
    if (tid == 0) {
      int nr = 0, nc = 0;
      for (int r = 0; r < G::BH; ++r)
        if (s_frow[r] != r) s_brow[nr++] = r;
      for (int c = 0; c < G::BW; ++c)
        if (s_fcol[c] != c) s_bcol[nc++] = c;
      s_nbr = nr;
      s_nbc = nc;
    }
  }
  if (tid == 0) {
    s_abort = 0;
    prefetch_tmap(&tmap);
    for (int s = 0; s < kPS; ++s) mbar_init(&bars[s], 1);
    fence_mbar_init();
  }
  __syncthreads();
  const int nbr = face ? s_nbr : 0, nbc = face ? s_nbc : 0;

  auto issue = [&](int n) {  // TMA load of input plane n into stage n % kPS
    const int zl = (int)(reflect(cz0 - R + n, Gz) - J.in.lo[0]);
    const int xl = (int)(cx0 - G::RA - J.in.lo[2]);
    const int yl = (int)(cy0 - R - J.in.lo[1]);
    uint64_t* bar = &bars[n % kPS];
    mbar_arrive_expect_tx(bar, G::BW * G::BH * 2);
    tma_load_3d(stages + (n % kPS) * G::SB, &tmap, xl, yl, zl, bar);
  };
  int next_issue = min(kPS, total);
  if (tid == 0) {
    fence_proxy_async();
    for (int n = 0; n < next_issue; ++n) issue(n);
  }

  // y/z role: pair column xp, rows yb .. yb + kPB - 1
  const int xp = tid % kPC, yb = (tid / kPC) * kPB;
  uint32_t acc[2 * R + 1][kPB];
#pragma unroll
  for (int j = 0; j <= 2 * R; ++j)
#pragma unroll
    for (int i = 0; i < kPB; ++i) acc[j][i] = O::id;
  // output addressing: rows of this thread, one plane further per store
  const DevOut& Ob = J.out;
  const int64_t gx = cx0 + 2 * xp;
  const int64_t pstride = Ob.dims[1] * Ob.dims[2], rstride = Ob.dims[2];
  uint16_t* optr = static_cast<uint16_t*>(Ob.ptr) +
                   ((cz0 - Ob.lo[0]) * Ob.dims[1] + (cy0 + yb - Ob.lo[1])) * Ob.dims[2] + (gx - Ob.lo[2]);
  const bool xok = gx < J.core_hi[2], xpair = gx + 1 < J.core_hi[2];
  const int nrow = xok ? (int)max((int64_t)0, min((int64_t)kPB, J.core_hi[1] - (cy0 + yb))) : 0;
  const bool full = xpair && nrow == kPB;

  // One phase p: x pass of plane p-1, disks + z push of plane p-2, store of
  // output plane cz0 + p - 2 - 2R. STEADY: all three parts are known to run.
  auto phase = [&](int p, auto steady) {
    constexpr bool ST = decltype(steady)::value;
    if (ST || (p >= 1 && p <= total)) {
      const int n = p - 1;
      if (!mbar_wait(&bars[n % kPS], (n / kPS) & 1)) atomicOr(&s_abort, 1);
      unsigned char* sb = stages + (n % kPS) * G::SB;
      if (face) {
        uint16_t* S16 = reinterpret_cast<uint16_t*>(sb);
        auto cell = [&](int r, int c) -> uint16_t& { return S16[r * G::BW + c]; };
        for (int i = tid; i < nbr * G::BW; i += kPT) {
          const int r = s_brow[i / G::BW], c = i % G::BW;
          const int sr = s_frow[r], sc = s_fcol[c];
          cell(r, c) = (sr >= 0 && sc >= 0) ? cell(sr, sc) : (uint16_t)0;
        }
        for (int i = tid; i < nbc * G::BH; i += kPT) {
          const int c = s_bcol[i / G::BH], r = i % G::BH;
          const int sr = s_frow[r], sc = s_fcol[c];
          cell(r, c) = (sr >= 0 && sc >= 0) ? cell(sr, sc) : (uint16_t)0;
        }
        fence_proxy_async();  // the stage is refilled by TMA later
        __syncthreads();
      }
      uint32_t* Mb = M + (n & 1) * G::MSZ;
      const uint32_t* S = reinterpret_cast<const uint32_t*>(sb);
      xpass_item<R, BALL, KIND, DIL>(Mb, S, tid / (kPX / kXI), tid % (kPX / kXI));
      if (G::NXI > kPT && tid < G::NXI - kPT)
        xpass_item<R, BALL, KIND, DIL>(Mb, S, (tid + kPT) / (kPX / kXI), (tid + kPT) % (kPX / kXI));
    }
    if (ST || p >= 2) {
      const int n = p - 2;
      uint32_t D[G::NDZ][kPB];
      disks<R, BALL, DIL>(D, M + (n & 1) * G::MSZ + (yb + R) * kPC + xp);
      uint32_t out[kPB];
#pragma unroll
      for (int i = 0; i < kPB; ++i) {
        out[i] = O::f2(acc[0][i], D[BALL ? R : 0][i]);
#pragma unroll
        for (int j = 1; j <= 2 * R; ++j) {
          const int d = j > R ? j - R : R - j;
          acc[j - 1][i] = O::f2(acc[j][i], D[BALL ? d : 0][i]);
        }
        acc[2 * R][i] = O::id;
      }
      if (ST || n >= 2 * R) {  // output plane cz0 + n - 2R is complete
        if (full) {
#pragma unroll
          for (int i = 0; i < kPB; ++i)
            *reinterpret_cast<uint32_t*>(optr + i * rstride) = from_keys<KIND>(out[i]);
        } else {
#pragma unroll
          for (int i = 0; i < kPB; ++i) {
            if (i < nrow) {
              const uint32_t v = from_keys<KIND>(out[i]);
              if (xpair)
                *reinterpret_cast<uint32_t*>(optr + i * rstride) = v;
              else
                optr[i * rstride] = (uint16_t)v;
            }
          }
        }
        optr += pstride;
      }
    }
    __syncthreads();
    if (s_abort) return false;
    if (p >= 1 && p - 1 + kPS < total) {  // plane p-1's stage is free again
      if (tid == 0) {
        fence_proxy_async();
        issue(p - 1 + kPS);
      }
      next_issue = p + kPS;
    }
    return true;
  };
  static_assert(G::NXI <= 2 * kPT, "at most two x items per thread");

  // head (pipeline fill), steady state, tail (pipeline drain)
  const int s0 = 2 * R + 2, s1 = total + 1;  // steady phases: s0 <= p < s1
  int p = 0;
  bool ok = true;
  for (; ok && p < min(s0, total + 2); ++p) ok = phase(p, std::false_type());
  for (; ok && p < s1; ++p) ok = phase(p, std::true_type());
  for (; ok && p < total + 2; ++p) ok = phase(p, std::false_type());
  if (!ok) {
    --p;  // the phase that saw the abort
    set_device_error(P.err, kErrTimeout);
    // drain the TMA loads still in flight into this CTA's shared memory
    if (tid == 0)
      for (int n = max(0, p - 1); n < next_issue; ++n) (void)mbar_wait(&bars[n % kPS], (n / kPS) & 1);
    __syncthreads();
  }
}

template <int R, int BALL, int KIND, int DIL>
cudaError_t launch_t(const Morph16Params& P0, const CUtensorMap& map, int64_t tiles, int64_t cz,
                     cudaStream_t s) {
  using G = PG<R, BALL>;
  static int slots_per_sm = 0;  // per instantiation, set once per process
  if (!slots_per_sm) {
    cudaError_t e = cudaFuncSetAttribute(k_morph16<R, BALL, KIND, DIL>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM);
    if (e != cudaSuccess) return e;
    int nb = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_morph16<R, BALL, KIND, DIL>, kPT, G::SMEM);
    if (e != cudaSuccess) return e;
    slots_per_sm = std::max(1, nb);
  }
  Morph16Params P = P0;
  P.zchunk = (int)pick_zchunk(cz, tiles, (int64_t)slots_per_sm * num_sms(), 2 * R + 2, 1);
  dim3 grid((unsigned)tiles, (unsigned)((cz + P.zchunk - 1) / P.zchunk));
  if (log_level() > 0)
    fprintf(stderr, "[hp] morph16 r=%d ball=%d kind=%d dilate=%d grid=%ux%u zchunk=%d slots/SM=%d\n",
            R, BALL, KIND, DIL, grid.x, grid.y, P.zchunk, slots_per_sm);
  k_morph16<R, BALL, KIND, DIL><<<grid, kPT, G::SMEM, s>>>(P, map);
  return cudaGetLastError();
}

template <int BALL, int KIND, int DIL>
cudaError_t dispatch16(int r, const Morph16Params& P, const CUtensorMap& map, int64_t tiles,
                       int64_t cz, cudaStream_t s) {
  switch (r) {
    case 1: return launch_t<1, BALL, KIND, DIL>(P, map, tiles, cz, s);
    case 2: return launch_t<2, BALL, KIND, DIL>(P, map, tiles, cz, s);
    case 3: return launch_t<3, BALL, KIND, DIL>(P, map, tiles, cz, s);
    case 4: return launch_t<4, BALL, KIND, DIL>(P, map, tiles, cz, s);
    case 5: return launch_t<5, BALL, KIND, DIL>(P, map, tiles, cz, s);
    case 6: return launch_t<6, BALL, KIND, DIL>(P, map, tiles, cz, s);
  }
  return cudaErrorInvalidValue;
}

template <int KIND, int DIL>
cudaError_t dispatch_se(int ball, int r, const Morph16Params& P, const CUtensorMap& map,
                        int64_t tiles, int64_t cz, cudaStream_t s) {
  return ball ? dispatch16<1, KIND, DIL>(r, P, map, tiles, cz, s)
              : dispatch16<0, KIND, DIL>(r, P, map, tiles, cz, s);
}

// --------------------------------------------------------------------------
// Strip variant (radius <= 3): no line-minimum buffer in shared memory. A
// thread owns one pair column and kSS consecutive output rows of a 64 x 32
// tile; for each input plane it reads its (1 + 2HP)-word window of the
// kSS + 2R stage rows it needs, forms the x-line minima of its pair per row,
// the disk minima of its rows from the last 2R + 1 rows (registers), and
// pushes them into its z ring. Four input planes per phase arrive in one
// four-deep TMA box (single-plane loads where z reflects), two groups in
// flight; face tiles patch the out-of-volume stage cells from a per-thread
// list of (cell, source) offsets before the barrier that precedes use.
constexpr int kSS = 8;                       // output rows per thread
constexpr int kSKP = 4;                      // input planes per phase (TMA box depth)
constexpr int kSNSG = 2;                     // plane groups in flight
constexpr int kSThreads = kPC * (kPY / kSS);  // 128
constexpr int kSFix = 8;                     // face cells per thread in registers
constexpr int kSDrift = 96;                  // z-chunk length that keeps halo reuse in L2

__host__ __device__ constexpr int gcd_i(int a, int b) { return b == 0 ? a : gcd_i(b, a % b); }

template <int R>
struct SG {
  static constexpr int BH = kPY + 2 * R;                      // stage rows used
  static constexpr int RA = rup(R, 8);
  static constexpr int BW = rup(kPX + RA + R, 8);             // stage row, elements
  static constexpr int BWW = BW / 2;                          // stage row, words
  static constexpr int BHP = rup(BH, 128 / gcd_i(BW * 2, 128));  // rows loaded
  static constexpr int PB = BW * BHP * 2;                     // bytes per stage plane
  static constexpr int GB = kSKP * PB;
  static constexpr int HP = (R + 1) / 2;
  static constexpr int NW = 1 + 2 * HP;                       // window words per row
  static constexpr int NR = kSS + 2 * R;                      // stage rows per strip
  static constexpr int NC = kPX + 2 * R;                      // stage columns read
  static constexpr int SMEM = 128 + kSNSG * GB;
  static_assert(PB % 128 == 0, "stage planes on 128-byte boundaries");
  static_assert(RA / 2 - HP >= 0 && RA / 2 + kPC - 1 + HP < BWW, "windows inside the row");
};

// x-line minima M[L] (L = 0..R) of one pair from its window w[0..NW) of keys
// (pair at w[HP]).
template <int R, int DIL>
__device__ __forceinline__ void xline1(const uint32_t (&w)[SG<R>::NW], uint32_t (&M)[R + 1]) {
  using O = Op<DIL>;
  constexpr int NW = SG<R>::NW, H = SG<R>::HP;
  uint32_t lv[R + 1][NW];
#pragma unroll
  for (int k = 0; k < NW; ++k) lv[0][k] = w[k];
  uint32_t q[NW - 1];
#pragma unroll
  for (int k = 0; k + 1 < NW; ++k) q[k] = __byte_perm(w[k], w[k + 1], 0x5432);
#pragma unroll
  for (int k = 1; k + 1 < NW; ++k) lv[1][k] = O::f3(q[k - 1], w[k], q[k]);
  if constexpr (R >= 2) {
#pragma unroll
    for (int k = 1; k + 1 < NW; ++k) lv[2][k] = O::f3(w[k - 1], lv[1][k], w[k + 1]);
  }
#pragma unroll
  for (int L = 3; L <= R; ++L) {
    const int c = (L + 1) / 2;
#pragma unroll
    for (int k = c; k < NW - c; ++k) lv[L][k] = O::f3(lv[L - 2][k - 1], lv[L - 2][k], lv[L - 2][k + 1]);
  }
#pragma unroll
  for (int L = 0; L <= R; ++L) M[L] = lv[L][H];
}

template <int R, int BALL, int KIND, int DIL>
__global__ void __launch_bounds__(kSThreads, 4)
    k_morph16s(const __grid_constant__ Morph16Params P, const __grid_constant__ CUtensorMap tmap_deep,
               const __grid_constant__ CUtensorMap tmap_one) {
  using G = SG<R>;
  using O = Op<DIL>;
  constexpr int NDZ = BALL ? R + 1 : 1;
  constexpr int KP = kSKP, NSG = kSNSG, NT = kSThreads;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ int s_abort, s_fixovf;
  __shared__ int s_frow[G::BH], s_fcol[G::BW], s_brow[G::BH], s_bcol[G::BW];
  __shared__ int s_nbr, s_nbc;

  const Job& J = P.job;
  const int tid = threadIdx.x;
  const int tx = blockIdx.x % P.tiles_x, ty = blockIdx.x / P.tiles_x;
  const int64_t cx0 = J.core_lo[2] + (int64_t)tx * kPX;
  const int64_t cy0 = J.core_lo[1] + (int64_t)ty * kPY;
  const int64_t cz0 = J.core_lo[0] + (int64_t)blockIdx.y * P.zchunk;
  const int64_t cz1 = min(cz0 + (int64_t)P.zchunk, J.core_hi[0]);
  if (cz0 >= cz1) return;
  const int nout = (int)(cz1 - cz0);
  const int total = nout + 2 * R;  // input planes cz0-R .. cz1+R-1
  const int ngroups = (total + KP - 1) / KP;
  const int64_t Gz = J.gdims[0], Gy = J.gdims[1], Gx = J.gdims[2];
  const bool face = (cx0 - R < 0) || (cx0 + kPX + R > Gx) || (cy0 - R < 0) || (cy0 + kPY + R > Gy);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
  unsigned char* stages = smem + 128;

  // face patch list: stage row r <-> y = cy0 - R + r, col c <-> x = cx0 - RA + c
  int fix_d[kSFix], fix_s[kSFix];
  int nfix = 0;
  if (face) {
    for (int r = tid; r < G::BH; r += NT) {
      const int64_t sr = reflect(cy0 - R + r, Gy) - (cy0 - R);
      s_frow[r] = (sr >= 0 && sr < G::BH) ? (int)sr : -1;
    }
    for (int c = tid; c < G::BW; c += NT) {
      const int64_t sc = reflect(cx0 - G::RA + c, Gx) - (cx0 - G::RA);
      s_fcol[c] = (sc >= 0 && sc < G::BW) ? (int)sc : -1;
    }
    if (tid == 0) s_fixovf = 0;
    __syncthreads();
    if (tid == 0) {
      int nr = 0, nc = 0;
      for (int r = 0; r < G::BH; ++r)
        if (s_frow[r] != r) s_brow[nr++] = r;
      for (int c = G::RA - R; c < G::RA + kPX + R; ++c)
        if (s_fcol[c] != c) s_bcol[nc++] = c;
      s_nbr = nr;
      s_nbc = nc;
    }
    __syncthreads();
    const int ncell = s_nbr * G::NC + s_nbc * G::BH;
    for (int i = tid; i < ncell; i += NT) {
      int r, c;
      if (i < s_nbr * G::NC) {
        r = s_brow[i / G::NC];
        c = G::RA - R + i % G::NC;
      } else {
        const int k = i - s_nbr * G::NC;
        c = s_bcol[k / G::BH];
        r = k % G::BH;
      }
      const int sr = s_frow[r], sc = s_fcol[c];
      if (sr < 0 || sc < 0) continue;
      if (nfix < kSFix) {
#pragma unroll
        for (int m = 0; m < kSFix; ++m)
          if (m == nfix) {
            fix_d[m] = r * G::BW + c;
            fix_s[m] = sr * G::BW + sc;
          }
        ++nfix;
      } else {
        s_fixovf = 1;
      }
    }
  }
  if (tid == 0) {
    s_abort = 0;
    prefetch_tmap(&tmap_deep);
    prefetch_tmap(&tmap_one);
    for (int b = 0; b < NSG; ++b) mbar_init(&bars[b], 1);
    fence_mbar_init();
  }
  __syncthreads();
  const bool fixovf = face && s_fixovf;

  const int xl = (int)(cx0 - G::RA - J.in.lo[2]);
  const int yl = (int)(cy0 - R - J.in.lo[1]);
  auto issue = [&](int g) {
    uint64_t* bar = &bars[g % NSG];
    unsigned char* dst = stages + (g % NSG) * G::GB;
    const int n0 = g * KP;
    const int nv = min(KP, total - n0);
    const int64_t z0 = cz0 - R + n0;
    if (z0 >= 0 && z0 + nv <= Gz) {
      mbar_arrive_expect_tx(bar, G::GB);
      tma_load_3d(dst, &tmap_deep, xl, yl, (int)(z0 - J.in.lo[0]), bar);
    } else {
      mbar_arrive_expect_tx(bar, nv * G::PB);
      for (int k = 0; k < nv; ++k)
        tma_load_3d(dst + k * G::PB, &tmap_one, xl, yl, (int)(reflect(z0 + k, Gz) - J.in.lo[0]), bar);
    }
  };
  if (tid == 0)
    for (int g = 0; g < min(NSG, ngroups); ++g) issue(g);

  // this thread: pair column xp, output rows ys .. ys + kSS - 1 of the tile
  const int xp = tid % kPC, ys = (tid / kPC) * kSS;
  uint32_t acc[2 * R + 1][kSS];
#pragma unroll
  for (int j = 0; j <= 2 * R; ++j)
#pragma unroll
    for (int i = 0; i < kSS; ++i) acc[j][i] = O::id;
  const DevOut& Ob = J.out;
  const int64_t gx = cx0 + 2 * xp;
  const int64_t pstride = Ob.dims[1] * Ob.dims[2], rstride = Ob.dims[2];
  uint16_t* optr = static_cast<uint16_t*>(Ob.ptr) +
                   ((cz0 - Ob.lo[0]) * Ob.dims[1] + (cy0 + ys - Ob.lo[1])) * Ob.dims[2] + (gx - Ob.lo[2]);
  const bool xok = gx < J.core_hi[2], xpair = gx + 1 < J.core_hi[2];
  const int nrow = xok ? (int)max((int64_t)0, min((int64_t)kSS, J.core_hi[1] - (cy0 + ys))) : 0;
  const bool full = xpair && nrow == kSS;
  // word of this thread's window in a stage row
  const int wofs = G::RA / 2 + xp - G::HP;

  int j = 0;
  for (; j < ngroups; ++j) {
    if (!mbar_wait(&bars[j % NSG], (j / NSG) & 1)) atomicOr(&s_abort, 1);
    unsigned char* sg = stages + (j % NSG) * G::GB;
    const int nv = min(KP, total - j * KP);
    if (face) {
      for (int k = 0; k < nv; ++k) {
        uint16_t* pl = reinterpret_cast<uint16_t*>(sg + k * G::PB);
#pragma unroll
        for (int c = 0; c < kSFix; ++c)
          if (c < nfix) pl[fix_d[c]] = pl[fix_s[c]];
        if (fixovf) {
          int seen = 0;
          const int ncell = s_nbr * G::NC + s_nbc * G::BH;
          for (int i = tid; i < ncell; i += NT) {
            int r, c;
            if (i < s_nbr * G::NC) {
              r = s_brow[i / G::NC];
              c = G::RA - R + i % G::NC;
            } else {
              const int q = i - s_nbr * G::NC;
              c = s_bcol[q / G::BH];
              r = q % G::BH;
            }
            const int sr = s_frow[r], sc = s_fcol[c];
            if (sr < 0 || sc < 0) continue;
            if (seen++ < kSFix) continue;
            pl[r * G::BW + c] = pl[sr * G::BW + sc];
          }
        }
      }
      fence_proxy_async();
      __syncthreads();
    }
#pragma unroll 1
    for (int k = 0; k < nv; ++k) {
      const uint32_t* S = reinterpret_cast<const uint32_t*>(sg + k * G::PB) + ys * G::BWW + wofs;
      // x-line minima of the strip's stage rows; disks of output row i once
      // rows i .. i + 2R are in
      uint32_t Mw[G::NR][R + 1];
      uint32_t D[NDZ][kSS];
#pragma unroll
      for (int rr = 0; rr < G::NR; ++rr) {
        uint32_t w[G::NW];
#pragma unroll
        for (int q = 0; q < G::NW; ++q) w[q] = to_keys<KIND>(S[rr * G::BWW + q]);
        xline1<R, DIL>(w, Mw[rr]);
        if (rr >= 2 * R) {
          const int i = rr - 2 * R;
          // row i + R + dy holds dy
          auto m = [&](int L, int dy) { return Mw[i + R + dy][L]; };
          if constexpr (BALL && R == 3) {
            // line lengths of the r = 3 ball: dz = 1 takes M_2 on dy -2..2;
            // dz = 2 M_2 on -1..1 and M_1 at +-2; dz = 0 M_3 at 0, M_2 on
            // +-1, +-2 and M_0 at +-3 (M_2 at 0 is no smaller than M_3); dz = 3
            // M_0 at 0. The three-row minimum of M_2 is shared.
            const uint32_t a = O::f3(m(2, -1), m(2, 0), m(2, 1));
            const uint32_t d1 = O::f3(a, m(2, -2), m(2, 2));
            D[1][i] = d1;
            D[0][i] = O::f3(d1, m(3, 0), O::f2(m(0, -3), m(0, 3)));
            D[2][i] = O::f3(a, m(1, -2), m(1, 2));
            D[3][i] = m(0, 0);
          } else {
#pragma unroll
            for (int dz = 0; dz < NDZ; ++dz) {
              // extreme of the disk's lines, three operands per instruction
              uint32_t d = O::id, pend = 0u;
              int cnt = 0;
#pragma unroll
              for (int dy = -R; dy <= R; ++dy) {
                const int L = BALL ? line_len(R, dz, dy) : R;
                if (L >= 0) {
                  const uint32_t t = m(L, dy);
                  if (cnt == 0)
                    d = t;
                  else if (cnt & 1)
                    pend = t;
                  else
                    d = O::f3(d, pend, t);
                  ++cnt;
                }
              }
              if (cnt >= 2 && !(cnt & 1)) d = O::f2(d, pend);
              D[dz][i] = d;
            }
          }
        }
      }
      // z ring: plane n = j*KP + k completes output plane cz0 + n - 2R
      uint32_t out[kSS];
#pragma unroll
      for (int i = 0; i < kSS; ++i) {
        out[i] = O::f2(acc[0][i], D[BALL ? R : 0][i]);
#pragma unroll
        for (int jj = 1; jj <= 2 * R; ++jj) {
          const int d = jj > R ? jj - R : R - jj;
          acc[jj - 1][i] = O::f2(acc[jj][i], D[BALL ? d : 0][i]);
        }
        acc[2 * R][i] = O::id;
      }
      const int n = j * KP + k;
      if (n >= 2 * R) {
        uint16_t* o = optr + (int64_t)(n - 2 * R) * pstride;
        if (full) {
          // evict-first: L2 keeps the input rows neighbouring tiles still read
#pragma unroll
          for (int i = 0; i < kSS; ++i)
            __stcs(reinterpret_cast<unsigned int*>(o + i * rstride), (unsigned int)from_keys<KIND>(out[i]));
        } else {
#pragma unroll
          for (int i = 0; i < kSS; ++i) {
            if (i < nrow) {
              const uint32_t v = from_keys<KIND>(out[i]);
              if (xpair)
                *reinterpret_cast<uint32_t*>(o + i * rstride) = v;
              else
                o[i * rstride] = (uint16_t)v;
            }
          }
        }
      }
    }
    __syncthreads();
    if (s_abort) break;
    if (tid == 0 && j + NSG < ngroups) issue(j + NSG);
  }
  if (s_abort) {
    set_device_error(P.err, kErrTimeout);
    if (tid == 0)
      for (int g = j + 1; g < min(j + NSG, ngroups); ++g)
        (void)mbar_wait(&bars[g % NSG], (g / NSG) & 1);
    __syncthreads();
  }
}

template <int R, int BALL, int KIND, int DIL>
cudaError_t launch_s(const Morph16Params& P0, const Job& job, int64_t tiles, int64_t cz,
                     cudaStream_t s) {
  using G = SG<R>;
  static int slots_per_sm = 0;
  if (!slots_per_sm) {
    cudaError_t e = cudaFuncSetAttribute(k_morph16s<R, BALL, KIND, DIL>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM);
    if (e != cudaSuccess) return e;
    int nb = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_morph16s<R, BALL, KIND, DIL>,
                                                      kSThreads, G::SMEM);
    if (e != cudaSuccess) return e;
    slots_per_sm = std::max(1, nb);
  }
  CUtensorMap deep, one;
  memset(&deep, 0, sizeof(deep));
  memset(&one, 0, sizeof(one));
  const int64_t dims[3] = {job.in.dims[2], job.in.dims[1], job.in.dims[0]};
  if (!make_tmap_3d(&deep, job.in.ptr, job.in.dtype, dims, G::BW, G::BHP, kSKP) ||
      !make_tmap_3d(&one, job.in.ptr, job.in.dtype, dims, G::BW, G::BHP, 1))
    return cudaErrorNotSupported;
  Morph16Params P = P0;
  const int64_t slots = (int64_t)slots_per_sm * num_sms();
  P.zchunk = (int)pick_zchunk(cz, tiles, slots, 2 * R + kSKP, kSKP);
  // Over a long chunk, CTAs that started together drift apart in z, until
  // L2 no longer holds the halo rows one of them read for its neighbour
  // (1024^3 ball-3 erosion: 128-plane chunks read 1.56x the input from
  // DRAM, 96-plane chunks 1.40x, 64-plane chunks 1.19x but pay more
  // pipeline fill). Where the grid runs many waves anyway, chunks are cut
  // to about kSDrift planes.
  if (P.zchunk > kSDrift) {
    const int64_t n = (cz + kSDrift - 1) / kSDrift;
    const int64_t zc = ((cz + n - 1) / n + kSKP - 1) / kSKP * kSKP;
    if (tiles * ((cz + zc - 1) / zc) >= 4 * slots) P.zchunk = (int)zc;
  }
  dim3 grid((unsigned)tiles, (unsigned)((cz + P.zchunk - 1) / P.zchunk));
  if (log_level() > 0)
    fprintf(stderr, "[hp] morph16 strip r=%d ball=%d kind=%d dilate=%d grid=%ux%u zchunk=%d slots/SM=%d\n",
            R, BALL, KIND, DIL, grid.x, grid.y, P.zchunk, slots_per_sm);
  k_morph16s<R, BALL, KIND, DIL><<<grid, kSThreads, G::SMEM, s>>>(P, deep, one);
  return cudaGetLastError();
}

template <int KIND, int DIL>
cudaError_t dispatch_s(int ball, int r, const Morph16Params& P, const Job& job, int64_t tiles,
                       int64_t cz, cudaStream_t s) {
  switch (r) {
#define HP_MS(RR)                                                                   \
  case RR:                                                                          \
    return ball ? launch_s<RR, 1, KIND, DIL>(P, job, tiles, cz, s)                  \
                : launch_s<RR, 0, KIND, DIL>(P, job, tiles, cz, s);
    HP_MS(1) HP_MS(2) HP_MS(3)
#undef HP_MS
  }
  return cudaErrorNotSupported;
}

}  // namespace

// Returns cudaErrorNotSupported (nothing enqueued) when the job does not fit
// this kernel: other dtypes, radius > 6, layouts TMA or the paired stores
// cannot take.
cudaError_t launch_morph16(const Job& job, int se, int rad, int is_dilate, cudaStream_t s) {
  const int dt = job.in.dtype;
  if ((dt != HP_U16 && dt != HP_F16) || job.out.dtype != dt) return cudaErrorNotSupported;
  if (rad < 1 || rad > kMaxR16 || job.gdims[2] < rad || job.gdims[1] < rad)
    return cudaErrorNotSupported;
  const int64_t cx = job.core_hi[2] - job.core_lo[2];
  const int64_t cy = job.core_hi[1] - job.core_lo[1];
  const int64_t cz = job.core_hi[0] - job.core_lo[0];
  if (cx <= 0 || cy <= 0 || cz <= 0) return cudaErrorNotSupported;
  // TMA: 16-byte aligned base and row pitch, tile origins on 8-element
  // boundaries; paired stores: 4-byte aligned output pairs.
  if ((uintptr_t)job.in.ptr % 16 || (job.in.dims[2] * 2) % 16 || (job.core_lo[2] - job.in.lo[2]) % 8)
    return cudaErrorNotSupported;
  if ((uintptr_t)job.out.ptr % 4 || job.out.dims[2] % 2 || (job.core_lo[2] - job.out.lo[2]) % 2)
    return cudaErrorNotSupported;
  if (rad <= 3) {
    // strip kernel: no line-minimum buffer in shared memory
    Morph16Params P;
    P.job = job;
    P.tiles_x = (int)((cx + kPX - 1) / kPX);
    P.zchunk = 0;
    P.err = device_error_word();
    const int64_t tiles = (int64_t)P.tiles_x * ((cy + kPY - 1) / kPY);
    const int ball = se == HP_SE_BALL;
    cudaError_t e;
    if (dt == HP_U16)
      e = is_dilate ? dispatch_s<0, 1>(ball, rad, P, job, tiles, cz, s)
                    : dispatch_s<0, 0>(ball, rad, P, job, tiles, cz, s);
    else
      e = is_dilate ? dispatch_s<1, 1>(ball, rad, P, job, tiles, cz, s)
                    : dispatch_s<1, 0>(ball, rad, P, job, tiles, cz, s);
    if (e != cudaErrorNotSupported) return e;
  }
  CUtensorMap map;
  memset(&map, 0, sizeof(map));
  const int64_t dims[3] = {job.in.dims[2], job.in.dims[1], job.in.dims[0]};
  const int ra = rup(rad, 8);
  if (!make_tmap_3d(&map, job.in.ptr, dt, dims, rup(kPX + ra + rad, 8), kPY + 2 * rad))
    return cudaErrorNotSupported;
  Morph16Params P;
  P.job = job;
  P.tiles_x = (int)((cx + kPX - 1) / kPX);
  P.zchunk = 0;
  P.err = device_error_word();
  const int64_t tiles = (int64_t)P.tiles_x * ((cy + kPY - 1) / kPY);
  const int ball = se == HP_SE_BALL;
  if (dt == HP_U16)
    return is_dilate ? dispatch_se<0, 1>(ball, rad, P, map, tiles, cz, s)
                     : dispatch_se<0, 0>(ball, rad, P, map, tiles, cz, s);
  return is_dilate ? dispatch_se<1, 1>(ball, rad, P, map, tiles, cz, s)
                   : dispatch_se<1, 0>(ball, rad, P, map, tiles, cz, s);
}

}  // namespace hp
