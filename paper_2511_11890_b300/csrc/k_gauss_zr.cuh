// Separable Gaussian / derivative-of-Gaussian filtering (Harpia Sec. III-C)
// over a core box, reflect boundaries on global coordinates (so halo-padded
// bricks of Sec. III-D reproduce the whole volume bit for bit): z-march with
// the z pass held in registers.
//
// A CTA owns a TX x TY column of the core and marches along z, KP input
// planes per pipeline phase and one barrier per phase:
//   stage  one TMA box of KP consecutive planes per phase ((TY+2R) x
//          (TX+2RA) x KP raw input; single-plane loads where the group needs
//          z reflection), NSG-deep mbarrier ring. A CTA's TMA loads complete
//          one after another, so deep boxes are what keeps HBM busy. Tiles at
//          a volume face patch the reflected cells in place one phase ahead
//          of use, from a per-thread list of (cell, source) offsets;
//   P1     x pass on row pairs read straight from the raw stage (element ->
//          FP32 inline), packed f32x2 FMAs over the row pair, into X;
//   P2     y pass on x pairs (packed f32x2 over the two columns), NY (8 or 16) rows
//          per item, into the z feed buffer Zb;
//   Z      each thread owns ZP x pairs of one row and keeps 2R+1 partial
//          outputs per pair in registers: input plane q adds tap i to the
//          output q-2R+i, whose slot is (q+1+i) mod (2R+1); the slot of
//          output q-2R is then complete, stored and cleared. The slot
//          rotation is a switch on q mod (2R+1) over compile-time slot maps.
// Phase j runs P1 on plane group j and Z on group j-1, then (after a
// barrier) P2 on group j; X and Zb are single-buffered (each is written and
// read on opposite sides of a barrier), and the P1 and P2 items of a group
// are spread over all threads.
//
// Every output is accumulated in FP32 with fma, starting from 0, over the
// taps of each axis in increasing input coordinate (x, then y, then z). That
// order does not depend on the tile, chunk or launch shape, so chunked ==
// unchunked exactly.
#pragma once

#include <cuda_fp16.h>

#include <stdio.h>
#include <string.h>

#include <algorithm>

#include "hp_device.cuh"
#include "hp_internal.h"

namespace hp {
namespace zr {


typedef unsigned long long u64;

constexpr int kKP = 4;   // input planes per pipeline phase (= TMA box depth)
constexpr int kNSG = 3;  // plane groups in flight (stage ring depth)
constexpr int kFixC = 4; // face cells a thread patches from its register list

// CTAs started per SM. At radii 5 and 6 (two CTAs per SM) the x-pass items
// of a phase give two of an SM's four schedulers one warp-round more than
// the other two; every other CTA an SM starts shifts its item map by two
// warps, so that two co-resident CTAs load the schedulers in complementary
// ways (warp w issues on scheduler w mod 4).
static __device__ unsigned g_sm_ctas[1024];

struct ZrParams {
  Job job;
  u64 w2[3][2 * kMaxR + 1];  // taps per axis (z, y, x), each as an FP32 pair (w, w)
  int zchunk;
  int tiles_x;
  int* err;
};

__host__ __device__ constexpr int rup(int a, int b) { return (a + b - 1) / b * b; }
__host__ __device__ constexpr int gcd_c(int a, int b) { return b == 0 ? a : gcd_c(b, a % b); }

inline uint32_t f32_bits(float f) {
  uint32_t u;
  memcpy(&u, &f, 4);
  return u;
}

// Tile and thread shape per radius: wide, short tiles for small radii (the x
// pass repeats 2R halo rows; two CTAs of 256 threads per SM, two x pairs of
// z state per thread), square tiles for larger ones (one CTA of 512 threads
// per SM, one x pair per thread). NY rows per y-pass item: 8 spreads the y
// pass over twice the threads (measured at 1024^3: r = 3 and r = 12 3 %
// faster than 16-row items, r = 6 1 % slower; 4-row items slower at all
// three); the per-output sums are the same either way.
template <int R>
struct ZrShape {
  static constexpr int TX = R <= 6 ? 64 : 32;
  static constexpr int TY = R <= 6 ? 16 : 32;
  static constexpr int ZP = R <= 6 ? 2 : 1;
  static constexpr int NT = TX * TY / (2 * ZP);
  static constexpr int NY = (R <= 3 || R >= 7) ? 8 : 16;
  // radii <= 3 (HBM-bound): a two-group stage ring, so that three CTAs fit
  // an SM; larger radii keep three groups in flight
  static constexpr int MINB = NT >= 512 ? 1 : (R <= 3 ? 3 : 2);
  static constexpr int NSG = R <= 3 ? 2 : kNSG;
};

template <int R, typename TIN>
struct ZrGeom {
  using S = ZrShape<R>;
  static constexpr int TX = S::TX, TY = S::TY, ZP = S::ZP, NT = S::NT, NY = S::NY;
  static constexpr int L = 2 * R + 1;
  static constexpr int ES = (int)sizeof(TIN);
  static constexpr int AL = 16 / ES;          // elements per 16 bytes
  static constexpr int RA = rup(R, AL);       // left halo of the raw patch
  // Raw patch width (elements): TX + 2RA, widened until a row is 32 mod 64
  // bytes, so that the x-pass loads of 8 consecutive threads (4 column groups
  // x 2 row pairs, rows 2 apart) fall in 8 distinct 16-byte bank groups.
  static constexpr int bw_pad(int w) { return (w * ES) % 64 == 32 ? w : bw_pad(w + AL); }
  static constexpr int BW = bw_pad(TX + 2 * RA);
  static constexpr int BH = TY + 2 * R;       // raw patch rows used
  // rows loaded: BH rounded up so that stage planes (written by one deep
  // box or by single-plane loads) start on 128-byte boundaries
  static constexpr int BHP = rup(BH, 128 / gcd_c(BW * ES, 128));
  static constexpr int PB = BW * BHP * ES;    // bytes per stage plane (multiple of 128)
  static constexpr int GB = kKP * PB;         // bytes per stage group
  static constexpr int RPN = BH / 2;          // row pairs
  // X holds row pairs: row r at (r/2)*RPS + (r%2)*XS floats. XS keeps rows
  // 16-byte aligned; RPS/4 odd puts the float4 stores of the 8 threads of a
  // quarter warp (4 column groups x 2 row pairs) in 8 distinct bank groups.
  static constexpr int XS = TX + 4;           // row stride within a pair (floats)
  static constexpr int RPS = 2 * XS + ((2 * XS / 4) % 2 == 0 ? 4 : 0);  // row-pair stride
  static constexpr int XP = (BH / 2) * RPS;   // X floats per plane
  static constexpr int ZW = TX / 2;           // x pairs per row
  static constexpr int ZPL = TY * ZW;         // Zb pairs per plane
  static constexpr int NV = (8 + 2 * RA) * ES / 16;  // 16-byte loads per P1 row
  static constexpr int G1 = TX / 8;           // 8-column groups
  static constexpr int GH = G1 / 4;
  static constexpr int NI1 = 8 * GH * ((RPN + 1) / 2);  // P1 slots per plane
  static constexpr int NI2 = ZW * (TY / NY);             // P2 items per plane
  static constexpr int NC = TX + 2 * R;       // raw columns P1 reads
  static constexpr int MI1 = (kKP * NI1 + NT - 1) / NT;  // P1 items per thread and group
  static constexpr int MI2 = (kKP * NI2 + NT - 1) / NT;  // P2 items per thread and group
  static constexpr int NSG = S::NSG;
  static constexpr int SMEM = 128 + NSG * GB + kKP * XP * 4 + kKP * ZPL * 8;
  static_assert(BH % 2 == 0 && TY % NY == 0 && NY % 2 == 0 && G1 % 4 == 0 && NI1 % 8 == 0, "tile shape");
  static_assert((RPS / 4) % 2 == 1 && XS % 4 == 0, "X layout");
  static_assert(PB % 128 == 0, "stage planes on 128-byte boundaries");
  static_assert((8 + 2 * RA) * ES % 16 == 0, "P1 window in whole 16-byte words");
  static_assert(BW <= 256 && BHP <= 256, "TMA box");
  static_assert(SMEM <= 227 * 1024, "shared memory");
};

__device__ __forceinline__ u64 pack2f(float a, float b) {
  u64 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}

__device__ __forceinline__ u64 add2(u64 a, u64 b) {
  u64 d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

// Element e of a window held as 16-byte words -> FP32, for two rows at
// once: returns (row0[e], row1[e]). uint16 uses the exact 2^23 bias (byte
// permute into 0x4B000000 | v, one packed subtract).
template <typename TIN, int NV>
struct PairOf;
template <int NV>
struct PairOf<uint16_t, NV> {
  static __device__ __forceinline__ u64 get(const uint4 (&a)[NV], const uint4 (&b)[NV], int e) {
    const int q = e >> 3, w = (e >> 1) & 3;
    const uint32_t wa = w == 0 ? a[q].x : w == 1 ? a[q].y : w == 2 ? a[q].z : a[q].w;
    const uint32_t wb = w == 0 ? b[q].x : w == 1 ? b[q].y : w == 2 ? b[q].z : b[q].w;
    const uint32_t sel = (e & 1) ? 0x7432u : 0x7410u;
    const float fa = __uint_as_float(__byte_perm(wa, 0x4B000000u, sel));
    const float fb = __uint_as_float(__byte_perm(wb, 0x4B000000u, sel));
    return add2(pack2f(fa, fb), pack2f(-8388608.0f, -8388608.0f));
  }
};
template <int NV>
struct PairOf<__half, NV> {
  static __device__ __forceinline__ u64 get(const uint4 (&a)[NV], const uint4 (&b)[NV], int e) {
    const int q = e >> 3, w = (e >> 1) & 3;
    const uint32_t wa = w == 0 ? a[q].x : w == 1 ? a[q].y : w == 2 ? a[q].z : a[q].w;
    const uint32_t wb = w == 0 ? b[q].x : w == 1 ? b[q].y : w == 2 ? b[q].z : b[q].w;
    const __half2 ha = *reinterpret_cast<const __half2*>(&wa);
    const __half2 hb = *reinterpret_cast<const __half2*>(&wb);
    const float fa = (e & 1) ? __high2float(ha) : __low2float(ha);
    const float fb = (e & 1) ? __high2float(hb) : __low2float(hb);
    return pack2f(fa, fb);
  }
};
template <int NV>
struct PairOf<float, NV> {
  static __device__ __forceinline__ u64 get(const uint4 (&a)[NV], const uint4 (&b)[NV], int e) {
    const int q = e >> 2, w = e & 3;
    const uint32_t wa = w == 0 ? a[q].x : w == 1 ? a[q].y : w == 2 ? a[q].z : a[q].w;
    const uint32_t wb = w == 0 ? b[q].x : w == 1 ? b[q].y : w == 2 ? b[q].z : b[q].w;
    return pack2f(__uint_as_float(wa), __uint_as_float(wb));
  }
};

// One z step for an input plane q with q mod L == K: tap i goes to the
// output q-2R+i in slot (K+1+i) mod L; the output q-2R (slot (K+1) mod L)
// is complete: it is moved to done[] and its slot cleared.
template <int K, int L, int ZP>
__device__ __forceinline__ void zstep(u64 (&acc)[ZP][L], const u64 (&v)[ZP], const ZrParams& P,
                                      u64 (&done)[ZP]) {
#pragma unroll
  for (int i = 0; i < L; ++i) {
    const int s = (K + 1 + i) % L;
#pragma unroll
    for (int zp = 0; zp < ZP; ++zp) acc[zp][s] = ffma2(P.w2[0][i], v[zp], acc[zp][s]);
  }
  constexpr int sd = (K + 1) % L;
#pragma unroll
  for (int zp = 0; zp < ZP; ++zp) {
    done[zp] = acc[zp][sd];
    acc[zp][sd] = 0ull;
  }
}

// Where a z thread stores its completed outputs: ZP x pairs of one row,
// one output plane further per step.
struct ZSink {
  unsigned char* ob;   // output plane oz = 0 of this thread's row and pairs
  int64_t pstride_b;   // bytes between output planes
  int xrem;            // valid columns from the first pair (<= 2*ZP)
  bool zrow, ovec, of32;
};

template <int ZP>
__device__ __forceinline__ void zstore(const ZSink& S, int oz, const u64 (&done)[ZP]) {
  if (oz < 0 || !S.zrow) return;
  unsigned char* dstb = S.ob + (int64_t)oz * S.pstride_b;
  if (S.ovec) {
    if (S.of32) {
      if constexpr (ZP == 2)
        *reinterpret_cast<ulonglong2*>(dstb) = make_ulonglong2(done[0], done[1]);
      else
        *reinterpret_cast<u64*>(dstb) = done[0];
    } else {
#pragma unroll
      for (int zp = 0; zp < ZP; ++zp) {
        const float2 f = unpack2(done[zp]);
        reinterpret_cast<__half2*>(dstb)[zp] = __floats2half2_rn(f.x, f.y);
      }
    }
    return;
  }
#pragma unroll
  for (int zp = 0; zp < ZP; ++zp) {
    const float2 f = unpack2(done[zp]);
    const float fv[2] = {f.x, f.y};
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      if (S.xrem > 2 * zp + e) {
        if (S.of32)
          reinterpret_cast<float*>(dstb)[2 * zp + e] = fv[e];
        else
          reinterpret_cast<__half*>(dstb)[2 * zp + e] = __float2half_rn(fv[e]);
      }
    }
  }
}

// The kKP z steps of one plane group whose first plane q0 has q0 mod L == C:
// plane q0+k takes the compile-time slot map of phase (C+k) mod L. zs points
// at this thread's z input of plane q0; planes are zpl pairs apart.
template <int C, int K, int L, int ZP, int KP>
__device__ __forceinline__ void zgroup_from(u64 (&acc)[ZP][L], const u64* zs, int zpl,
                                           const ZrParams& P, const ZSink& S, int oz0, int nv) {
  if constexpr (K < KP) {
    if (K < nv) {
      u64 v[ZP];
      if constexpr (ZP == 2) {
        const ulonglong2 t = *reinterpret_cast<const ulonglong2*>(zs + K * zpl);
        v[0] = t.x;
        v[1] = t.y;
      } else {
        v[0] = zs[K * zpl];
      }
      u64 done[ZP];
      zstep<(C + K) % L, L, ZP>(acc, v, P, done);
      zstore<ZP>(S, oz0 + K, done);
      zgroup_from<C, K + 1, L, ZP, KP>(acc, zs, zpl, P, S, oz0, nv);
    }
  }
}

// Steady-state group: all kKP planes present, every output complete and
// stored at ob + K * pstride: one FP32 vector where the row allows (vec),
// else one FP32 store per output (rows of an odd number of floats).
template <int C, int L, int ZP, int KP, bool VEC>
__device__ __forceinline__ void zgroup_fast(u64 (&acc)[ZP][L], const u64* zs, int zpl,
                                           const ZrParams& P, unsigned char* ob,
                                           int64_t pstride) {
  static_assert(KP == 4, "four spelled-out slot maps");
#pragma unroll
  for (int K = 0; K < KP; ++K) {
    u64 v[ZP];
    if constexpr (ZP == 2) {
      const ulonglong2 t = *reinterpret_cast<const ulonglong2*>(zs + K * zpl);
      v[0] = t.x;
      v[1] = t.y;
    } else {
      v[0] = zs[K * zpl];
    }
    u64 done[ZP];
    // (C + K) % L for a loop index K: spelled out per K so it stays constant
    if (K == 0) zstep<(C + 0) % L, L, ZP>(acc, v, P, done);
    if (K == 1) zstep<(C + 1) % L, L, ZP>(acc, v, P, done);
    if (K == 2) zstep<(C + 2) % L, L, ZP>(acc, v, P, done);
    if (K == 3) zstep<(C + 3) % L, L, ZP>(acc, v, P, done);
    // evict-first stores: the outputs are not read again here, and L2
    // keeps the input rows that neighbouring tiles still have to read
    unsigned char* d = ob + K * pstride;
    if constexpr (VEC) {
      if constexpr (ZP == 2)
        __stcs(reinterpret_cast<ulonglong2*>(d), make_ulonglong2(done[0], done[1]));
      else
        __stcs(reinterpret_cast<float2*>(d), unpack2(done[0]));
    } else {
#pragma unroll
      for (int zp = 0; zp < ZP; ++zp) {
        const float2 f = unpack2(done[zp]);
        __stcs(reinterpret_cast<float*>(d) + 2 * zp, f.x);
        __stcs(reinterpret_cast<float*>(d) + 2 * zp + 1, f.y);
      }
    }
  }
}

template <int R, typename TIN>
__global__ void __launch_bounds__(ZrShape<R>::NT, ZrShape<R>::MINB)
    k_gauss_zr(const __grid_constant__ ZrParams P, const __grid_constant__ CUtensorMap tmap_deep,
               const __grid_constant__ CUtensorMap tmap_one) {
  using G = ZrGeom<R, TIN>;
  constexpr int NT = G::NT, TX = G::TX, TY = G::TY, ZP = G::ZP, NY = G::NY, L = G::L;
  constexpr int BW = G::BW, BH = G::BH, RA = G::RA, ES = G::ES, XS = G::XS, ZW = G::ZW;
  constexpr int KP = kKP, NSG = G::NSG;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ int s_abort, s_fixovf, s_rot;
  __shared__ int s_frow[BH], s_fcol[BW], s_brow[BH], s_bcol[BW];
  __shared__ int s_nbr, s_nbc;

  const Job& J = P.job;
  const int tid = threadIdx.x;
  const int tx = blockIdx.x % P.tiles_x, ty = blockIdx.x / P.tiles_x;
  const int64_t cx0 = J.core_lo[2] + (int64_t)tx * TX;
  const int64_t cy0 = J.core_lo[1] + (int64_t)ty * TY;
  const int64_t cz0 = J.core_lo[0] + (int64_t)blockIdx.y * P.zchunk;
  const int64_t cz1 = min(cz0 + (int64_t)P.zchunk, J.core_hi[0]);
  if (cz0 >= cz1) return;
  const int nout = (int)(cz1 - cz0);
  const int total = nout + 2 * R;  // input planes cz0-R .. cz1+R-1
  const int ngroups = (total + KP - 1) / KP;
  const int64_t Gz = J.gdims[0], Gy = J.gdims[1], Gx = J.gdims[2];
  const bool face = (cx0 - R < 0) || (cx0 + TX + R > Gx) || (cy0 - R < 0) || (cy0 + TY + R > Gy);

  uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
  unsigned char* stages = smem + 128;
  float* Xb = reinterpret_cast<float*>(stages + NSG * G::GB);
  u64* Zb = reinterpret_cast<u64*>(Xb + KP * G::XP);

  // Face tiles: stage cells outside the volume (TMA zero fill) take the
  // value of their reflected source, which lies inside the volume and the
  // patch. Each thread keeps up to kFixC (cell, source) element offsets.
  int fix_d[kFixC], fix_s[kFixC];
  int nfix = 0;
  if (face) {
    for (int r = tid; r < BH; r += NT) {
      const int64_t s = reflect(cy0 - R + r, Gy) - (cy0 - R);
      s_frow[r] = (s >= 0 && s < BH) ? (int)s : -1;
    }
    for (int c = tid; c < BW; c += NT) {
      const int64_t s = reflect(cx0 - RA + c, Gx) - (cx0 - RA);
      s_fcol[c] = (s >= 0 && s < BW) ? (int)s : -1;
    }
    if (tid == 0) s_fixovf = 0;
    __syncthreads();
    if (tid == 0) {
      int nr = 0, nc = 0;
      for (int r = 0; r < BH; ++r)
        if (s_frow[r] != r) s_brow[nr++] = r;
      for (int c = RA - R; c < RA + TX + R; ++c)
        if (s_fcol[c] != c) s_bcol[nc++] = c;
      s_nbr = nr;
      s_nbc = nc;
    }
    __syncthreads();
    const int ncell = s_nbr * G::NC + s_nbc * BH;
    for (int i = tid; i < ncell; i += NT) {
      int r, c;
      if (i < s_nbr * G::NC) {
        r = s_brow[i / G::NC];
        c = RA - R + i % G::NC;
      } else {
        const int k = i - s_nbr * G::NC;
        c = s_bcol[k / BH];
        r = k % BH;
      }
      const int sr = s_frow[r], sc = s_fcol[c];
      if (sr < 0 || sc < 0) continue;  // no stored output reads this cell
      if (nfix < kFixC) {
#pragma unroll
        for (int m = 0; m < kFixC; ++m)  // constant indices keep the list in registers
          if (m == nfix) {
            fix_d[m] = r * BW + c;
            fix_s[m] = sr * BW + sc;
          }
        ++nfix;
      } else {
        s_fixovf = 1;
      }
    }
  }
  if (tid == 0) {
    s_abort = 0;
    int rot = 0;
    if constexpr (R == 5 || R == 6) {
      unsigned sm;
      asm volatile("mov.u32 %0, %%smid;" : "=r"(sm));
      rot = (atomicAdd(&g_sm_ctas[sm & 1023u], 1u) & 1u) ? 64 : 0;
    }
    s_rot = rot;
    prefetch_tmap(&tmap_deep);
    prefetch_tmap(&tmap_one);
    for (int s = 0; s < NSG; ++s) mbar_init(&bars[s], 1);
    fence_mbar_init();
  }
  __syncthreads();
  const bool fixovf = face && s_fixovf;

  // TMA loads of plane group g: one KP-deep box where its planes need no z
  // reflection, else one load per valid plane.
  const int xl = (int)(cx0 - RA - J.in.lo[2]);
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
  auto wait_group = [&](int g) {
    if (!mbar_wait(&bars[g % NSG], (g / NSG) & 1)) atomicOr(&s_abort, 1);
  };
  auto fix_group = [&](int g) {
    wait_group(g);
    TIN* st = reinterpret_cast<TIN*>(stages + (g % NSG) * G::GB);
    const int nv = min(KP, total - g * KP);
#pragma unroll
    for (int k = 0; k < KP; ++k) {
      if (k < nv) {
        TIN* pl = st + k * (G::PB / ES);
#pragma unroll
        for (int c = 0; c < kFixC; ++c)
          if (c < nfix) pl[fix_d[c]] = pl[fix_s[c]];
      }
    }
    if (fixovf) {  // cells beyond the register lists (tiles covering small volumes)
      for (int k = 0; k < nv; ++k) {
        TIN* pl = st + k * (G::PB / ES);
        int seen = 0;
        const int ncell = s_nbr * G::NC + s_nbc * BH;
        for (int i = tid; i < ncell; i += NT) {
          int r, c;
          if (i < s_nbr * G::NC) {
            r = s_brow[i / G::NC];
            c = RA - R + i % G::NC;
          } else {
            const int q = i - s_nbr * G::NC;
            c = s_bcol[q / BH];
            r = q % BH;
          }
          const int sr = s_frow[r], sc = s_fcol[c];
          if (sr < 0 || sc < 0) continue;
          if (seen++ < kFixC) continue;  // already patched from the register list
          pl[r * BW + c] = pl[sr * BW + sc];
        }
      }
    }
    fence_proxy_async();  // generic writes before the stage's next TMA fill
  };
  if (tid == 0)
    for (int g = 0; g < min(NSG, ngroups); ++g) issue(g);
  if (face) {
    fix_group(0);
    __syncthreads();
  }

  // Z: ZP consecutive x pairs of row zy
  constexpr int ZT = ZW / ZP;  // z threads per row
  const int zxg = tid % ZT, zy = tid / ZT;
  const int64_t gy = cy0 + zy, gx = cx0 + 2 * ZP * zxg;
  const DevOut& O = J.out;
  ZSink S;
  {
    const int64_t xrem64 = J.core_hi[2] - gx;  // valid columns from gx (may be <= 0)
    const int oes = O.dtype == HP_F32 ? 4 : 2;
    S.xrem = xrem64 < 2 * ZP ? (int)xrem64 : 2 * ZP;
    S.zrow = gy < J.core_hi[1];
    S.of32 = O.dtype == HP_F32;
    S.pstride_b = O.dims[1] * O.dims[2] * oes;
    S.ob = static_cast<unsigned char*>(O.ptr) +
           (((cz0 - O.lo[0]) * O.dims[1] + (gy - O.lo[1])) * O.dims[2] + (gx - O.lo[2])) * oes;
    S.ovec = ((reinterpret_cast<uintptr_t>(S.ob) | (uintptr_t)S.pstride_b) &
              (uintptr_t)(2 * ZP * oes - 1)) == 0 && S.xrem == 2 * ZP;
  }

  // Per-thread work items, decoded once. P1 slot -> (row pair rp, 8-column
  // group g): 8 consecutive threads cover 4 groups of 2 row pairs
  // (conflict-free stage loads). P2 item -> (x pair xp, row block b).
  // Offsets: stage bytes and X floats (P1), X floats and Zb pairs (P2);
  // plane index KP marks an empty slot.
  int p1_k[G::MI1], p1_s[G::MI1], p1_x[G::MI1];
  bool p1_any = false;  // the thread reads stages (and so waits for them)
#pragma unroll
  for (int m = 0; m < G::MI1; ++m) {
    const int i1 = (tid + s_rot) % NT + m * NT;  // a permutation of the threads
    const int k = i1 / G::NI1, sl = i1 - k * G::NI1;
    const int g = ((sl >> 3) % G::GH) * 4 + (sl & 3);
    const int rp = ((sl >> 3) / G::GH) * 2 + ((sl >> 2) & 1);
    const bool ok = i1 < KP * G::NI1 && rp < G::RPN;
    p1_any |= ok;
    p1_k[m] = ok ? k : KP;
    p1_s[m] = ok ? k * G::PB + (2 * rp * BW + 8 * g) * ES : 0;
    p1_x[m] = ok ? k * G::XP + rp * G::RPS + 8 * g : 0;
  }
  int p2_k[G::MI2], p2_x[G::MI2], p2_z[G::MI2];
#pragma unroll
  for (int m = 0; m < G::MI2; ++m) {
    const int i2 = tid + m * NT;
    const int k = i2 / G::NI2, t2 = i2 - k * G::NI2;
    const int xp = t2 % ZW, b = t2 / ZW;
    const bool ok = i2 < KP * G::NI2;
    p2_k[m] = ok ? k : KP;
    p2_x[m] = ok ? k * G::XP + (NY * b / 2) * G::RPS + 2 * xp : 0;
    p2_z[m] = ok ? k * G::ZPL + (NY * b) * ZW + xp : 0;
  }
  const bool zfast = S.zrow && S.of32 && S.xrem == 2 * ZP;  // full FP32 outputs
  const u64* zsrc = Zb + zy * ZW + ZP * zxg;

  u64 acc[ZP][L];
#pragma unroll
  for (int zp = 0; zp < ZP; ++zp)
#pragma unroll
    for (int i = 0; i < L; ++i) acc[zp][i] = 0ull;
  int ph = 0;  // index of the next z input plane, mod L

  // Phase j, part 1: P1 (x pass) of group j into X, Z of group j-1 from Zb;
  // part 2 (after a barrier): P2 (y pass) of group j from X into Zb, and the
  // face patch of group j+1. The TMA refill of stage j%NSG is issued at the
  // mid-phase barrier, right after P1 has read it.
  int j = 0;
  for (; j < ngroups + 1; ++j) {
    if (j < ngroups) {
      // P1: x pass of the thread's items of group j
      if (!face && p1_any) wait_group(j);
      const unsigned char* sg = stages + (j % NSG) * G::GB;
      const int nv = min(KP, total - j * KP);
#pragma unroll
      for (int m = 0; m < G::MI1; ++m) {
        if (p1_k[m] >= nv) continue;
        // outputs x = 8g+i (raw column RA+8g+i) of rows 2rp, 2rp+1; window
        // raw columns [8g, 8g + 8 + 2RA)
        const unsigned char* s0 = sg + p1_s[m];
        uint4 a[G::NV], b[G::NV];
#pragma unroll
        for (int q = 0; q < G::NV; ++q) {
          a[q] = reinterpret_cast<const uint4*>(s0)[q];
          b[q] = reinterpret_cast<const uint4*>(s0 + BW * ES)[q];
        }
        u64 o[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) o[i] = 0ull;
#pragma unroll
        for (int e = RA - R; e < RA + 8 + R; ++e) {
          const u64 v = PairOf<TIN, G::NV>::get(a, b, e);
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const int t = R + RA + i - e;  // tap index: input x - output x = e - RA - i
            if (t >= 0 && t <= 2 * R) o[i] = ffma2(P.w2[2][t], v, o[i]);
          }
        }
        float* x0 = Xb + p1_x[m];
        float2 u[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) u[i] = unpack2(o[i]);
        reinterpret_cast<float4*>(x0)[0] = make_float4(u[0].x, u[1].x, u[2].x, u[3].x);
        reinterpret_cast<float4*>(x0)[1] = make_float4(u[4].x, u[5].x, u[6].x, u[7].x);
        reinterpret_cast<float4*>(x0 + XS)[0] = make_float4(u[0].y, u[1].y, u[2].y, u[3].y);
        reinterpret_cast<float4*>(x0 + XS)[1] = make_float4(u[4].y, u[5].y, u[6].y, u[7].y);
      }
    }
    if (j >= 1) {
      // Z: planes of group j-1; one dispatch per group: ph = q0 mod L
      // selects the slot maps of all its planes
      const int q0 = (j - 1) * KP;
      const int nv = min(KP, total - q0);
      const int oz0 = q0 - 2 * R;  // output plane completed by plane q0
      if (zfast && nv == KP && oz0 >= 0) {
        unsigned char* ob = S.ob + (int64_t)oz0 * S.pstride_b;
        if (S.ovec) {
          switch (ph) {
#define HP_ZC(kk)                                                                              \
  case kk:                                                                                     \
    if constexpr (kk < L) zgroup_fast<(kk < L ? kk : 0), L, ZP, KP, true>(acc, zsrc, G::ZPL, P, ob, S.pstride_b); \
    break;
            HP_ZC(0) HP_ZC(1) HP_ZC(2) HP_ZC(3) HP_ZC(4) HP_ZC(5) HP_ZC(6) HP_ZC(7) HP_ZC(8)
            HP_ZC(9) HP_ZC(10) HP_ZC(11) HP_ZC(12) HP_ZC(13) HP_ZC(14) HP_ZC(15) HP_ZC(16)
            HP_ZC(17) HP_ZC(18) HP_ZC(19) HP_ZC(20) HP_ZC(21) HP_ZC(22) HP_ZC(23) HP_ZC(24)
#undef HP_ZC
            default: break;
          }
        } else {
          switch (ph) {
#define HP_ZC(kk)                                                                              \
  case kk:                                                                                     \
    if constexpr (kk < L) zgroup_fast<(kk < L ? kk : 0), L, ZP, KP, false>(acc, zsrc, G::ZPL, P, ob, S.pstride_b); \
    break;
            HP_ZC(0) HP_ZC(1) HP_ZC(2) HP_ZC(3) HP_ZC(4) HP_ZC(5) HP_ZC(6) HP_ZC(7) HP_ZC(8)
            HP_ZC(9) HP_ZC(10) HP_ZC(11) HP_ZC(12) HP_ZC(13) HP_ZC(14) HP_ZC(15) HP_ZC(16)
            HP_ZC(17) HP_ZC(18) HP_ZC(19) HP_ZC(20) HP_ZC(21) HP_ZC(22) HP_ZC(23) HP_ZC(24)
#undef HP_ZC
            default: break;
          }
        }
      } else {
        switch (ph) {
#define HP_ZC(kk)                                                                       \
  case kk:                                                                              \
    if constexpr (kk < L) zgroup_from<(kk < L ? kk : 0), 0, L, ZP, KP>(acc, zsrc, G::ZPL, P, S, oz0, nv); \
    break;
          HP_ZC(0) HP_ZC(1) HP_ZC(2) HP_ZC(3) HP_ZC(4) HP_ZC(5) HP_ZC(6) HP_ZC(7) HP_ZC(8)
          HP_ZC(9) HP_ZC(10) HP_ZC(11) HP_ZC(12) HP_ZC(13) HP_ZC(14) HP_ZC(15) HP_ZC(16)
          HP_ZC(17) HP_ZC(18) HP_ZC(19) HP_ZC(20) HP_ZC(21) HP_ZC(22) HP_ZC(23) HP_ZC(24)
#undef HP_ZC
          default: break;
        }
      }
      ph = (ph + KP) % L;
    }
    __syncthreads();
    if (s_abort) break;
    if (tid == 0 && j + NSG < ngroups) issue(j + NSG);
    if (j < ngroups) {
      // P2: y pass of the thread's items of group j
      const int nv = min(KP, total - j * KP);
#pragma unroll
      for (int m = 0; m < G::MI2; ++m) {
        if (p2_k[m] >= nv) continue;
        // rows NY*b .. NY*b+NY-1 of x pair xp; X row j' <-> y - R
        const float* xs = Xb + p2_x[m];
        u64 o[NY];
#pragma unroll
        for (int i = 0; i < NY; ++i) o[i] = 0ull;
#pragma unroll
        for (int jj = 0; jj < NY + 2 * R; ++jj) {
          // X row NY*b + jj (NY even: the pair parity is that of jj)
          const u64 v = *reinterpret_cast<const u64*>(xs + (jj >> 1) * G::RPS + (jj & 1) * XS);
#pragma unroll
          for (int i = 0; i < NY; ++i) {
            const int t = 2 * R + i - jj;
            if (t >= 0 && t <= 2 * R) o[i] = ffma2(P.w2[1][t], v, o[i]);
          }
        }
        u64* zd = Zb + p2_z[m];
#pragma unroll
        for (int i = 0; i < NY; ++i) zd[i * ZW] = o[i];
      }
    }
    if (face && j + 1 < ngroups) fix_group(j + 1);
    __syncthreads();
  }
  if (s_abort) {
    set_device_error(P.err, kErrTimeout);
    // drain TMA loads still in flight into this CTA's shared memory
    if (tid == 0)
      for (int g = j + 1; g < min(j + NSG, ngroups); ++g)
        (void)mbar_wait(&bars[g % NSG], (g / NSG) & 1);
    __syncthreads();
  }
}

template <int R, typename TIN>
cudaError_t launch_zr_t(const ZrParams& P0, const Job& job, cudaStream_t s) {
  using G = ZrGeom<R, TIN>;
  static int occ = 0;  // resident CTAs per SM, per instantiation
  if (!occ) {
    cudaError_t e = cudaFuncSetAttribute(k_gauss_zr<R, TIN>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM);
    if (e != cudaSuccess) return e;
    int n = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_gauss_zr<R, TIN>, G::NT, G::SMEM);
    if (e != cudaSuccess) return e;
    occ = std::max(1, n);
  }
  CUtensorMap deep, one;
  memset(&deep, 0, sizeof(deep));
  memset(&one, 0, sizeof(one));
  const int64_t dims[3] = {job.in.dims[2], job.in.dims[1], job.in.dims[0]};
  if (!make_tmap_3d(&deep, job.in.ptr, job.in.dtype, dims, G::BW, G::BHP, kKP) ||
      !make_tmap_3d(&one, job.in.ptr, job.in.dtype, dims, G::BW, G::BHP, 1))
    return cudaErrorNotSupported;
  ZrParams P = P0;
  const int64_t cx = job.core_hi[2] - job.core_lo[2];
  const int64_t cy = job.core_hi[1] - job.core_lo[1];
  const int64_t cz = job.core_hi[0] - job.core_lo[0];
  P.tiles_x = (int)((cx + G::TX - 1) / G::TX);
  const int64_t tiles = (int64_t)P.tiles_x * ((cy + G::TY - 1) / G::TY);
  // z chunks in whole plane groups (the halo is 2R planes plus the two
  // pipeline phases)
  P.zchunk = (int)pick_zchunk(cz, tiles, (int64_t)num_sms() * occ, 2 * R + 2 * kKP, kKP);
  dim3 grid((unsigned)tiles, (unsigned)((cz + P.zchunk - 1) / P.zchunk));
  if (log_level() > 0)
    fprintf(stderr, "[hp] gauss zr r=%d tile=%dx%d threads=%d occ=%d grid=%ux%u zchunk=%d\n", R,
            G::TX, G::TY, G::NT, occ, grid.x, grid.y, P.zchunk);
  k_gauss_zr<R, TIN><<<grid, G::NT, G::SMEM, s>>>(P, deep, one);
  return cudaGetLastError();
}

template <typename TIN>
cudaError_t dispatch_zr_t(int r, const ZrParams& P, const Job& job, cudaStream_t s) {
  switch (r) {
#define HP_CASE(RR) \
  case RR: return launch_zr_t<RR, TIN>(P, job, s);
    HP_CASE(1) HP_CASE(2) HP_CASE(3) HP_CASE(4) HP_CASE(5) HP_CASE(6)
    HP_CASE(7) HP_CASE(8) HP_CASE(9) HP_CASE(10) HP_CASE(11) HP_CASE(12)
#undef HP_CASE
    default: return cudaErrorNotSupported;
  }
}

// One instantiation set per input element type (k_gauss_zr_<type>.cu).
cudaError_t dispatch_u16(int r, const ZrParams& P, const Job& job, cudaStream_t s);
cudaError_t dispatch_f16(int r, const ZrParams& P, const Job& job, cudaStream_t s);
cudaError_t dispatch_f32(int r, const ZrParams& P, const Job& job, cudaStream_t s);

}  // namespace zr
}  // namespace hp
