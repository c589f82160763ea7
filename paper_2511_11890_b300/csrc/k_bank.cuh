// Multi-sigma derivative-of-Gaussian filter bank: shared work-list types and
// the four-plane z-march kernel (k_bank2).
//
// Per sigma the bank needs seven separable filters that share intermediates
// (Harpia Sec. III-C, Gaussian smoothing and the "Hessian" texture features):
// the x pass applies g0, g1, g2; the y pass forms y0(X0), y0(X1), y1(X0) and
// the Laplacian plane L = y2(X0) + y0(X2); the z pass yields
//   G = z0 y0 x0,  Dz = z1 y0 x0,  Dzz = z2 y0 x0,  Dx = z0 y0 x1,
//   Dy = z0 y1 x0,  Dxx + Dyy = z0 L,
// from which it writes G, GM = sqrt(Dx^2 + Dy^2 + Dz^2) and
// LoG = (Dxx + Dyy) + Dzz.
//
// k_bank2 marches a TX x TY tile column through z four planes per phase:
//   A(g): wait for the TMA group g (one 4-deep box, or four single reflected
//         planes at the z faces); x pass of its planes (all three orders per
//         task, raw input converted in registers) into X; then every block
//         of four output planes whose inputs are all in the ring.
//   B(g): y pass of group g from X into the ring (four planes per input
//         plane: y00, y10, y01, L); thread 0 issues group g + kNSG.
// The 3 x (2R+1) taps of the item's sigma stay in registers for the whole
// item. Every output sums its taps in increasing input coordinate from 0 on
// each axis, so any brick partition gives the whole-volume result bit for
// bit.
#pragma once

#include <cuda_fp16.h>

#include "hp_device.cuh"
#include "hp_internal.h"

namespace hp {

constexpr int kBankMaxGroups = 8;

struct BankItem {
  int group;    // sigma group
  int tile_x0;  // tile origin (global)
  int tile_y0;
  int z0, z1;   // output z range (global)
  int x1, y1;   // exclusive bounds of the brick core in x, y
  int cfg;      // tile configuration (0: 16x16, 1: 32x16)
};

struct BankGroup {
  int r;
  float w[3][2 * kMaxR + 1];  // taps of orders 0, 1, 2
  void* out[3];               // G, GM, LoG (nullptr when not requested)
};

struct BankParams {
  const void* in;  // planes [in_z0, in_z0 + nz) of the volume (whole x/y planes)
  int dtype;
  int out_dtype;
  int64_t G[3];    // global volume (z, y, x)
  int64_t in_z0;   // global z of the input's first plane
  int64_t out_z0;  // global z of the outputs' first plane
  int ngroups;
  BankGroup grp[kBankMaxGroups];
  const BankItem* items;
  int nitems;
  int* counter;
  int* err;
  int use_tma;
};

// TMA maps per sigma group: m (the first kernel's one-plane box, or the
// four-plane kernel's 4-deep box) and m1 (the four-plane kernel's one-plane
// box for reflected z planes).
struct BankMaps {
  CUtensorMap m[kBankMaxGroups];
  CUtensorMap m1[kBankMaxGroups];
};

__device__ __forceinline__ void bank_store(void* base, int dt, int64_t idx, float v) {
  if (dt == HP_F32)
    static_cast<float*>(base)[idx] = v;
  else
    static_cast<__half*>(base)[idx] = __float2half_rn(v);
}

// Kernel entry of the four-plane bank for one input type (uint16, float16,
// float32) and residency (1: all radii, one CTA per SM; 2: r <= 6 on 16 x 16
// tiles, two CTAs per SM); defined in k_bank2_<type>.cu.
const void* bank2_kernel(int dtype, int minb);

namespace b2 {

constexpr int kKP = 4;       // planes per phase (one TMA group)
constexpr int kNSG = 2;      // TMA groups in flight
// Threads per CTA of the one-CTA-per-SM kernel (MINB = 1) and of the
// two-CTAs-per-SM kernel (MINB = 2).
constexpr int kThreads1 = 256;
constexpr int kThreads2 = 256;
__host__ __device__ constexpr int threads_of(int minb) { return minb == 2 ? kThreads2 : kThreads1; }

__host__ __device__ constexpr int rup(int a, int b) { return (a + b - 1) / b * b; }
__host__ __device__ constexpr int gcdi(int a, int b) { return b == 0 ? a : gcdi(b, a % b); }

// Geometry of one (radius, tile, input type) instance; shared by host
// (maps, shared-memory size) and device.
struct Geo {
  int R, TX, TY, ES, AL;
  int RA;    // left margin of the box: R rounded up to a 16-byte word
  int BW;    // box width: an odd number of 16-byte words covering TX + 2 RA
  int BH;    // rows the x pass reads: TY + 2R
  int BHP;   // box height: BH padded so that a plane is a multiple of 128 bytes
  int PB;    // bytes of one staged plane
  int GB;    // bytes of one staged group (kKP planes)
  int XS;    // row stride (floats) of the x-pass output
  int NR;    // ring planes: round_up(2R, 4) + 4
  int PL;    // positions per plane
  int OFF_X, OFF_RING, OFF_TAB, SMEM;
};

__host__ __device__ constexpr Geo geo(int R, int TX, int TY, int ES) {
  Geo g{};
  g.R = R;
  g.TX = TX;
  g.TY = TY;
  g.ES = ES;
  g.AL = 16 / ES;
  g.RA = rup(R, g.AL);
  int words = (TX + 2 * g.RA) / g.AL;
  if (words % 2 == 0) ++words;
  g.BW = words * g.AL;
  g.BH = TY + 2 * R;
  g.BHP = rup(g.BH, 128 / gcdi(g.BW * ES, 128));
  g.PB = g.BW * g.BHP * ES;
  g.GB = kKP * g.PB;
  g.XS = TX + 4;
  g.NR = rup(2 * R, 4) + 4;
  g.PL = TX * TY;
  g.OFF_X = 128 + kNSG * g.GB;
  g.OFF_RING = g.OFF_X + 4 * 3 * kKP * g.BH * g.XS;
  g.OFF_TAB = g.OFF_RING + 4 * 4 * g.NR * g.PL;
  g.SMEM = g.OFF_TAB + 4 * (g.BH + TX + 2 * R);
  return g;
}

// Raw 16-byte word -> 16/ES floats (exact for every input type).
template <typename T>
struct Unpack;
template <>
struct Unpack<uint16_t> {
  static __device__ __forceinline__ void run(const uint4 v, float (&e)[8]) {
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      e[2 * i] = __uint_as_float(__byte_perm(w[i], 0x4B000000u, 0x7410u)) - 8388608.0f;
      e[2 * i + 1] = __uint_as_float(__byte_perm(w[i], 0x4B000000u, 0x7432u)) - 8388608.0f;
    }
  }
};
template <>
struct Unpack<__half> {
  static __device__ __forceinline__ void run(const uint4 v, float (&e)[8]) {
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&w[i]));
      e[2 * i] = f.x;
      e[2 * i + 1] = f.y;
    }
  }
};
template <>
struct Unpack<float> {
  static __device__ __forceinline__ void run(const uint4 v, float (&e)[4]) {
    e[0] = __uint_as_float(v.x);
    e[1] = __uint_as_float(v.y);
    e[2] = __uint_as_float(v.z);
    e[3] = __uint_as_float(v.w);
  }
};

// Taps of the item's sigma, orders 0..2, in registers.
template <int R>
struct Taps3 {
  float w[3][2 * R + 1];
};

// Ring word of tile position (y, x). With 16-column tiles the two half warps
// of a y-pass task write rows 4 apart, which fall on the same banks; flipping
// the half-row of rows with bit 2 of y set puts them on opposite halves, and
// keeps the z pass's reads of 32 consecutive positions conflict-free.
template <int TX>
__device__ __forceinline__ int ring_pos(int y, int x) {
  if constexpr (TX == 16)
    return (y * 16 + x) ^ (((y >> 2) & 1) << 4);
  else
    return y * TX + x;
}

// x pass of one task: 8 outputs of one row of one plane, all three orders.
template <int R, int TX, int TY, typename TIN>
__device__ __forceinline__ void x_task(const unsigned char* plane, int srow, int seg, bool face,
                                       const int* scol, const Taps3<R>& T, float* Xp) {
  constexpr Geo g = geo(R, TX, TY, sizeof(TIN));
  constexpr int NW = 8 + 2 * R;
  const TIN* rowp = reinterpret_cast<const TIN*>(plane) + srow * g.BW;
  float w[NW];
  if (!face) {
    constexpr int D = g.RA - R;
    constexpr int NWORDS = (D + NW + g.AL - 1) / g.AL;
    const uint4* src = reinterpret_cast<const uint4*>(rowp + 8 * seg);
#pragma unroll
    for (int q = 0; q < NWORDS; ++q) {
      float e[g.AL];
      Unpack<TIN>::run(src[q], e);
#pragma unroll
      for (int k = 0; k < g.AL; ++k) {
        const int j = q * g.AL + k - D;
        if (j >= 0 && j < NW) w[j] = e[k];
      }
    }
  } else {
#pragma unroll
    for (int j = 0; j < NW; ++j) w[j] = to_f32<TIN>(rowp[scol[8 * seg + j]]);
  }
  constexpr int XPLANE = kKP * g.BH * g.XS;  // floats between orders
#pragma unroll
  for (int f = 0; f < 3; ++f) {
    float o[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      float acc = 0.0f;
#pragma unroll
      for (int j = i; j <= i + 2 * R; ++j) acc = fmaf(T.w[f][i - j + 2 * R], w[j], acc);
      o[i] = acc;
    }
    float4* dst = reinterpret_cast<float4*>(Xp + f * XPLANE + 8 * seg);
    dst[0] = make_float4(o[0], o[1], o[2], o[3]);
    dst[1] = make_float4(o[4], o[5], o[6], o[7]);
  }
}

// One item: z-march over a TX x TY tile column for one sigma group.
template <int R, int TX, int TY, typename TIN, int NT>
__device__ void run_item2(const BankParams& P, const BankMaps& maps, const BankItem& it,
                          unsigned char* smem, int& gbase, int* s_abort) {
  constexpr Geo g = geo(R, TX, TY, sizeof(TIN));
  const BankGroup& grp = P.grp[it.group];
  const CUtensorMap* md = &maps.m[it.group];
  const CUtensorMap* m1 = &maps.m1[it.group];
  const int tid = threadIdx.x;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
  unsigned char* stg = smem + 128;
  float* X = reinterpret_cast<float*>(smem + g.OFF_X);
  float* ring = reinterpret_cast<float*>(smem + g.OFF_RING);
  int* srow = reinterpret_cast<int*>(smem + g.OFF_TAB);
  int* scol = srow + g.BH;
  const int64_t Gz = P.G[0], Gy = P.G[1], Gx = P.G[2];
  const int cx0 = it.tile_x0, cy0 = it.tile_y0, cz0 = it.z0;
  const int nout = it.z1 - it.z0;
  const int total = nout + 2 * R;
  const int ngr = (total + kKP - 1) / kKP;
  const bool xface = (cx0 - R < 0) || (cx0 + TX + R > Gx);

  // Staged row / column of each reflected input coordinate. Every input a
  // stored output reads reflects into the staged box (the volume is wider
  // than R in x and y); rows and columns that feed only outputs beyond the
  // volume (a ragged last tile, reflected twice) are clamped into the box so
  // that every shared-memory read stays in bounds.
  for (int row = tid; row < g.BH; row += NT) {
    const int64_t sr = reflect(cy0 - R + row, Gy) - (cy0 - R);
    srow[row] = (int)(sr < 0 ? 0 : (sr >= g.BH ? g.BH - 1 : sr));
  }
  for (int c = tid; c < TX + 2 * R; c += NT) {
    const int64_t sc = reflect(cx0 - R + c, Gx) - (cx0 - g.RA);
    scol[c] = (int)(sc < 0 ? 0 : (sc >= g.BW ? g.BW - 1 : sc));
  }
  Taps3<R> T;
#pragma unroll
  for (int f = 0; f < 3; ++f)
#pragma unroll
    for (int k = 0; k <= 2 * R; ++k) T.w[f][k] = grp.w[f][k];

  int issued = 0;
  auto issue = [&](int gi) {
    const int G = gbase + gi, b = G % kNSG;
    unsigned char* dst = stg + b * g.GB;
    const int n0 = kKP * gi;
    const int z0 = cz0 - R + n0;
    if (n0 + kKP <= total && z0 >= 0 && z0 + kKP <= Gz) {
      mbar_arrive_expect_tx(&bars[b], g.GB);
      tma_load_3d(dst, md, cx0 - g.RA, cy0 - R, (int)(z0 - P.in_z0), &bars[b]);
    } else {
      const int cnt = min(kKP, total - n0);
      mbar_arrive_expect_tx(&bars[b], cnt * g.PB);
      for (int p = 0; p < cnt; ++p)
        tma_load_3d(dst + p * g.PB, m1, cx0 - g.RA, cy0 - R, (int)(reflect(z0 + p, Gz) - P.in_z0),
                    &bars[b]);
    }
  };
  __syncthreads();  // tables ready; the previous item's stage reads are done
  if (tid == 0) {
    fence_proxy_async();
    for (; issued < min(kNSG, ngr); ++issued) issue(issued);
  }

  int zb = 0, gi = 0;
  for (; gi <= ngr; ++gi) {
    const int np = min(kKP, total - kKP * gi);
    if (gi < ngr) {
      const int G = gbase + gi, b = G % kNSG;
      if (!mbar_wait(&bars[b], (G / kNSG) & 1)) atomicOr(s_abort, 1);
      const unsigned char* sb = stg + b * g.GB;
      constexpr int NXT = kKP * (TX / 8) * g.BH;
      for (int t = tid; t < NXT; t += NT) {
        const int row = t % g.BH;
        const int rest = t / g.BH;
        const int seg = rest % (TX / 8), pl = rest / (TX / 8);
        if (pl < np)
          x_task<R, TX, TY, TIN>(sb + pl * g.PB, srow[row], seg, xface, scol, T,
                                 X + (pl * g.BH + row) * g.XS);
      }
    }
    // z blocks of four output planes whose inputs are all in the ring
    const int done = min(kKP * gi, total);
    while (zb < nout && done >= min(zb + kKP + 2 * R, total)) {
      const int s0 = zb % g.NR;
      for (int pos = tid; pos < g.PL; pos += NT) {
        const int rpos = ring_pos<TX>(pos / TX, pos % TX);
        float aG[kKP], aDz[kKP], aDzz[kKP], aDx[kKP], aDy[kKP], aL[kKP];
#pragma unroll
        for (int j = 0; j < kKP; ++j) aG[j] = aDz[j] = aDzz[j] = aDx[j] = aDy[j] = aL[j] = 0.0f;
        int slot = s0;
#pragma unroll
        for (int m = 0; m < kKP + 2 * R; ++m) {
          const float* rp = ring + slot * g.PL + rpos;
          const float y00 = rp[0];
          const float y10 = rp[1 * g.NR * g.PL];
          const float y01 = rp[2 * g.NR * g.PL];
          const float yl = rp[3 * g.NR * g.PL];
          slot = slot + 1 == g.NR ? 0 : slot + 1;
#pragma unroll
          for (int j = 0; j < kKP; ++j) {
            if (m >= j && m <= j + 2 * R) {
              const int k = j - m + 2 * R;
              aG[j] = fmaf(T.w[0][k], y00, aG[j]);
              aDz[j] = fmaf(T.w[1][k], y00, aDz[j]);
              aDzz[j] = fmaf(T.w[2][k], y00, aDzz[j]);
              aDx[j] = fmaf(T.w[0][k], y10, aDx[j]);
              aDy[j] = fmaf(T.w[0][k], y01, aDy[j]);
              aL[j] = fmaf(T.w[0][k], yl, aL[j]);
            }
          }
        }
        const int py = pos / TX, px = pos % TX;
        const int64_t gy = cy0 + py, gx = cx0 + px;
        if (gy < it.y1 && gx < it.x1) {
          const int64_t pstride = Gy * Gx;
          int64_t idx = ((int64_t)(cz0 + zb - P.out_z0) * Gy + gy) * Gx + gx;
#pragma unroll
          for (int j = 0; j < kKP; ++j, idx += pstride) {
            if (zb + j >= nout) break;
            if (grp.out[0]) bank_store(grp.out[0], P.out_dtype, idx, aG[j]);
            if (grp.out[1]) {
              const float s2 = fmaf(aDz[j], aDz[j], fmaf(aDy[j], aDy[j], aDx[j] * aDx[j]));
              bank_store(grp.out[1], P.out_dtype, idx, sqrtf(s2));
            }
            if (grp.out[2]) bank_store(grp.out[2], P.out_dtype, idx, aL[j] + aDzz[j]);
          }
        }
      }
      zb += kKP;
    }
    __syncthreads();
    if (*s_abort) break;
    if (gi < ngr) {
      if (tid == 0 && issued < ngr) {
        fence_proxy_async();
        issue(issued);
        ++issued;
      }
      // y pass: four rows of one column of one plane per task
      constexpr int NYT = kKP * TX * (TY / 4);
      constexpr int OS = kKP * g.BH * g.XS;  // floats between x-pass orders
      for (int t = tid; t < NYT; t += NT) {
        const int x = t % TX;
        const int rest = t / TX;
        const int ys = rest % (TY / 4), pl = rest / (TY / 4);
        if (pl >= np) continue;
        const float* x0 = X + (pl * g.BH + 4 * ys) * g.XS + x;
        float a00[4], a01[4], al[4], a10[4];
        {
          float v[4 + 2 * R];
#pragma unroll
          for (int j = 0; j < 4 + 2 * R; ++j) v[j] = x0[j * g.XS];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f;
#pragma unroll
            for (int j = i; j <= i + 2 * R; ++j) {
              s0 = fmaf(T.w[0][i - j + 2 * R], v[j], s0);
              s1 = fmaf(T.w[1][i - j + 2 * R], v[j], s1);
              s2 = fmaf(T.w[2][i - j + 2 * R], v[j], s2);
            }
            a00[i] = s0;
            a01[i] = s1;
            al[i] = s2;
          }
        }
        {
          float v[4 + 2 * R];
#pragma unroll
          for (int j = 0; j < 4 + 2 * R; ++j) v[j] = x0[OS + j * g.XS];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            float s = 0.0f;
#pragma unroll
            for (int j = i; j <= i + 2 * R; ++j) s = fmaf(T.w[0][i - j + 2 * R], v[j], s);
            a10[i] = s;
          }
        }
        {
          float v[4 + 2 * R];
#pragma unroll
          for (int j = 0; j < 4 + 2 * R; ++j) v[j] = x0[2 * OS + j * g.XS];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            float s = al[i];
#pragma unroll
            for (int j = i; j <= i + 2 * R; ++j) s = fmaf(T.w[0][i - j + 2 * R], v[j], s);
            al[i] = s;
          }
        }
        const int slot = (kKP * gi + pl) % g.NR;
        float* rp = ring + slot * g.PL;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int o = ring_pos<TX>(4 * ys + i, x);
          rp[o] = a00[i];
          rp[1 * g.NR * g.PL + o] = a10[i];
          rp[2 * g.NR * g.PL + o] = a01[i];
          rp[3 * g.NR * g.PL + o] = al[i];
        }
      }
    }
    __syncthreads();
  }
  if (*s_abort && tid == 0)  // let the loads in flight land before the CTA exits
    for (int q = gi; q < issued; ++q)
      (void)mbar_wait(&bars[(gbase + q) % kNSG], ((gbase + q) / kNSG) & 1);
  gbase += ngr;
}

template <int TX, int TY, typename TIN, int NT>
__device__ __forceinline__ void dispatch2(int r, const BankParams& P, const BankMaps& maps,
                                          const BankItem& it, unsigned char* smem, int& gb,
                                          int* s_abort) {
  switch (r) {
#define HP_B2(RR) \
  case RR: run_item2<RR, TX, TY, TIN, NT>(P, maps, it, smem, gb, s_abort); break;
    HP_B2(1) HP_B2(2) HP_B2(3) HP_B2(4) HP_B2(5) HP_B2(6)
    HP_B2(7) HP_B2(8) HP_B2(9) HP_B2(10) HP_B2(11) HP_B2(12)
#undef HP_B2
  }
}

template <typename TIN, int NT>
__device__ __forceinline__ void dispatch2_wide(int r, const BankParams& P, const BankMaps& maps,
                                               const BankItem& it, unsigned char* smem, int& gb,
                                               int* s_abort) {
  switch (r) {
#define HP_B2(RR) \
  case RR: run_item2<RR, 32, 16, TIN, NT>(P, maps, it, smem, gb, s_abort); break;
    HP_B2(1) HP_B2(2) HP_B2(3) HP_B2(4) HP_B2(5) HP_B2(6)
#undef HP_B2
  }
}

// Largest radius the 32 x 16 tile takes.
constexpr int kWideMaxR = 6;

// Persistent kernel: CTAs take items from the counter until the list ends.
// MINB = 1: every radius, 16 x 16 or 32 x 16 tiles, one CTA per SM.
// MINB = 2: radii up to kWideMaxR on 16 x 16 tiles only (at most ~113 KB of
// shared memory for 16-bit inputs), two CTAs per SM and at most 128
// registers per thread.
template <typename TIN, int MINB>
__global__ void __launch_bounds__(threads_of(MINB), MINB)
    k_bank2(const __grid_constant__ BankParams P, const __grid_constant__ BankMaps maps) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ int s_item;
  __shared__ int s_abort;
  if (threadIdx.x == 0) {
    s_abort = 0;
    for (int s = 0; s < kNSG; ++s) mbar_init(reinterpret_cast<uint64_t*>(smem) + s, 1);
    fence_mbar_init();
  }
  int gbase = 0;
  while (true) {
    __syncthreads();
    if (threadIdx.x == 0) s_item = atomicAdd(P.counter, 1);
    __syncthreads();
    const int i = s_item;
    if (i >= P.nitems || s_abort) break;
    const BankItem it = P.items[i];
    const int r = P.grp[it.group].r;
    if constexpr (MINB == 1) {
      if (it.cfg == 1)
        dispatch2_wide<TIN, kThreads1>(r, P, maps, it, smem, gbase, &s_abort);
      else
        dispatch2<16, 16, TIN, kThreads1>(r, P, maps, it, smem, gbase, &s_abort);
    } else {
      switch (r) {
#define HP_B2(RR) \
  case RR: run_item2<RR, 16, 16, TIN, kThreads2>(P, maps, it, smem, gbase, &s_abort); break;
        HP_B2(1) HP_B2(2) HP_B2(3) HP_B2(4) HP_B2(5) HP_B2(6)
#undef HP_B2
      }
    }
  }
  if (s_abort && threadIdx.x == 0) set_device_error(P.err, kErrTimeout);
}

}  // namespace b2
}  // namespace hp
