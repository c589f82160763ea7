// Multi-sigma derivative-of-Gaussian filter bank (Harpia Sec. III-C:
// Gaussian smoothing and "Hessian" texture features) in one persistent
// launch: work list, autotuner, CUDA graph, and the single-plane kernel
// k_bank for inputs the four-plane kernel (k_bank2, k_bank.cuh) does not
// take (rows or brick origins TMA cannot address, uint8, volumes not wider
// than the largest radius in x or y).
//
// Per sigma the bank needs seven separable filters that share
// intermediates: the x pass applies g0, g1, g2 (3 planes), the y pass forms
// y0(X0), y0(X1), y1(X0), y0(X2), y2(X0) (5 ring planes), and the z pass
// yields G = z0 y0 x0, Dz = z1 y0 x0, Dzz = z2 y0 x0, Dx = z0 y0 x1,
// Dy = z0 y1 x0, Dxx = z0 y0 x2, Dyy = z0 y2 x0, from which it writes
// G, GM = sqrt(Dx^2 + Dy^2 + Dz^2) and LoG = Dxx + Dyy + Dzz.
//
// The work list holds (sigma group, tile, z range) items over a set of
// bricks; persistent CTAs take items from an atomic counter, heaviest sigma
// first. Halos come from the whole device volume, so any brick set gives the
// whole-volume result bit for bit. The single-plane kernel is the z-march of
// the Gaussian kernel (plane loads, one barrier per plane) widened to 3/5/7
// planes; tile shape and z-chunk length come from the autotuner.
#include <cuda_fp16.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <map>
#include <memory>
#include <string>
#include <mutex>
#include <tuple>
#include <vector>

#include "hp_device.cuh"
#include "hp_internal.h"
#include "k_bank.cuh"

namespace hp {

namespace {

constexpr int kThreads = 256;
constexpr int kNS = 4;
constexpr int kMaxGroups = kBankMaxGroups;
constexpr int kBZ = 8;

__host__ __device__ constexpr int round_up(int a, int b) { return (a + b - 1) / b * b; }
__host__ __device__ constexpr int patch_stride(int n) {
  int f = n;
  while (f % 8 != 4) ++f;
  return f;
}

template <int R, int TX, int TY>
struct BGeom {
  static constexpr int R4 = round_up(R, 4);
  static constexpr int WL = round_up(R4 + R + 8, 4);
  static constexpr int FWN = (TX - 8) + WL;
  static constexpr int FW = patch_stride(FWN);
  static constexpr int BH = TY + 2 * R;
  static constexpr int NC = (FWN + 31) / 32;
  static constexpr int XS = TX + 4;
  static constexpr int NRING = kBZ + 2 * R;
  static constexpr int FSZ = BH * FW;
  static constexpr int XSZ = BH * XS;
  static constexpr int PL = TX * TY;  // positions per plane
  static constexpr int TAIL = (2 * FSZ + 2 * 3 * XSZ + 5 * NRING * PL) * 4 + BH * 4;
  static_assert(FWN % 4 == 0, "patch width must be a multiple of 4");
};

__host__ __device__ inline void bbox_geom(int r, int tx, int es, int* ra, int* bw) {
  const int al = 16 / es;
  *ra = round_up(r, al);
  *bw = round_up(tx + *ra + r, al);
}

__host__ __device__ inline int bstage_bytes(int r, int tx, int ty, int es) {
  int ra, bw;
  bbox_geom(r, tx, es, &ra, &bw);
  return round_up(bw * (ty + 2 * r) * es, 128);
}

template <int R, int TX, int TY>
__host__ __device__ inline int item_smem(int es) {
  return 128 + kNS * bstage_bytes(R, TX, TY, es) + BGeom<R, TX, TY>::TAIL;
}

__device__ __forceinline__ void store_val(void* base, int dt, int64_t idx, float v) {
  if (dt == HP_F32)
    static_cast<float*>(base)[idx] = v;
  else
    static_cast<__half*>(base)[idx] = __float2half_rn(v);
}

// One item: z-march over a TX x TY tile column for sigma group g.
template <int R, int TX, int TY>
__device__ void run_item(const BankParams& P, const CUtensorMap* tmap, const BankItem& it,
                         unsigned char* smem, int& phase_base, int* s_abort) {
  using Gm = BGeom<R, TX, TY>;
  const BankGroup& grp = P.grp[it.group];
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const int64_t cx0 = it.tile_x0, cy0 = it.tile_y0, cz0 = it.z0;
  const int nout = it.z1 - it.z0;
  const int total = nout + 2 * R;
  const int64_t Gz = P.G[0], Gy = P.G[1], Gx = P.G[2];
  const int dt = P.dtype;
  const int es = dt == HP_U8 ? 1 : (dt == HP_F32 ? 4 : 2);
  int ra, bw;
  bbox_geom(R, TX, es, &ra, &bw);
  const int sbytes = bstage_bytes(R, TX, TY, es);
  const bool tma = P.use_tma != 0;
  const bool face = (cx0 - R < 0) || (cx0 + TX + R > Gx) || (cy0 - R < 0) || (cy0 + TY + R > Gy);

  uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
  unsigned char* stages = smem + 128;
  float* F = reinterpret_cast<float*>(stages + kNS * sbytes);
  float* X = F + 2 * Gm::FSZ;                 // [2][3][XSZ]
  float* ring = X + 2 * 3 * Gm::XSZ;          // [5][NRING][PL]
  int* srow = reinterpret_cast<int*>(ring + 5 * Gm::NRING * Gm::PL);

  for (int row = tid; row < Gm::BH; row += kThreads) {
    const int64_t sy = reflect(cy0 - R + row, Gy);
    const int64_t s = tma ? sy - (cy0 - R) : sy;
    srow[row] = (s >= 0 && s < (tma ? Gm::BH : Gy)) ? (int)s : -1;
  }
  int scol[Gm::NC];
#pragma unroll
  for (int k = 0; k < Gm::NC; ++k) {
    const int col = lane + 32 * k;
    const int64_t sx = reflect(cx0 - Gm::R4 + col, Gx);
    const int64_t s = tma ? sx - (cx0 - ra) : sx;
    scol[k] = (col < Gm::FWN && s >= 0 && s < (tma ? bw : Gx)) ? (int)s : -1;
  }
  // barrier phases continue across items: plane n uses barrier (base+n)%kNS
  const int base = phase_base;
  auto issue = [&](int n) {
    const int b = (base + n) % kNS;
    const int zl = (int)(reflect(cz0 - R + n, Gz) - P.in_z0);
    uint64_t* bar = &bars[b];
    mbar_arrive_expect_tx(bar, bw * Gm::BH * es);
    tma_load_3d(stages + b * sbytes, tmap, (int)(cx0 - ra), (int)(cy0 - R), zl, bar);
  };
  __syncthreads();  // tables ready, previous item's buffers free
  if (tma && tid == 0) {
    fence_proxy_async();
    for (int n = 0; n < min(kNS, total); ++n) issue(n);
  }

  int zb = 0, p = 0;
  for (; p < total + 2; ++p) {
    if (p < total) {
      float* Fb = F + (p & 1) * Gm::FSZ;
      if (tma) {
        const int b = (base + p) % kNS;
        if (!mbar_wait(&bars[b], ((base + p) / kNS) & 1)) atomicOr(s_abort, 1);
        const unsigned char* rawb = stages + b * sbytes;
        if (!face) {
          constexpr int Q = Gm::FWN / 4;
          for (int i = tid; i < Gm::BH * Q; i += kThreads) {
            const int row = i / Q, q = i - row * Q;
            float4 v;
            switch (dt) {
              case HP_U8: v = load4_f32<uint8_t>(reinterpret_cast<const uint8_t*>(rawb) + (ra - Gm::R4) + row * bw + 4 * q); break;
              case HP_U16: v = load4_f32<uint16_t>(reinterpret_cast<const uint16_t*>(rawb) + (ra - Gm::R4) + row * bw + 4 * q); break;
              case HP_F16: v = load4_f32<__half>(reinterpret_cast<const __half*>(rawb) + (ra - Gm::R4) + row * bw + 4 * q); break;
              default: v = load4_f32<float>(reinterpret_cast<const float*>(rawb) + (ra - Gm::R4) + row * bw + 4 * q); break;
            }
            *reinterpret_cast<float4*>(Fb + row * Gm::FW + 4 * q) = v;
          }
        } else {
          for (int row = warp; row < Gm::BH; row += kThreads / 32) {
            const int sr = srow[row];
#pragma unroll
            for (int k = 0; k < Gm::NC; ++k) {
              const int col = lane + 32 * k;
              if (col < Gm::FWN) {
                const int sc = scol[k];
                float v = 0.0f;
                if (sr >= 0 && sc >= 0) {
                  const int e = sr * bw + sc;
                  switch (dt) {
                    case HP_U8: v = to_f32<uint8_t>(reinterpret_cast<const uint8_t*>(rawb)[e]); break;
                    case HP_U16: v = to_f32<uint16_t>(reinterpret_cast<const uint16_t*>(rawb)[e]); break;
                    case HP_F16: v = to_f32<__half>(reinterpret_cast<const __half*>(rawb)[e]); break;
                    default: v = reinterpret_cast<const float*>(rawb)[e]; break;
                  }
                }
                Fb[row * Gm::FW + col] = v;
              }
            }
          }
        }
      } else {
        const int64_t sz = reflect(cz0 - R + p, Gz);
        for (int row = warp; row < Gm::BH; row += kThreads / 32) {
          const int sr = srow[row];
#pragma unroll
          for (int k = 0; k < Gm::NC; ++k) {
            const int col = lane + 32 * k;
            if (col < Gm::FWN) {
              const int sc = scol[k];
              float v = 0.0f;
              if (sr >= 0 && sc >= 0) {
                const int64_t e = ((sz - P.in_z0) * Gy + sr) * Gx + sc;
                switch (dt) {
                  case HP_U8: v = to_f32<uint8_t>(static_cast<const uint8_t*>(P.in)[e]); break;
                  case HP_U16: v = to_f32<uint16_t>(static_cast<const uint16_t*>(P.in)[e]); break;
                  case HP_F16: v = to_f32<__half>(static_cast<const __half*>(P.in)[e]); break;
                  default: v = static_cast<const float*>(P.in)[e]; break;
                }
              }
              Fb[row * Gm::FW + col] = v;
            }
          }
        }
      }
    }
    if (p >= 1 && p - 1 < total) {
      // x pass: three orders, 8 outputs per task
      const float* Fb = F + ((p - 1) & 1) * Gm::FSZ;
      float* Xb = X + ((p - 1) & 1) * 3 * Gm::XSZ;
      constexpr int NT = 3 * Gm::BH * (TX / 8);
      for (int t = tid; t < NT; t += kThreads) {
        const int f = t / (Gm::BH * (TX / 8));
        const int rr = t - f * (Gm::BH * (TX / 8));
        const int row = rr / (TX / 8), xg = (rr % (TX / 8)) * 8;
        float w[Gm::WL];
        const float4* src = reinterpret_cast<const float4*>(Fb + row * Gm::FW + xg);
#pragma unroll
        for (int j = 0; j < Gm::WL / 4; ++j) {
          const float4 v = src[j];
          w[4 * j] = v.x;
          w[4 * j + 1] = v.y;
          w[4 * j + 2] = v.z;
          w[4 * j + 3] = v.w;
        }
        const float* wx = grp.w[f];
        float o[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          float acc = 0.0f;
#pragma unroll
          for (int j = i + Gm::R4 - R; j <= i + Gm::R4 + R; ++j)
            acc = fmaf(wx[i + Gm::R4 - j + R], w[j], acc);
          o[i] = acc;
        }
        float4* dst = reinterpret_cast<float4*>(Xb + f * Gm::XSZ + row * Gm::XS + xg);
        dst[0] = make_float4(o[0], o[1], o[2], o[3]);
        dst[1] = make_float4(o[4], o[5], o[6], o[7]);
      }
    }
    if (p >= 2) {
      // y pass: five combinations, 4 rows per task
      const float* Xb = X + ((p - 2) & 1) * 3 * Gm::XSZ;
      const int slot = (p - 2) % Gm::NRING;
      constexpr int NT = 5 * TX * (TY / 4);
      for (int t = tid; t < NT; t += kThreads) {
        const int c = t / (TX * (TY / 4));
        const int rr = t - c * (TX * (TY / 4));
        const int x = rr % TX, yb = (rr / TX) * 4;
        // c: 0 y0(X0), 1 y0(X1), 2 y1(X0), 3 y0(X2), 4 y2(X0)
        const int xs = c == 1 ? 1 : (c == 3 ? 2 : 0);
        const int yo = c == 2 ? 1 : (c == 4 ? 2 : 0);
        const float* src = Xb + xs * Gm::XSZ;
        const float* wy = grp.w[yo];
        float w[4 + 2 * R];
#pragma unroll
        for (int j = 0; j < 4 + 2 * R; ++j) w[j] = src[(yb + j) * Gm::XS + x];
        float* dst = ring + (c * Gm::NRING + slot) * Gm::PL;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          float acc = 0.0f;
#pragma unroll
          for (int j = i; j <= i + 2 * R; ++j) acc = fmaf(wy[i - j + 2 * R], w[j], acc);
          dst[(yb + i) * TX + x] = acc;
        }
      }
    }
    __syncthreads();
    if (*s_abort) break;
    if (tma && tid == 0 && p + kNS < total) {
      fence_proxy_async();
      issue(p + kNS);
    }
    const int done = min(p - 1, total);
    while (zb < nout && done >= min(zb + kBZ + 2 * R, total)) {
      for (int pos = tid; pos < Gm::PL; pos += kThreads) {
        float a[7][kBZ];
#pragma unroll
        for (int q = 0; q < 7; ++q)
#pragma unroll
          for (int j = 0; j < kBZ; ++j) a[q][j] = 0.0f;
        int slot = zb % Gm::NRING;
#pragma unroll
        for (int m = 0; m < kBZ + 2 * R; ++m) {
          const float y00 = ring[(0 * Gm::NRING + slot) * Gm::PL + pos];
          const float y10 = ring[(1 * Gm::NRING + slot) * Gm::PL + pos];
          const float y01 = ring[(2 * Gm::NRING + slot) * Gm::PL + pos];
          const float y20 = ring[(3 * Gm::NRING + slot) * Gm::PL + pos];
          const float y02 = ring[(4 * Gm::NRING + slot) * Gm::PL + pos];
          slot = slot + 1 == Gm::NRING ? 0 : slot + 1;
#pragma unroll
          for (int j = 0; j < kBZ; ++j) {
            if (m >= j && m <= j + 2 * R) {
              const int k = j - m + 2 * R;
              a[0][j] = fmaf(grp.w[0][k], y00, a[0][j]);  // G
              a[1][j] = fmaf(grp.w[1][k], y00, a[1][j]);  // Dz
              a[2][j] = fmaf(grp.w[2][k], y00, a[2][j]);  // Dzz
              a[3][j] = fmaf(grp.w[0][k], y10, a[3][j]);  // Dx
              a[4][j] = fmaf(grp.w[0][k], y01, a[4][j]);  // Dy
              a[5][j] = fmaf(grp.w[0][k], y20, a[5][j]);  // Dxx
              a[6][j] = fmaf(grp.w[0][k], y02, a[6][j]);  // Dyy
            }
          }
        }
        const int py = pos / TX, px = pos % TX;
        const int64_t gy = cy0 + py, gx = cx0 + px;
        if (gy < it.y1 && gx < it.x1) {
          const int64_t pstride = Gy * Gx;
          int64_t idx = ((cz0 + zb - P.out_z0) * Gy + gy) * Gx + gx;
#pragma unroll
          for (int j = 0; j < kBZ; ++j, idx += pstride) {
            if (zb + j >= nout) break;
            if (grp.out[0]) store_val(grp.out[0], P.out_dtype, idx, a[0][j]);
            if (grp.out[1]) {
              const float s2 = fmaf(a[1][j], a[1][j], fmaf(a[4][j], a[4][j], a[3][j] * a[3][j]));
              store_val(grp.out[1], P.out_dtype, idx, sqrtf(s2));
            }
            if (grp.out[2]) store_val(grp.out[2], P.out_dtype, idx, (a[5][j] + a[6][j]) + a[2][j]);
          }
        }
      }
      zb += kBZ;
      __syncthreads();
    }
  }
  if (*s_abort && tma && tid == 0)
    for (int n = p; n < min(p + kNS, total); ++n)
      (void)mbar_wait(&bars[(base + n) % kNS], ((base + n) / kNS) & 1);
  phase_base = base + total;
}

template <int TX, int TY>
__device__ __forceinline__ void dispatch_item(int r, const BankParams& P, const CUtensorMap* tmap,
                                              const BankItem& it, unsigned char* smem, int& pb,
                                              int* s_abort) {
  switch (r) {
#define HP_BI(RR) \
  case RR: run_item<RR, TX, TY>(P, tmap, it, smem, pb, s_abort); break;
    HP_BI(1) HP_BI(2) HP_BI(3) HP_BI(4) HP_BI(5) HP_BI(6)
    HP_BI(7) HP_BI(8) HP_BI(9) HP_BI(10) HP_BI(11) HP_BI(12)
#undef HP_BI
  }
}

template <int TX, int TY>
__device__ __forceinline__ void dispatch_item_small(int r, const BankParams& P,
                                                    const CUtensorMap* tmap, const BankItem& it,
                                                    unsigned char* smem, int& pb, int* s_abort) {
  switch (r) {
    case 1: run_item<1, TX, TY>(P, tmap, it, smem, pb, s_abort); break;
    case 2: run_item<2, TX, TY>(P, tmap, it, smem, pb, s_abort); break;
    case 3: run_item<3, TX, TY>(P, tmap, it, smem, pb, s_abort); break;
    case 4: run_item<4, TX, TY>(P, tmap, it, smem, pb, s_abort); break;
  }
}

// Persistent kernel: CTAs take items from the counter until the list ends.
__global__ void __launch_bounds__(kThreads, 1)
    k_bank(const __grid_constant__ BankParams P, const __grid_constant__ BankMaps maps) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ int s_item;
  __shared__ int s_abort;
  if (threadIdx.x == 0) {
    s_abort = 0;
    if (P.use_tma) {
      for (int s = 0; s < kNS; ++s) mbar_init(reinterpret_cast<uint64_t*>(smem) + s, 1);
      fence_mbar_init();
    }
  }
  int phase_base = 0;
  while (true) {
    __syncthreads();
    if (threadIdx.x == 0) s_item = atomicAdd(P.counter, 1);
    __syncthreads();
    const int i = s_item;
    if (i >= P.nitems || s_abort) break;
    const BankItem it = P.items[i];
    const int r = P.grp[it.group].r;
    const CUtensorMap* tm = &maps.m[it.group];
    if (it.cfg == 1)
      dispatch_item_small<32, 16>(r, P, tm, it, smem, phase_base, &s_abort);
    else
      dispatch_item<16, 16>(r, P, tm, it, smem, phase_base, &s_abort);
  }
  if (s_abort && threadIdx.x == 0) set_device_error(P.err, kErrTimeout);
}

template <int TX, int TY>
int max_item_smem(int r, int es) {
  switch (r) {
#define HP_MS(RR) \
  case RR: return item_smem<RR, TX, TY>(es);
    HP_MS(1) HP_MS(2) HP_MS(3) HP_MS(4) HP_MS(5) HP_MS(6)
    HP_MS(7) HP_MS(8) HP_MS(9) HP_MS(10) HP_MS(11) HP_MS(12)
#undef HP_MS
  }
  return 0;
}

int cfg_smem(int cfg, int r, int es) {
  return cfg == 1 ? max_item_smem<32, 16>(r, es) : max_item_smem<16, 16>(r, es);
}

}  // namespace

// ----------------------------------------------------------------- host side

// Tuning knobs picked by the autotuner: tile configuration for small radii
// and z-chunk length.
struct BankTune {
  // 0: 16x16 tiles for all radii; 1: 32x16 tiles for small radii (r <= 4 on
  // the single-plane kernel, r <= 6 where it fits on the four-plane kernel);
  // 2: four-plane kernel only: radii <= 6 in a second launch of 16x16 tiles
  // at two CTAs per SM, beside the one-CTA-per-SM launch of the rest.
  int small_cfg;
  int zchunk;
};

struct BankPlan {
  BankParams P;
  BankItem* d_items = nullptr;
  int* d_counter = nullptr;  // [2]: one per launch
  bool owns = true;          // false: work list in caller memory, no graph
  BankMaps maps;
  int smem = 0;
  int grid = 0;
  int threads = 0;
  const void* kernel = nullptr;
  // second launch (small radii at two CTAs per SM), when split
  BankParams P2;
  int smem2 = 0;
  int grid2 = 0;
  const void* kernel2 = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  size_t bytes = 0;
  ~BankPlan() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (owns && d_items) cudaFree(d_items);
    if (owns && d_counter) cudaFree(d_counter);
  }
};

static std::mutex g_bank_mu;
static std::map<std::string, std::unique_ptr<BankPlan>> g_plans;
static std::map<std::string, BankTune> g_tuned;
static std::atomic<int64_t> g_plan_bytes{0};

static std::atomic<int> g_last_kernels{0};

int64_t bank_cache_bytes() { return g_plan_bytes.load(); }
int bank_last_kernels() { return g_last_kernels.load(); }

void bank_release_cache() {
  std::lock_guard<std::mutex> lk(g_bank_mu);
  g_plans.clear();
  g_plan_bytes.store(0);
}

static std::string key_of(const BankRequest& q, const BankTune* t, bool with_ptrs) {
  char buf[128];
  std::string k;
  snprintf(buf, sizeof(buf), "%d/%d/%lld,%lld,%lld|", q.dtype, q.out_dtype, (long long)q.G[0],
           (long long)q.G[1], (long long)q.G[2]);
  k += buf;
  for (auto& f : q.filters) {
    snprintf(buf, sizeof(buf), "%d:%.17g;", f.first, f.second);
    k += buf;
  }
  for (auto& b : q.bricks) {
    snprintf(buf, sizeof(buf), "[%lld %lld %lld %lld %lld %lld]", (long long)b.lo[0],
             (long long)b.lo[1], (long long)b.lo[2], (long long)b.hi[0], (long long)b.hi[1],
             (long long)b.hi[2]);
    k += buf;
  }
  if (t) {
    snprintf(buf, sizeof(buf), "|t%d,%d", t->small_cfg, t->zchunk);
    k += buf;
  }
  if (with_ptrs) {
    snprintf(buf, sizeof(buf), "|%p", q.in);
    k += buf;
    for (void* o : q.outs) {
      snprintf(buf, sizeof(buf), ",%p", o);
      k += buf;
    }
  }
  return k;
}

// Build a plan (work list, TMA maps, graph) for one tuning choice. With
// `wl` set, the counters and the work list go into that caller device
// memory (wl_bytes), copied on stream s from the caller's page-locked
// buffer hwl (wl_bytes, not reused until the copy has run), and no graph
// is made: the plan is launched directly (launch_direct) and owns no
// device memory.
static int build_plan(const BankRequest& q, const BankTune& t, std::unique_ptr<BankPlan>* out,
                      void* wl = nullptr, size_t wl_bytes = 0, cudaStream_t s = nullptr,
                      void* hwl = nullptr) {
  auto plan = std::make_unique<BankPlan>();
  plan->owns = wl == nullptr;
  BankParams& P = plan->P;
  memset(&P, 0, sizeof(P));
  P.in = q.in;
  P.dtype = q.dtype;
  P.out_dtype = q.out_dtype;
  for (int a = 0; a < 3; ++a) P.G[a] = q.G[a];
  P.in_z0 = q.in_z0;
  P.out_z0 = q.out_z0;
  // sigma groups, heaviest first
  std::vector<double> sigmas;
  for (auto& f : q.filters)
    if (std::find(sigmas.begin(), sigmas.end(), f.second) == sigmas.end()) sigmas.push_back(f.second);
  std::sort(sigmas.begin(), sigmas.end(), [](double a, double b) { return a > b; });
  if ((int)sigmas.size() > kMaxGroups)
    return set_error(HP_ERR_UNSUPPORTED, "filter bank: at most 8 distinct sigmas");
  P.ngroups = (int)sigmas.size();
  for (int g = 0; g < P.ngroups; ++g) {
    BankGroup& G = P.grp[g];
    G.r = radius_of(sigmas[g], 3.0);
    if (G.r < 1 || G.r > kMaxR)
      return set_error(HP_ERR_UNSUPPORTED, "filter bank: radius must be in [1, 12] (sigma in ~[0.17, 4.16])");
    std::vector<double> w(2 * G.r + 1);
    for (int o = 0; o < 3; ++o) {
      taps1d_f64(sigmas[g], G.r, o, w.data());
      for (int k = 0; k < 2 * kMaxR + 1; ++k) G.w[o][k] = k <= 2 * G.r ? (float)w[k] : 0.0f;
    }
    for (int o = 0; o < 3; ++o) G.out[o] = nullptr;
  }
  for (size_t i = 0; i < q.filters.size(); ++i) {
    const int g = (int)(std::find(sigmas.begin(), sigmas.end(), q.filters[i].second) - sigmas.begin());
    void*& slot = P.grp[g].out[q.filters[i].first];
    if (slot) return set_error(HP_ERR_INVALID_ARG, "filter bank: duplicate (kind, sigma)");
    slot = q.outs[i];
  }
  // Kernel choice. The four-plane kernel (k_bank2) takes uint16, float16
  // and float32 inputs that TMA can address (16-byte aligned base and rows,
  // brick x origins on multiples of 16) in volumes at least r_max + 1 wide in
  // x and y (one reflection lands inside the staged box); the first kernel
  // takes everything else.
  const int es = (int)dtype_size(q.dtype);
  int rmax = 0;
  for (int g = 0; g < P.ngroups; ++g) rmax = std::max(rmax, P.grp[g].r);
  bool tma = ((uintptr_t)q.in % 16 == 0) && ((q.G[2] * es) % 16 == 0) && getenv("HP_NO_TMA") == nullptr;
  for (auto& b : q.bricks) tma = tma && (b.lo[2] % 16 == 0);
  const bool v2 = tma && (q.dtype == HP_U16 || q.dtype == HP_F16 || q.dtype == HP_F32) &&
                  q.G[1] > rmax && q.G[2] > rmax && getenv("HP_BANK_V1") == nullptr;
  auto cfg_of = [&](int r) {
    if (t.small_cfg != 1) return 0;
    if (v2) return (r <= b2::kWideMaxR && b2::geo(r, 32, 16, es).SMEM <= max_dyn_smem()) ? 1 : 0;
    return r <= 4 ? 1 : 0;
  };
  // split: the radii <= kWideMaxR whose 16 x 16 tiles fit two CTAs per SM
  // go to the two-CTAs-per-SM launch
  const void* kfn2 = v2 ? bank2_kernel(q.dtype, 2) : nullptr;
  bool split = false;
  bool second_of[kMaxGroups] = {false};
  if (v2 && t.small_cfg == 2) {
    const int sm_smem = max_smem_per_sm();
    int s2 = 0;
    for (int g = 0; g < P.ngroups; ++g) {
      const int r = P.grp[g].r;
      const int need = b2::geo(r, 16, 16, es).SMEM;
      if (r <= b2::kWideMaxR && 2 * (need + 1024) <= sm_smem) {
        second_of[g] = true;
        s2 = std::max(s2, need);
      }
    }
    int per_sm2 = 0;
    if (s2 > 0 && cudaFuncSetAttribute(kfn2, cudaFuncAttributeMaxDynamicSharedMemorySize, s2) == cudaSuccess &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm2, kfn2, b2::kThreads2, s2) == cudaSuccess && per_sm2 >= 2) {
      split = true;
      plan->smem2 = s2;
      plan->grid2 = num_sms() * per_sm2;
    }
    (void)cudaGetLastError();
  }
  // work list over bricks: groups (heaviest first) x bricks x tiles x z chunks
  std::vector<BankItem> items, items2;
  int smem = 0;
  for (int g = 0; g < P.ngroups; ++g) {
    const int r = P.grp[g].r;
    const int cfg = cfg_of(r);
    const int TX = cfg == 1 ? 32 : 16, TY = 16;
    const bool second = split && second_of[g];
    if (!second) smem = std::max(smem, v2 ? b2::geo(r, TX, TY, es).SMEM : cfg_smem(cfg, r, es));
    std::vector<BankItem>& list = second ? items2 : items;
    for (auto& b : q.bricks)
      for (int64_t y0 = b.lo[1]; y0 < b.hi[1]; y0 += TY)
        for (int64_t x0 = b.lo[2]; x0 < b.hi[2]; x0 += TX)
          for (int64_t z0 = b.lo[0]; z0 < b.hi[0]; z0 += t.zchunk) {
            BankItem it;
            it.group = g;
            it.tile_x0 = (int)x0;
            it.tile_y0 = (int)y0;
            it.z0 = (int)z0;
            it.z1 = (int)std::min<int64_t>(z0 + t.zchunk, b.hi[0]);
            it.x1 = (int)b.hi[2];
            it.y1 = (int)b.hi[1];
            it.cfg = cfg;
            list.push_back(it);
          }
  }
  if (smem > max_dyn_smem()) return set_error(HP_ERR_UNSUPPORTED, "filter bank: tile does not fit in shared memory");
  P.nitems = (int)items.size();
  cudaError_t e;
  const size_t nall = items.size() + items2.size();
  items.insert(items.end(), items2.begin(), items2.end());
  if (wl) {
    // counters in the first 256 bytes, the work list after them
    if (256 + sizeof(BankItem) * nall > wl_bytes)
      return set_error(HP_ERR_INTERNAL, "filter bank: work list exceeds its buffer");
    if (!hwl) return set_error(HP_ERR_INTERNAL, "filter bank: no staging buffer for the work list");
    plan->d_counter = static_cast<int*>(wl);
    plan->d_items = reinterpret_cast<BankItem*>(static_cast<char*>(wl) + 256);
    if (nall) {
      memcpy(static_cast<char*>(hwl) + 256, items.data(), sizeof(BankItem) * nall);
      if ((e = cudaMemcpyAsync(plan->d_items, static_cast<char*>(hwl) + 256, sizeof(BankItem) * nall,
                               cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return cuda_fail(e, "copy work list");
    }
  } else {
    if ((e = cudaMalloc(&plan->d_items, sizeof(BankItem) * std::max<size_t>(1, nall))) != cudaSuccess)
      return cuda_fail(e, "cudaMalloc(work list)");
    if ((e = cudaMalloc(&plan->d_counter, 2 * sizeof(int))) != cudaSuccess)
      return cuda_fail(e, "cudaMalloc(counter)");
    plan->bytes = sizeof(BankItem) * nall + 2 * sizeof(int);
    if (nall && (e = cudaMemcpy(plan->d_items, items.data(), sizeof(BankItem) * nall,
                                cudaMemcpyHostToDevice)) != cudaSuccess)
      return cuda_fail(e, "copy work list");
  }
  P.items = plan->d_items;
  P.counter = plan->d_counter;
  P.err = device_error_word();
  // TMA maps, per sigma group.
  memset(&plan->maps, 0, sizeof(plan->maps));
  const int64_t dims[3] = {q.G[2], q.G[1], q.in_nz > 0 ? q.in_nz : q.G[0]};
  for (int g = 0; g < P.ngroups && tma; ++g) {
    const int r = P.grp[g].r;
    const int tx = cfg_of(r) == 1 ? 32 : 16;
    if (v2) {
      const b2::Geo gm = b2::geo(r, tx, 16, es);
      tma = make_tmap_3d(&plan->maps.m[g], q.in, q.dtype, dims, gm.BW, gm.BHP, b2::kKP) &&
            make_tmap_3d(&plan->maps.m1[g], q.in, q.dtype, dims, gm.BW, gm.BHP, 1);
    } else {
      int ra = 0, bw = 0;
      bbox_geom(r, tx, es, &ra, &bw);
      tma = make_tmap_3d(&plan->maps.m[g], q.in, q.dtype, dims, bw, 16 + 2 * r);
    }
  }
  if (v2 && !tma) return set_error(HP_ERR_CUDA, "filter bank: TMA map encoding failed");
  P.use_tma = tma ? 1 : 0;
  plan->P2 = P;
  plan->P2.items = plan->d_items + P.nitems;
  plan->P2.nitems = (int)items2.size();
  plan->P2.counter = plan->d_counter + 1;
  if (split && !items2.empty()) {
    plan->kernel2 = kfn2;
    plan->grid2 = std::max(1, std::min(plan->P2.nitems, plan->grid2));
  }
  plan->smem = smem;
  const void* kfn = v2 ? bank2_kernel(q.dtype, 1) : reinterpret_cast<const void*>(&k_bank);
  const int nt1 = v2 ? b2::kThreads1 : kThreads;
  plan->kernel = kfn;
  plan->threads = nt1;
  const int sms = num_sms();
  if ((e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess)
    return cuda_fail(e, "cudaFuncSetAttribute(filter bank)");
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, nt1, smem);
  plan->grid = std::max(1, std::min(P.nitems, sms * std::max(1, per_sm)));
  if (wl) {
    *out = std::move(plan);
    return HP_OK;
  }
  // graph: reset the counters, then the persistent launch(es); two launches
  // are sibling nodes, so the second fills SMs as the first drains
  if ((e = cudaGraphCreate(&plan->graph, 0)) != cudaSuccess) return cuda_fail(e, "cudaGraphCreate");
  cudaGraphNode_t mset, kern;
  cudaMemsetParams mp;
  memset(&mp, 0, sizeof(mp));
  mp.dst = plan->d_counter;
  mp.value = 0;
  mp.elementSize = 4;
  mp.width = 2;
  mp.height = 1;
  if ((e = cudaGraphAddMemsetNode(&mset, plan->graph, nullptr, 0, &mp)) != cudaSuccess)
    return cuda_fail(e, "cudaGraphAddMemsetNode");
  if (P.nitems > 0 || !plan->kernel2) {
    cudaKernelNodeParams kp;
    memset(&kp, 0, sizeof(kp));
    void* args[2] = {&plan->P, &plan->maps};
    kp.func = const_cast<void*>(plan->kernel);
    kp.gridDim = dim3(plan->grid);
    kp.blockDim = dim3(plan->threads);
    kp.sharedMemBytes = smem;
    kp.kernelParams = args;
    if ((e = cudaGraphAddKernelNode(&kern, plan->graph, &mset, 1, &kp)) != cudaSuccess)
      return cuda_fail(e, "cudaGraphAddKernelNode");
  }
  if (plan->kernel2) {
    cudaKernelNodeParams kp;
    memset(&kp, 0, sizeof(kp));
    void* args[2] = {&plan->P2, &plan->maps};
    kp.func = const_cast<void*>(plan->kernel2);
    kp.gridDim = dim3(plan->grid2);
    kp.blockDim = dim3(b2::kThreads2);
    kp.sharedMemBytes = plan->smem2;
    kp.kernelParams = args;
    if ((e = cudaGraphAddKernelNode(&kern, plan->graph, &mset, 1, &kp)) != cudaSuccess)
      return cuda_fail(e, "cudaGraphAddKernelNode");
  }
  if ((e = cudaGraphInstantiate(&plan->exec, plan->graph, 0)) != cudaSuccess)
    return cuda_fail(e, "cudaGraphInstantiate");
  *out = std::move(plan);
  return HP_OK;
}

// Launch of a plan without a graph: counters reset, then the launch(es) in
// stream order (the second follows the first).
static int launch_direct(BankPlan& pl, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(pl.d_counter, 0, 2 * sizeof(int), s);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(bank counters)");
  if (pl.P.nitems > 0 || !pl.kernel2) {
    void* args[2] = {&pl.P, &pl.maps};
    e = cudaLaunchKernel(pl.kernel, dim3(pl.grid), dim3(pl.threads), args, pl.smem, s);
    if (e != cudaSuccess) return cuda_fail(e, "filter bank launch");
  }
  if (pl.kernel2) {
    void* args[2] = {&pl.P2, &pl.maps};
    e = cudaLaunchKernel(pl.kernel2, dim3(pl.grid2), dim3(b2::kThreads2), args, pl.smem2, s);
    if (e != cudaSuccess) return cuda_fail(e, "filter bank launch");
  }
  g_last_kernels.store((pl.P.nitems > 0 || !pl.kernel2 ? 1 : 0) + (pl.kernel2 ? 1 : 0));
  return HP_OK;
}

static int launch_plan(BankPlan& pl, cudaStream_t s) {
  cudaError_t e = cudaGraphLaunch(pl.exec, s);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch(filter bank)");
  g_last_kernels.store((pl.P.nitems > 0 || !pl.kernel2 ? 1 : 0) + (pl.kernel2 ? 1 : 0));
  return HP_OK;
}

// Autotuner: time each candidate once (after a warm-up launch) on the
// caller's data and keep the fastest per (shape, dtype, filters, bricks).
// Every candidate computes the same values bit for bit, so tuning on the
// real outputs is harmless.
static int tune(const BankRequest& q, cudaStream_t s, BankTune* best) {
  const std::string k = key_of(q, nullptr, false);
  {
    std::lock_guard<std::mutex> lk(g_bank_mu);
    auto it = g_tuned.find(k);
    if (it != g_tuned.end()) {
      *best = it->second;
      return HP_OK;
    }
  }
  // HP_BANK_TUNE=0 skips tuning (32 x 16 tiles where they fit, z chunks of
  // 256); HP_BANK_TUNE=<cfg>,<zchunk> pins one candidate (cfg 0, 1 or 2 as
  // in BankTune, zchunk >= 4).
  const char* env = getenv("HP_BANK_TUNE");
  std::vector<BankTune> cands = {{1, 64}, {1, 128}, {1, 256}, {0, 256}, {2, 128}, {2, 256}};
  if (env && !strcmp(env, "0")) cands = {{1, 256}};
  int pin_cfg = -1, pin_z = 0;
  if (env && sscanf(env, "%d,%d", &pin_cfg, &pin_z) == 2 && pin_cfg >= 0 && pin_cfg <= 2 && pin_z >= 4)
    cands = {{pin_cfg, pin_z}};
  float best_ms = 1e30f;
  BankTune bt = cands[0];
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  int rc = HP_OK;
  for (auto& c : cands) {
    std::unique_ptr<BankPlan> pl;
    rc = build_plan(q, c, &pl);
    if (rc != HP_OK) break;
    if (cands.size() == 1) break;
    if ((rc = launch_plan(*pl, s)) != HP_OK) break;
    cudaEventRecord(a, s);
    if ((rc = launch_plan(*pl, s)) != HP_OK) break;
    cudaEventRecord(b, s);
    cudaEventSynchronize(b);
    float ms = 0;
    cudaEventElapsedTime(&ms, a, b);
    if (log_level() > 0)
      fprintf(stderr, "[hp] bank tune cfg=%d zchunk=%d tma=%d kernel=%s grid=%d items=%d (+%d on %d CTAs at 2/SM): %.3f ms\n",
              c.small_cfg, c.zchunk, pl->P.use_tma,
              pl->kernel == reinterpret_cast<const void*>(&k_bank) ? "k_bank" : "k_bank2", pl->grid,
              pl->P.nitems, pl->kernel2 ? pl->P2.nitems : 0, pl->kernel2 ? pl->grid2 : 0, ms);
    if (ms < best_ms) {
      best_ms = ms;
      bt = c;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (rc != HP_OK) return rc;
  std::lock_guard<std::mutex> lk(g_bank_mu);
  g_tuned[k] = bt;
  *best = bt;
  return HP_OK;
}

int run_filterbank(const BankRequest& q, cudaStream_t s) {
  BankTune t;
  int rc = tune(q, s, &t);
  if (rc != HP_OK) return rc;
  const std::string k = key_of(q, &t, true);
  BankPlan* pl = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_bank_mu);
    auto it = g_plans.find(k);
    if (it != g_plans.end()) pl = it->second.get();
  }
  if (!pl) {
    std::unique_ptr<BankPlan> np;
    rc = build_plan(q, t, &np);
    if (rc != HP_OK) return rc;
    std::lock_guard<std::mutex> lk(g_bank_mu);
    if (g_plans.size() >= 16) {  // bounded cache
      for (auto& kv : g_plans) g_plan_bytes.fetch_sub((int64_t)kv.second->bytes);
      g_plans.clear();
    }
    g_plan_bytes.fetch_add((int64_t)np->bytes);
    pl = np.get();
    g_plans[k] = std::move(np);
  }
  return launch_plan(*pl, s);
}

// Out-of-core tuning choice: 16 x 16 tiles, radii <= 6 in a second launch
// at two CTAs per SM where they fit, z chunks of 128 planes.
static const BankTune kHostTune = {2, 128};

size_t bank_worklist_bytes(const BankRequest& q) {
  // items of 16 x 16 tiles and 128-plane chunks per distinct sigma and
  // brick (32 x 16 tiles need fewer), after 256 bytes of counters
  int ng = 0;
  std::vector<double> seen;
  for (auto& f : q.filters)
    if (std::find(seen.begin(), seen.end(), f.second) == seen.end()) {
      seen.push_back(f.second);
      ++ng;
    }
  size_t items = 0;
  for (auto& b : q.bricks)
    items += (size_t)((b.hi[1] - b.lo[1] + 15) / 16) * (size_t)((b.hi[2] - b.lo[2] + 15) / 16) *
             (size_t)((b.hi[0] - b.lo[0] + kHostTune.zchunk - 1) / kHostTune.zchunk);
  return 256 + sizeof(BankItem) * items * (size_t)ng;
}

// One out-of-core brick: the bank over q.bricks (the brick's core) with the
// input and outputs as plane ranges of the volume (in_z0, out_z0), the work
// list in caller device memory wl staged through the caller's page-locked
// hwl (both bank_worklist_bytes), launched without a graph.
int run_filterbank_brick(const BankRequest& q, void* wl, void* hwl, size_t wl_bytes, cudaStream_t s) {
  std::unique_ptr<BankPlan> pl;
  int rc = build_plan(q, kHostTune, &pl, wl, wl_bytes, s, hwl);
  if (rc != HP_OK) return rc;
  return launch_direct(*pl, s);
}

const void* bank2_kernel_u16(int minb);
const void* bank2_kernel_f16(int minb);
const void* bank2_kernel_f32(int minb);

const void* bank2_kernel(int dtype, int minb) {
  switch (dtype) {
    case HP_U16: return bank2_kernel_u16(minb);
    case HP_F16: return bank2_kernel_f16(minb);
    case HP_F32: return bank2_kernel_f32(minb);
    default: return nullptr;
  }
}

}  // namespace hp
