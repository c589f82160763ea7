// C ABI of libhp: volumes, memory budget, chunk planner, out-of-core
// executor and dispatch of the filtering kernels.
//
// The chunked execution model follows Harpia Sec. III-D:
//   step 1 (resource profiling): the budget is the user value or a fixed
//           fraction (0.8) of cudaMemGetInfo's free bytes;
//   step 2 (chunk size estimation): hp_plan_bricks sizes halo-padded bricks
//           so that the stages in flight fit the budget;
//   step 3 (independent chunk execution): bricks stream through the device
//           on several CUDA streams (H2D of the halo box, kernel, D2H of the
//           core), each brick independent given its halo.
// Library memory is allocated per call and released before return
// (Sec. IV-C).
#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <functional>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "hp_device.cuh"
#include "hp_internal.h"

namespace hp {

// ------------------------------------------------------------------ errors
static thread_local std::string t_msg;

int set_error(int status, const std::string& msg) {
  t_msg = msg;
  return status;
}

int cuda_fail(cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  if (e == cudaErrorMemoryAllocation) return set_error(HP_ERR_OOM, m);
  return set_error(HP_ERR_CUDA, m);
}

// ------------------------------------------------------------------ state
static std::mutex g_mu;
static size_t g_budget = 0;
static bool g_budget_init = false;
static hp_stats g_stats;
static std::atomic<int64_t> g_live{0};
static std::atomic<int64_t> g_peak{0};
static std::atomic<int64_t> g_cached{0};

static void track_alloc(int64_t b) {
  int64_t now = g_live.fetch_add(b) + b;
  int64_t p = g_peak.load();
  while (now > p && !g_peak.compare_exchange_weak(p, now)) {
  }
}
static void track_free(int64_t b) { g_live.fetch_sub(b); }

// Stream-ordered scratch of device-mode calls (positive on allocation,
// negative on release).
void note_scratch(int64_t bytes) {
  if (bytes > 0) track_alloc(bytes);
  else track_free(-bytes);
}

size_t budget_setting() {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_budget_init) {
    g_budget_init = true;
    const char* e = getenv("HP_BUDGET");
    if (e) g_budget = (size_t)strtoull(e, nullptr, 10);
  }
  return g_budget;
}

static int effective_budget(size_t* out) {
  size_t b = budget_setting();
  if (b == 0) {
    size_t fr = 0, tot = 0;
    cudaError_t e = cudaMemGetInfo(&fr, &tot);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemGetInfo");
    b = (size_t)(0.8 * (double)fr);
  }
  *out = b;
  return HP_OK;
}

int check_scratch_budget(size_t need) {
  size_t b = 0;
  const int st = effective_budget(&b);
  if (st != HP_OK) return st;
  if (need > b)
    return set_error(HP_ERR_BUDGET, "scratch of " + std::to_string(need) +
                                        " bytes exceeds the budget of " + std::to_string(b) +
                                        " bytes");
  return HP_OK;
}

// Device error word: one int per device, set by kernels whose bounded waits
// give up. Its device address is looked up once per device.
__device__ int g_error_word;
static int* g_err_ptr[64];
static std::mutex g_err_mu;

int64_t bank_cache_bytes();
int bank_last_kernels();

// Drops the cached error-word addresses (hp_release_cache), so that after a
// cudaDeviceReset the next call looks the word up in the new context.
void error_word_forget() {
  std::lock_guard<std::mutex> lk(g_err_mu);
  for (auto& p : g_err_ptr) p = nullptr;
}

int* device_error_word() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(g_err_mu);
  if (!g_err_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_error_word) != cudaSuccess) return nullptr;
    g_err_ptr[dev] = static_cast<int*>(p);
  }
  return g_err_ptr[dev];
}

// A bounded mbarrier wait on a barrier that nothing completes: the wait
// gives up after its poll limit and records a timeout in the error word.
__global__ void k_wait_selftest(int* err) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait(&bar, 0)) set_device_error(err, kErrTimeout);
}

int log_level() {
  static int lv = [] {
    const char* e = getenv("HP_LOG");
    return e ? atoi(e) : 0;
  }();
  return lv;
}

int num_sms() {
  static int cached[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return 148;
  if (!cached[dev]) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
      n = 148;
    cached[dev] = n;
  }
  return cached[dev];
}

int max_dyn_smem() {
  static int cached[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return 227 * 1024 - 1024;
  if (!cached[dev]) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess || n <= 0)
      n = 227 * 1024;
    cached[dev] = n - 1024;
  }
  return cached[dev];
}

int max_smem_per_sm() {
  static int cached[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return 228 * 1024;
  if (!cached[dev]) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess || n <= 0)
      n = 228 * 1024;
    cached[dev] = n;
  }
  return cached[dev];
}

int64_t pick_zchunk(int64_t cz, int64_t tiles, int64_t slots, int halo, int align) {
  if (cz <= 0) return align;
  slots = std::max<int64_t>(1, slots);
  int64_t best_zc = (cz + align - 1) / align * align;
  double best = 1e300;
  for (int64_t n = 1; n <= 512; ++n) {
    int64_t zc = (cz + n - 1) / n;
    zc = (zc + align - 1) / align * align;
    const int64_t chunks = (cz + zc - 1) / zc;
    const int64_t waves = (tiles * chunks + slots - 1) / slots;
    const double cost = (double)waves * (double)(zc + halo);
    if (cost < best * 0.999) {
      best = cost;
      best_zc = zc;
    }
    if (zc <= align) break;
  }
  return best_zc;
}

// ------------------------------------------------------------ TMA maps
typedef CUresult (*PFN_encodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                    const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                    const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                    CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static PFN_encodeTiled get_encode() {
  static PFN_encodeTiled fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_encodeTiled>(p);
  });
  return fn;
}

bool make_tmap_3d(CUtensorMap* map, const void* base, int dtype, const int64_t dims[3], int bw,
                  int bh, int bd) {
  PFN_encodeTiled enc = get_encode();
  if (!enc) return false;
  CUtensorMapDataType t;
  switch (dtype) {
    case HP_U8: t = CU_TENSOR_MAP_DATA_TYPE_UINT8; break;
    case HP_U16: t = CU_TENSOR_MAP_DATA_TYPE_UINT16; break;
    case HP_F16: t = CU_TENSOR_MAP_DATA_TYPE_FLOAT16; break;
    case HP_F32: t = CU_TENSOR_MAP_DATA_TYPE_FLOAT32; break;
    default: return false;
  }
  const size_t es = dtype_size(dtype);
  if ((uintptr_t)base % 16 != 0) return false;
  if (dims[0] > (1LL << 31) || dims[1] > (1LL << 31) || dims[2] > (1LL << 31)) return false;
  cuuint64_t gdim[3] = {(cuuint64_t)dims[0], (cuuint64_t)dims[1], (cuuint64_t)dims[2]};
  cuuint64_t gstride[2] = {(cuuint64_t)(dims[0] * es), (cuuint64_t)(dims[0] * dims[1] * es)};
  if (gstride[0] % 16 || gstride[1] % 16) return false;
  cuuint32_t box[3] = {(cuuint32_t)bw, (cuuint32_t)bh, (cuuint32_t)bd};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(map, t, 3, const_cast<void*>(base), gdim, gstride, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// ------------------------------------------------------------ weights
int radius_of(double sigma, double truncate) {
  return (int)std::floor(truncate * sigma + 0.5);
}

// FP64 taps of the sampled Gaussian (order 0) and its analytic derivatives
// (orders 1, 2), normalised by the sum of the order-0 samples.
void taps1d_f64(double sigma, int r, int order, double* w) {
  const double s2 = sigma * sigma;
  double norm = 0.0;
  for (int k = -r; k <= r; ++k) norm += std::exp(-0.5 * (double)k * (double)k / s2);
  for (int k = -r; k <= r; ++k) {
    const double g = std::exp(-0.5 * (double)k * (double)k / s2) / norm;
    const double kk = (double)k;
    double v = g;
    if (order == 1) v = -kk / s2 * g;
    if (order == 2) v = (kk * kk / (s2 * s2) - 1.0 / s2) * g;
    w[k + r] = v;
  }
}

void make_taps(double sigma, double truncate, const int order[3], Taps* t) {
  const int r = radius_of(sigma, truncate);
  t->r = r;
  if (r < 0 || r > kMaxRGeneric) return;  // rejected by the caller
  std::vector<double> w(2 * r + 1);
  for (int a = 0; a < 3; ++a) {
    for (int k = 0; k < kMaxTaps; ++k) t->w[a][k] = 0.0f;
    taps1d_f64(sigma, r, order[a], w.data());
    for (int k = 0; k <= 2 * r; ++k) t->w[a][k] = (float)w[k];
  }
}

// ------------------------------------------------------------ planner
static void reflect_hull(int64_t a, int64_t b, int64_t n, int64_t* lo, int64_t* hi) {
  // hull of {R(c) : c in [a, b)}
  if (b - a >= 2 * n) {
    *lo = 0;
    *hi = n;
    return;
  }
  if (a >= 0 && b <= n) {
    *lo = a;
    *hi = b;
    return;
  }
  int64_t mn = n, mx = -1;
  for (int64_t c = a; c < b; ++c) {
    int64_t s = reflect(c, n);
    mn = std::min(mn, s);
    mx = std::max(mx, s);
  }
  *lo = mn;
  *hi = mx + 1;
}

struct Brick {
  hp_box core;
  hp_box in;
};

// Device bytes of one stage: its input box (in_b per voxel, plus scr_b per
// voxel of kernel scratch) and its core output box.
static size_t stage_bytes(const int64_t ext[3], const int64_t n[3], int halo, size_t in_b,
                          size_t out_b, size_t scr_b) {
  size_t inv = 1, outv = 1;
  for (int a = 0; a < 3; ++a) {
    int64_t e = std::min<int64_t>(ext[a] + 2 * (int64_t)halo + (a == 2 ? 32 : 0), n[a]);
    inv *= (size_t)e;
    outv *= (size_t)ext[a];
  }
  return inv * (in_b + scr_b) + outv * out_b;
}

// Plan bricks; returns HP_OK or HP_ERR_BUDGET / HP_ERR_INVALID_ARG.
static int plan(const int64_t n[3], int halo, size_t in_b, size_t out_b, size_t scr_b,
                size_t budget, int stages, int min_bricks, bool z_only, std::vector<Brick>* out) {
  if (n[0] < 1 || n[1] < 1 || n[2] < 1 || halo < 0 || stages < 1)
    return set_error(HP_ERR_INVALID_ARG, "plan: bad extents, halo or stages");
  const size_t per = budget / (size_t)stages;
  int64_t ext[3] = {n[0], n[1], n[2]};
  // Prefer Z slabs (contiguous planes); split y, then x, only when one
  // plane plus halos does not fit.
  int axis_split = -1;
  for (int a = 0; a < (z_only ? 1 : 3) && axis_split < 0; ++a) {
    for (int b = 0; b < a; ++b) ext[b] = 1;
    for (int b = a; b < 3; ++b) ext[b] = n[b];
    ext[a] = 1;
    if (stage_bytes(ext, n, halo, in_b, out_b, scr_b) > per) continue;
    // largest extent along a that fits
    int64_t lo = 1, hi = n[a];
    while (lo < hi) {
      int64_t mid = (lo + hi + 1) / 2;
      ext[a] = mid;
      if (stage_bytes(ext, n, halo, in_b, out_b, scr_b) <= per) lo = mid;
      else hi = mid - 1;
    }
    ext[a] = lo;
    axis_split = a;
  }
  if (axis_split < 0)
    return set_error(HP_ERR_BUDGET, "budget too small for the smallest brick (" +
                                        std::to_string(budget) + " bytes, " +
                                        std::to_string(stages) + " stages)");
  // at least min_bricks bricks along the split axis (for pipelining) when
  // the volume allows it; then balance the brick lengths
  const int a = axis_split;
  int64_t nb = (n[a] + ext[a] - 1) / ext[a];
  if (a == 0 && nb < min_bricks) nb = std::min<int64_t>(min_bricks, n[a]);
  int64_t len = (n[a] + nb - 1) / nb;
  if (a == 2) len = std::max<int64_t>(16, len / 16 * 16);  // 16-aligned x cores (TMA)
  ext[a] = std::min<int64_t>(len, n[a]);
  out->clear();
  for (int64_t z0 = 0; z0 < n[0]; z0 += ext[0])
    for (int64_t y0 = 0; y0 < n[1]; y0 += ext[1])
      for (int64_t x0 = 0; x0 < n[2]; x0 += ext[2]) {
        Brick b;
        const int64_t lo[3] = {z0, y0, x0};
        for (int k = 0; k < 3; ++k) {
          b.core.lo[k] = lo[k];
          b.core.hi[k] = std::min(lo[k] + ext[k], n[k]);
          reflect_hull(b.core.lo[k] - halo, b.core.hi[k] + halo, n[k], &b.in.lo[k], &b.in.hi[k]);
        }
        if (ext[2] < n[2]) {  // align the x origin of the input box to 16 elements
          b.in.lo[2] = b.in.lo[2] / 16 * 16;
        }
        out->push_back(b);
      }
  return HP_OK;
}

// ------------------------------------------------------------ executor
struct Op {
  int halo;
  int out_dtype;
  int nout = 1;         // outputs per voxel (filter bank: one per filter)
  std::vector<int> out_dtypes;  // per-output dtypes when they differ (else out_dtype)
  bool z_only = false;  // plan Z slabs only (whole x/y planes per brick)
  // planning bound of the kernel scratch, bytes per voxel of the input box
  size_t scratch_per_in_voxel = 0;
  // exact scratch bytes of one job (null: none)
  std::function<size_t(const Job&)> scratch_bytes;
  // host-mode bricks also get a page-locked host buffer of the same size
  bool host_scratch = false;
  // the kernels stage the input with TMA where its rows allow: device inputs
  // whose rows do not are copied with padded rows first (pad_device_input)
  bool pad_rows = true;
  // enqueue the op for one job: job.out is output 0, outs[k] output k (each
  // a dense box like job.out); job.scratch is set when scratch_bytes > 0.
  // Returns an hp_status.
  std::function<int(const Job&, void* const* outs, cudaStream_t)> launch;
};

// Wraps a cudaError_t launcher as an Op launch.
static int launched(cudaError_t e) { return e == cudaSuccess ? HP_OK : cuda_fail(e, "kernel launch"); }

// Out-of-core placement (Sec. III-D step 3 and Sec. V: round-robin chunk
// scheduling without inter-GPU communication): the devices host-mode calls
// spread their bricks over, and the shard of the brick list this process
// executes.
static std::vector<int> g_devices;  // empty: the current device
static int g_shard_rank = 0, g_shard_world = 1;

static bool is_pinned(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeHost;
}

static void host_copy_box(void* dst, const void* src, size_t es, const int64_t src_dims[3],
                          const int64_t src_lo[3], const int64_t dst_dims[3],
                          const int64_t dst_lo[3], const int64_t box_lo[3],
                          const int64_t box_hi[3]) {
  // copy box [box_lo, box_hi) (global coords) between two dense boxes,
  // row by row, on several host threads
  const int64_t nzb = box_hi[0] - box_lo[0], nyb = box_hi[1] - box_lo[1],
                nxb = box_hi[2] - box_lo[2];
  const int64_t rows = nzb * nyb;
  const unsigned nt = std::max(1u, std::min(8u, std::thread::hardware_concurrency()));
  auto work = [&](unsigned t) {
    for (int64_t r = t; r < rows; r += nt) {
      const int64_t z = box_lo[0] + r / nyb, y = box_lo[1] + r % nyb;
      const char* s = (const char*)src +
                      (((z - src_lo[0]) * src_dims[1] + (y - src_lo[1])) * src_dims[2] +
                       (box_lo[2] - src_lo[2])) * es;
      char* d = (char*)dst + (((z - dst_lo[0]) * dst_dims[1] + (y - dst_lo[1])) * dst_dims[2] +
                              (box_lo[2] - dst_lo[2])) * es;
      memcpy(d, s, (size_t)nxb * es);
    }
  };
  if (rows * nxb * (int64_t)es < (8 << 20) || nt == 1) {
    work(0);
    for (unsigned t = 1; t < nt; ++t) work(t);
    return;
  }
  std::vector<std::thread> th;
  for (unsigned t = 0; t < nt; ++t) th.emplace_back(work, t);
  for (auto& x : th) x.join();
}

// cudaMemcpy3DAsync of box [lo, hi) between a dense host box and a dense
// device box (both described in global coordinates).
static cudaError_t copy_box_async(void* dst, const int64_t dst_dims[3], const int64_t dst_lo[3],
                                  const void* src, const int64_t src_dims[3],
                                  const int64_t src_lo[3], const int64_t lo[3], const int64_t hi[3],
                                  size_t es, cudaMemcpyKind kind, cudaStream_t s) {
  const bool full_rows = lo[2] == src_lo[2] && hi[2] == src_lo[2] + src_dims[2] &&
                         lo[2] == dst_lo[2] && hi[2] == dst_lo[2] + dst_dims[2];
  const bool full_planes = full_rows && lo[1] == src_lo[1] && hi[1] == src_lo[1] + src_dims[1] &&
                           lo[1] == dst_lo[1] && hi[1] == dst_lo[1] + dst_dims[1];
  if (full_planes) {
    const size_t plane = (size_t)src_dims[1] * src_dims[2] * es;
    const char* sp = (const char*)src + (size_t)(lo[0] - src_lo[0]) * plane;
    char* dp = (char*)dst + (size_t)(lo[0] - dst_lo[0]) * plane;
    return cudaMemcpyAsync(dp, sp, (size_t)(hi[0] - lo[0]) * plane, kind, s);
  }
  cudaMemcpy3DParms p;
  memset(&p, 0, sizeof(p));
  p.srcPtr = make_cudaPitchedPtr(const_cast<void*>(src), (size_t)src_dims[2] * es, (size_t)src_dims[2],
                                 (size_t)src_dims[1]);
  p.dstPtr = make_cudaPitchedPtr(dst, (size_t)dst_dims[2] * es, (size_t)dst_dims[2], (size_t)dst_dims[1]);
  p.srcPos = make_cudaPos((size_t)(lo[2] - src_lo[2]) * es, (size_t)(lo[1] - src_lo[1]),
                          (size_t)(lo[0] - src_lo[0]));
  p.dstPos = make_cudaPos((size_t)(lo[2] - dst_lo[2]) * es, (size_t)(lo[1] - dst_lo[1]),
                          (size_t)(lo[0] - dst_lo[0]));
  p.extent = make_cudaExtent((size_t)(hi[2] - lo[2]) * es, (size_t)(hi[1] - lo[1]),
                             (size_t)(hi[0] - lo[0]));
  p.kind = kind;
  return cudaMemcpy3DAsync(&p, s);
}

// Fault injection on the host (HP_FAULT=alloc:N | memcpy:N | budget): the
// N-th library allocation / copy of a call reports failure. Used by tests.
struct Faults {
  int alloc_at = -1, memcpy_at = -1;
  bool budget = false;
  int allocs = 0, copies = 0;
  Faults() {
    const char* e = getenv("HP_FAULT");
    if (!e) return;
    if (!strncmp(e, "alloc:", 6)) alloc_at = atoi(e + 6);
    else if (!strncmp(e, "memcpy:", 7)) memcpy_at = atoi(e + 7);
    else if (!strcmp(e, "budget")) budget = true;
  }
  bool fail_alloc() { return alloc_at >= 0 && allocs++ == alloc_at; }
  bool fail_copy() { return memcpy_at >= 0 && copies++ == memcpy_at; }
};

// Host-mode execution: plan halo-padded bricks for the budget, keep the
// bricks of this process's shard (i mod world == rank), deal them
// round-robin over the device list (brick k of the shard to device
// k mod ndev), and stream each through one of S stages of its device: H2D
// of the halo box, the kernels, D2H of the core box(es). Each device has its
// own streams and buffers; no device talks to another. Slots that name the
// same device share its budget.
static int run_host(const Op& op, const hp_volume* in, hp_volume* const* outs) {
  auto t0 = std::chrono::steady_clock::now();
  Faults faults;
  const int64_t n[3] = {in->nz, in->ny, in->nx};
  const int nout = op.nout;
  const size_t ies = dtype_size(in->dtype);
  std::vector<int> odt(nout, op.out_dtype);
  if ((int)op.out_dtypes.size() == nout) odt = op.out_dtypes;
  size_t out_bpv = 0;  // output bytes per voxel, all outputs
  for (int k = 0; k < nout; ++k) out_bpv += dtype_size(odt[k]);
  int caller_dev = 0;
  cudaError_t ce = cudaGetDevice(&caller_dev);
  if (ce != cudaSuccess) return cuda_fail(ce, "cudaGetDevice");
  std::vector<int> devs;
  int rank = 0, world = 1;
  size_t user_budget = 0;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    devs = g_devices;
    rank = g_shard_rank;
    world = g_shard_world;
  }
  user_budget = budget_setting();
  if (devs.empty()) devs.push_back(caller_dev);
  const int ndev = (int)devs.size();
  // per-slot budget: each device's budget split over the slots naming it
  size_t budget = SIZE_MAX;
  for (int k = 0; k < ndev; ++k) {
    int same = 0;
    for (int d : devs) same += d == devs[k];
    size_t b = user_budget;
    if (b == 0) {
      size_t fr = 0, tot = 0;
      if ((ce = cudaSetDevice(devs[k])) != cudaSuccess || (ce = cudaMemGetInfo(&fr, &tot)) != cudaSuccess) {
        cudaSetDevice(caller_dev);
        return cuda_fail(ce, "cudaMemGetInfo");
      }
      b = (size_t)(0.8 * (double)fr);
    }
    budget = std::min(budget, b / (size_t)same);
  }
  cudaSetDevice(caller_dev);
  if (faults.budget) budget = 1;
  if (world > 1 && user_budget == 0)
    return set_error(HP_ERR_INVALID_ARG,
                     "a brick shard needs an explicit memory budget (hp_set_memory_budget), so "
                     "that every process plans the same bricks");
  const int S = 3;
  std::vector<Brick> all;
  int st = plan(n, op.halo, ies, out_bpv, op.scratch_per_in_voxel, budget, S, 8 * ndev * world,
                op.z_only, &all);
  if (st != HP_OK) return st;
  std::vector<Brick> bricks;  // this process's shard
  for (size_t i = 0; i < all.size(); ++i)
    if ((int)(i % (size_t)world) == rank) bricks.push_back(all[i]);

  const int64_t vol_lo[3] = {0, 0, 0};
  // the job of brick b with stage buffers din / dout
  auto brick_job = [&](const Brick& b, void* din, void* dout) {
    Job job;
    job.in = DevBox{din, in->dtype, {b.in.lo[0], b.in.lo[1], b.in.lo[2]},
                    {b.in.hi[0] - b.in.lo[0], b.in.hi[1] - b.in.lo[1], b.in.hi[2] - b.in.lo[2]}};
    job.out = DevOut{dout, op.out_dtype, {b.core.lo[0], b.core.lo[1], b.core.lo[2]},
                     {b.core.hi[0] - b.core.lo[0], b.core.hi[1] - b.core.lo[1],
                      b.core.hi[2] - b.core.lo[2]}};
    for (int a = 0; a < 3; ++a) {
      job.gdims[a] = n[a];
      job.core_lo[a] = b.core.lo[a];
      job.core_hi[a] = b.core.hi[a];
    }
    return job;
  };
  size_t max_in = 0, max_vox = 0, max_scr = 0;
  for (auto& b : bricks) {
    size_t vi = ies, vo = 1;
    for (int a = 0; a < 3; ++a) {
      vi *= (size_t)(b.in.hi[a] - b.in.lo[a]);
      vo *= (size_t)(b.core.hi[a] - b.core.lo[a]);
    }
    max_in = std::max(max_in, vi);
    max_vox = std::max(max_vox, vo);
    if (op.scratch_bytes) max_scr = std::max(max_scr, op.scratch_bytes(brick_job(b, nullptr, nullptr)));
  }
  // stage output layout: output k at off[k] (256-byte aligned), max_vox voxels each
  std::vector<size_t> off(nout + 1, 0);
  for (int k = 0; k < nout; ++k)
    off[k + 1] = (off[k] + max_vox * dtype_size(odt[k]) + 255) / 256 * 256;
  const size_t out_stage = off[nout];
  const bool in_pinned = is_pinned(in->data);
  bool out_pinned = true;
  for (int k = 0; k < nout; ++k) out_pinned = out_pinned && is_pinned(outs[k]->data);

  struct Stage {
    int dev = 0;
    void* din = nullptr;
    void* dout = nullptr;  // nout core boxes (layout off[])
    void* dscr = nullptr;
    void* hscr = nullptr;
    void* hin = nullptr;
    void* hout = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t ev = nullptr;
    int brick = -1;
  };
  // slot k (device devs[k]) owns stages [k * nst, (k + 1) * nst)
  const int per_slot = (int)((bricks.size() + ndev - 1) / ndev);
  const int nst = std::max(1, std::min(S, per_slot));
  const int nslot = bricks.empty() ? 0 : std::min<int>(ndev, (int)bricks.size());
  std::vector<Stage> sg((size_t)nslot * nst);
  uint64_t h2d = 0, d2h = 0;
  size_t pinned = 0;
  int rc = HP_OK;
  auto fail = [&](int code, const std::string& m) {
    if (rc == HP_OK) rc = set_error(code, m);
  };
  auto cfail = [&](cudaError_t e, const char* what) {
    if (rc == HP_OK) rc = cuda_fail(e, what);
  };
  for (size_t i = 0; i < sg.size(); ++i) {
    Stage& x = sg[i];
    x.dev = devs[i / nst];
    if (rc != HP_OK) break;
    cudaError_t e;
    if ((e = cudaSetDevice(x.dev)) != cudaSuccess) { cfail(e, "cudaSetDevice"); break; }
    if (faults.fail_alloc()) { fail(HP_ERR_OOM, "injected allocation failure"); break; }
    if ((e = cudaMalloc(&x.din, max_in)) != cudaSuccess) { cfail(e, "cudaMalloc(in stage)"); x.din = nullptr; break; }
    track_alloc((int64_t)max_in);
    if (faults.fail_alloc()) { fail(HP_ERR_OOM, "injected allocation failure"); break; }
    if ((e = cudaMalloc(&x.dout, out_stage)) != cudaSuccess) { cfail(e, "cudaMalloc(out stage)"); x.dout = nullptr; break; }
    track_alloc((int64_t)out_stage);
    if (max_scr > 0) {
      if (faults.fail_alloc()) { fail(HP_ERR_OOM, "injected allocation failure"); break; }
      if ((e = cudaMalloc(&x.dscr, max_scr)) != cudaSuccess) { cfail(e, "cudaMalloc(scratch stage)"); x.dscr = nullptr; break; }
      track_alloc((int64_t)max_scr);
      if (op.host_scratch) {
        if ((e = cudaHostAlloc(&x.hscr, max_scr, cudaHostAllocDefault)) != cudaSuccess) { cfail(e, "cudaHostAlloc"); x.hscr = nullptr; break; }
        pinned += max_scr;
      }
    }
    if (!in_pinned) {
      if ((e = cudaHostAlloc(&x.hin, max_in, cudaHostAllocDefault)) != cudaSuccess) { cfail(e, "cudaHostAlloc"); x.hin = nullptr; break; }
      pinned += max_in;
    }
    if (!out_pinned) {
      if ((e = cudaHostAlloc(&x.hout, out_stage, cudaHostAllocDefault)) != cudaSuccess) { cfail(e, "cudaHostAlloc"); x.hout = nullptr; break; }
      pinned += out_stage;
    }
    if ((e = cudaStreamCreateWithFlags(&x.s, cudaStreamNonBlocking)) != cudaSuccess) { cfail(e, "cudaStreamCreate"); x.s = nullptr; break; }
    if ((e = cudaEventCreateWithFlags(&x.ev, cudaEventDisableTiming)) != cudaSuccess) { cfail(e, "cudaEventCreate"); x.ev = nullptr; break; }
  }

  // completes the brick of stage x: copy its staged outputs to the user arrays
  auto retire = [&](Stage& x) {
    if (x.brick < 0) return;
    cudaError_t e = cudaEventSynchronize(x.ev);
    if (e != cudaSuccess) cfail(e, "brick execution");
    if (rc == HP_OK && !out_pinned) {
      const Brick& b = bricks[x.brick];
      const int64_t cd[3] = {b.core.hi[0] - b.core.lo[0], b.core.hi[1] - b.core.lo[1],
                             b.core.hi[2] - b.core.lo[2]};
      for (int k = 0; k < nout; ++k)
        host_copy_box(outs[k]->data, (const char*)x.hout + off[k], dtype_size(odt[k]), cd, b.core.lo, n,
                      vol_lo, b.core.lo, b.core.hi);
    }
    x.brick = -1;
  };

  std::vector<int> next_stage(nslot, 0);
  for (size_t i = 0; i < bricks.size() && rc == HP_OK; ++i) {
    const int slot = (int)(i % (size_t)nslot);
    Stage& x = sg[(size_t)slot * nst + (next_stage[slot]++ % nst)];
    retire(x);
    if (rc != HP_OK) break;
    cudaError_t e;
    if ((e = cudaSetDevice(x.dev)) != cudaSuccess) { cfail(e, "cudaSetDevice"); break; }
    const Brick& b = bricks[i];
    const int64_t idims[3] = {b.in.hi[0] - b.in.lo[0], b.in.hi[1] - b.in.lo[1], b.in.hi[2] - b.in.lo[2]};
    const int64_t cdims[3] = {b.core.hi[0] - b.core.lo[0], b.core.hi[1] - b.core.lo[1],
                              b.core.hi[2] - b.core.lo[2]};
    const size_t cvox = (size_t)(cdims[0] * cdims[1] * cdims[2]);
    if (faults.fail_copy()) { fail(HP_ERR_CUDA, "injected memcpy failure"); break; }
    if (in_pinned) {
      e = copy_box_async(x.din, idims, b.in.lo, in->data, n, vol_lo, b.in.lo, b.in.hi, ies,
                         cudaMemcpyHostToDevice, x.s);
    } else {
      host_copy_box(x.hin, in->data, ies, n, vol_lo, idims, b.in.lo, b.in.lo, b.in.hi);
      size_t bytes = ies * idims[0] * idims[1] * idims[2];
      e = cudaMemcpyAsync(x.din, x.hin, bytes, cudaMemcpyHostToDevice, x.s);
    }
    if (e != cudaSuccess) { cfail(e, "H2D copy"); break; }
    h2d += ies * (uint64_t)(idims[0] * idims[1] * idims[2]);
    Job job = brick_job(b, x.din, x.dout);
    job.scratch = x.dscr;
    job.scratch_bytes = max_scr;
    job.host_scratch = x.hscr;
    std::vector<void*> souts(nout);
    for (int k = 0; k < nout; ++k) souts[k] = (char*)x.dout + off[k];
    if ((st = op.launch(job, souts.data(), x.s)) != HP_OK) { if (rc == HP_OK) rc = st; break; }
    if (faults.fail_copy()) { fail(HP_ERR_CUDA, "injected memcpy failure"); break; }
    for (int k = 0; k < nout && e == cudaSuccess; ++k) {
      const size_t es = dtype_size(odt[k]);
      if (out_pinned)
        e = copy_box_async(outs[k]->data, n, vol_lo, souts[k], cdims, b.core.lo, b.core.lo,
                           b.core.hi, es, cudaMemcpyDeviceToHost, x.s);
      else
        e = cudaMemcpyAsync((char*)x.hout + off[k], souts[k], es * cvox, cudaMemcpyDeviceToHost, x.s);
      d2h += es * cvox;
    }
    if (e != cudaSuccess) { cfail(e, "D2H copy"); break; }
    if ((e = cudaEventRecord(x.ev, x.s)) != cudaSuccess) { cfail(e, "cudaEventRecord"); break; }
    x.brick = (int)i;
  }
  for (auto& x : sg) {
    if (rc == HP_OK) retire(x);
    else if (x.s) cudaStreamSynchronize(x.s);
  }
  // kernels whose bounded waits gave up leave a mark in their device's error word
  for (int k = 0; k < nslot && rc == HP_OK; ++k) {
    if (cudaSetDevice(devs[k]) != cudaSuccess) continue;
    int* ew = device_error_word();
    int hv = 0;
    if (ew && cudaMemcpy(&hv, ew, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess && hv) {
      cudaMemset(ew, 0, sizeof(int));
      rc = set_error(HP_ERR_TIMEOUT, "a device-side wait gave up");
    }
  }
  for (auto& x : sg) {
    cudaSetDevice(x.dev);
    if (x.ev) cudaEventDestroy(x.ev);
    if (x.s) cudaStreamDestroy(x.s);
    if (x.din) { cudaFree(x.din); track_free((int64_t)max_in); }
    if (x.dout) { cudaFree(x.dout); track_free((int64_t)out_stage); }
    if (x.dscr) { cudaFree(x.dscr); track_free((int64_t)max_scr); }
    if (x.hscr) cudaFreeHost(x.hscr);
    if (x.hin) cudaFreeHost(x.hin);
    if (x.hout) cudaFreeHost(x.hout);
  }
  cudaSetDevice(caller_dev);
  cudaError_t le = cudaGetLastError();
  if (rc == HP_OK && le != cudaSuccess) rc = cuda_fail(le, "executor");
  {
    std::lock_guard<std::mutex> lk(g_mu);
    g_stats.budget_bytes = budget;
    g_stats.bricks = bricks.size();
    g_stats.h2d_bytes = h2d;
    g_stats.d2h_bytes = d2h;
    g_stats.pinned_host_bytes = pinned;
    g_stats.wall_ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  return rc;
}

static Job whole_job(const hp_volume* in, hp_volume* out, int out_dtype) {
  Job j;
  const int64_t n[3] = {in->nz, in->ny, in->nx};
  j.in = DevBox{in->data, in->dtype, {0, 0, 0}, {n[0], n[1], n[2]}};
  j.out = DevOut{out->data, out_dtype, {0, 0, 0}, {n[0], n[1], n[2]}};
  for (int a = 0; a < 3; ++a) {
    j.gdims[a] = n[a];
    j.core_lo[a] = 0;
    j.core_hi[a] = n[a];
  }
  return j;
}

static int check_pair(const hp_volume* in, const hp_volume* out) {
  if (!in || !out) return set_error(HP_ERR_INVALID_ARG, "null volume");
  if (!in->data || !out->data) return set_error(HP_ERR_INVALID_ARG, "null data pointer");
  if (in->nx != out->nx || in->ny != out->ny || in->nz != out->nz)
    return set_error(HP_ERR_INVALID_ARG, "input and output extents differ");
  if (in->loc != out->loc) return set_error(HP_ERR_UNSUPPORTED, "mixed host/device locations");
  const char* a = (const char*)in->data;
  const char* b = (const char*)out->data;
  const size_t na = dtype_size(in->dtype) * (size_t)(in->nx * in->ny * in->nz);
  const size_t nb = dtype_size(out->dtype) * (size_t)(out->nx * out->ny * out->nz);
  if (a < b + nb && b < a + na) return set_error(HP_ERR_INVALID_ARG, "input and output alias");
  return HP_OK;
}

static void begin_call() {
  g_peak.store(g_live.load());
  std::lock_guard<std::mutex> lk(g_mu);
  g_stats.bricks = 0;
  g_stats.h2d_bytes = g_stats.d2h_bytes = 0;
  g_stats.pinned_host_bytes = 0;
  g_stats.wall_ms = 0;
}

// Device inputs whose rows the TMA kernels cannot address (a base that is
// not 16-byte aligned, or rows that are not a whole number of 16-byte words,
// e.g. 2052 uint16 samples) would take the kernels' element-load paths,
// 6-15x slower at 1024^3. Such an input is first copied, with rows padded to
// 16 bytes, into library scratch (k_pad_rows on the stream); the job's
// input box then describes the padded copy. The kernels never read the pad:
// every source x reflects into [0, nx). pad_bytes returns the bytes of the
// padded copy (0: none needed).
static int64_t padded_nx(int64_t nx) { return (nx + 15) / 16 * 16; }  // a 16-byte row for every dtype

static bool rows_aligned(const void* p, int64_t nx, size_t es) {
  return (uintptr_t)p % 16 == 0 && ((size_t)nx * es) % 16 == 0;
}

static size_t pad_bytes(const Op& op, const hp_volume* in) {
  const size_t es = dtype_size(in->dtype);
  if (!op.pad_rows || es == 0 || rows_aligned(in->data, in->nx, es)) return 0;
  return (size_t)padded_nx(in->nx) * es * (size_t)in->ny * (size_t)in->nz;
}

static int pad_device_input(Job& j, const hp_volume* in, Scratch& sc, size_t bytes,
                            cudaStream_t s) {
  void* p = nullptr;
  cudaError_t e = sc.alloc(&p, bytes);
  if (e != cudaSuccess) return cuda_fail(e, "padded input copy");
  const int64_t px = padded_nx(in->nx);
  e = launch_pad_rows(in->data, p, in->dtype, in->nx, px, in->ny * in->nz, s);
  if (e != cudaSuccess) return cuda_fail(e, "padded input copy");
  j.in.ptr = p;
  j.in.dims[2] = px;
  return HP_OK;
}

// Runs op on a device job: the input padding where needed, kernel scratch
// and the launch.
static int run_device(const Op& op, const hp_volume* in, hp_volume* const* outs, int nout,
                      cudaStream_t s) {
  Job j = whole_job(in, outs[0], op.out_dtype);
  Scratch sc(s);
  const size_t need = op.scratch_bytes ? op.scratch_bytes(j) : 0;
  const size_t padb = pad_bytes(op, in);
  if (need + padb > 0) {
    const int st = check_scratch_budget(need + padb);
    if (st != HP_OK) return st;
  }
  if (padb > 0) {
    const int st = pad_device_input(j, in, sc, padb, s);
    if (st != HP_OK) return st;
  }
  if (need > 0) {
    cudaError_t e = sc.alloc(&j.scratch, need);
    if (e != cudaSuccess) return cuda_fail(e, "kernel scratch");
    j.scratch_bytes = need;
  }
  std::vector<void*> ptrs(nout);
  for (int k = 0; k < nout; ++k) ptrs[k] = outs[k]->data;
  const int st = op.launch(j, ptrs.data(), s);
  if (st != HP_OK) return st;
  std::lock_guard<std::mutex> lk(g_mu);
  g_stats.bricks = 1;
  return HP_OK;
}

static int run_multi(const Op& op, const hp_volume* in, hp_volume* const* outs, void* stream) {
  begin_call();
  if (in->loc == HP_HOST) return run_host(op, in, outs);
  return run_device(op, in, outs, op.nout, (cudaStream_t)stream);
}

static int run(const Op& op, const hp_volume* in, hp_volume* out, void* stream) {
  begin_call();
  if (in->loc == HP_HOST) return run_host(op, in, &out);
  return run_device(op, in, &out, 1, (cudaStream_t)stream);
}

// Out-of-core filter bank (Sec. III-D applied to the bank): Z slabs whose
// input (halo = the largest radius) crosses the host link once for all the
// bank's outputs; each slab runs the bank kernels on its core planes.
int run_bank_host(const hp_volume* in, hp_volume* const* outs, const BankRequest& proto) {
  begin_call();
  int rmax = 0;
  for (auto& f : proto.filters) rmax = std::max(rmax, radius_of(f.second, 3.0));
  Op op;
  op.halo = rmax;
  op.out_dtype = proto.out_dtype;
  op.nout = (int)proto.filters.size();
  op.z_only = true;
  op.scratch_per_in_voxel = 1;  // bound of the work list (32 B per >= 256-voxel tile item)
  op.host_scratch = true;
  auto request = [proto](const Job& j) {
    BankRequest q = proto;
    q.in = j.in.ptr;
    q.in_z0 = j.in.lo[0];
    q.in_nz = j.in.dims[0];
    q.out_z0 = j.core_lo[0];
    hp_box core;
    for (int a = 0; a < 3; ++a) {
      core.lo[a] = j.core_lo[a];
      core.hi[a] = j.core_hi[a];
    }
    q.bricks.assign(1, core);
    return q;
  };
  op.scratch_bytes = [request](const Job& j) { return bank_worklist_bytes(request(j)); };
  op.launch = [request](const Job& j, void* const* souts, cudaStream_t s) {
    BankRequest q = request(j);
    for (size_t k = 0; k < q.outs.size(); ++k) q.outs[k] = souts[k];
    return run_filterbank_brick(q, j.scratch, j.host_scratch, j.scratch_bytes, s);
  };
  return run_host(op, in, outs);
}

}  // namespace hp

using namespace hp;

// ===================================================================== ABI
extern "C" {

const char* hp_last_error(void) { return t_msg.c_str(); }
const char* hp_version(void) { return "hp 0.1 (sm_103a)"; }

int hp_volume_create(hp_volume** out, void* data, hp_dtype dtype, hp_loc loc, int64_t nx,
                     int64_t ny, int64_t nz) {
  if (!out) return set_error(HP_ERR_INVALID_ARG, "null output handle");
  *out = nullptr;
  if (nx < 1 || ny < 1 || nz < 1) return set_error(HP_ERR_INVALID_ARG, "extents must be >= 1");
  if (dtype_size(dtype) == 0) return set_error(HP_ERR_INVALID_ARG, "unknown dtype");
  if (loc != HP_HOST && loc != HP_DEVICE) return set_error(HP_ERR_INVALID_ARG, "unknown location");
  hp_volume* v = new (std::nothrow) hp_volume;
  if (!v) return set_error(HP_ERR_OOM, "out of host memory");
  *v = hp_volume{data, (int)dtype, (int)loc, nx, ny, nz};
  *out = v;
  return HP_OK;
}

int hp_volume_destroy(hp_volume* v) {
  delete v;
  return HP_OK;
}

int hp_set_memory_budget(size_t bytes) {
  budget_setting();
  std::lock_guard<std::mutex> lk(g_mu);
  g_budget = bytes;
  return HP_OK;
}

int hp_get_memory_budget(size_t* bytes) {
  if (!bytes) return set_error(HP_ERR_INVALID_ARG, "null pointer");
  *bytes = budget_setting();
  return HP_OK;
}

int hp_gaussian3d(const hp_volume* in, hp_volume* out, double sigma, double truncate,
                  const int order[3], void* stream) {
  int st = check_pair(in, out);
  if (st != HP_OK) return st;
  if (!(sigma > 0) || !std::isfinite(sigma)) return set_error(HP_ERR_INVALID_ARG, "sigma must be > 0");
  if (truncate <= 0) truncate = 3.0;
  int ord[3] = {0, 0, 0};
  if (order)
    for (int a = 0; a < 3; ++a) {
      if (order[a] < 0 || order[a] > 2) return set_error(HP_ERR_INVALID_ARG, "order must be 0, 1 or 2");
      ord[a] = order[a];
    }
  if (out->dtype != HP_F32 && out->dtype != HP_F16)
    return set_error(HP_ERR_UNSUPPORTED, "Gaussian output dtype must be f32 or f16");
  auto taps = std::make_shared<Taps>();
  make_taps(sigma, truncate, ord, taps.get());
  if (taps->r > kMaxRGeneric)
    return set_error(HP_ERR_UNSUPPORTED, "radius " + std::to_string(taps->r) + " exceeds 32");
  Op op;
  op.halo = taps->r;
  op.out_dtype = out->dtype;
  const int r = taps->r;
  {
    Job probe = whole_job(in, out, out->dtype);
    if (gauss_scratch_bytes(probe, r) > 0) {
      op.scratch_per_in_voxel = 2 * sizeof(float);
      op.scratch_bytes = [r](const Job& j) { return gauss_scratch_bytes(j, r); };
    }
  }
  op.launch = [taps](const Job& j, void* const*, cudaStream_t s) { return launched(launch_gauss(j, *taps, s)); };
  return run(op, in, out, stream);
}

static int morph(const hp_volume* in, hp_volume* out, hp_se se, int radius, void* stream,
                 int dil) {
  int st = check_pair(in, out);
  if (st != HP_OK) return st;
  if (in->dtype != out->dtype) return set_error(HP_ERR_UNSUPPORTED, "morphology output dtype must equal input dtype");
  if (se != HP_SE_CUBE && se != HP_SE_BALL) return set_error(HP_ERR_INVALID_ARG, "unknown structuring element");
  if (radius < 0 || radius > kMaxMorphR) return set_error(HP_ERR_INVALID_ARG, "radius must be in [0, 16]");
  Op op;
  op.halo = radius;
  op.out_dtype = out->dtype;
  if (morph_scratch_bytes(whole_job(in, out, out->dtype), (int)se, radius) > 0) {
    op.scratch_per_in_voxel = 8;
    op.scratch_bytes = [se, radius](const Job& j) { return morph_scratch_bytes(j, (int)se, radius); };
  }
  op.launch = [se, radius, dil](const Job& j, void* const*, cudaStream_t s) {
    return launched(launch_morph(j, (int)se, radius, dil, s));
  };
  return run(op, in, out, stream);
}

int hp_erode3d(const hp_volume* in, hp_volume* out, hp_se se, int radius, void* stream) {
  return morph(in, out, se, radius, stream, 0);
}

int hp_dilate3d(const hp_volume* in, hp_volume* out, hp_se se, int radius, void* stream) {
  return morph(in, out, se, radius, stream, 1);
}

int hp_threshold3d(const hp_volume* in, hp_volume* out, double t, void* stream) {
  int st = check_pair(in, out);
  if (st != HP_OK) return st;
  if (out->dtype != HP_U8) return set_error(HP_ERR_UNSUPPORTED, "threshold output dtype must be u8");
  if (std::isnan(t)) return set_error(HP_ERR_INVALID_ARG, "threshold must not be NaN");
  Op op;
  op.halo = 0;
  op.out_dtype = HP_U8;
  op.pad_rows = false;  // an elementwise comparison: no staging to gain from
  op.launch = [t](const Job& j, void* const*, cudaStream_t s) { return launched(launch_threshold(j, t, s)); };
  return run(op, in, out, stream);
}

int hp_threshold_box3d(const hp_volume* in, hp_volume* out, int method, int radius, double k,
                       double c, void* stream) {
  int st = check_pair(in, out);
  if (st != HP_OK) return st;
  if (out->dtype != HP_U8) return set_error(HP_ERR_UNSUPPORTED, "local threshold output dtype must be u8");
  if (method < HP_LOCAL_MEAN || method > HP_LOCAL_SAUVOLA)
    return set_error(HP_ERR_INVALID_ARG, "unknown local threshold method");
  if (radius < 0 || radius > 15) return set_error(HP_ERR_INVALID_ARG, "radius must be in [0, 15]");
  if (!std::isfinite(k) || !std::isfinite(c)) return set_error(HP_ERR_INVALID_ARG, "k and c must be finite");
  if (method == HP_LOCAL_SAUVOLA && !(c > 0)) return set_error(HP_ERR_INVALID_ARG, "Sauvola needs c = R > 0");
  Op op;
  op.halo = radius;
  op.out_dtype = HP_U8;
  const bool fp = in->dtype == HP_F16 || in->dtype == HP_F32;
  op.scratch_per_in_voxel = fp ? 32 : 24;
  op.scratch_bytes = [radius](const Job& j) { return box_scratch_bytes(j, radius); };
  op.launch = [method, radius, k, c](const Job& j, void* const*, cudaStream_t s) {
    return launched(launch_threshold_box(j, method, radius, k, c, s));
  };
  return run(op, in, out, stream);
}

int hp_hessian3d(const hp_volume* in, hp_volume* const* outs, int what, double sigma,
                 void* stream) {
  if (what != HP_HESSIAN_COMPONENTS && what != HP_HESSIAN_EIGENVALUES)
    return set_error(HP_ERR_INVALID_ARG, "what must be HP_HESSIAN_COMPONENTS or HP_HESSIAN_EIGENVALUES");
  const int nout = what == HP_HESSIAN_COMPONENTS ? 6 : 3;
  if (!outs) return set_error(HP_ERR_INVALID_ARG, "null outputs");
  for (int k = 0; k < nout; ++k) {
    int st = check_pair(in, outs[k]);
    if (st != HP_OK) return st;
    if (outs[k]->dtype != HP_F32 && outs[k]->dtype != HP_F16)
      return set_error(HP_ERR_UNSUPPORTED, "Hessian outputs must be f32 or f16");
    if (outs[k]->dtype != outs[0]->dtype)
      return set_error(HP_ERR_UNSUPPORTED, "Hessian outputs must share one dtype");
  }
  if (!(sigma > 0) || !std::isfinite(sigma)) return set_error(HP_ERR_INVALID_ARG, "sigma must be > 0");
  const int r = radius_of(sigma, 3.0);
  if (r > kMaxRGeneric) return set_error(HP_ERR_UNSUPPORTED, "radius exceeds 32");
  static const int kOrders[6][3] = {{2, 0, 0}, {0, 2, 0}, {0, 0, 2}, {1, 1, 0}, {1, 0, 1}, {0, 1, 1}};
  auto taps = std::make_shared<std::vector<Taps>>(6);
  for (int k = 0; k < 6; ++k) make_taps(sigma, 3.0, kOrders[k], &(*taps)[k]);
  const bool eig = what == HP_HESSIAN_EIGENVALUES;
  Op op;
  op.halo = r;
  op.out_dtype = outs[0]->dtype;
  op.nout = nout;
  Job probe = whole_job(in, outs[0], outs[0]->dtype);
  const bool gen = gauss_scratch_bytes(probe, r) > 0;
  op.scratch_per_in_voxel = (eig ? 24 : 0) + (gen ? 8 : 0);
  auto core_voxels = [](const Job& j) {
    return (j.core_hi[0] - j.core_lo[0]) * (j.core_hi[1] - j.core_lo[1]) * (j.core_hi[2] - j.core_lo[2]);
  };
  if (op.scratch_per_in_voxel > 0)
    op.scratch_bytes = [eig, r, core_voxels](const Job& j) {
      return (eig ? hessian_eig_scratch(core_voxels(j)) : 0) + gauss_scratch_bytes(j, r);
    };
  op.launch = [taps, eig, core_voxels](const Job& j, void* const* o, cudaStream_t s) -> int {
    const int64_t nv = core_voxels(j);
    const size_t comp_bytes = eig ? hessian_eig_scratch(nv) : 0;
    float* comps = static_cast<float*>(j.scratch);
    for (int k = 0; k < 6; ++k) {
      Job jk = j;
      if (eig) {
        jk.out.ptr = comps + (size_t)k * nv;
        jk.out.dtype = HP_F32;
      } else {
        jk.out.ptr = o[k];
      }
      // generic-path scratch after the components
      jk.scratch = j.scratch ? static_cast<char*>(j.scratch) + comp_bytes : nullptr;
      jk.scratch_bytes = j.scratch_bytes - comp_bytes;
      const cudaError_t e = launch_gauss(jk, (*taps)[k], s);
      if (e != cudaSuccess) return cuda_fail(e, "Hessian component launch");
    }
    if (eig) return launched(launch_hessian_eig(comps, nv, o, j.out.dtype, s));
    return HP_OK;
  };
  return run_multi(op, in, outs, stream);
}

int hp_multi3d(const hp_volume* in, hp_volume* const* outs, const hp_op* ops, int n,
               void* stream) {
  if (!in || !outs || !ops || n < 1 || n > 64)
    return set_error(HP_ERR_INVALID_ARG, "multi: null argument or n outside [1, 64]");
  auto taps = std::make_shared<std::vector<Taps>>(n);
  std::vector<int> odt(n);
  int halo = 0;
  bool scratch = false;
  for (int k = 0; k < n; ++k) {
    int st = check_pair(in, outs[k]);
    if (st != HP_OK) return st;
    const hp_op& q = ops[k];
    odt[k] = outs[k]->dtype;
    if (q.kind == HP_OP_GAUSSIAN) {
      if (!(q.sigma > 0) || !std::isfinite(q.sigma)) return set_error(HP_ERR_INVALID_ARG, "multi: sigma must be > 0");
      for (int a = 0; a < 3; ++a)
        if (q.order[a] < 0 || q.order[a] > 2) return set_error(HP_ERR_INVALID_ARG, "multi: order must be 0, 1 or 2");
      if (odt[k] != HP_F32 && odt[k] != HP_F16)
        return set_error(HP_ERR_UNSUPPORTED, "multi: Gaussian outputs must be f32 or f16");
      make_taps(q.sigma, 3.0, q.order, &(*taps)[k]);
      if ((*taps)[k].r > kMaxRGeneric) return set_error(HP_ERR_UNSUPPORTED, "multi: radius exceeds 32");
      halo = std::max(halo, (*taps)[k].r);
      scratch = scratch || gauss_scratch_bytes(whole_job(in, outs[k], odt[k]), (*taps)[k].r) > 0;
    } else if (q.kind == HP_OP_ERODE || q.kind == HP_OP_DILATE) {
      if (q.se != HP_SE_CUBE && q.se != HP_SE_BALL) return set_error(HP_ERR_INVALID_ARG, "multi: unknown structuring element");
      if (q.radius < 0 || q.radius > kMaxMorphR) return set_error(HP_ERR_INVALID_ARG, "multi: radius must be in [0, 16]");
      if (odt[k] != in->dtype) return set_error(HP_ERR_UNSUPPORTED, "multi: morphology output dtype must equal the input's");
      halo = std::max(halo, q.radius);
      scratch = scratch || morph_scratch_bytes(whole_job(in, outs[k], odt[k]), q.se, q.radius) > 0;
    } else {
      return set_error(HP_ERR_INVALID_ARG, "multi: unknown op kind");
    }
  }
  auto opsv = std::make_shared<std::vector<hp_op>>(ops, ops + n);
  Op op;
  op.halo = halo;
  op.out_dtype = odt[0];
  op.out_dtypes = odt;
  op.nout = n;
  if (scratch) {
    op.scratch_per_in_voxel = 8;
    op.scratch_bytes = [opsv, taps](const Job& j) {
      size_t m = 0;
      for (size_t k = 0; k < opsv->size(); ++k) {
        const hp_op& q = (*opsv)[k];
        m = std::max(m, q.kind == HP_OP_GAUSSIAN ? gauss_scratch_bytes(j, (*taps)[k].r)
                                                 : morph_scratch_bytes(j, q.se, q.radius));
      }
      return m;
    };
  }
  op.launch = [opsv, taps, odt](const Job& j, void* const* o, cudaStream_t s) -> int {
    for (size_t k = 0; k < opsv->size(); ++k) {
      const hp_op& q = (*opsv)[k];
      Job jk = j;
      jk.out.ptr = o[k];
      jk.out.dtype = odt[k];
      const cudaError_t e = q.kind == HP_OP_GAUSSIAN
                                ? launch_gauss(jk, (*taps)[k], s)
                                : launch_morph(jk, q.se, q.radius, q.kind == HP_OP_DILATE, s);
      if (e != cudaSuccess) return cuda_fail(e, "multi: kernel launch");
    }
    return HP_OK;
  };
  return run_multi(op, in, outs, stream);
}

int hp_set_devices(const int* devices, int n) {
  if (n < 0 || (n > 0 && !devices)) return set_error(HP_ERR_INVALID_ARG, "bad device list");
  int count = 0;
  cudaError_t e = cudaGetDeviceCount(&count);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
  for (int i = 0; i < n; ++i)
    if (devices[i] < 0 || devices[i] >= count)
      return set_error(HP_ERR_INVALID_ARG, "device " + std::to_string(devices[i]) + " does not exist");
  std::lock_guard<std::mutex> lk(g_mu);
  g_devices.assign(devices, devices + n);
  return HP_OK;
}

int hp_get_devices(int* devices, int max_n, int* n) {
  if (!n) return set_error(HP_ERR_INVALID_ARG, "null count");
  std::lock_guard<std::mutex> lk(g_mu);
  *n = (int)g_devices.size();
  for (int i = 0; i < *n && i < max_n; ++i)
    if (devices) devices[i] = g_devices[i];
  return HP_OK;
}

int hp_set_brick_shard(int rank, int world) {
  if (world < 1 || rank < 0 || rank >= world)
    return set_error(HP_ERR_INVALID_ARG, "shard needs 0 <= rank < world");
  std::lock_guard<std::mutex> lk(g_mu);
  g_shard_rank = rank;
  g_shard_world = world;
  return HP_OK;
}

int hp_plan_bricks(int64_t nx, int64_t ny, int64_t nz, int halo, size_t in_bytes,
                   size_t out_bytes, size_t budget, int stages, int min_bricks, hp_box* cores,
                   hp_box* in_boxes, int max_bricks, int* nbricks) {
  if (!nbricks) return set_error(HP_ERR_INVALID_ARG, "null nbricks");
  const int64_t n[3] = {nz, ny, nx};
  std::vector<Brick> b;
  int st = plan(n, halo, in_bytes, out_bytes, 0, budget, stages, min_bricks, false, &b);
  if (st != HP_OK) return st;
  *nbricks = (int)b.size();
  for (int i = 0; i < (int)b.size() && i < max_bricks; ++i) {
    if (cores) cores[i] = b[i].core;
    if (in_boxes) in_boxes[i] = b[i].in;
  }
  return HP_OK;
}

int hp_selftest_wait_timeout(void* stream) {
  int* ew = device_error_word();
  if (!ew) return set_error(HP_ERR_CUDA, "no device error word");
  k_wait_selftest<<<1, 32, 0, (cudaStream_t)stream>>>(ew);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "wait self-test launch");
  return HP_OK;
}

int hp_stream_status(void* stream) {
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  int* ew = device_error_word();
  if (!ew) return set_error(HP_ERR_CUDA, "no device error word");
  int hv = 0;
  e = cudaMemcpy(&hv, ew, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "read device error word");
  if (hv) {
    cudaMemset(ew, 0, sizeof(int));
    return set_error(HP_ERR_TIMEOUT, "a device-side wait gave up");
  }
  return HP_OK;
}

int hp_get_stats(hp_stats* s) {
  if (!s) return set_error(HP_ERR_INVALID_ARG, "null pointer");
  std::lock_guard<std::mutex> lk(g_mu);
  *s = g_stats;
  s->live_device_bytes = (size_t)std::max<int64_t>(0, g_live.load());
  s->peak_device_bytes = (size_t)std::max<int64_t>(0, g_peak.load());
  s->cached_device_bytes = (size_t)std::max<int64_t>(0, bank_cache_bytes());
  s->bank_kernels = (uint64_t)bank_last_kernels();
  return HP_OK;
}

}  // extern "C"
