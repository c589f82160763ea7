// Internal declarations shared by the C ABI layer, the planner, the
// executor and the kernel launchers of libhp.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <string>
#include <utility>
#include <vector>

#include "hp.h"

// The opaque volume view of the C ABI (hp.h): a non-owning pointer to a
// dense C-order volume with its dtype, location and extents.
struct hp_volume {
  void* data;
  int dtype;
  int loc;
  int64_t nx, ny, nz;
};

namespace hp {

constexpr int kMaxR = 12;        // largest radius with a tiled z-march kernel
constexpr int kMaxRGeneric = 32; // largest radius overall (generic kernel)
constexpr int kMaxTaps = 2 * kMaxRGeneric + 1;
constexpr int kMaxMorphR = 16;

// Reflect (half-sample symmetric) index, valid for any i and n >= 1. The
// in-range and single-fold cases avoid the 64-bit remainder.
__host__ __device__ inline int64_t reflect(int64_t i, int64_t n) {
  if (i >= 0 && i < n) return i;
  if (i < 0 && i >= -n) return -1 - i;
  if (i >= n && i < 2 * n) return 2 * n - 1 - i;
  int64_t p = 2 * n;
  int64_t m = i % p;
  if (m < 0) m += p;
  return m < n ? m : p - 1 - m;
}

inline size_t dtype_size(int dt) {
  switch (dt) {
    case HP_U8: return 1;
    case HP_U16: case HP_F16: return 2;
    case HP_F32: return 4;
    default: return 0;
  }
}

// A dense box of a global volume held in device memory: element (z, y, x)
// of the global volume lives at ptr[((z-lo0)*d1 + (y-lo1))*d2 + (x-lo2)].
struct DevBox {
  const void* ptr;
  int dtype;
  int64_t lo[3];
  int64_t dims[3];
};

struct DevOut {
  void* ptr;
  int dtype;
  int64_t lo[3];
  int64_t dims[3];
};

// One filtering job over a core box of the global volume. `scratch` is
// device memory the caller provides for kernels that need it (the generic
// Gaussian path: gauss_scratch_bytes); launchers never allocate.
struct Job {
  DevBox in;
  DevOut out;
  int64_t gdims[3];
  int64_t core_lo[3];
  int64_t core_hi[3];
  void* scratch = nullptr;
  size_t scratch_bytes = 0;
  void* host_scratch = nullptr;  // page-locked, scratch_bytes long (host-mode bricks only)
};

// FP32 taps per axis (z, y, x), index k + r for k in [-r, r].
struct Taps {
  int r;
  float w[3][kMaxTaps];
};

// Kernel-weight generation (FP64, rounded once to FP32).
int radius_of(double sigma, double truncate);
void make_taps(double sigma, double truncate, const int order[3], Taps* t);
void taps1d_f64(double sigma, int r, int order, double* w);

// Device-side error word (per device), set by bounded waits that give up.
int* device_error_word();

// Hessian eigenvalue epilogue: comps = six dense FP32 volumes of n voxels
// (Dzz, Dyy, Dxx, Dzy, Dzx, Dyx) one after another; outs[0..2] = ascending
// eigenvalues in out_dtype.
size_t hessian_eig_scratch(int64_t core_voxels);
cudaError_t launch_hessian_eig(const float* comps, int64_t n, void* const* outs, int out_dtype,
                               cudaStream_t s);
// Box-window local threshold (mean / Niblack / Sauvola) of a job: window
// sums through job.scratch (box_scratch_bytes), decision into job.out (u8).
size_t box_scratch_bytes(const Job& job, int w);
cudaError_t launch_threshold_box(const Job& job, int method, int w, double k, double c,
                                 cudaStream_t s);

// Regions of a separable three-pass job of radius r (Gaussian generic path,
// box sums): after the x pass, z and y cover the hull of the reflected
// sources of the core grown by r (from rlo) and x the core; after the y
// pass, z as before and y, x the core.
struct SepRegions {
  int64_t rlo[2];
  int64_t n_x[3], n_y[3];
};
SepRegions sep_regions(const Job& job, int r);

// Launchers (enqueue only). Return a cudaError_t.
// Scratch bytes launch_gauss needs in job.scratch for radius r (nonzero only
// on the generic three-pass path: r > kMaxR, r = 0, or a volume thinner than
// r in x or y); at most 8 bytes per voxel of the job's input box.
size_t gauss_scratch_bytes(const Job& job, int r);
cudaError_t launch_gauss(const Job& job, const Taps& taps, cudaStream_t s);
cudaError_t launch_gauss_zr(const Job& job, const Taps& taps, cudaStream_t s);
cudaError_t launch_morph(const Job& job, int se, int rad, int is_dilate, cudaStream_t s);
// Scratch bytes launch_morph needs in job.scratch: the van Herk / Gil-Werman
// cube passes (radii above the tiled kernels' limit, or volumes thinner than
// the radius) keep two key regions (sep_regions), 8 bytes per input voxel at
// most; 0 on the other paths.
size_t morph_scratch_bytes(const Job& job, int se, int rad);
cudaError_t launch_morph16(const Job& job, int se, int rad, int is_dilate, cudaStream_t s);
cudaError_t launch_threshold(const Job& job, double t, cudaStream_t s);

// Error reporting (thread-local message).
int set_error(int status, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);

// TMA tensor map over a dense 3D box (x, y, z extents), box (bw, bh, bd).
// Returns false when the layout does not meet TMA rules.
bool make_tmap_3d(CUtensorMap* map, const void* base, int dtype, const int64_t dims[3], int bw,
                  int bh, int bd = 1);

int num_sms();

// Copy `rows` dense rows of n elements of dtype into rows of `pitch`
// elements at dst (16-byte aligned; pitch * element size a multiple of 16),
// the elements past n zero; on stream s.
cudaError_t launch_pad_rows(const void* src, void* dst, int dtype, int64_t n, int64_t pitch,
                            int64_t rows, cudaStream_t s);

// out[i] = in[i] - out[i] over n elements of dtype (FP32 difference rounded
// to the dtype), on stream s.
cudaError_t launch_difference(const void* in, void* out, int dtype, int64_t n, cudaStream_t s);

// g[i] = fma(amount, f[i] - g[i], f[i]) over n elements (f of dtype, g f32),
// on stream s.
cudaError_t launch_unsharp(const void* f, int dtype, float* g, float amount, int64_t n, cudaStream_t s);

// out[i] = f[i] > m[i] - offset (FP32 comparison), over n elements.
cudaError_t launch_local_threshold(const void* f, int dtype, const float* m, float offset,
                                   uint8_t* out, int64_t n, cudaStream_t s);

// Largest dynamic shared memory a block may opt into on the current device,
// less 1 KB for the kernels' static shared variables.
int max_dyn_smem();

// Shared memory of one SM on the current device (all resident CTAs).
int max_smem_per_sm();

// z-chunk length for a z-march grid of `tiles` columns: CTAs run in waves
// of `slots` (resident CTAs on the whole GPU) and each costs about its
// planes plus `halo`; returns the multiple of `align` that minimises
// waves x (chunk + halo).
int64_t pick_zchunk(int64_t cz, int64_t tiles, int64_t slots, int halo, int align);

// A filter-bank request: the input and each output are whole x/y planes of
// the volume G, starting at planes in_z0 / out_z0 (0: the whole volume);
// the work list covers `bricks` (core boxes in global coordinates).
struct BankRequest {
  const void* in;
  int dtype, out_dtype;
  int64_t G[3];
  std::vector<std::pair<int, double>> filters;  // (kind, sigma)
  std::vector<void*> outs;
  std::vector<hp_box> bricks;
  int64_t in_z0 = 0, in_nz = 0, out_z0 = 0;  // in_nz = 0: the whole volume
};
// Device-mode bank: autotuned, cached, CUDA-graph launch.
int run_filterbank(const BankRequest& q, cudaStream_t s);
// Out-of-core brick: work list in caller device memory wl, staged through
// the caller's page-locked hwl, both bank_worklist_bytes(q) long; no graph.
size_t bank_worklist_bytes(const BankRequest& q);
int run_filterbank_brick(const BankRequest& q, void* wl, void* hwl, size_t wl_bytes, cudaStream_t s);
// Host-mode (out-of-core) bank over Z slabs; outs are host volumes.
int run_bank_host(const hp_volume* in, hp_volume* const* outs, const BankRequest& proto);

// HP_LOG >= 1 prints the kernel path chosen for each launch to stderr.
int log_level();

// Library device-byte counters (hp_stats): bytes > 0 on allocation, < 0 on
// release.
void note_scratch(int64_t bytes);
size_t budget_setting();
// HP_OK when `need` bytes fit the effective budget (the user value, or 0.8 x
// free device memory), else HP_ERR_BUDGET with a message.
int check_scratch_budget(size_t need);

// Stream-ordered scratch of device-mode calls, counted in the library's
// device-byte statistics and released in stream order when it goes out of
// scope.
struct Scratch {
  cudaStream_t s;
  std::vector<std::pair<void*, size_t>> bufs;
  explicit Scratch(cudaStream_t st) : s(st) {}
  Scratch(const Scratch&) = delete;
  Scratch& operator=(const Scratch&) = delete;
  cudaError_t alloc(void** p, size_t bytes) {
    cudaError_t e = cudaMallocAsync(p, bytes, s);
    if (e == cudaSuccess) {
      bufs.push_back({*p, bytes});
      note_scratch((int64_t)bytes);
    }
    return e;
  }
  ~Scratch() {
    for (auto& b : bufs) {
      cudaFreeAsync(b.first, s);
      note_scratch(-(int64_t)b.second);
    }
  }
};

}  // namespace hp
