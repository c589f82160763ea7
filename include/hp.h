/*
 * hp.h -- C ABI of the B300-native chunked 3D filtering library (libhp).
 *
 * The operations are the filtering core of the Harpia library described in
 * "Advancing Annotat3D with Harpia" (arXiv 2511.11890):
 *   - Sec. III-C lists the filters: Gaussian smoothing, "Hessian" texture
 *     features (here: Gaussian gradient magnitude and Laplacian of
 *     Gaussian), erosion, dilation and thresholds.
 *   - Sec. III-D gives the execution model: query free device memory and
 *     reserve a fixed fraction (step 1), size chunks including padding
 *     (step 2), and process overlapping, context-preserving chunks one by
 *     one (step 3).
 *   - Sec. IV-C fixes the memory contract: the library allocates and frees
 *     its own device memory and never hands library-owned device memory to
 *     the caller.
 * The paper prints no formulas. The conventions used by every call:
 *   - Volumes are dense, C order, f[z][y][x] with x fastest.
 *   - Reflect boundary, half-sample symmetric (d c b a | a b c d).
 *   - Gaussian radius r = floor(truncate * sigma + 0.5); taps are the
 *     normalised sampled Gaussian g0 and its analytic derivatives
 *     g1 = -k/sigma^2 g0, g2 = (k^2/sigma^4 - 1/sigma^2) g0 (not
 *     re-normalised); a 1D filter is the convolution y[i] = sum_k g(k) x[i-k].
 *   - Arithmetic is FP32 with FP32 accumulation; taps are generated and
 *     normalised in FP64 and rounded once to FP32.
 *   - Erosion takes the min over the structuring element B of f(p + o),
 *     dilation the max of f(p - o); B is a cube of half-width radius or the
 *     digital ball dz^2 + dy^2 + dx^2 <= radius^2. Morphology is exact and
 *     orders floating-point values by IEEE 754 totalOrder (-0 < +0; a NaN
 *     with the sign bit clear above +inf, with it set below -inf).
 *
 * Execution mode follows where the volumes live:
 *   - HP_DEVICE in and out: the data stays in device memory. The call
 *     enqueues its kernels on `stream` (a cudaStream_t; NULL = legacy
 *     default stream) and returns without synchronising. Use
 *     hp_stream_status() to collect asynchronous failures.
 *   - HP_HOST in and out: out-of-core. The volume is cut into halo-padded
 *     bricks sized to the memory budget and streamed through the device on
 *     several CUDA streams. The call is synchronous. Host buffers that are
 *     page-locked (cudaHostAlloc / cudaHostRegister, torch pin_memory) are
 *     copied directly; other host buffers go through a pinned staging ring.
 *     `stream` is ignored.
 *   - Mixed locations return HP_ERR_UNSUPPORTED.
 *
 * Ownership: hp_volume is a non-owning view of caller memory. The caller
 * keeps the memory alive and unchanged until the call (device mode: the
 * enqueued work) completes. Every library-internal buffer is released
 * before a host-mode call returns and, in device mode, freed in stream order
 * on `stream`. The only memory kept across calls is the small cache of
 * filter-bank launch plans (see hp_release_cache).
 *
 * Errors: every call returns an hp_status. On failure hp_last_error()
 * returns a thread-local message; outputs are then unspecified. Input and
 * output must not alias.
 */
#ifndef HP_H
#define HP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HP_OK = 0,
  HP_ERR_INVALID_ARG = 1, /* null pointer, bad dims, aliasing, bad sigma/radius */
  HP_ERR_UNSUPPORTED = 2, /* dtype / structuring element / location combination */
  HP_ERR_BUDGET = 3,      /* smallest legal brick does not fit the memory budget */
  HP_ERR_OOM = 4,         /* device or pinned host allocation failed */
  HP_ERR_CUDA = 5,        /* a CUDA runtime call failed */
  HP_ERR_TIMEOUT = 6,     /* a bounded device-side wait gave up */
  HP_ERR_INTERNAL = 7
} hp_status;

typedef enum { HP_U8 = 0, HP_U16 = 1, HP_F16 = 2, HP_F32 = 3 } hp_dtype;
typedef enum { HP_HOST = 0, HP_DEVICE = 1 } hp_loc;
typedef enum { HP_SE_CUBE = 0, HP_SE_BALL = 1 } hp_se;
typedef enum { HP_FILTER_G = 0, HP_FILTER_GM = 1, HP_FILTER_LOG = 2 } hp_filter_kind;
typedef enum { HP_LOCAL_MEAN = 0, HP_LOCAL_NIBLACK = 1, HP_LOCAL_SAUVOLA = 2 } hp_local_method;
typedef enum { HP_HESSIAN_COMPONENTS = 0, HP_HESSIAN_EIGENVALUES = 1 } hp_hessian_output;

/* Opaque, non-owning view of a dense C-order volume. */
typedef struct hp_volume hp_volume;

/* One output of a filter bank: kind = hp_filter_kind, sigma > 0.
 * G = Gaussian; GM = sqrt(Dx^2 + Dy^2 + Dz^2) with D_a the first Gaussian
 * derivative along axis a; LOG = Dxx + Dyy + Dzz. */
typedef struct {
  int kind;
  double sigma;
} hp_filter;

/* Half-open box [lo, hi) in (z, y, x) order. */
typedef struct {
  int64_t lo[3];
  int64_t hi[3];
} hp_box;

/* Library counters. Sizes in bytes; times in milliseconds. */
typedef struct {
  size_t budget_bytes;        /* effective budget used by the last host-mode call */
  size_t peak_device_bytes;   /* peak library-owned device bytes during the last call */
  size_t live_device_bytes;   /* library-owned device bytes now (excluding plan cache) */
  size_t cached_device_bytes; /* device bytes held by cached filter-bank plans */
  size_t pinned_host_bytes;   /* pinned staging bytes allocated by the last call */
  uint64_t bricks;            /* bricks executed by the last call */
  uint64_t h2d_bytes;         /* host-to-device bytes of the last call */
  uint64_t d2h_bytes;         /* device-to-host bytes of the last call */
  double wall_ms;             /* wall time of the last host-mode call */
  uint64_t bank_kernels;      /* kernels one launch of the last filter-bank plan runs (1 or 2) */
} hp_stats;

/* Create a view of `data` (dtype, location) with extents nx (fastest), ny,
 * nz, each >= 1. `data` may be NULL only if the view is never used as an
 * input or output. Returns HP_ERR_INVALID_ARG on bad extents. */
int hp_volume_create(hp_volume** out, void* data, hp_dtype dtype, hp_loc loc, int64_t nx,
                     int64_t ny, int64_t nz);
/* Destroy a view (never frees `data`). NULL is accepted. */
int hp_volume_destroy(hp_volume* v);

/* Device-memory budget for library-owned buffers (Sec. III-D step 1).
 * bytes = 0 selects the default: 0.8 x the free device memory reported by
 * cudaMemGetInfo at the start of each call. Process-wide and thread-safe.
 * The environment variable HP_BUDGET (bytes) sets the initial value. */
int hp_set_memory_budget(size_t bytes);
int hp_get_memory_budget(size_t* bytes);

/* Separable Gaussian or derivative-of-Gaussian filter (Sec. III-C, Gaussian
 * smoothing and derivative features). order = {oz, oy, ox}, each in
 * {0, 1, 2}; NULL means {0, 0, 0}. truncate <= 0 selects 3.0. Input dtype
 * u8/u16/f16/f32; output dtype f32 or f16 (rounded to nearest even once).
 * Radius up to 32. Radii above 12 (and volumes thinner than the radius in x
 * or y) take a three-pass path with two FP32 scratch volumes (at most 8
 * bytes per voxel of the input, or of each brick's input box out of core),
 * counted against the memory budget. */
int hp_gaussian3d(const hp_volume* in, hp_volume* out, double sigma, double truncate,
                  const int order[3], void* stream);

/* Multi-sigma filter bank: n outputs, outs[i] holds filter f[i]. All outputs
 * have the input's extents, its location, and one dtype, f16 or f32.
 * truncate is 3.0; radii 1..12; at most 8 distinct sigmas; each
 * (kind, sigma) at most once.
 *   - Device mode runs one persistent, CUDA-graph-captured launch over a
 *     work list of (brick, tile, sigma) items; the launch plan (graph + work
 *     list) is cached per shape, filter set, brick set and buffer addresses.
 *   - Host mode (Sec. III-D) streams Z slabs (halo = the largest radius)
 *     through the device under the memory budget: each slab's input crosses
 *     the host link once for all n outputs, and the bank kernels run on it
 *     with a per-slab work list (no graph, nothing cached). Results equal
 *     device mode bit for bit. HP_ERR_BUDGET when one plane with its halo
 *     and outputs does not fit. */
int hp_filterbank3d(const hp_volume* in, hp_volume* const* outs, const hp_filter* f, int n,
                    void* stream);
/* As hp_filterbank3d, with the work list built over the given bricks
 * (disjoint boxes covering the volume; halos are read from neighbouring
 * bricks, so the result equals the whole-volume result bit for bit).
 * Device mode only. */
int hp_filterbank3d_bricks(const hp_volume* in, hp_volume* const* outs, const hp_filter* f, int n,
                           const hp_box* bricks, int nbricks, void* stream);

/* Several filters of one volume in one pass (Sec. III-D applied to a set
 * of filters): out k holds op k. Host volumes run out of core with one
 * brick plan for all ops (halo = the largest radius): each brick's input
 * crosses the host link once and every op runs on it; device volumes run
 * the ops one after another on `stream`. Results equal the single-op calls
 * bit for bit.
 *   HP_OP_GAUSSIAN: as hp_gaussian3d (sigma, order {oz, oy, ox}, truncate
 *     3); output f32 or f16.
 *   HP_OP_ERODE / HP_OP_DILATE: as hp_erode3d / hp_dilate3d (se, radius);
 *     output dtype = input dtype.
 * 1 <= n <= 64; every output has the input's extents and location. */
typedef enum { HP_OP_GAUSSIAN = 0, HP_OP_ERODE = 1, HP_OP_DILATE = 2 } hp_op_kind;
typedef struct {
  int kind;     /* hp_op_kind */
  double sigma; /* Gaussian: sigma > 0 */
  int order[3]; /* Gaussian: derivative orders (z, y, x), each 0..2 */
  int se;       /* morphology: hp_se */
  int radius;   /* morphology: 0..16 */
} hp_op;
int hp_multi3d(const hp_volume* in, hp_volume* const* outs, const hp_op* ops, int n,
               void* stream);

/* Grayscale erosion / dilation with a cube (half-width radius) or ball
 * (radius) structuring element (Sec. III-C, label-editing morphology).
 * Output dtype equals input dtype; results are exact. radius in [0, 16]. */
int hp_erode3d(const hp_volume* in, hp_volume* out, hp_se se, int radius, void* stream);
int hp_dilate3d(const hp_volume* in, hp_volume* out, hp_se se, int radius, void* stream);

/* Opening (erosion, then dilation), closing (dilation, then erosion) and
 * white top-hat (in - opening) with the same structuring elements and
 * reflect boundaries as hp_erode3d / hp_dilate3d (Sec. III-C, label-editing
 * morphology: compositions of the two). Device volumes only (in and out on
 * the device, out may not alias in); the intermediate volume is library
 * scratch, allocated and freed on `stream`. Output dtype equals input dtype;
 * results are exact (the top-hat difference is taken in FP32 and rounded to
 * the dtype). HP_ERR_UNSUPPORTED for host volumes, HP_ERR_BUDGET when the
 * scratch volume exceeds the memory budget. */
int hp_open3d(const hp_volume* in, hp_volume* out, hp_se se, int radius, void* stream);
int hp_close3d(const hp_volume* in, hp_volume* out, hp_se se, int radius, void* stream);
int hp_tophat3d(const hp_volume* in, hp_volume* out, hp_se se, int radius, void* stream);

/* Unsharp mask (Sec. III-C, Harpia filtering suite: edge enhancement on
 * the Gaussian): out (f32) =
 * in + amount * (in - G_sigma in), the Gaussian as hp_gaussian3d (truncate
 * 3, reflect), the sum in FP32 as fma(amount, in - G, in). Device volumes
 * only (in and out on the device, out f32 of the input's extents, no
 * aliasing); HP_ERR_UNSUPPORTED for host volumes. */
int hp_unsharp3d(const hp_volume* in, hp_volume* out, double sigma, double amount, void* stream);

/* Gaussian local threshold (Sec. III-C, threshold algorithms): out (u8) =
 * in > G_sigma in - offset, the Gaussian as hp_gaussian3d (truncate 3,
 * reflect, FP32) and the comparison in FP32. Device volumes only (out u8 of
 * the input's extents); the local mean is library scratch on `stream`.
 * HP_ERR_UNSUPPORTED for host volumes. */
int hp_threshold_local3d(const hp_volume* in, hp_volume* out, double sigma, double offset,
                         void* stream);

/* Box-window local threshold (Sec. III-C, threshold algorithms: mean,
 * Niblack, Sauvola): out (u8) = in > T, with m and s the mean and standard
 * deviation of the input over the (2 radius + 1)^3 cube around each voxel
 * (reflect boundary) and
 *   HP_LOCAL_MEAN:    T = m - c
 *   HP_LOCAL_NIBLACK: T = m + k s
 *   HP_LOCAL_SAUVOLA: T = m (1 + k (s / c - 1))   (c = the dynamic range R)
 * Window sums run separably (x, then y, then z): exactly in integers for
 * u8 / u16 input (running sums along each line), in FP64 for f16 / f32 (each
 * window in increasing source coordinate); the decision is that of
 * m = S1/N, s = sqrt(max(S2/N - m^2, 0)), T and f > T in FP64, one rounded
 * operation at a time, so it is reproducible bit for bit. For integer input
 * an FP32 evaluation with a proven error margin settles every voxel whose
 * value is clear of T, and the FP64 sequence decides the rest.
 * radius in [0, 15]; c > 0 for Sauvola. Host volumes run out of core (halo
 * = radius); device volumes use library scratch of 24 (integer input) or 32
 * (floating-point input) bytes per voxel. */
int hp_threshold_box3d(const hp_volume* in, hp_volume* out, int method, int radius, double k,
                       double c, void* stream);

/* Hessian texture features (Sec. III-C, "Hessian"): the second derivatives
 * of the Gaussian-smoothed volume, each the hp_gaussian3d derivative filter
 * whose orders sum to 2 (truncate 3, reflect, FP32).
 *   HP_HESSIAN_COMPONENTS: n = 6 outputs Dzz, Dyy, Dxx, Dzy, Dzx, Dyx;
 *   HP_HESSIAN_EIGENVALUES: n = 3 outputs, the eigenvalues of the symmetric
 *     3x3 Hessian per voxel in ascending order, solved in FP32 in closed form
 *     (trigonometric solution of the characteristic cubic); the components
 *     live in library scratch (24 bytes per voxel).
 * Outputs f32 or f16 (one dtype), the input's extents and location; host
 * volumes run out of core. */
int hp_hessian3d(const hp_volume* in, hp_volume* const* outs, int what, double sigma,
                 void* stream);

/* Global threshold (Sec. III-C, threshold algorithms): out (u8) = in > t,
 * decided exactly for every input dtype: the kernels compare against the
 * largest value of the input's type that is <= t, so a t that is not
 * representable in that type (0.1 for f32, 7499.7 for u16) is never rounded
 * up. NaN inputs give 0. HP_ERR_INVALID_ARG when t is NaN. */
int hp_threshold3d(const hp_volume* in, hp_volume* out, double t, void* stream);

/* Adjoint of the filter bank (device mode, f32): gin = sum_i J_i^T gouts[i],
 * J_i the Jacobian of filter i at input `in`. Linear filters use the
 * flipped-kernel correlation followed by the reflect fold-back;
 * GM routes through D_a / GM (0 where GM = 0). Uses library scratch. */
int hp_filterbank3d_adjoint(const hp_volume* in, const hp_volume* const* gouts,
                            const hp_filter* f, int n, hp_volume* gin, void* stream);

/* Subgradient of erosion (is_dilate = 0) or dilation (1), device mode, f32
 * gradients, input of any dtype: gin[q] = sum of gout[p] over outputs p whose
 * extreme source is q; among equal values the source with the smallest linear
 * index wins. With accumulate != 0 the sum is added to gin instead of
 * overwriting it. Deterministic (an argmin map, then a gather; no atomics).
 * Uses library scratch: an int32 source index per voxel, so at most
 * 2^31 - 1 voxels. */
int hp_morph3d_backward(const hp_volume* in, const hp_volume* gout, int is_dilate, hp_se se,
                        int radius, hp_volume* gin, int accumulate, void* stream);

/* Allocation-free variant of hp_morph3d_backward (same arguments, same
 * result). The paper has no counterpart; it exists for callers that must not
 * allocate device memory while this step runs -- for example code that runs
 * inside a fixed memory arena, a loop with real-time limits that may not
 * enter the allocator, or a process whose device memory is already handed to
 * another pool. Instead of a per-call scratch buffer it uses one int32 index
 * array of 16,777,216 entries (64 MiB, enough for 256^3 voxels) that the
 * library holds in device memory on every GPU that loads it, until the
 * process exits. Larger volumes return HP_ERR_UNSUPPORTED; use
 * hp_morph3d_backward for them.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress, with that device current), which may also load
 *     the library's device code; make that first call before any stream
 *     capture. The address is cached per device; after cudaDeviceReset call
 *     hp_release_cache() so that the next call looks it up again.
 *   - Every call uses the same array: calls that overlap on the GPU (other
 *     streams, other host threads) race and give wrong results. Order them.
 *   - No state needs clearing between calls: each call rewrites every index
 *     it later reads.
 *   - The call itself performs no cudaMalloc, cudaFree or other device
 *     allocation. */
int hp_morph3d_backward_noalloc(const hp_volume* in, const hp_volume* gout, int is_dilate,
                                hp_se se, int radius, hp_volume* gin, int accumulate,
                                void* stream);

/* Devices that host-mode (out-of-core) calls spread their bricks over
 * (Sec. III-D step 3 and Sec. V: round-robin chunk scheduling without
 * inter-GPU communication): brick k of a call runs on devices[k mod n], each
 * device with its own streams and stage buffers, no peer access and no
 * collective. The budget (hp_set_memory_budget, or 0.8 x that device's free
 * memory) applies per device; entries naming the same device share it.
 * n = 0 (the default) means the current device only. Device-mode calls are
 * not affected. Process-wide; HP_ERR_INVALID_ARG for an index that is not a
 * device. hp_get_devices writes up to max_n entries and the count. */
int hp_set_devices(const int* devices, int n);
int hp_get_devices(int* devices, int max_n, int* n);

/* Brick shard of this process for host-mode calls: of the planned bricks
 * (in the planner's order) only those with index i mod world == rank run,
 * and only their core boxes of the output are written; the rest of the
 * output is left as it was. Processes that run the same call with
 * rank = 0..world-1 together write every output voxel exactly once, with
 * no communication between them. The planned brick list depends on the
 * budget, so a shard with world > 1 requires an explicit
 * hp_set_memory_budget (else HP_ERR_INVALID_ARG); rank 0 of world 1 (the
 * default) runs every brick. Process-wide. */
int hp_set_brick_shard(int rank, int world);

/* Chunk planner (Sec. III-D step 2), host only, no device work. Splits an
 * (nz, ny, nx) volume into bricks whose core boxes tile it exactly; box i's
 * input box is the hull of the reflected sources of its core grown by
 * `halo`. Sized so that `stages` bricks in flight, each holding its input
 * box (in_bytes per voxel) and core (out_bytes per voxel), fit `budget`
 * bytes, with at least `min_bricks` bricks when the volume allows it.
 * Writes up to max_bricks entries; *nbricks receives the count needed (call
 * with max_bricks = 0 to size the arrays). */
int hp_plan_bricks(int64_t nx, int64_t ny, int64_t nz, int halo, size_t in_bytes,
                   size_t out_bytes, size_t budget, int stages, int min_bricks, hp_box* cores,
                   hp_box* in_boxes, int max_bricks, int* nbricks);

/* Synchronise `stream`, then read and clear the device error word that
 * kernels set when a bounded wait gives up. Returns HP_OK, HP_ERR_TIMEOUT or
 * HP_ERR_CUDA. */
int hp_stream_status(void* stream);

/* Diagnostic for the failure path of bounded device-side waits (the paper
 * has no counterpart): enqueues on `stream` one small kernel that waits, with
 * the same bounded mbarrier wait the filtering kernels use, on a barrier that
 * nothing ever completes. The wait gives up after its poll limit and sets the
 * device error word, so a following hp_stream_status(stream) returns
 * HP_ERR_TIMEOUT and clears it; the CUDA context stays usable. No fault, trap
 * or unbounded spin is involved. Returns HP_OK or HP_ERR_CUDA (launch). */
int hp_selftest_wait_timeout(void* stream);

/* Diagnostic (the paper has no counterpart): measures the FP32 FMA
 * throughput of the current device, the ceiling the FMA-bound filters
 * (large-radius Gaussians, the filter bank) are compared against. Runs
 * independent packed fma.rn.f32x2 chains on every SM, `repeats` timed
 * launches on `stream` (after one warm-up), and writes the best rate in
 * FLOP/s (2 per FMA). Synchronises `stream`. */
int hp_probe_fp32_fma(void* stream, int repeats, double* flops_per_s);

/* Free cached filter-bank launch plans (graphs and work lists) and forget
 * cached per-device addresses of library device variables (call it after a
 * cudaDeviceReset). */
int hp_release_cache(void);

/* Counters of the last call; see hp_stats. */
int hp_get_stats(hp_stats* s);

/* Thread-local message for the last failing call on this thread. */
const char* hp_last_error(void);

/* Library version string. */
const char* hp_version(void);

#ifdef __cplusplus
}
#endif

#endif /* HP_H */
