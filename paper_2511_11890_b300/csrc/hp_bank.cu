// C entry points of the filter bank, its adjoint and the morphology
// subgradient.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <cmath>

#include <string>
#include <vector>

#include "hp_internal.h"

namespace hp {

void bank_release_cache();
cudaError_t launch_sep_adjoint(const float* w, float* dst, const int64_t dims[3],
                               const Taps& taps, float* t1, float* t2, int accumulate,
                               cudaStream_t s);
cudaError_t launch_gm_chain3(const float* w, float* dz, float* dy, float* dx, int64_t total,
                             cudaStream_t s);
cudaError_t launch_morph_arg(const void* in, int dt, const int64_t dims[3], int ball, int rad,
                             int is_dilate, int32_t* arg, cudaStream_t s);
cudaError_t launch_morph_gather(const int32_t* arg, const float* gout, float* gin,
                                const int64_t dims[3], int rad, int accumulate, cudaStream_t s);
void noalloc_forget();
void error_word_forget();

static Job whole_job_of(const hp_volume* in, void* out, int out_dtype) {
  Job j;
  const int64_t n[3] = {in->nz, in->ny, in->nx};
  j.in = DevBox{in->data, in->dtype, {0, 0, 0}, {n[0], n[1], n[2]}};
  j.out = DevOut{out, out_dtype, {0, 0, 0}, {n[0], n[1], n[2]}};
  for (int a = 0; a < 3; ++a) {
    j.gdims[a] = n[a];
    j.core_lo[a] = 0;
    j.core_hi[a] = n[a];
  }
  return j;
}

static int check_bricks(const std::vector<hp_box>& b, const int64_t G[3]) {
  int64_t vol = 0;
  for (size_t i = 0; i < b.size(); ++i) {
    int64_t v = 1;
    for (int a = 0; a < 3; ++a) {
      if (b[i].lo[a] < 0 || b[i].hi[a] > G[a] || b[i].lo[a] >= b[i].hi[a])
        return set_error(HP_ERR_INVALID_ARG, "brick " + std::to_string(i) + " is empty or outside the volume");
      v *= b[i].hi[a] - b[i].lo[a];
    }
    vol += v;
    for (size_t j = 0; j < i; ++j) {
      bool overlap = true;
      for (int a = 0; a < 3; ++a)
        overlap = overlap && b[i].lo[a] < b[j].hi[a] && b[j].lo[a] < b[i].hi[a];
      if (overlap) return set_error(HP_ERR_INVALID_ARG, "bricks overlap");
    }
  }
  if (vol != G[0] * G[1] * G[2]) return set_error(HP_ERR_INVALID_ARG, "bricks do not cover the volume");
  return HP_OK;
}

static int bank_common(const hp_volume* in, hp_volume* const* outs, const hp_filter* f, int n,
                       const hp_box* bricks, int nbricks, void* stream) {
  if (!in || !in->data || !outs || !f || n < 1)
    return set_error(HP_ERR_INVALID_ARG, "filter bank: null argument or n < 1");
  if (in->loc != HP_HOST && in->loc != HP_DEVICE)
    return set_error(HP_ERR_INVALID_ARG, "filter bank: unknown location");
  if (in->loc == HP_HOST && bricks)
    return set_error(HP_ERR_UNSUPPORTED, "filter bank: brick lists are for device volumes (host volumes are planned by the library)");
  BankRequest q;
  q.in = in->data;
  q.dtype = in->dtype;
  q.G[0] = in->nz;
  q.G[1] = in->ny;
  q.G[2] = in->nx;
  q.out_dtype = -1;
  const size_t in_bytes = dtype_size(in->dtype) * (size_t)(in->nx * in->ny * in->nz);
  for (int i = 0; i < n; ++i) {
    const hp_volume* o = outs[i];
    if (!o || !o->data) return set_error(HP_ERR_INVALID_ARG, "filter bank: null output");
    if (o->loc != in->loc) return set_error(HP_ERR_UNSUPPORTED, "filter bank: mixed host/device locations");
    if (o->nx != in->nx || o->ny != in->ny || o->nz != in->nz)
      return set_error(HP_ERR_INVALID_ARG, "filter bank: output extents differ from the input");
    if (o->dtype != HP_F16 && o->dtype != HP_F32)
      return set_error(HP_ERR_UNSUPPORTED, "filter bank: outputs must be f16 or f32");
    if (q.out_dtype >= 0 && o->dtype != q.out_dtype)
      return set_error(HP_ERR_UNSUPPORTED, "filter bank: all outputs must share one dtype");
    q.out_dtype = o->dtype;
    const char* a = (const char*)in->data;
    const char* b = (const char*)o->data;
    const size_t ob = dtype_size(o->dtype) * (size_t)(o->nx * o->ny * o->nz);
    if (a < b + ob && b < a + in_bytes) return set_error(HP_ERR_INVALID_ARG, "filter bank: input and output alias");
    if (f[i].kind < HP_FILTER_G || f[i].kind > HP_FILTER_LOG)
      return set_error(HP_ERR_INVALID_ARG, "filter bank: unknown filter kind");
    if (!(f[i].sigma > 0)) return set_error(HP_ERR_INVALID_ARG, "filter bank: sigma must be > 0");
    q.filters.push_back({f[i].kind, f[i].sigma});
    q.outs.push_back(o->data);
  }
  if (in->loc == HP_HOST) {
    for (auto& f : q.filters)
      if (radius_of(f.second, 3.0) < 1 || radius_of(f.second, 3.0) > kMaxR)
        return set_error(HP_ERR_UNSUPPORTED, "filter bank: radius must be in [1, 12] (sigma in ~[0.17, 4.16])");
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < i; ++j)
        if (f[i].kind == f[j].kind && f[i].sigma == f[j].sigma)
          return set_error(HP_ERR_INVALID_ARG, "filter bank: duplicate (kind, sigma)");
    return run_bank_host(in, outs, q);
  }
  if (bricks && nbricks > 0) {
    q.bricks.assign(bricks, bricks + nbricks);
    int st = check_bricks(q.bricks, q.G);
    if (st != HP_OK) return st;
  } else {
    hp_box whole;
    for (int a = 0; a < 3; ++a) {
      whole.lo[a] = 0;
      whole.hi[a] = q.G[a];
    }
    q.bricks.push_back(whole);
  }
  return run_filterbank(q, (cudaStream_t)stream);
}

}  // namespace hp

using namespace hp;

extern "C" {

int hp_filterbank3d(const hp_volume* in, hp_volume* const* outs, const hp_filter* f, int n,
                    void* stream) {
  return bank_common(in, outs, f, n, nullptr, 0, stream);
}

int hp_filterbank3d_bricks(const hp_volume* in, hp_volume* const* outs, const hp_filter* f, int n,
                           const hp_box* bricks, int nbricks, void* stream) {
  if (!bricks || nbricks < 1) return set_error(HP_ERR_INVALID_ARG, "filter bank: no bricks");
  return bank_common(in, outs, f, n, bricks, nbricks, stream);
}

int hp_filterbank3d_adjoint(const hp_volume* in, const hp_volume* const* gouts,
                            const hp_filter* f, int n, hp_volume* gin, void* stream) {
  if (!in || !in->data || !gouts || !f || n < 1 || !gin || !gin->data)
    return set_error(HP_ERR_INVALID_ARG, "adjoint: null argument or n < 1");
  if (in->loc != HP_DEVICE || gin->loc != HP_DEVICE)
    return set_error(HP_ERR_UNSUPPORTED, "adjoint runs on device volumes only");
  if (gin->dtype != HP_F32) return set_error(HP_ERR_UNSUPPORTED, "adjoint: gin must be f32");
  if (gin->nx != in->nx || gin->ny != in->ny || gin->nz != in->nz)
    return set_error(HP_ERR_INVALID_ARG, "adjoint: gin extents differ from the input");
  bool any_gm = false;
  for (int i = 0; i < n; ++i) {
    const hp_volume* g = gouts[i];
    if (!g || !g->data || g->loc != HP_DEVICE || g->dtype != HP_F32 || g->nx != in->nx ||
        g->ny != in->ny || g->nz != in->nz)
      return set_error(HP_ERR_INVALID_ARG, "adjoint: every output gradient must be an f32 device volume of the input's extents");
    if (f[i].kind < HP_FILTER_G || f[i].kind > HP_FILTER_LOG || !(f[i].sigma > 0))
      return set_error(HP_ERR_INVALID_ARG, "adjoint: bad filter");
    if (radius_of(f[i].sigma, 3.0) > kMaxRGeneric)
      return set_error(HP_ERR_UNSUPPORTED, "adjoint: radius exceeds 32");
    any_gm = any_gm || f[i].kind == HP_FILTER_GM;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t dims[3] = {in->nz, in->ny, in->nx};
  const int64_t total = dims[0] * dims[1] * dims[2];
  const size_t vb = sizeof(float) * (size_t)total;
  // GM forms its derivatives with the Gaussian kernels; the generic path
  // (large radii, thin volumes) needs scratch of its own
  size_t gscr = 0;
  for (int i = 0; i < n; ++i)
    if (f[i].kind == HP_FILTER_GM)
      gscr = std::max(gscr, gauss_scratch_bytes(whole_job_of(in, gin->data, HP_F32),
                                                radius_of(f[i].sigma, 3.0)));
  int st = check_scratch_budget(vb * (any_gm ? 5 : 2) + gscr);
  if (st != HP_OK) return st;
  Scratch sc(s);
  float *t1 = nullptr, *t2 = nullptr, *dz = nullptr, *dy = nullptr, *dx = nullptr;
  void* gs = nullptr;
  cudaError_t e = sc.alloc((void**)&t1, vb);
  if (e == cudaSuccess && gscr > 0) e = sc.alloc(&gs, gscr);
  if (e == cudaSuccess) e = sc.alloc((void**)&t2, vb);
  if (e == cudaSuccess && any_gm) e = sc.alloc((void**)&dz, vb);
  if (e == cudaSuccess && any_gm) e = sc.alloc((void**)&dy, vb);
  if (e == cudaSuccess && any_gm) e = sc.alloc((void**)&dx, vb);
  if (e != cudaSuccess) return cuda_fail(e, "adjoint scratch");
  float* g = static_cast<float*>(gin->data);
  if ((e = cudaMemsetAsync(g, 0, vb, s)) != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
  for (int i = 0; i < n && e == cudaSuccess; ++i) {
    const float* w = static_cast<const float*>(gouts[i]->data);
    const double sigma = f[i].sigma;
    Taps taps;
    if (f[i].kind == HP_FILTER_G) {
      const int ord[3] = {0, 0, 0};
      make_taps(sigma, 3.0, ord, &taps);
      e = launch_sep_adjoint(w, g, dims, taps, t1, t2, 1, s);
    } else if (f[i].kind == HP_FILTER_LOG) {
      for (int a = 0; a < 3 && e == cudaSuccess; ++a) {
        int ord[3] = {0, 0, 0};
        ord[a] = 2;
        make_taps(sigma, 3.0, ord, &taps);
        e = launch_sep_adjoint(w, g, dims, taps, t1, t2, 1, s);
      }
    } else {
      float* D[3] = {dz, dy, dx};
      for (int a = 0; a < 3 && e == cudaSuccess; ++a) {
        int ord[3] = {0, 0, 0};
        ord[a] = 1;
        make_taps(sigma, 3.0, ord, &taps);
        Job j = whole_job_of(in, D[a], HP_F32);
        j.scratch = gs;
        j.scratch_bytes = gscr;
        e = launch_gauss(j, taps, s);
      }
      // the chain rule through GM for all three axes in one pass, in place
      if (e == cudaSuccess) e = launch_gm_chain3(w, dz, dy, dx, total, s);
      for (int a = 0; a < 3 && e == cudaSuccess; ++a) {
        int ord[3] = {0, 0, 0};
        ord[a] = 1;
        make_taps(sigma, 3.0, ord, &taps);
        e = launch_sep_adjoint(D[a], g, dims, taps, t1, t2, 1, s);
      }
    }
  }
  if (e != cudaSuccess) return cuda_fail(e, "adjoint launch");
  return HP_OK;
}

int hp_morph3d_backward(const hp_volume* in, const hp_volume* gout, int is_dilate, hp_se se,
                        int radius, hp_volume* gin, int accumulate, void* stream) {
  if (!in || !in->data || !gout || !gout->data || !gin || !gin->data)
    return set_error(HP_ERR_INVALID_ARG, "morphology backward: null argument");
  if (in->loc != HP_DEVICE || gout->loc != HP_DEVICE || gin->loc != HP_DEVICE)
    return set_error(HP_ERR_UNSUPPORTED, "morphology backward runs on device volumes only");
  if (gout->dtype != HP_F32 || gin->dtype != HP_F32)
    return set_error(HP_ERR_UNSUPPORTED, "morphology backward: gradients must be f32");
  if (gout->nx != in->nx || gout->ny != in->ny || gout->nz != in->nz || gin->nx != in->nx ||
      gin->ny != in->ny || gin->nz != in->nz)
    return set_error(HP_ERR_INVALID_ARG, "morphology backward: extents differ");
  if (se != HP_SE_CUBE && se != HP_SE_BALL) return set_error(HP_ERR_INVALID_ARG, "unknown structuring element");
  if (radius < 0 || radius > kMaxMorphR) return set_error(HP_ERR_INVALID_ARG, "radius must be in [0, 16]");
  const int64_t dims[3] = {in->nz, in->ny, in->nx};
  const int64_t total = dims[0] * dims[1] * dims[2];
  if (total >= (int64_t)1 << 31)
    return set_error(HP_ERR_UNSUPPORTED, "morphology backward: more than 2^31 - 1 voxels");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t ab = sizeof(int32_t) * (size_t)total;
  int st = check_scratch_budget(ab);
  if (st != HP_OK) return st;
  Scratch sc(s);
  int32_t* arg = nullptr;
  cudaError_t e = sc.alloc((void**)&arg, ab);
  if (e != cudaSuccess) return cuda_fail(e, "morphology backward scratch");
  e = launch_morph_arg(in->data, in->dtype, dims, se == HP_SE_BALL, radius, is_dilate, arg, s);
  if (e == cudaSuccess)
    e = launch_morph_gather(arg, static_cast<const float*>(gout->data), static_cast<float*>(gin->data),
                            dims, radius, accumulate, s);
  if (e != cudaSuccess) return cuda_fail(e, "morphology backward launch");
  return HP_OK;
}

// Opening / closing / white top-hat on device volumes: two morphology
// passes through a scratch volume (and, for the top-hat, in - opening).
static int morph_compose(const hp_volume* in, hp_volume* out, hp_se se, int radius, void* stream,
                         int kind /* 0 open, 1 close, 2 white top-hat */) {
  if (!in || !in->data || !out || !out->data) return set_error(HP_ERR_INVALID_ARG, "null argument");
  if (in->loc != HP_DEVICE || out->loc != HP_DEVICE)
    return set_error(HP_ERR_UNSUPPORTED, "opening / closing / top-hat run on device volumes only");
  if (in->data == out->data) return set_error(HP_ERR_INVALID_ARG, "output may not alias the input");
  if (out->dtype != in->dtype || out->nx != in->nx || out->ny != in->ny || out->nz != in->nz)
    return set_error(HP_ERR_INVALID_ARG, "output must match the input's dtype and extents");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t vb = dtype_size(in->dtype) * (size_t)(in->nx * in->ny * in->nz);
  int st = check_scratch_budget(vb);
  if (st != HP_OK) return st;
  Scratch sc(s);
  void* tmp = nullptr;
  cudaError_t e = sc.alloc(&tmp, vb);
  if (e != cudaSuccess) return cuda_fail(e, "opening / closing scratch");
  hp_volume t = *in;
  t.data = tmp;
  const bool erode_first = kind != 1;
  st = erode_first ? hp_erode3d(in, &t, se, radius, stream) : hp_dilate3d(in, &t, se, radius, stream);
  if (st != HP_OK) return st;
  st = erode_first ? hp_dilate3d(&t, out, se, radius, stream) : hp_erode3d(&t, out, se, radius, stream);
  if (st != HP_OK) return st;
  if (kind == 2) {
    e = launch_difference(in->data, out->data, in->dtype, (int64_t)(in->nx * in->ny * in->nz), s);
    if (e != cudaSuccess) return cuda_fail(e, "top-hat difference");
  }
  return HP_OK;
}

int hp_open3d(const hp_volume* in, hp_volume* out, hp_se se, int radius, void* stream) {
  return morph_compose(in, out, se, radius, stream, 0);
}

int hp_close3d(const hp_volume* in, hp_volume* out, hp_se se, int radius, void* stream) {
  return morph_compose(in, out, se, radius, stream, 1);
}

int hp_tophat3d(const hp_volume* in, hp_volume* out, hp_se se, int radius, void* stream) {
  return morph_compose(in, out, se, radius, stream, 2);
}

int hp_unsharp3d(const hp_volume* in, hp_volume* out, double sigma, double amount, void* stream) {
  if (!in || !in->data || !out || !out->data) return set_error(HP_ERR_INVALID_ARG, "null argument");
  if (in->loc != HP_DEVICE || out->loc != HP_DEVICE)
    return set_error(HP_ERR_UNSUPPORTED, "unsharp mask runs on device volumes only");
  if (out->dtype != HP_F32) return set_error(HP_ERR_UNSUPPORTED, "unsharp mask output must be f32");
  if (!std::isfinite(amount)) return set_error(HP_ERR_INVALID_ARG, "amount must be finite");
  int st = hp_gaussian3d(in, out, sigma, 3.0, nullptr, stream);
  if (st != HP_OK) return st;
  const cudaError_t e = launch_unsharp(in->data, in->dtype, static_cast<float*>(out->data), (float)amount,
                                       (int64_t)(in->nx * in->ny * in->nz), (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "unsharp mask epilogue");
  return HP_OK;
}

int hp_threshold_local3d(const hp_volume* in, hp_volume* out, double sigma, double offset,
                         void* stream) {
  if (!in || !in->data || !out || !out->data) return set_error(HP_ERR_INVALID_ARG, "null argument");
  if (in->loc != HP_DEVICE || out->loc != HP_DEVICE)
    return set_error(HP_ERR_UNSUPPORTED, "local threshold runs on device volumes only");
  if (out->dtype != HP_U8) return set_error(HP_ERR_UNSUPPORTED, "local threshold output must be u8");
  if (out->nx != in->nx || out->ny != in->ny || out->nz != in->nz || out->data == in->data)
    return set_error(HP_ERR_INVALID_ARG, "output must match the input's extents and not alias it");
  if (!std::isfinite(offset)) return set_error(HP_ERR_INVALID_ARG, "offset must be finite");
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = in->nx * in->ny * in->nz;
  int st = check_scratch_budget(4 * (size_t)n);
  if (st != HP_OK) return st;
  Scratch sc(s);
  void* m = nullptr;
  cudaError_t e = sc.alloc(&m, 4 * (size_t)n);
  if (e != cudaSuccess) return cuda_fail(e, "local threshold scratch");
  hp_volume mv = *in;
  mv.data = m;
  mv.dtype = HP_F32;
  st = hp_gaussian3d(in, &mv, sigma, 3.0, nullptr, stream);
  if (st != HP_OK) return st;
  e = launch_local_threshold(in->data, in->dtype, static_cast<const float*>(m), (float)offset,
                             static_cast<uint8_t*>(out->data), n, s);
  if (e != cudaSuccess) return cuda_fail(e, "local threshold");
  return HP_OK;
}

int hp_release_cache(void) {
  bank_release_cache();
  noalloc_forget();
  error_word_forget();
  return HP_OK;
}

}  // extern "C"
