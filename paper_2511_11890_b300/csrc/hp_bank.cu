// C entry points of the filter bank, its adjoint and the morphology
// subgradient.
#include <cuda_runtime.h>
#include <string.h>

#include <string>
#include <vector>

#include "hp_internal.h"

struct hp_volume {
  void* data;
  int dtype;
  int loc;
  int64_t nx, ny, nz;
};

namespace hp {

struct BankRequest {
  const void* in;
  int dtype, out_dtype;
  int64_t G[3];
  std::vector<std::pair<int, double>> filters;
  std::vector<void*> outs;
  std::vector<hp_box> bricks;
};
int run_filterbank(const BankRequest& q, cudaStream_t s);
void bank_release_cache();

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
  if (in->loc != HP_DEVICE)
    return set_error(HP_ERR_UNSUPPORTED, "filter bank runs on device volumes only");
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
    if (o->loc != HP_DEVICE) return set_error(HP_ERR_UNSUPPORTED, "filter bank: outputs must be device volumes");
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

int hp_filterbank3d_adjoint(const hp_volume*, const hp_volume* const*, const hp_filter*, int,
                            hp_volume*, void*) {
  return set_error(HP_ERR_UNSUPPORTED, "adjoint not built yet");
}

int hp_morph3d_backward(const hp_volume*, const hp_volume*, int, hp_se, int, hp_volume*, void*) {
  return set_error(HP_ERR_UNSUPPORTED, "morphology backward not built yet");
}

int hp_release_cache(void) {
  bank_release_cache();
  return HP_OK;
}

}  // extern "C"
