/*
 * CPU oracle for chunked, halo-padded 3D filtering (Harpia, Sec. III-C/III-D).
 *
 * TEST INFRASTRUCTURE ONLY. Plain, slow, single-threaded FP64 C written from
 * the definitions below. It shares no code with the CUDA library and is
 * called only by the tests, the smoke check and the CPU-baseline leg of the
 * benchmark. The same source built with -fopenmp splits the outermost (z)
 * loops of the Gaussian, morphology and box-sum passes over threads (the
 * multi-core CPU baseline); every output is still computed by the same
 * operations in the same order, so both builds give identical results.
 *
 * Conventions (the paper names the filters -- Sec. III-C: erosion,
 * dilation, Gaussian, "Hessian" feature extraction -- but prints no formula;
 * the readings below are the ones this project fixes):
 *   - Volume f[z][y][x], x fastest. Every coordinate triple is (z, y, x).
 *   - Reflect boundary, half-sample symmetric ("d c b a | a b c d"):
 *       R(i, n) = m < n ? m : 2n - 1 - m,  m = i mod 2n taken in [0, 2n).
 *   - Radius r = floor(truncate * sigma + 0.5).
 *   - Weights, k in [-r, r]: phi(k) = exp(-k^2 / (2 sigma^2)),
 *       g0 = phi / sum(phi), g1 = -k / sigma^2 * g0,
 *       g2 = (k^2 / sigma^4 - 1 / sigma^2) * g0   (no re-normalisation).
 *   - 1D filter of order o: y[i] = sum_k g_o(k) * x[R(i - k)]  (convolution).
 *   - 3D filter of orders (oz, oy, ox): x pass, then y, then z, all in FP64.
 *   - GM = sqrt(Dx^2 + Dy^2 + Dz^2), LoG = Dxx + Dyy + Dzz.
 *   - Erosion eps(f)(p) = min over o in B of f(R(p + o)); dilation
 *     delta(f)(p) = max over o in B of f(R(p - o)). Cube of half-width rho:
 *     max(|dz|,|dy|,|dx|) <= rho. Ball of radius r: dz^2+dy^2+dx^2 <= r^2.
 *     Min and max follow IEEE 754 totalOrder: integers by value; floating
 *     point by value with -0 below +0, a NaN whose sign bit is clear above
 *     +inf, one whose sign bit is set below -inf, and NaNs of one sign by
 *     their trailing significand field (see total_cmp).
 *   - Threshold: u8 = (f > t).
 *   - Adjoint of a 1D filter: t[j] = sum_k g(k) w[j + k] over the
 *     zero-extended w, j in [-r, n-1+r]; then gin[R(j)] += t[j].
 *   - Morphology subgradient: each output routes its weight to the source
 *     q = R(p +- o) holding the extreme value (in totalOrder); ties (equal
 *     elements) go to the smallest linear index q.
 *
 * Chunking (Sec. III-D): every forward function reads its input from a box
 * [in_lo, in_lo + in_dims) of a global volume of size gdims and writes the
 * output for a box [out_lo, out_lo + out_dims). Reflection acts on global
 * coordinates. A function returns ORC_ERR_HALO when the input box lacks a
 * voxel that the output box needs -- that is how a too-small halo shows up.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { ORC_U8 = 0, ORC_U16 = 1, ORC_F16 = 2, ORC_F32 = 3, ORC_F64 = 4 };
enum { ORC_OK = 0, ORC_ERR_ARG = -1, ORC_ERR_NOMEM = -2, ORC_ERR_HALO = -3 };
enum { ORC_SE_CUBE = 0, ORC_SE_BALL = 1 };
enum { ORC_G = 0, ORC_GM = 1, ORC_LOG = 2 };

/* ---------------------------------------------------------------- basics */

int64_t orc_reflect(int64_t i, int64_t n) {
  int64_t p = 2 * n;
  int64_t m = i % p;
  if (m < 0) m += p;
  return m < n ? m : p - 1 - m;
}

int orc_radius(double sigma, double truncate) { return (int)floor(truncate * sigma + 0.5); }

int orc_kernel1d(double sigma, int r, int order, double* w) {
  if (sigma <= 0 || r < 0 || order < 0 || order > 2) return ORC_ERR_ARG;
  double s2 = sigma * sigma, sum = 0.0;
  for (int k = -r; k <= r; ++k) {
    w[k + r] = exp(-(double)k * (double)k / (2.0 * s2));
    sum += w[k + r];
  }
  for (int k = -r; k <= r; ++k) {
    double g0 = w[k + r] / sum;
    if (order == 0) w[k + r] = g0;
    else if (order == 1) w[k + r] = -(double)k / s2 * g0;
    else w[k + r] = ((double)k * (double)k / (s2 * s2) - 1.0 / s2) * g0;
  }
  return ORC_OK;
}

static double half_to_double(uint16_t h) {
  int s = h >> 15, e = (h >> 10) & 31, m = h & 1023;
  double v;
  if (e == 0) v = ldexp((double)m, -24);
  else if (e == 31) v = m ? NAN : INFINITY;
  else v = ldexp((double)(1024 + m), e - 25);
  return s ? -v : v;
}

static size_t dtype_size(int dt) {
  switch (dt) {
    case ORC_U8: return 1;
    case ORC_U16: case ORC_F16: return 2;
    case ORC_F32: return 4;
    case ORC_F64: return 8;
    default: return 0;
  }
}

static double load_elem(const void* p, int dt, int64_t i) {
  switch (dt) {
    case ORC_U8: return (double)((const uint8_t*)p)[i];
    case ORC_U16: return (double)((const uint16_t*)p)[i];
    case ORC_F16: return half_to_double(((const uint16_t*)p)[i]);
    case ORC_F32: return (double)((const float*)p)[i];
    default: return ((const double*)p)[i];
  }
}

/* IEEE 754 totalOrder of elements i and j of p (<0, 0 or >0). Integers
 * compare by value. A floating-point element is split into its sign bit,
 * whether it is a NaN, its trailing significand field and its value; then:
 *   - two non-NaNs compare by value, and equal values that are both zero
 *     by sign (-0 < +0);
 *   - a NaN with the sign bit clear is above every non-NaN, one with the
 *     sign bit set below every non-NaN;
 *   - NaNs of opposite signs: the negative one is below; NaNs of one sign
 *     compare by significand field, ascending for +, descending for -. */
typedef struct {
  int sign, nan;
  uint64_t sig;
  double v;
} orc_fp;

static orc_fp fp_split(const void* p, int dt, int64_t i) {
  orc_fp r;
  uint64_t bits = 0, expmask = 0, sigmask = 0;
  int sbit = 0;
  if (dt == ORC_F16) {
    bits = ((const uint16_t*)p)[i];
    sbit = 15; expmask = 0x7C00u; sigmask = 0x03FFu;
  } else if (dt == ORC_F32) {
    uint32_t b;
    memcpy(&b, (const char*)p + 4 * i, 4);
    bits = b;
    sbit = 31; expmask = 0x7F800000u; sigmask = 0x007FFFFFu;
  } else {
    memcpy(&bits, (const char*)p + 8 * i, 8);
    sbit = 63; expmask = 0x7FF0000000000000ull; sigmask = 0x000FFFFFFFFFFFFFull;
  }
  r.sign = (int)((bits >> sbit) & 1u);
  r.sig = bits & sigmask;
  r.nan = (bits & expmask) == expmask && r.sig != 0;
  r.v = load_elem(p, dt, i);
  return r;
}

static int total_cmp(const void* p, int dt, int64_t i, int64_t j) {
  if (dt == ORC_U8 || dt == ORC_U16) {
    double a = load_elem(p, dt, i), b = load_elem(p, dt, j);
    return a < b ? -1 : (a > b ? 1 : 0);
  }
  orc_fp a = fp_split(p, dt, i), b = fp_split(p, dt, j);
  if (!a.nan && !b.nan) {
    if (a.v < b.v) return -1;
    if (a.v > b.v) return 1;
    if (a.v == 0.0 && a.sign != b.sign) return a.sign ? -1 : 1;
    return 0;
  }
  if (a.nan && !b.nan) return a.sign ? -1 : 1;
  if (!a.nan && b.nan) return b.sign ? 1 : -1;
  if (a.sign != b.sign) return a.sign ? -1 : 1;
  if (a.sig == b.sig) return 0;
  return (a.sig < b.sig) == (a.sign == 0) ? -1 : 1;
}

/* Index of global voxel (z, y, x) inside the input box, or -1. */
static int64_t box_index(const int64_t lo[3], const int64_t dims[3], int64_t z, int64_t y,
                         int64_t x) {
  int64_t c[3] = {z - lo[0], y - lo[1], x - lo[2]};
  for (int a = 0; a < 3; ++a)
    if (c[a] < 0 || c[a] >= dims[a]) return -1;
  return (c[0] * dims[1] + c[1]) * dims[2] + c[2];
}

static int valid_boxes(const int64_t in_lo[3], const int64_t in_dims[3], const int64_t g[3],
                       const int64_t out_lo[3], const int64_t out_dims[3]) {
  for (int a = 0; a < 3; ++a) {
    if (g[a] < 1 || in_dims[a] < 1 || out_dims[a] < 0) return 0;
    if (in_lo[a] < 0 || in_lo[a] + in_dims[a] > g[a]) return 0;
    if (out_lo[a] < 0 || out_lo[a] + out_dims[a] > g[a]) return 0;
  }
  return 1;
}

/* ------------------------------------------------- Gaussian and derivatives */

/* Hull [lo, hi) of {R(c - k) : c in [o_lo, o_lo + o_n), k in [-r, r]}. */
static void source_hull(int64_t o_lo, int64_t o_n, int r, int64_t n, int64_t* lo, int64_t* hi) {
  int64_t a = n, b = -1;
  for (int64_t c = o_lo; c < o_lo + o_n; ++c)
    for (int k = -r; k <= r; ++k) {
      int64_t s = orc_reflect(c - k, n);
      if (s < a) a = s;
      if (s > b) b = s;
    }
  *lo = a;
  *hi = b + 1;
}

int orc_gaussian3d(const void* in, int dtype, const int64_t in_lo[3], const int64_t in_dims[3],
                   const int64_t gdims[3], const int64_t out_lo[3], const int64_t out_dims[3],
                   double sigma, double truncate, const int order[3], double* out) {
  if (!valid_boxes(in_lo, in_dims, gdims, out_lo, out_dims) || dtype_size(dtype) == 0)
    return ORC_ERR_ARG;
  if (out_dims[0] * out_dims[1] * out_dims[2] == 0) return ORC_OK;
  int r = orc_radius(sigma, truncate);
  if (r < 0 || sigma <= 0) return ORC_ERR_ARG;
  double* w[3];  /* per axis (z, y, x) */
  for (int a = 0; a < 3; ++a) {
    w[a] = (double*)malloc(sizeof(double) * (2 * r + 1));
    if (!w[a]) return ORC_ERR_NOMEM;
    orc_kernel1d(sigma, r, order[a], w[a]);
  }
  /* Source windows per axis: W_a = hull of the reflected sources of the
   * output box. Every intermediate below is indexed over these windows. */
  int64_t wlo[3], whi[3], wn[3];
  for (int a = 0; a < 3; ++a) {
    source_hull(out_lo[a], out_dims[a], r, gdims[a], &wlo[a], &whi[a]);
    wn[a] = whi[a] - wlo[a];
  }
  int64_t oz = out_dims[0], oy = out_dims[1], ox = out_dims[2];
  double* A = (double*)malloc(sizeof(double) * (size_t)(wn[0] * wn[1] * wn[2]));
  double* B = (double*)malloc(sizeof(double) * (size_t)(wn[0] * wn[1] * ox));
  double* C = (double*)malloc(sizeof(double) * (size_t)(wn[0] * oy * ox));
  int rc = ORC_OK;
  if (!A || !B || !C) { rc = ORC_ERR_NOMEM; goto done; }

  /* A = f over the source windows */
  int miss = 0;
  for (int64_t z = 0; z < wn[0]; ++z)
    for (int64_t y = 0; y < wn[1]; ++y)
      for (int64_t x = 0; x < wn[2]; ++x) {
        int64_t q = box_index(in_lo, in_dims, wlo[0] + z, wlo[1] + y, wlo[2] + x);
        if (q < 0) miss = 1;
        else A[(z * wn[1] + y) * wn[2] + x] = load_elem(in, dtype, q);
      }
  if (miss) { rc = ORC_ERR_HALO; goto done; }
  /* x pass: B[z][y][x] = sum_k g_x(k) A[z][y][R(x - k)] */
#pragma omp parallel for schedule(static)
  for (int64_t z = 0; z < wn[0]; ++z)
    for (int64_t y = 0; y < wn[1]; ++y)
      for (int64_t x = 0; x < ox; ++x) {
        double s = 0.0;
        for (int k = -r; k <= r; ++k) {
          int64_t src = orc_reflect(out_lo[2] + x - k, gdims[2]) - wlo[2];
          s += w[2][k + r] * A[(z * wn[1] + y) * wn[2] + src];
        }
        B[(z * wn[1] + y) * ox + x] = s;
      }
  /* y pass: C[z][y][x] = sum_k g_y(k) B[z][R(y - k)][x] */
#pragma omp parallel for schedule(static)
  for (int64_t z = 0; z < wn[0]; ++z)
    for (int64_t y = 0; y < oy; ++y)
      for (int64_t x = 0; x < ox; ++x) {
        double s = 0.0;
        for (int k = -r; k <= r; ++k) {
          int64_t src = orc_reflect(out_lo[1] + y - k, gdims[1]) - wlo[1];
          s += w[1][k + r] * B[(z * wn[1] + src) * ox + x];
        }
        C[(z * oy + y) * ox + x] = s;
      }
  /* z pass: out[z][y][x] = sum_k g_z(k) C[R(z - k)][y][x] */
#pragma omp parallel for schedule(static)
  for (int64_t z = 0; z < oz; ++z)
    for (int64_t y = 0; y < oy; ++y)
      for (int64_t x = 0; x < ox; ++x) {
        double s = 0.0;
        for (int k = -r; k <= r; ++k) {
          int64_t src = orc_reflect(out_lo[0] + z - k, gdims[0]) - wlo[0];
          s += w[0][k + r] * C[(src * oy + y) * ox + x];
        }
        out[(z * oy + y) * ox + x] = s;
      }
done:
  free(A); free(B); free(C);
  for (int a = 0; a < 3; ++a) free(w[a]);
  return rc;
}

/* Filter bank: outs[i] is the FP64 result of filter i = (kinds[i], sigmas[i])
 * over the output box. G = order (0,0,0); GM and LoG combine the first and
 * second derivatives along z, y and x. */
int orc_filterbank3d(const void* in, int dtype, const int64_t in_lo[3], const int64_t in_dims[3],
                     const int64_t gdims[3], const int64_t out_lo[3], const int64_t out_dims[3],
                     const int* kinds, const double* sigmas, int n, double truncate,
                     double* const* outs) {
  int64_t nv = out_dims[0] * out_dims[1] * out_dims[2];
  double* tmp = (double*)malloc(sizeof(double) * (size_t)(nv > 0 ? nv : 1));
  if (!tmp) return ORC_ERR_NOMEM;
  int rc = ORC_OK;
  for (int i = 0; i < n && rc == ORC_OK; ++i) {
    if (kinds[i] == ORC_G) {
      int ord[3] = {0, 0, 0};
      rc = orc_gaussian3d(in, dtype, in_lo, in_dims, gdims, out_lo, out_dims, sigmas[i], truncate,
                          ord, outs[i]);
      continue;
    }
    if (kinds[i] != ORC_GM && kinds[i] != ORC_LOG) { rc = ORC_ERR_ARG; break; }
    for (int64_t q = 0; q < nv; ++q) outs[i][q] = 0.0;
    for (int a = 0; a < 3 && rc == ORC_OK; ++a) {
      int ord[3] = {0, 0, 0};
      ord[a] = kinds[i] == ORC_GM ? 1 : 2;
      rc = orc_gaussian3d(in, dtype, in_lo, in_dims, gdims, out_lo, out_dims, sigmas[i], truncate,
                          ord, tmp);
      if (rc != ORC_OK) break;
      for (int64_t q = 0; q < nv; ++q)
        outs[i][q] += kinds[i] == ORC_GM ? tmp[q] * tmp[q] : tmp[q];
    }
    if (rc == ORC_OK && kinds[i] == ORC_GM)
      for (int64_t q = 0; q < nv; ++q) outs[i][q] = sqrt(outs[i][q]);
  }
  free(tmp);
  return rc;
}

/* ------------------------------------------------------------- morphology */

static int in_se(int se, int rad, int dz, int dy, int dx) {
  if (se == ORC_SE_CUBE) return abs(dz) <= rad && abs(dy) <= rad && abs(dx) <= rad;
  return dz * dz + dy * dy + dx * dx <= rad * rad;
}

/* Output element has the input's dtype and is a bitwise copy of the chosen
 * source element, so the result is exact. */
int orc_morph3d(const void* in, int dtype, const int64_t in_lo[3], const int64_t in_dims[3],
                const int64_t gdims[3], const int64_t out_lo[3], const int64_t out_dims[3],
                int se, int rad, int is_dilate, void* out) {
  if (!valid_boxes(in_lo, in_dims, gdims, out_lo, out_dims) || dtype_size(dtype) == 0 || rad < 0 ||
      (se != ORC_SE_CUBE && se != ORC_SE_BALL))
    return ORC_ERR_ARG;
  size_t es = dtype_size(dtype);
  int miss = 0;
#pragma omp parallel for schedule(static) reduction(| : miss)
  for (int64_t z = 0; z < out_dims[0]; ++z)
    for (int64_t y = 0; y < out_dims[1]; ++y)
      for (int64_t x = 0; x < out_dims[2]; ++x) {
        int64_t pz = out_lo[0] + z, py = out_lo[1] + y, px = out_lo[2] + x;
        int64_t best_q = -1;
        for (int dz = -rad; dz <= rad; ++dz)
          for (int dy = -rad; dy <= rad; ++dy)
            for (int dx = -rad; dx <= rad; ++dx) {
              if (!in_se(se, rad, dz, dy, dx)) continue;
              int64_t sz, sy, sx;
              if (is_dilate) {
                sz = orc_reflect(pz - dz, gdims[0]);
                sy = orc_reflect(py - dy, gdims[1]);
                sx = orc_reflect(px - dx, gdims[2]);
              } else {
                sz = orc_reflect(pz + dz, gdims[0]);
                sy = orc_reflect(py + dy, gdims[1]);
                sx = orc_reflect(px + dx, gdims[2]);
              }
              int64_t q = box_index(in_lo, in_dims, sz, sy, sx);
              if (q < 0) { miss = 1; continue; }
              int c = best_q < 0 ? 0 : total_cmp(in, dtype, q, best_q);
              if (best_q < 0 || (is_dilate ? c > 0 : c < 0)) best_q = q;
            }
        if (best_q >= 0)
          memcpy((char*)out + (size_t)((z * out_dims[1] + y) * out_dims[2] + x) * es,
                 (const char*)in + (size_t)best_q * es, es);
      }
  return miss ? ORC_ERR_HALO : ORC_OK;
}

/* u8 = (f > t) over n elements, compared in FP64 (exact for every input
 * dtype here, since each converts to double without rounding). */
int orc_threshold(const void* in, int dtype, int64_t n, double t, uint8_t* out) {
  if (dtype_size(dtype) == 0 || n < 0) return ORC_ERR_ARG;
  for (int64_t q = 0; q < n; ++q) out[q] = load_elem(in, dtype, q) > t ? 1 : 0;
  return ORC_OK;
}

/* --------------------------------------------------------------- adjoints */

/* Adjoint of one 1D filter along axis a (0 = z, 1 = y, 2 = x) of a whole
 * volume, in place from w to g (distinct buffers). */
static int adjoint_axis(const double* w, double* g, const int64_t d[3], int a, const double* gk,
                        int r) {
  int64_t n = d[a];
  int64_t stride = a == 2 ? 1 : (a == 1 ? d[2] : d[1] * d[2]);
  int64_t nlines = d[0] * d[1] * d[2] / n;
  double* t = (double*)malloc(sizeof(double) * (size_t)(n + 2 * r));
  if (!t) return ORC_ERR_NOMEM;
  for (int64_t l = 0; l < nlines; ++l) {
    /* base offset of line l: enumerate the other two axes */
    int64_t base;
    if (a == 2) base = l * d[2];
    else if (a == 1) base = (l / d[2]) * d[1] * d[2] + (l % d[2]);
    else base = l;
    /* K^T: t[j] = sum_k g(k) w[j + k], w zero outside [0, n) */
    for (int64_t j = -r; j < n + r; ++j) {
      double s = 0.0;
      for (int k = -r; k <= r; ++k) {
        int64_t i = j + k;
        if (i >= 0 && i < n) s += gk[k + r] * w[base + i * stride];
      }
      t[j + r] = s;
    }
    /* E^T: fold the extended line back through the reflection */
    for (int64_t i = 0; i < n; ++i) g[base + i * stride] = 0.0;
    for (int64_t j = -r; j < n + r; ++j) g[base + orc_reflect(j, n) * stride] += t[j + r];
  }
  free(t);
  return ORC_OK;
}

/* gin = A^T w for A = the 3D filter of orders (oz, oy, ox). Since
 * A = Z Y X, A^T = X^T Y^T Z^T: adjoint along z, then y, then x. */
int orc_gaussian3d_adjoint(const double* w, const int64_t dims[3], double sigma, double truncate,
                           const int order[3], double* gin) {
  int r = orc_radius(sigma, truncate);
  int64_t nv = dims[0] * dims[1] * dims[2];
  if (nv <= 0 || sigma <= 0) return ORC_ERR_ARG;
  double* gk = (double*)malloc(sizeof(double) * (2 * r + 1));
  double* t1 = (double*)malloc(sizeof(double) * (size_t)nv);
  double* t2 = (double*)malloc(sizeof(double) * (size_t)nv);
  int rc = ORC_OK;
  if (!gk || !t1 || !t2) { rc = ORC_ERR_NOMEM; goto done; }
  orc_kernel1d(sigma, r, order[0], gk);
  if ((rc = adjoint_axis(w, t1, dims, 0, gk, r)) != ORC_OK) goto done;
  orc_kernel1d(sigma, r, order[1], gk);
  if ((rc = adjoint_axis(t1, t2, dims, 1, gk, r)) != ORC_OK) goto done;
  orc_kernel1d(sigma, r, order[2], gk);
  rc = adjoint_axis(t2, gin, dims, 2, gk, r);
done:
  free(gk); free(t1); free(t2);
  return rc;
}

/* Vector-Jacobian product of the filter bank: gin = sum_i J_i^T w_i with
 * J_i the Jacobian of filter i at the whole input volume `in`. */
int orc_filterbank3d_vjp(const void* in, int dtype, const int64_t dims[3], const int* kinds,
                         const double* sigmas, int n, double truncate, const double* const* w,
                         double* gin) {
  int64_t nv = dims[0] * dims[1] * dims[2];
  int64_t zero[3] = {0, 0, 0};
  double* tmp = (double*)malloc(sizeof(double) * (size_t)nv);
  double* acc = (double*)malloc(sizeof(double) * (size_t)nv);
  double* gm = (double*)malloc(sizeof(double) * (size_t)nv);
  double* d[3] = {NULL, NULL, NULL};
  int rc = ORC_OK;
  if (!tmp || !acc || !gm) { rc = ORC_ERR_NOMEM; goto done; }
  for (int a = 0; a < 3; ++a)
    if (!(d[a] = (double*)malloc(sizeof(double) * (size_t)nv))) { rc = ORC_ERR_NOMEM; goto done; }
  for (int64_t q = 0; q < nv; ++q) gin[q] = 0.0;
  for (int i = 0; i < n && rc == ORC_OK; ++i) {
    if (kinds[i] == ORC_G) {
      int ord[3] = {0, 0, 0};
      rc = orc_gaussian3d_adjoint(w[i], dims, sigmas[i], truncate, ord, acc);
      for (int64_t q = 0; rc == ORC_OK && q < nv; ++q) gin[q] += acc[q];
    } else if (kinds[i] == ORC_LOG) {
      for (int a = 0; a < 3 && rc == ORC_OK; ++a) {
        int ord[3] = {0, 0, 0};
        ord[a] = 2;
        rc = orc_gaussian3d_adjoint(w[i], dims, sigmas[i], truncate, ord, acc);
        for (int64_t q = 0; rc == ORC_OK && q < nv; ++q) gin[q] += acc[q];
      }
    } else if (kinds[i] == ORC_GM) {
      for (int a = 0; a < 3 && rc == ORC_OK; ++a) {
        int ord[3] = {0, 0, 0};
        ord[a] = 1;
        rc = orc_gaussian3d(in, dtype, zero, dims, dims, zero, dims, sigmas[i], truncate, ord, d[a]);
      }
      if (rc != ORC_OK) break;
      for (int64_t q = 0; q < nv; ++q)
        gm[q] = sqrt(d[0][q] * d[0][q] + d[1][q] * d[1][q] + d[2][q] * d[2][q]);
      for (int a = 0; a < 3 && rc == ORC_OK; ++a) {
        int ord[3] = {0, 0, 0};
        ord[a] = 1;
        /* dGM/dD_a = D_a / GM, taken as 0 where GM = 0 */
        for (int64_t q = 0; q < nv; ++q) tmp[q] = gm[q] > 0.0 ? w[i][q] * d[a][q] / gm[q] : 0.0;
        rc = orc_gaussian3d_adjoint(tmp, dims, sigmas[i], truncate, ord, acc);
        for (int64_t q = 0; rc == ORC_OK && q < nv; ++q) gin[q] += acc[q];
      }
    } else {
      rc = ORC_ERR_ARG;
    }
  }
done:
  free(tmp); free(acc); free(gm);
  for (int a = 0; a < 3; ++a) free(d[a]);
  return rc;
}

/* Morphology subgradient routing over a whole volume: for every output p,
 * gin[q*] += w[p], with q* the source holding the extreme value and, among
 * equal values, the smallest linear index. Also writes q* per output to
 * `arg` when it is not NULL. */
int orc_morph3d_vjp(const void* in, int dtype, const int64_t dims[3], int se, int rad,
                    int is_dilate, const double* w, double* gin, int64_t* arg) {
  if (dtype_size(dtype) == 0 || rad < 0) return ORC_ERR_ARG;
  int64_t nv = dims[0] * dims[1] * dims[2];
  for (int64_t q = 0; q < nv; ++q) gin[q] = 0.0;
  for (int64_t pz = 0; pz < dims[0]; ++pz)
    for (int64_t py = 0; py < dims[1]; ++py)
      for (int64_t px = 0; px < dims[2]; ++px) {
        int64_t best_q = -1;
        for (int dz = -rad; dz <= rad; ++dz)
          for (int dy = -rad; dy <= rad; ++dy)
            for (int dx = -rad; dx <= rad; ++dx) {
              if (!in_se(se, rad, dz, dy, dx)) continue;
              int sg = is_dilate ? -1 : 1;
              int64_t q = (orc_reflect(pz + sg * dz, dims[0]) * dims[1] +
                           orc_reflect(py + sg * dy, dims[1])) * dims[2] +
                          orc_reflect(px + sg * dx, dims[2]);
              int c = best_q < 0 ? 0 : total_cmp(in, dtype, q, best_q);
              int better = best_q < 0 || (is_dilate ? c > 0 : c < 0) || (c == 0 && q < best_q);
              if (better) best_q = q;
            }
        int64_t p = (pz * dims[1] + py) * dims[2] + px;
        gin[best_q] += w[p];
        if (arg) arg[p] = best_q;
      }
  return ORC_OK;
}

/* ------------------------------------------------ box statistics, thresholds */

/* Local sums over the cube window of half-width w with reflect boundary
 * (Sec. III-C local thresholds): s1[p] = sum f(R(p + o)), s2[p] = sum
 * f(R(p + o))^2 over |o|_inf <= w, whole volume. Accumulated separably in
 * FP64, x then y then z, each 1D window in increasing source coordinate
 * (exact for u8 / u16 input, whose sums stay below 2^53). */
int orc_box_sums(const void* in, int dtype, const int64_t d[3], int w, double* s1, double* s2) {
  if (dtype_size(dtype) == 0 || w < 0) return ORC_ERR_ARG;
  int64_t nv = d[0] * d[1] * d[2];
  double* a1 = (double*)malloc(sizeof(double) * (size_t)nv);
  double* a2 = (double*)malloc(sizeof(double) * (size_t)nv);
  double* b1 = (double*)malloc(sizeof(double) * (size_t)nv);
  double* b2 = (double*)malloc(sizeof(double) * (size_t)nv);
  int rc = ORC_OK;
  if (!a1 || !a2 || !b1 || !b2) { rc = ORC_ERR_NOMEM; goto done; }
  /* x */
#pragma omp parallel for schedule(static)
  for (int64_t z = 0; z < d[0]; ++z)
    for (int64_t y = 0; y < d[1]; ++y)
      for (int64_t x = 0; x < d[2]; ++x) {
        double t1 = 0.0, t2 = 0.0;
        for (int k = -w; k <= w; ++k) {
          double v = load_elem(in, dtype, (z * d[1] + y) * d[2] + orc_reflect(x + k, d[2]));
          t1 += v;
          t2 += v * v;
        }
        a1[(z * d[1] + y) * d[2] + x] = t1;
        a2[(z * d[1] + y) * d[2] + x] = t2;
      }
  /* y */
#pragma omp parallel for schedule(static)
  for (int64_t z = 0; z < d[0]; ++z)
    for (int64_t y = 0; y < d[1]; ++y)
      for (int64_t x = 0; x < d[2]; ++x) {
        double t1 = 0.0, t2 = 0.0;
        for (int k = -w; k <= w; ++k) {
          int64_t q = (z * d[1] + orc_reflect(y + k, d[1])) * d[2] + x;
          t1 += a1[q];
          t2 += a2[q];
        }
        b1[(z * d[1] + y) * d[2] + x] = t1;
        b2[(z * d[1] + y) * d[2] + x] = t2;
      }
  /* z */
#pragma omp parallel for schedule(static)
  for (int64_t z = 0; z < d[0]; ++z)
    for (int64_t y = 0; y < d[1]; ++y)
      for (int64_t x = 0; x < d[2]; ++x) {
        double t1 = 0.0, t2 = 0.0;
        for (int k = -w; k <= w; ++k) {
          int64_t q = (orc_reflect(z + k, d[0]) * d[1] + y) * d[2] + x;
          t1 += b1[q];
          t2 += b2[q];
        }
        s1[(z * d[1] + y) * d[2] + x] = t1;
        s2[(z * d[1] + y) * d[2] + x] = t2;
      }
done:
  free(a1); free(a2); free(b1); free(b2);
  return rc;
}

enum { ORC_LOCAL_MEAN = 0, ORC_LOCAL_NIBLACK = 1, ORC_LOCAL_SAUVOLA = 2 };

/* Local threshold from the window statistics, all in FP64 in this order
 * (Sec. III-C threshold algorithms):
 *   m = s1 / N,  v = max(s2 / N - m * m, 0),  s = sqrt(v),  N = (2w + 1)^3;
 *   mean:    T = m - c
 *   Niblack: T = m + k * s
 *   Sauvola: T = m * (1 + k * (s / c - 1))     (c = the dynamic range R)
 * and out = f > T (u8). Also writes T when `thr` is not NULL. */
int orc_threshold_box(const void* in, int dtype, const int64_t d[3], int method, int w, double k,
                      double c, uint8_t* out, double* thr) {
  if (method < ORC_LOCAL_MEAN || method > ORC_LOCAL_SAUVOLA) return ORC_ERR_ARG;
  int64_t nv = d[0] * d[1] * d[2];
  double* s1 = (double*)malloc(sizeof(double) * (size_t)nv);
  double* s2 = (double*)malloc(sizeof(double) * (size_t)nv);
  if (!s1 || !s2) { free(s1); free(s2); return ORC_ERR_NOMEM; }
  int rc = orc_box_sums(in, dtype, d, w, s1, s2);
  double n = (double)(2 * w + 1) * (double)(2 * w + 1) * (double)(2 * w + 1);
  for (int64_t q = 0; rc == ORC_OK && q < nv; ++q) {
    double m = s1[q] / n;
    double v = s2[q] / n - m * m;
    if (v < 0.0) v = 0.0;
    double s = sqrt(v);
    double t;
    if (method == ORC_LOCAL_MEAN) t = m - c;
    else if (method == ORC_LOCAL_NIBLACK) t = m + k * s;
    else t = m * (1.0 + k * (s / c - 1.0));
    out[q] = load_elem(in, dtype, q) > t ? 1 : 0;
    if (thr) thr[q] = t;
  }
  free(s1); free(s2);
  return rc;
}
