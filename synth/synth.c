/*
 * Seeded synthetic volumes for the chunked 3D filtering workloads.
 *
 * This module only draws inputs. It holds none of the filtering or
 * morphology arithmetic, and both the CPU oracle and the CUDA path read the
 * arrays it writes.
 *
 * Random numbers: counter-based splitmix64. Draw i of stream s is
 *   mix64(seed_s + (i + 1) * 0x9E3779B97F4A7C15)
 * with seed_s = seed ^ (s << 56), so every value depends only on
 * (seed, stream, counter) and never on the thread count.
 *
 * Generators (the paper's real tomogram is not available; these stand in
 * for it at the sizes of its 1-32 GiB sweep, Sec. IV-A):
 *   - spheres: background 0.2, N balls of value 1.0 with real centres
 *     uniform in the volume and radius U[4,16], plus i.i.d. N(0, 0.05^2).
 *   - porous:  Boolean model of pore balls, radius U[2,30], centres uniform,
 *     count chosen for 35% expected porosity; Poisson-like intensities
 *     12000 (solid) / 3000 (pore) with a 1% linear gradient along z.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GAMMA64 0x9E3779B97F4A7C15ULL

enum { ST_SPHERE = 1, ST_NOISE = 2, ST_FIELD = 3, ST_SPLIT = 4, ST_PICK = 5 };

static inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

static inline uint64_t draw(uint64_t seed, int stream, uint64_t i) {
  return mix64((seed ^ ((uint64_t)stream << 56)) + (i + 1) * GAMMA64);
}

/* uniform in [0, 1) with 53 random bits */
static inline double unif(uint64_t seed, int stream, uint64_t i) {
  return (double)(draw(seed, stream, i) >> 11) * (1.0 / 9007199254740992.0);
}

/* standard normal by Box-Muller from draws 2i and 2i+1 */
static inline double normal(uint64_t seed, int stream, uint64_t i) {
  double u1 = ((double)(draw(seed, stream, 2 * i) >> 11) + 1.0) * (1.0 / 9007199254740992.0);
  double u2 = (double)(draw(seed, stream, 2 * i + 1) >> 11) * (1.0 / 9007199254740992.0);
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

uint64_t synth_draw_u64(uint64_t seed, int stream, uint64_t i) { return draw(seed, stream, i); }
double synth_uniform(uint64_t seed, int stream, uint64_t i) { return unif(seed, stream, i); }
double synth_normal(uint64_t seed, int stream, uint64_t i) { return normal(seed, stream, i); }

typedef struct { double cz, cy, cx, r; } ball_t;

/* Paint a 0/1 mask of the union of balls. A voxel (z,y,x) is inside when
 * (z-cz)^2 + (y-cy)^2 + (x-cx)^2 <= r^2 (voxel centres at integer
 * coordinates). Parallel over z planes only, so each plane is written by
 * one thread. */
static void paint_balls(uint8_t* mask, int64_t nx, int64_t ny, int64_t nz,
                        const ball_t* b, int64_t nb) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t z = 0; z < nz; ++z) {
    uint8_t* plane = mask + z * nx * ny;
    for (int64_t s = 0; s < nb; ++s) {
      double dz = (double)z - b[s].cz;
      double rr = b[s].r * b[s].r - dz * dz;
      if (rr < 0) continue;
      double ry = sqrt(rr);
      int64_t y0 = (int64_t)ceil(b[s].cy - ry), y1 = (int64_t)floor(b[s].cy + ry);
      if (y0 < 0) y0 = 0;
      if (y1 > ny - 1) y1 = ny - 1;
      for (int64_t y = y0; y <= y1; ++y) {
        double dy = (double)y - b[s].cy;
        double rx2 = rr - dy * dy;
        if (rx2 < 0) continue;
        double rx = sqrt(rx2);
        int64_t x0 = (int64_t)ceil(b[s].cx - rx), x1 = (int64_t)floor(b[s].cx + rx);
        if (x0 < 0) x0 = 0;
        if (x1 > nx - 1) x1 = nx - 1;
        for (int64_t x = x0; x <= x1; ++x) {
          double dx = (double)x - b[s].cx;
          if (dz * dz + dy * dy + dx * dx <= b[s].r * b[s].r) plane[y * nx + x] = 1;
        }
      }
    }
  }
}

static ball_t* draw_balls(uint64_t seed, int64_t nb, int64_t nx, int64_t ny, int64_t nz,
                          double rmin, double rmax) {
  ball_t* b = (ball_t*)malloc(sizeof(ball_t) * (size_t)(nb > 0 ? nb : 1));
  if (!b) return NULL;
  for (int64_t s = 0; s < nb; ++s) {
    b[s].cz = unif(seed, ST_SPHERE, 4 * s + 0) * (double)nz;
    b[s].cy = unif(seed, ST_SPHERE, 4 * s + 1) * (double)ny;
    b[s].cx = unif(seed, ST_SPHERE, 4 * s + 2) * (double)nx;
    b[s].r = rmin + (rmax - rmin) * unif(seed, ST_SPHERE, 4 * s + 3);
  }
  return b;
}

/* Spheres volume, float32. Returns 0 on success, -1 on allocation failure. */
int synth_spheres_f32(float* out, int64_t nx, int64_t ny, int64_t nz, int64_t nspheres,
                      uint64_t seed) {
  int64_t n = nx * ny * nz;
  uint8_t* mask = (uint8_t*)calloc((size_t)n, 1);
  ball_t* b = draw_balls(seed, nspheres, nx, ny, nz, 4.0, 16.0);
  if (!mask || !b) { free(mask); free(b); return -1; }
  paint_balls(mask, nx, ny, nz, b, nspheres);
#pragma omp parallel for schedule(static)
  for (int64_t q = 0; q < n; ++q) {
    double v = mask[q] ? 1.0 : 0.2;
    out[q] = (float)(v + 0.05 * normal(seed, ST_NOISE, (uint64_t)q));
  }
  free(mask);
  free(b);
  return 0;
}

/* Number of pore balls for the target porosity:
 * N = ceil(-ln(1 - phi) * V / E[4/3 pi r^3]), r ~ U[rmin, rmax],
 * E[r^3] = (rmax^4 - rmin^4) / (4 (rmax - rmin)). */
int64_t synth_porous_count(int64_t nx, int64_t ny, int64_t nz, double porosity) {
  const double rmin = 2.0, rmax = 30.0;
  double er3 = (pow(rmax, 4) - pow(rmin, 4)) / (4.0 * (rmax - rmin));
  double ev = 4.0 / 3.0 * 3.14159265358979323846 * er3;
  double v = (double)nx * (double)ny * (double)nz;
  return (int64_t)ceil(-log(1.0 - porosity) * v / ev);
}

/* Porous-media tomogram, uint16. Writes the pore fraction actually drawn to
 * *porosity_out (may be NULL). */
int synth_porous_u16(uint16_t* out, int64_t nx, int64_t ny, int64_t nz, uint64_t seed,
                     double* porosity_out) {
  int64_t n = nx * ny * nz;
  int64_t nb = synth_porous_count(nx, ny, nz, 0.35);
  uint8_t* mask = (uint8_t*)calloc((size_t)n, 1);
  ball_t* b = draw_balls(seed, nb, nx, ny, nz, 2.0, 30.0);
  if (!mask || !b) { free(mask); free(b); return -1; }
  paint_balls(mask, nx, ny, nz, b, nb);
  int64_t pores = 0;
#pragma omp parallel for schedule(static) reduction(+ : pores)
  for (int64_t q = 0; q < n; ++q) {
    int64_t z = q / (nx * ny);
    double grad = 1.0 + 0.01 * ((nz > 1 ? (double)z / (double)(nz - 1) : 0.0) - 0.5);
    double lam = (mask[q] ? 3000.0 : 12000.0) * grad;
    double v = lam + sqrt(lam) * normal(seed, ST_NOISE, (uint64_t)q);
    v = floor(v + 0.5);
    if (v < 0) v = 0;
    if (v > 65535) v = 65535;
    out[q] = (uint16_t)v;
    pores += mask[q];
  }
  if (porosity_out) *porosity_out = (double)pores / (double)n;
  free(mask);
  free(b);
  return 0;
}

/* i.i.d. N(0,1) field in float32 (seeded weight fields for a scalar loss). */
void synth_normal_f32(float* out, int64_t n, uint64_t seed) {
#pragma omp parallel for schedule(static)
  for (int64_t q = 0; q < n; ++q) out[q] = (float)normal(seed, ST_FIELD, (uint64_t)q);
}

/* i.i.d. N(0,1) field in float64. */
void synth_normal_f64(double* out, int64_t n, uint64_t seed) {
#pragma omp parallel for schedule(static)
  for (int64_t q = 0; q < n; ++q) out[q] = normal(seed, ST_FIELD, (uint64_t)q);
}

/* Seeded k-d partition of a volume into `nbricks` disjoint boxes.
 * Start from the 8 octants, then repeatedly split the brick with the largest
 * side (lowest index on ties) along that side, at a uniformly drawn multiple
 * of `quantum` that leaves both parts at least `minside` long. Boxes are
 * written as [z0, y0, x0, z1, y1, x1] (half-open). Returns the number of
 * boxes written (< nbricks if no further legal split exists), or -1 on bad
 * arguments. */
int synth_kd_bricks(int64_t* boxes, int nbricks, int64_t nx, int64_t ny, int64_t nz,
                    int64_t minside, int64_t quantum, uint64_t seed) {
  if (nbricks < 8 || quantum <= 0 || minside <= 0) return -1;
  int64_t dims[3] = {nz, ny, nx};
  int count = 0;
  for (int o = 0; o < 8; ++o) {
    int64_t* b = boxes + 6 * count;
    for (int a = 0; a < 3; ++a) {
      int64_t half = dims[a] / 2;
      int bit = (o >> (2 - a)) & 1;
      b[a] = bit ? half : 0;
      b[3 + a] = bit ? dims[a] : half;
    }
    ++count;
  }
  uint64_t ctr = 0;
  while (count < nbricks) {
    int best = -1, best_axis = 0;
    int64_t best_len = -1;
    for (int i = 0; i < count; ++i)
      for (int a = 0; a < 3; ++a) {
        int64_t len = boxes[6 * i + 3 + a] - boxes[6 * i + a];
        if (len > best_len) { best_len = len; best = i; best_axis = a; }
      }
    int64_t lo = boxes[6 * best + best_axis], hi = boxes[6 * best + 3 + best_axis];
    /* legal cut offsets c (relative to lo): multiple of quantum, c >= minside,
     * (hi - lo) - c >= minside */
    int64_t cmin = (minside + quantum - 1) / quantum * quantum;
    int64_t cmax = ((hi - lo) - minside) / quantum * quantum;
    if (cmax < cmin) break;
    int64_t nchoice = (cmax - cmin) / quantum + 1;
    int64_t pick = (int64_t)(unif(seed, ST_SPLIT, ctr++) * (double)nchoice);
    if (pick >= nchoice) pick = nchoice - 1;
    int64_t cut = lo + cmin + pick * quantum;
    int64_t* nb = boxes + 6 * count;
    memcpy(nb, boxes + 6 * best, 6 * sizeof(int64_t));
    boxes[6 * best + 3 + best_axis] = cut;
    nb[best_axis] = cut;
    ++count;
  }
  return count;
}

/* Distinct random voxel indices are not required; this draws m linear
 * indices uniformly (with replacement) from [0, n). */
void synth_pick(int64_t* out, int64_t m, int64_t n, uint64_t seed) {
  for (int64_t i = 0; i < m; ++i) {
    int64_t v = (int64_t)(unif(seed, ST_PICK, (uint64_t)i) * (double)n);
    out[i] = v < n ? v : n - 1;
  }
}
