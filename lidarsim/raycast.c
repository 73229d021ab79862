/*
 * raycast.c - seeded FP64 ray-caster that produces synthetic spinning-Lidar scans.
 *
 * This is the input generator shared by the tests, the oracle checks and the
 * benchmark.  It models the sensor of Sec. 2 of Mukherjee et al. (PReMI 2019,
 * "Fast Geometric Surface based Segmentation of Point Cloud from Lidar Data"):
 * a vertical array of lasers at fixed elevations theta, spun about the z axis,
 * firing W times per revolution at azimuths phi_c = phi0 + c * dphi, each shot
 * returning a range r.  The paper's own scans come from the Blensor simulator
 * (Sec. 3), which needs a graphics stack; this file replaces it with plain ray
 * / primitive intersection over analytic planes, axis-aligned boxes and
 * vertical cylinders.
 *
 * It holds none of the segmentation method's arithmetic (meshing, normals,
 * labelling).  All random numbers are drawn from SplitMix64 (Steele, Lea and
 * Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014), keyed
 * by (seed, ring, column, stream), so a scan depends only on its inputs and not
 * on the thread schedule.
 *
 * Build: gcc -O2 -fPIC -shared [-fopenmp] raycast.c -lm -o liblidarsim.so
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define PRIM_PLANE 0
#define PRIM_BOX 1
#define PRIM_CYL 2
#define PRIM_STRIDE 10 /* kind, id, a[0..7] */

static const double kPi = 3.14159265358979323846;

/* SplitMix64 output function applied to a counter. */
static uint64_t smix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

/* Uniform double in (0, 1): 53 random bits, never exactly 0. */
static double u01(uint64_t key) {
  uint64_t v = smix64(key) >> 11;
  return ((double)v + 0.5) * (1.0 / 9007199254740992.0);
}

static uint64_t ray_key(uint64_t seed, int ring, int col, int stream) {
  uint64_t k = smix64(seed ^ 0xA0761D6478BD642Full);
  k = smix64(k ^ ((uint64_t)(uint32_t)ring << 32 | (uint32_t)col));
  return k ^ ((uint64_t)stream * 0xE7037ED1A0B428DBull);
}

static double wrap_pi(double a) {
  while (a > kPi) a -= 2.0 * kPi;
  while (a <= -kPi) a += 2.0 * kPi;
  return a;
}

/* Nearest hit t > 0 of the ray t*d (origin at the sensor) with one primitive.
 * Returns 1 on a hit and sets *t and *face. */
static int hit_plane(const double* a, const double d[3], double* t, int* face) {
  double nd = a[0] * d[0] + a[1] * d[1] + a[2] * d[2];
  if (fabs(nd) < 1e-300) return 0;
  double tt = a[3] / nd;
  if (!(tt > 1e-9)) return 0;
  *t = tt;
  *face = 0;
  return 1;
}

static int hit_box(const double* a, const double d[3], double* t, int* face) {
  double tn = -INFINITY, tf = INFINITY;
  int fn = -1;
  for (int k = 0; k < 3; ++k) {
    double lo = a[k], hi = a[3 + k];
    if (fabs(d[k]) < 1e-300) {
      if (0.0 < lo || 0.0 > hi) return 0;
      continue;
    }
    double t1 = lo / d[k], t2 = hi / d[k];
    int f1 = 2 * k, f2 = 2 * k + 1; /* 2k: min face of axis k, 2k+1: max face */
    if (t1 > t2) {
      double tmp = t1; t1 = t2; t2 = tmp;
      int ft = f1; f1 = f2; f2 = ft;
    }
    if (t1 > tn) { tn = t1; fn = f1; }
    if (t2 < tf) tf = t2;
    if (tn > tf) return 0;
  }
  if (!(tn > 1e-9) || fn < 0) return 0; /* sensor inside or behind */
  *t = tn;
  *face = fn;
  return 1;
}

static int hit_cyl(const double* a, const double d[3], double* t, int* face) {
  double cx = a[0], cy = a[1], rho = a[2], z0 = a[3], z1 = a[4];
  double best = INFINITY;
  int bf = -1;
  double qa = d[0] * d[0] + d[1] * d[1];
  if (qa > 1e-300) {
    double qb = -2.0 * (d[0] * cx + d[1] * cy);
    double qc = cx * cx + cy * cy - rho * rho;
    double disc = qb * qb - 4.0 * qa * qc;
    if (disc >= 0.0) {
      double sq = sqrt(disc);
      double r0 = (-qb - sq) / (2.0 * qa), r1 = (-qb + sq) / (2.0 * qa);
      double cand[2] = {r0, r1};
      for (int k = 0; k < 2; ++k) {
        double tt = cand[k];
        if (tt > 1e-9 && tt < best) {
          double z = tt * d[2];
          if (z >= z0 && z <= z1) { best = tt; bf = 0; }
        }
      }
    }
  }
  if (fabs(d[2]) > 1e-300) {
    double caps[2] = {z1, z0};
    for (int k = 0; k < 2; ++k) {
      double tt = caps[k] / d[2];
      if (tt > 1e-9 && tt < best) {
        double x = tt * d[0] - cx, y = tt * d[1] - cy;
        if (x * x + y * y <= rho * rho) { best = tt; bf = 1 + k; }
      }
    }
  }
  if (bf < 0) return 0;
  *t = best;
  *face = bf;
  return 1;
}

/* Azimuth interval of a primitive as (centre, lo, hi) offsets; planes are
 * always candidates (flag 0). */
static int prim_interval(const double* p, double* ac, double* lo, double* hi) {
  int kind = (int)p[0];
  const double* a = p + 2;
  if (kind == PRIM_BOX) {
    double cx = 0.5 * (a[0] + a[3]), cy = 0.5 * (a[1] + a[4]);
    if (a[0] <= 0.0 && a[3] >= 0.0 && a[1] <= 0.0 && a[4] >= 0.0) return 0;
    *ac = atan2(cy, cx);
    double mn = 0.0, mx = 0.0;
    double xs[2] = {a[0], a[3]}, ys[2] = {a[1], a[4]};
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 2; ++j) {
        double dl = wrap_pi(atan2(ys[j], xs[i]) - *ac);
        if (dl < mn) mn = dl;
        if (dl > mx) mx = dl;
      }
    *lo = mn - 1e-9;
    *hi = mx + 1e-9;
    return 1;
  }
  if (kind == PRIM_CYL) {
    double dist = sqrt(a[0] * a[0] + a[1] * a[1]);
    if (dist <= a[2] * 1.0000001) return 0;
    *ac = atan2(a[1], a[0]);
    double half = asin(a[2] / dist) + 1e-9;
    *lo = -half;
    *hi = half;
    return 1;
  }
  return 0;
}

/*
 * Ray-cast one scan.
 *   H, W          rings and shots per revolution
 *   elev[H]       ring elevations (radians), in the order rows are written
 *   az0, daz      azimuth of column 0 and step (radians)
 *   prims[n*10]   primitives: kind, id, a[0..7]
 *   sigma         Gaussian range noise (m); p_drop dropout probability
 *   r_max         returns beyond this range are dropped (range 0)
 *   seed          noise / dropout seed
 * Outputs (caller-allocated):
 *   xyzr[H*W*4]   float x, y, z, range (range 0 = no return, xyz 0)
 *   gt[H*W]       primitive id * 8 + face of the surface hit, -1 if none
 */
int lidarsim_raycast(int H, int W, const double* elev, double az0, double daz,
                     int nprims, const double* prims, double sigma, double p_drop,
                     double r_max, uint64_t seed, float* xyzr, int32_t* gt) {
  if (H < 0 || W < 0 || nprims < 0) return -1;
  /* per-primitive azimuth intervals */
  double* iv = (double*)malloc(sizeof(double) * 4 * (size_t)(nprims > 0 ? nprims : 1));
  if (!iv) return -2;
  for (int k = 0; k < nprims; ++k) {
    double ac = 0, lo = 0, hi = 0;
    int f = prim_interval(prims + (size_t)k * PRIM_STRIDE, &ac, &lo, &hi);
    iv[4 * k + 0] = f;
    iv[4 * k + 1] = ac;
    iv[4 * k + 2] = lo;
    iv[4 * k + 3] = hi;
  }
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 16)
#endif
  for (int c = 0; c < W; ++c) {
    double phi = az0 + (double)c * daz;
    double cphi = cos(phi), sphi = sin(phi);
    for (int i = 0; i < H; ++i) {
      double ce = cos(elev[i]), se = sin(elev[i]);
      double d[3] = {ce * cphi, ce * sphi, se};
      double best = INFINITY;
      int bid = -1;
      for (int k = 0; k < nprims; ++k) {
        const double* p = prims + (size_t)k * PRIM_STRIDE;
        if (iv[4 * k] != 0.0) {
          double dl = wrap_pi(phi - iv[4 * k + 1]);
          if (dl < iv[4 * k + 2] || dl > iv[4 * k + 3]) continue;
        }
        double t = 0;
        int face = 0, h = 0;
        switch ((int)p[0]) {
          case PRIM_PLANE: h = hit_plane(p + 2, d, &t, &face); break;
          case PRIM_BOX: h = hit_box(p + 2, d, &t, &face); break;
          case PRIM_CYL: h = hit_cyl(p + 2, d, &t, &face); break;
          default: h = 0;
        }
        if (h && t < best) {
          best = t;
          bid = (int)p[1] * 8 + face;
        }
      }
      size_t o = (size_t)i * W + c;
      float r = 0.0f;
      int id = -1;
      if (bid >= 0 && best <= r_max) {
        uint64_t key = ray_key(seed, i, c, 0);
        double u1 = u01(key), u2 = u01(key ^ 0x5851F42D4C957F2Dull);
        double ud = u01(key ^ 0x14057B7EF767814Full);
        double g = sqrt(-2.0 * log(u1)) * cos(2.0 * kPi * u2); /* Box-Muller */
        double rn = best + sigma * g;
        if (ud >= p_drop && rn > 0.0 && rn <= r_max) {
          r = (float)rn;
          id = bid;
        }
      }
      if (r > 0.0f) {
        double rd = (double)r;
        xyzr[4 * o + 0] = (float)(rd * d[0]);
        xyzr[4 * o + 1] = (float)(rd * d[1]);
        xyzr[4 * o + 2] = (float)(rd * d[2]);
      } else {
        xyzr[4 * o + 0] = xyzr[4 * o + 1] = xyzr[4 * o + 2] = 0.0f;
      }
      xyzr[4 * o + 3] = r;
      gt[o] = id;
    }
  }
  free(iv);
  return 0;
}
