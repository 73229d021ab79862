/*
 * lsg_raycast.h - synthetic spinning-Lidar scans generated on the GPU.
 *
 * Data generation for tests and load, not part of the segmentation method.
 * Mukherjee et al. (PReMI 2019) evaluate on scans from a Lidar simulator
 * (Sec. 3: a Velodyne-32E-like sensor over scenes of primitives on a floor,
 * with Gaussian range noise).  This entry point produces scans of that kind
 * from an analytic scene, on the device, in the input layout lsg_segment
 * takes (lsg.h: x, y, z, r float32 per point, rows in the order of the given
 * elevations).
 *
 * Sensor model (Sec. 2): ring i fires along elevation theta_i; shot c of a
 * revolution along azimuth phi_c = azimuth0 + c * azimuth_step; the return of
 * a ray is the nearest intersection with the scene, plus noise.
 *
 * Scene: a table of primitives, one row of ten float64 per primitive:
 *   row[0] kind (LSG_PRIM_*), row[1] id (an integer >= 0), row[2..9] a[0..7]:
 *     LSG_PRIM_PLANE  a = n_x, n_y, n_z, d         points p with n . p = d
 *     LSG_PRIM_BOX    a = lo_x, lo_y, lo_z, hi_x, hi_y, hi_z   axis-aligned
 *     LSG_PRIM_CYL    a = c_x, c_y, rho, z0, z1    vertical axis through
 *                                                   (c_x, c_y), radius rho,
 *                                                   z0 <= z <= z1, capped
 * Ground truth of a return: id * 8 + face, face = 0 for a plane or a
 * cylinder's side, 1 / 2 for its top (z1) / bottom (z0) cap, 2k / 2k+1 for a
 * box's min / max face along axis k; -1 where the ray returns nothing.
 *
 * Noise: a hit at distance t <= r_max returns r = t + sigma * g, with g a
 * standard Gaussian (Box-Muller), unless a dropout (probability p_drop)
 * removes it; returns with r <= 0 or r > r_max are removed too.  A removed
 * return has r = 0 and x = y = z = 0.  The random numbers of ray (i, c) are
 * SplitMix64 outputs (Steele, Lea and Flood, OOPSLA 2014) keyed by
 * (seed, i, c): u = (top 53 bits + 1/2) / 2^53 of smix64(key), smix64(key ^
 * 0x5851F42D4C957F2D) and smix64(key ^ 0x14057B7EF767814F) for the two
 * Box-Muller uniforms and the dropout uniform, where key =
 * smix64(smix64(seed ^ 0xA0761D6478BD642F) ^ (i << 32 | c)).
 *
 * Precision: directions are formed in float64 from the float32 angles, the
 * intersections and the Gaussian in float32, the dropout test in float64.
 */
#ifndef LSG_RAYCAST_H
#define LSG_RAYCAST_H

#include "lsg.h"

#ifdef __cplusplus
extern "C" {
#endif

#define LSG_RAYCAST_MAX_PRIMS 256

enum { LSG_PRIM_PLANE = 0, LSG_PRIM_BOX = 1, LSG_PRIM_CYL = 2 };

typedef struct {
  int32_t rings, cols;     /* H, W */
  const float* elevation;  /* device [rings], radians, in output row order */
  float azimuth0;          /* radians */
  float azimuth_step;      /* radians */
  int32_t nprims;          /* 0 .. LSG_RAYCAST_MAX_PRIMS */
  const double* prims;     /* device [nprims][10], the table above */
  double sigma;            /* range noise, >= 0 */
  double p_drop;           /* dropout probability, 0 .. 1 */
  double r_max;            /* farthest return, > 0 */
  uint64_t seed;
} lsg_raycast_spec;

/* Ray-casts one scan into caller-owned device buffers:
 *   xyzr  float32 [rings][cols][4], 16-byte aligned (x, y, z, r)
 *   gt    int32 [rings][cols] ground-truth face ids, or NULL
 * Stream-ordered and asynchronous on the current CUDA device; the spec is
 * read at call time.  Returns LSG_E_ARG for a NULL spec / xyzr, negative
 * sizes, nprims outside 0 .. LSG_RAYCAST_MAX_PRIMS, a misaligned xyzr or
 * noise parameters out of range; LSG_E_SHAPE for more than LSG_MAX_POINTS
 * points; LSG_E_CUDA if the launch fails.  An empty scan launches nothing. */
lsg_status lsg_raycast(const lsg_raycast_spec* spec, float* xyzr, int32_t* gt, lsg_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* LSG_RAYCAST_H */
