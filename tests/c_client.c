/*
 * A plain C client of liblsg: no Python and no torch in the process, only
 * include/lsg.h, liblsg.so and the CUDA runtime for device memory.
 *
 *   c_client host   host-side calls: status strings, default parameters,
 *                   NULL handles refused with LSG_E_ARG.
 *   c_client gpu    one scan segmented on device 0 through lsg_segment.
 *
 * The scan of the gpu mode is a wall x = 10 m seen by 16 rings at
 * -15, -13, .., +15 degrees (given bottom ring first, so the library has to
 * sort them) over 96 shots from -24 to +23.5 degrees of azimuth, without
 * noise or dropouts.  Every point is in range and every mesh edge joins two
 * points of one plane, so (Sec. 2, Algorithm 1) the scan is a single segment
 * whose label is the smallest point index, 0, and every vertex has the wall's
 * normal facing the sensor, (-1, 0, 0).  Prints "ok" and exits 0 when all of
 * that holds.
 */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cuda_runtime_api.h>

#include "lsg.h"

#define H 16
#define W 96

static int fail(const char* what) {
  fprintf(stderr, "c_client: %s\n", what);
  return 1;
}

static int host_mode(void) {
  lsg_params p;
  lsg_ctx* ctx = NULL;
  if (strcmp(lsg_status_str(LSG_OK), "ok") != 0) return fail("status string of LSG_OK");
  for (int s = LSG_OK; s <= LSG_E_DEVICE; ++s)
    if (!lsg_status_str((lsg_status)s) || !lsg_status_str((lsg_status)s)[0]) return fail("empty status string");
  lsg_default_params(&p);
  if (p.subsample != 1 || p.wrap != 1 || p.predicate != LSG_PRED_ANGLE || !(p.r_max > p.r_min))
    return fail("default parameters");
  if (lsg_segment(NULL, NULL, NULL, NULL, NULL) != LSG_E_ARG) return fail("NULL context accepted");
  if (lsg_destroy(NULL) != LSG_E_ARG) return fail("NULL destroy accepted");
  if (lsg_create(-1, 0, &ctx) != LSG_E_ARG || ctx != NULL) return fail("device -1 accepted");
  printf("ok\n");
  return 0;
}

static int gpu_mode(void) {
  const double pi = 3.14159265358979323846;
  static float elev[H], xyzr[H * W * 4], normals[H * W * 3];
  static int32_t labels[H * W];
  static uint8_t mb[H * W];
  int32_t nseg = -1;
  const float az0 = (float)(-24.0 * pi / 180.0), daz = (float)(0.5 * pi / 180.0);
  for (int i = 0; i < H; ++i) {
    const double th = (double)(float)((-15.0 + 2.0 * i) * pi / 180.0);
    elev[i] = (float)th;
    for (int c = 0; c < W; ++c) {
      const double ph = (double)az0 + c * (double)daz;
      const double dx = cos(th) * cos(ph), dy = cos(th) * sin(ph), dz = sin(th);
      const double r = 10.0 / dx;  /* the ray meets the wall x = 10 */
      float* q = xyzr + 4 * (i * W + c);
      q[0] = (float)(r * dx);
      q[1] = (float)(r * dy);
      q[2] = (float)(r * dz);
      q[3] = (float)r;
    }
  }
  float *d_elev = NULL, *d_xyzr = NULL, *d_nrm = NULL;
  int32_t *d_lab = NULL, *d_nseg = NULL;
  uint8_t* d_mb = NULL;
  if (cudaMalloc((void**)&d_elev, sizeof elev) != cudaSuccess ||
      cudaMalloc((void**)&d_xyzr, sizeof xyzr) != cudaSuccess ||
      cudaMalloc((void**)&d_nrm, sizeof normals) != cudaSuccess ||
      cudaMalloc((void**)&d_lab, sizeof labels) != cudaSuccess ||
      cudaMalloc((void**)&d_mb, sizeof mb) != cudaSuccess || cudaMalloc((void**)&d_nseg, sizeof nseg) != cudaSuccess)
    return fail("cudaMalloc");
  if (cudaMemcpy(d_elev, elev, sizeof elev, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(d_xyzr, xyzr, sizeof xyzr, cudaMemcpyHostToDevice) != cudaSuccess)
    return fail("cudaMemcpy in");

  lsg_ctx* ctx = NULL;
  lsg_status st = lsg_create(0, 0, &ctx);
  if (st != LSG_OK) return fail(lsg_status_str(st));
  lsg_scan scan = {H, W, d_elev, az0, daz, d_xyzr, NULL};
  lsg_params p;
  lsg_default_params(&p);
  p.wrap = 0; /* a partial sweep */
  lsg_out out = {d_mb, d_nrm, d_lab, d_nseg};
  st = lsg_segment(ctx, &scan, &p, &out, NULL);
  if (st != LSG_OK) return fail(lsg_status_str(st));
  if (cudaDeviceSynchronize() != cudaSuccess) return fail("cudaDeviceSynchronize");
  st = lsg_get_error(ctx);
  if (st != LSG_OK) return fail(lsg_status_str(st));
  if (cudaMemcpy(mb, d_mb, sizeof mb, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(normals, d_nrm, sizeof normals, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(labels, d_lab, sizeof labels, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(&nseg, d_nseg, sizeof nseg, cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail("cudaMemcpy out");
  lsg_destroy(ctx);

  if (nseg != 1) return fail("the wall is not one segment");
  for (int v = 0; v < H * W; ++v) {
    if (labels[v] != 0) return fail("a label other than 0");
    if ((mb[v] & (LSG_BIT_VALID | LSG_BIT_HASN)) != (LSG_BIT_VALID | LSG_BIT_HASN))
      return fail("a vertex without the valid or normal bit");
    const float* n = normals + 3 * v;
    if (!(n[0] < -0.999f) || fabsf(n[1]) > 1e-3f || fabsf(n[2]) > 1e-3f)
      return fail("a normal other than (-1, 0, 0)");
  }
  cudaFree(d_elev);
  cudaFree(d_xyzr);
  cudaFree(d_nrm);
  cudaFree(d_lab);
  cudaFree(d_mb);
  cudaFree(d_nseg);
  printf("ok\n");
  return 0;
}

int main(int argc, char** argv) {
  if (argc == 2 && strcmp(argv[1], "host") == 0) return host_mode();
  if (argc == 2 && strcmp(argv[1], "gpu") == 0) return gpu_mode();
  fprintf(stderr, "usage: c_client host|gpu\n");
  return 2;
}
