// lsg_raycast.cu - synthetic spinning-Lidar scans generated on the GPU.
//
// Data generation, not part of the segmentation method.  The paper's scans
// come from a Lidar simulator (Sec. 3: Velodyne-32E-like, 0.2 deg azimuth
// step, primitives on a floor, Gaussian range noise); this kernel produces
// the same kind of scan from an analytic scene (planes, axis-aligned boxes,
// capped vertical cylinders) fast enough to feed the segmentation at its own
// rate.
//
// One thread per azimuth column and group of 8 rings: it culls the
// primitives whose azimuth interval misses the column once (a bit mask over
// at most 256 primitives), then walks its rings.  Ray directions are formed in double from the
// float32 elevation and azimuth, the intersections run in binary32.  Noise
// and dropouts come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
// pseudorandom number generators", OOPSLA 2014) keyed by (seed, ring,
// column, stream): each ray's draws depend only on those keys, so any other
// generator keyed the same way draws the same numbers.  The dropout test is
// made on the 53-bit uniform in double; the Gaussian (Box-Muller) in
// binary32.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "lsg_raycast.h"

namespace {

constexpr int PSTRIDE = 10;     // table row: kind, id, a[0..7]
constexpr int SROW = 14;        // shared row: kind, id, a[0..7], flag, centre, lo, hi
constexpr int NT_RAY = 128;
constexpr int RG = 8;     // rings per thread (grid: columns x ring groups)
constexpr float kPiF = 3.14159265358979f;

__device__ __forceinline__ uint64_t smix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

// Uniform in (0, 1) from 53 random bits, never 0.
__device__ __forceinline__ double u01(uint64_t key) {
  const uint64_t v = smix64(key) >> 11;
  return ((double)v + 0.5) * (1.0 / 9007199254740992.0);
}

__device__ __forceinline__ uint64_t ray_key(uint64_t seed, int ring, int col) {
  uint64_t k = smix64(seed ^ 0xA0761D6478BD642Full);
  return smix64(k ^ ((uint64_t)(uint32_t)ring << 32 | (uint32_t)col));
}

__device__ __forceinline__ float wrap_pi(float a) {
  while (a > kPiF) a -= 2.f * kPiF;
  while (a <= -kPiF) a += 2.f * kPiF;
  return a;
}

// Azimuth interval (centre, lo, hi offsets) of a box or cylinder seen from
// the origin, widened by 1e-4 rad; flag 0 = always a candidate (planes, and
// primitives around the sensor).
__device__ void prim_interval(const float* p, float* out) {
  const int kind = (int)p[0];
  const float* a = p + 2;
  out[0] = 0.f;
  out[1] = out[2] = out[3] = 0.f;
  if (kind == LSG_PRIM_BOX) {
    if (a[0] <= 0.f && a[3] >= 0.f && a[1] <= 0.f && a[4] >= 0.f) return;
    const float cx = 0.5f * (a[0] + a[3]), cy = 0.5f * (a[1] + a[4]);
    const float ac = atan2f(cy, cx);
    float mn = 0.f, mx = 0.f;
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 2; ++j) {
        const float dl = wrap_pi(atan2f(a[1 + 3 * j], a[3 * i]) - ac);
        mn = fminf(mn, dl);
        mx = fmaxf(mx, dl);
      }
    out[0] = 1.f;
    out[1] = ac;
    out[2] = mn - 1e-4f;
    out[3] = mx + 1e-4f;
  } else if (kind == LSG_PRIM_CYL) {
    const float dist = sqrtf(a[0] * a[0] + a[1] * a[1]);
    if (dist <= a[2] * 1.001f) return;
    const float half = asinf(fminf(1.f, a[2] / dist)) + 1e-4f;
    out[0] = 1.f;
    out[1] = atan2f(a[1], a[0]);
    out[2] = -half;
    out[3] = half;
  }
}

// Nearest hit t > 0 of the ray t*d with one primitive (binary32).
__device__ __forceinline__ bool hit_plane(const float* a, float dx, float dy, float dz, float& t, int& face) {
  const float nd = fmaf(a[0], dx, fmaf(a[1], dy, a[2] * dz));
  if (!(fabsf(nd) > 1e-30f)) return false;
  const float tt = a[3] / nd;
  if (!(tt > 1e-6f)) return false;
  t = tt;
  face = 0;
  return true;
}

__device__ __forceinline__ bool hit_box(const float* a, float dx, float dy, float dz, float& t, int& face) {
  const float d[3] = {dx, dy, dz};
  float tn = -INFINITY, tf = INFINITY;
  int fn = -1;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float lo = a[k], hi = a[3 + k];
    if (!(fabsf(d[k]) > 1e-30f)) {
      if (0.f < lo || 0.f > hi) return false;
      continue;
    }
    float t1 = lo / d[k], t2 = hi / d[k];
    int f1 = 2 * k, f2 = 2 * k + 1;  // 2k: the min face of axis k, 2k+1: the max face
    if (t1 > t2) {
      const float tmp = t1;
      t1 = t2;
      t2 = tmp;
      const int ft = f1;
      f1 = f2;
      f2 = ft;
    }
    if (t1 > tn) {
      tn = t1;
      fn = f1;
    }
    tf = fminf(tf, t2);
  }
  if (tn > tf || !(tn > 1e-6f) || fn < 0) return false;
  t = tn;
  face = fn;
  return true;
}

// Capped vertical cylinder.  The side is intersected in the horizontal
// plane around the closest approach of the ray to the axis (no difference
// of large squares), the caps as planes z = z0, z1.
__device__ __forceinline__ bool hit_cyl(const float* a, float dx, float dy, float dz, float& t, int& face) {
  const float cx = a[0], cy = a[1], rho = a[2], z0 = a[3], z1 = a[4];
  float best = INFINITY;
  int bf = -1;
  const float qa = fmaf(dx, dx, dy * dy);
  if (qa > 1e-30f) {
    const float tm = fmaf(dx, cx, dy * cy) / qa;   // closest approach
    const float cr = fmaf(cx, dy, -cy * dx);       // |C x D|
    const float h2 = cr * cr / qa;                  // squared distance of closest approach
    const float e = rho * rho - h2;
    if (e >= 0.f) {
      const float hc = sqrtf(e / qa);
      const float cand[2] = {tm - hc, tm + hc};
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const float tt = cand[k];
        if (tt > 1e-6f && tt < best) {
          const float z = tt * dz;
          if (z >= z0 && z <= z1) {
            best = tt;
            bf = 0;
          }
        }
      }
    }
  }
  if (fabsf(dz) > 1e-30f) {
    const float caps[2] = {z1, z0};
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const float tt = caps[k] / dz;
      if (tt > 1e-6f && tt < best) {
        const float x = fmaf(tt, dx, -cx), y = fmaf(tt, dy, -cy);
        if (fmaf(x, x, y * y) <= rho * rho) {
          best = tt;
          bf = 1 + k;
        }
      }
    }
  }
  if (bf < 0) return false;
  t = best;
  face = bf;
  return true;
}

struct RayArgs {
  int H, W, n;
  const float* elev;
  double az0, daz;
  const double* prims;
  float sigma, r_max;
  double p_drop, r_max_d;
  uint64_t seed;
  float* xyzr;
  int32_t* gt;
};

__global__ void __launch_bounds__(NT_RAY) k_raycast(const __grid_constant__ RayArgs a) {
  extern __shared__ double2 dyn[];  // [RG] (cos, sin) of the group's elevations, then [n][SROW] floats
  const int i0 = blockIdx.y * RG, i1 = min(a.H, i0 + RG);
  double2* trig = dyn;
  float* sp = reinterpret_cast<float*>(dyn + RG);
  for (int i = i0 + (int)threadIdx.x; i < i1; i += NT_RAY) {
    double se, ce;
    sincos((double)a.elev[i], &se, &ce);
    trig[i - i0] = make_double2(ce, se);
  }
  for (int k = threadIdx.x; k < a.n; k += NT_RAY) {
    float* row = sp + k * SROW;
    for (int q = 0; q < PSTRIDE; ++q) row[q] = (float)a.prims[(size_t)k * PSTRIDE + q];
    prim_interval(row, row + PSTRIDE);
  }
  __syncthreads();
  const int c = blockIdx.x * NT_RAY + threadIdx.x;
  if (c >= a.W) return;
  const double phi = a.az0 + (double)c * a.daz;
  double sphi, cphi;
  sincos(phi, &sphi, &cphi);
  const float phif = (float)phi;
  // primitives whose azimuth interval holds this column
  uint32_t cand[LSG_RAYCAST_MAX_PRIMS / 32];
#pragma unroll
  for (int w = 0; w < LSG_RAYCAST_MAX_PRIMS / 32; ++w) {
    uint32_t m = 0;
    for (int b = 0; b < 32; ++b) {
      const int k = 32 * w + b;
      if (k >= a.n) break;
      const float* iv = sp + k * SROW + PSTRIDE;
      bool in = true;
      if (iv[0] != 0.f) {
        const float dl = wrap_pi(phif - iv[1]);
        in = dl >= iv[2] && dl <= iv[3];
      }
      m |= (uint32_t)in << b;
    }
    cand[w] = m;
  }
  for (int i = i0; i < i1; ++i) {
    const double2 t2 = trig[i - i0];
    const double ce = t2.x, se = t2.y;
    const double d0 = ce * cphi, d1 = ce * sphi, d2 = se;
    const float dx = (float)d0, dy = (float)d1, dz = (float)d2;
    float best = INFINITY;
    int bid = -1;
#pragma unroll
    for (int w = 0; w < LSG_RAYCAST_MAX_PRIMS / 32; ++w) {
      uint32_t m = cand[w];
      while (m) {
        const int k = 32 * w + __ffs(m) - 1;
        m &= m - 1;
        const float* p = sp + k * SROW;
        float t = 0.f;
        int face = 0;
        bool h = false;
        switch ((int)p[0]) {
          case LSG_PRIM_PLANE: h = hit_plane(p + 2, dx, dy, dz, t, face); break;
          case LSG_PRIM_BOX: h = hit_box(p + 2, dx, dy, dz, t, face); break;
          case LSG_PRIM_CYL: h = hit_cyl(p + 2, dx, dy, dz, t, face); break;
          default: break;
        }
        if (h && t < best) {
          best = t;
          bid = (int)p[1] * 8 + face;
        }
      }
    }
    const size_t o = (size_t)i * a.W + c;
    float r = 0.f;
    int id = -1;
    if (bid >= 0 && (double)best <= a.r_max_d) {
      const uint64_t key = ray_key(a.seed, i, c);
      const float u1 = (float)u01(key), u2 = (float)u01(key ^ 0x5851F42D4C957F2Dull);
      const double ud = u01(key ^ 0x14057B7EF767814Full);
      const float g = sqrtf(-2.f * logf(u1)) * cosf(2.f * kPiF * u2);  // Box-Muller
      const float rn = fmaf(a.sigma, g, best);
      if (ud >= a.p_drop && rn > 0.f && rn <= a.r_max) {
        r = rn;
        id = bid;
      }
    }
    float4 out = make_float4(0.f, 0.f, 0.f, r);
    if (r > 0.f) {
      const double rd = (double)r;
      out.x = (float)(rd * d0);
      out.y = (float)(rd * d1);
      out.z = (float)(rd * d2);
    }
    reinterpret_cast<float4*>(a.xyzr)[o] = out;
    if (a.gt) a.gt[o] = id;
  }
}

}  // namespace

extern "C" lsg_status lsg_raycast(const lsg_raycast_spec* spec, float* xyzr, int32_t* gt, lsg_stream stream) {
  if (!spec || !xyzr) return LSG_E_ARG;
  const lsg_raycast_spec& s = *spec;
  if (s.rings < 0 || s.cols < 0 || s.nprims < 0) return LSG_E_ARG;
  if (s.nprims > LSG_RAYCAST_MAX_PRIMS || (s.nprims > 0 && !s.prims)) return LSG_E_ARG;
  if ((size_t)s.rings * (size_t)s.cols > (size_t)LSG_MAX_POINTS) return LSG_E_SHAPE;
  if (s.rings == 0 || s.cols == 0) return LSG_OK;
  if (!s.elevation) return LSG_E_ARG;
  if (reinterpret_cast<uintptr_t>(xyzr) % 16) return LSG_E_ARG;
  if (!(s.sigma >= 0.0) || !(s.r_max > 0.0) || !(s.p_drop >= 0.0 && s.p_drop <= 1.0)) return LSG_E_ARG;
  RayArgs a;
  a.H = s.rings;
  a.W = s.cols;
  a.n = s.nprims;
  a.elev = s.elevation;
  a.az0 = (double)s.azimuth0;
  a.daz = (double)s.azimuth_step;
  a.prims = s.prims;
  a.sigma = (float)s.sigma;
  a.r_max = (float)s.r_max;
  a.r_max_d = s.r_max;
  a.p_drop = s.p_drop;
  a.seed = s.seed;
  a.xyzr = xyzr;
  a.gt = gt;
  const dim3 grid((s.cols + NT_RAY - 1) / NT_RAY, (s.rings + RG - 1) / RG);
  const size_t smem = sizeof(double2) * RG + sizeof(float) * SROW * (size_t)(s.nprims > 0 ? s.nprims : 1);
  k_raycast<<<grid, NT_RAY, smem, reinterpret_cast<cudaStream_t>(stream)>>>(a);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LSG_OK : LSG_E_CUDA;
}
