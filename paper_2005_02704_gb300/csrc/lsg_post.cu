// lsg_post.cu - optional post-processing of a segmentation (Sec. 2, last
// paragraph: segments with too few points may be eliminated): per-segment
// point counts and normal sums, and removal of small segments.
//
// Labels are point indices (the smallest point index of the segment), so the
// per-segment arrays are indexed directly by label.  Counting uses one
// atomic per run of equal labels in a warp (__match_any_sync groups the
// lanes that share a label), which cuts the atomics on large segments by up
// to 32x.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "lsg_internal.h"

namespace {

constexpr int NT = 256;
constexpr unsigned FULL = 0xffffffffu;

__global__ void __launch_bounds__(NT) k_count(const int32_t* __restrict__ labels, int64_t npts, int32_t* sizes) {
  for (int64_t base = (int64_t)blockIdx.x * NT; base < npts; base += (int64_t)gridDim.x * NT) {
    const int64_t p = base + threadIdx.x;
    int32_t lab = p < npts ? labels[p] : -1;
    if (lab >= npts) lab = -1;  // not a label of this scan
    const unsigned grp = __match_any_sync(FULL, lab);
    const int lane = threadIdx.x & 31;
    if (lab >= 0 && lane == __ffs(grp) - 1) atomicAdd(sizes + lab, __popc(grp));
  }
}

__global__ void __launch_bounds__(NT) k_normal_sums(const int32_t* __restrict__ labels, const float* __restrict__ nrm,
                                                    const uint8_t* __restrict__ mb, int H, int W, int Ws, int s,
                                                    float* nsum) {
  const int64_t nv = (int64_t)H * Ws;
  for (int64_t v = (int64_t)blockIdx.x * NT + threadIdx.x; v < nv; v += (int64_t)gridDim.x * NT) {
    if (!(mb[v] & LSG_BIT_HASN)) continue;
    const int i = (int)(v / Ws), j = (int)(v - (int64_t)i * Ws);
    const int32_t lab = labels[(int64_t)i * W + (int64_t)j * s];
    if (lab < 0 || lab >= (int64_t)H * W) continue;
    atomicAdd(nsum + 3 * (int64_t)lab + 0, nrm[3 * v + 0]);
    atomicAdd(nsum + 3 * (int64_t)lab + 1, nrm[3 * v + 1]);
    atomicAdd(nsum + 3 * (int64_t)lab + 2, nrm[3 * v + 2]);
  }
}

__global__ void __launch_bounds__(NT) k_filter(int32_t* labels, int64_t npts, const int32_t* __restrict__ sizes,
                                               int32_t min_points, int32_t* nseg) {
  for (int64_t base = (int64_t)blockIdx.x * NT; base < npts; base += (int64_t)gridDim.x * NT) {
    const int64_t p = base + threadIdx.x;
    int kept_root = 0;
    if (p < npts) {
      const int32_t lab = labels[p];
      if (lab >= npts) {
        labels[p] = -1;  // not a label of this scan
      } else if (lab >= 0) {
        const bool keep = sizes[lab] >= min_points;
        if (!keep) labels[p] = -1;
        kept_root = keep && (int64_t)lab == p;
      }
    }
    const int cnt = __reduce_add_sync(FULL, kept_root);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(nseg, cnt);
  }
}

int grid_for(int64_t n) {
  const int64_t g = (n + NT - 1) / NT;
  return (int)(g < 1 ? 1 : (g > 65535 ? 65535 : g));
}

}  // namespace

extern "C" lsg_status lsg_segment_stats(lsg_ctx* ctx, int32_t H, int32_t W, int32_t s, int32_t min_points,
                                        int32_t* labels, const float* normals, const uint8_t* meshbits,
                                        int32_t* sizes, float* nsum, int32_t* nseg, lsg_stream stream) {
  if (!ctx || !nseg) return LSG_E_ARG;
  if (H < 0 || W < 0 || H > LSG_MAX_RINGS || W > LSG_MAX_COLS) return LSG_E_SHAPE;
  if ((int64_t)H * W > (int64_t)LSG_MAX_POINTS) return LSG_E_SHAPE;
  if (s < 1 || min_points < 0) return LSG_E_ARG;
  cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
  const int64_t npts = (int64_t)H * W;
  cudaError_t e = cudaMemsetAsync(nseg, 0, sizeof(int32_t), cs);
  if (npts == 0) return e == cudaSuccess ? LSG_OK : LSG_E_CUDA;
  if (!labels || !sizes || (nsum && (!normals || !meshbits))) return LSG_E_ARG;
  const int Ws = (W + s - 1) / s;
  if (e == cudaSuccess) e = cudaMemsetAsync(sizes, 0, sizeof(int32_t) * npts, cs);
  if (e == cudaSuccess && nsum) e = cudaMemsetAsync(nsum, 0, sizeof(float) * 3 * npts, cs);
  if (e == cudaSuccess) {
    k_count<<<grid_for(npts), NT, 0, cs>>>(labels, npts, sizes);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && nsum) {
    k_normal_sums<<<grid_for((int64_t)H * Ws), NT, 0, cs>>>(labels, normals, meshbits, H, W, Ws, s, nsum);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    k_filter<<<grid_for(npts), NT, 0, cs>>>(labels, npts, sizes, min_points, nseg);
    e = cudaGetLastError();
  }
  return e == cudaSuccess ? LSG_OK : LSG_E_CUDA;
}
