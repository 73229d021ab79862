// lsg_kernels.cu - CUDA kernels (sm_103a) of the Lidar surface-segmentation path.
//
// Mukherjee et al., "Fast Geometric Surface based Segmentation of Point Cloud
// from Lidar Data" (PReMI 2019), Sec. 2 and Algorithm 1.  One pass over a scan
// (or a batch of scans) is four launches:
//
//   k_prep     ring order by elevation (rank counting), sin/cos of the sorted
//              elevations, segment counter reset.                 [Sec. 2 point model]
//   k_tile     one CTA per tile of TR x TC mesh vertices: stage the tile and a
//              halo (1 ring above, 2 below, 1 column left, 2 right) of x,y,z,r in
//              shared memory, then mesh bits, normals, the homogeneity mask and a
//              tile-local union-find, all in shared memory; writes the mesh byte,
//              the normal and each vertex's tile-local root.   [Sec. 2 mesh, normals;
//                                                              Algorithm 1 predicate]
//   k_merge    joins tile-local components across tile borders (and the 360 deg
//              seam) with a lock-free atomicMin union-find in global memory.
//   k_flatten  label = smallest full-resolution index of the component
//              (path to the root), back-fill of non-sampled points, segment
//              count with warp-aggregated atomics.              [Algorithm 1; Sec. 2 end]
//
// Labels are exact: the union-find always hooks the larger root under the
// smaller, so every component's root is its smallest vertex index, whatever
// the order in which threads run.
#include <cuda_runtime.h>
#include <stdint.h>

#include "lsg_internal.h"

namespace lsg {

constexpr int NT = 256;

constexpr uint8_t B_R = LSG_BIT_R, B_D = LSG_BIT_D, B_G = LSG_BIT_G;
constexpr uint8_t B_HR = LSG_BIT_HR, B_HD = LSG_BIT_HD, B_HG = LSG_BIT_HG;
constexpr uint8_t B_VALID = LSG_BIT_VALID, B_HASN = LSG_BIT_HASN;

TileShape tile_shape(int tile) {
  switch (tile) {
    case LSG_TILE_4x256: return {4, 256};
    case LSG_TILE_16x64: return {16, 64};
    case LSG_TILE_2x512: return {2, 512};
    case LSG_TILE_8x64: return {8, 64};
    case LSG_TILE_8x128:
    default: return {8, 128};
  }
}

// ---------------------------------------------------------------------------
// small device helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool in_range(float r, float rmin, float rmax) {
  return rmin < r && r <= rmax;
}

// Depth-jump cut |r_p - r_q| > tau * min(r_p, r_q) in binary32, round to
// nearest, never contracted into an FMA (the decision must be reproducible).
__device__ __forceinline__ bool jump_cut(float rp, float rq, float tau) {
  float d = fabsf(__fsub_rn(rp, rq));
  float m = fminf(rp, rq);
  return d > __fmul_rn(tau, m);
}

__device__ __forceinline__ const ScanDesc* tile_desc(const KArgs& a, int t, int& lt) {
  if (a.scans) {
    const ScanDesc* d = a.scans + a.tile_scan[t];
    lt = t - d->tile0;
    return d;
  }
  lt = t;
  return &a.one;
}

// Union-find on shared memory.  P[x] <= x always holds, so the forest has no
// cycles and the root of every tree is its smallest index.
__device__ __forceinline__ int find_s(volatile int* P, int x, int limit) {
  int p = P[x];
  while (p != x && limit-- > 0) {
    x = p;
    p = P[x];
  }
  return x;
}

__device__ void union_s(int* P, int a, int b, int limit, int32_t* err) {
  volatile int* V = P;
  for (int it = 0; it < limit; ++it) {
    a = find_s(V, a, limit);
    b = find_s(V, b, limit);
    if (a == b) return;
    if (a > b) {
      int t = a;
      a = b;
      b = t;
    }
    int old = atomicMin(P + b, a);
    if (old == b) return;
    b = old;
  }
  atomicOr(err, DERR_TIMEOUT);
}

// Union-find on global memory: loads bypass L1 (ld.global.cg) so they see the
// atomics, which resolve in L2.
__device__ __forceinline__ int find_g(const int32_t* P, int x, int limit) {
  int p = __ldcg(P + x);
  while (p != x && limit-- > 0) {
    x = p;
    p = __ldcg(P + x);
  }
  return x;
}

__device__ void union_g(int32_t* P, int a, int b, int limit, int32_t* err) {
  for (int it = 0; it < limit; ++it) {
    a = find_g(P, a, limit);
    b = find_g(P, b, limit);
    if (a == b) return;
    if (a > b) {
      int t = a;
      a = b;
      b = t;
    }
    int old = atomicMin(P + b, a);
    if (old == b) return;
    b = old;
  }
  atomicOr(err, DERR_TIMEOUT);
}

// ---------------------------------------------------------------------------
// k_prep: ring order (Sec. 2: rings counted from the topmost sensor down)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(NT) k_prep(const __grid_constant__ KArgs a) {
  __shared__ float se[LSG_MAX_RINGS];
  const ScanDesc* d = a.scans ? a.scans + blockIdx.x : &a.one;
  const int H = d->H;
  for (int k = threadIdx.x; k < H; k += NT) {
    se[k] = d->elev[k];
    d->order[k] = -1;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < H; k += NT) {
    float e = se[k];
    if (e != e) atomicOr(a.err, DERR_NAN_ELEV);
    int rank = 0;
    for (int m = 0; m < H; ++m) {
      float em = se[m];
      rank += (em > e) || (em == e && m < k);
    }
    if (rank < H) {
      d->order[rank] = k;
      float sn, cs;
      sincosf(e, &sn, &cs);
      d->trig[rank] = make_float2(sn, cs);
    }
  }
  if (threadIdx.x == 0) *d->nseg = 0;
}

// ---------------------------------------------------------------------------
// tile geometry in shared memory
// ---------------------------------------------------------------------------
template <int TR, int TC>
struct Geo {
  static constexpr int HR = TR + 3, HC = TC + 3;  // halo: rows r0-1..r0+TR+1, cols c0-1..c0+TC+1
  static constexpr int NR = TR + 1, NC = TC + 1;  // normals: rows r0..r0+TR, cols c0..c0+TC
  static constexpr int NH = HR * HC, NN = NR * NC, NV = TR * TC;
  static constexpr size_t off_hx = 0;
  static constexpr size_t off_hn = off_hx + sizeof(float4) * NH;
  static constexpr size_t off_lp = off_hn + sizeof(float4) * NN;
  static constexpr size_t off_hm = off_lp + sizeof(int) * NV;
  static constexpr size_t off_tb = off_hm + ((NH + 15) / 16) * 16;
  static constexpr size_t bytes = off_tb + ((NV + 15) / 16) * 16;
};

// Weighted normal of the vertex at halo position k (Sec. 2, normal
// estimation).  Spokes in the paper's anticlockwise order
// A=(i+1,j) B=(i+1,j+1) C=(i,j+1) D=(i-1,j) E=(i-1,j-1) F=(i,j-1); triangle
// (p, q_k, q_k+1) counts when its three edges are mesh edges; its term is
// w_k (V_k x V_k+1), w_k = 1/(|V_k| + |V_k+1|).  Returns (n, 1) or (0, 0).
template <int HC>
__device__ __forceinline__ float4 vertex_normal(const float4* __restrict__ hx,
                                                const uint8_t* __restrict__ hm, int k,
                                                float nsign) {
  const uint8_t bp = hm[k];
  if (!(bp & B_VALID)) return make_float4(0.f, 0.f, 0.f, 0.f);
  const int kq[6] = {k + HC, k + HC + 1, k + 1, k - HC, k - HC - 1, k - 1};
  const uint8_t bA = hm[kq[0]], bC = hm[kq[2]], bD = hm[kq[3]], bE = hm[kq[4]], bF = hm[kq[5]];
  bool spoke[6] = {(bp & B_D) != 0, (bp & B_G) != 0, (bp & B_R) != 0,
                   (bD & B_D) != 0, (bE & B_G) != 0, (bF & B_R) != 0};
  bool rim[6] = {(bA & B_R) != 0, (bC & B_D) != 0, (bD & B_G) != 0,
                 (bE & B_R) != 0, (bE & B_D) != 0, (bF & B_G) != 0};
  const float4 p = hx[k];
  float vx[6], vy[6], vz[6], vl[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    if (spoke[q]) {
      float4 o = hx[kq[q]];
      vx[q] = o.x - p.x;
      vy[q] = o.y - p.y;
      vz[q] = o.z - p.z;
      vl[q] = norm3df(vx[q], vy[q], vz[q]);
    } else {
      vx[q] = vy[q] = vz[q] = vl[q] = 0.f;
    }
  }
  float sx = 0.f, sy = 0.f, sz = 0.f;
  int ntri = 0;
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    const int q1 = (q + 1) % 6;
    if (spoke[q] && spoke[q1] && rim[q]) {
      const float w = 1.0f / (vl[q] + vl[q1]);
      sx += w * (vy[q] * vz[q1] - vz[q] * vy[q1]);
      sy += w * (vz[q] * vx[q1] - vx[q] * vz[q1]);
      sz += w * (vx[q] * vy[q1] - vy[q] * vx[q1]);
      ++ntri;
    }
  }
  if (ntri == 0) return make_float4(0.f, 0.f, 0.f, 0.f);
  const float inv = rnorm3df(sx, sy, sz);
  if (!(inv > 0.f) || !isfinite(inv)) return make_float4(0.f, 0.f, 0.f, 0.f);
  const float f = nsign * inv;
  return make_float4(sx * f, sy * f, sz * f, 1.f);
}

// Homogeneity predicate of Algorithm 1 between two vertices' normals.
__device__ __forceinline__ bool homog(const float4 a, const float4 b, const ScanDesc* d) {
  if (a.w == 0.f || b.w == 0.f) return false;
  if (d->pred == LSG_PRED_ANGLE) return a.x * b.x + a.y * b.y + a.z * b.z > d->cos_t;
  return fabsf(a.x - b.x) < d->comp_x && fabsf(a.y - b.y) < d->comp_y &&
         fabsf(a.z - b.z) < d->comp_z;
}

// Tile-local components over the homogeneous edges that stay inside the tile,
// then each vertex's root written as a scan-local vertex index into parent[].
// tb[] holds the final mesh byte of each tile vertex.
template <int TR, int TC>
__device__ void local_components(const ScanDesc* d, int r0, int c0, int rn, int cn,
                                 const uint8_t* tb, int* lp, int32_t* err) {
  using G = Geo<TR, TC>;
  const int tid = threadIdx.x;
  const bool full_ring = d->wrap && c0 == 0 && cn == d->Ws;  // seam inside the tile
  for (int k = tid; k < G::NV; k += NT) lp[k] = k;
  __syncthreads();
  for (int k = tid; k < G::NV; k += NT) {
    const int lr = k / TC, lc = k - (k / TC) * TC;
    if (lr >= rn || lc >= cn) continue;
    const uint8_t bits = tb[k];
    if (bits & B_HR) {
      if (lc + 1 < cn) union_s(lp, k, k + 1, G::NV + 1, err);
      else if (full_ring) union_s(lp, k, lr * TC, G::NV + 1, err);
    }
    if ((bits & B_HD) && lr + 1 < rn) union_s(lp, k, k + TC, G::NV + 1, err);
    if ((bits & B_HG) && lr + 1 < rn) {
      if (lc + 1 < cn) union_s(lp, k, k + TC + 1, G::NV + 1, err);
      else if (full_ring) union_s(lp, k, (lr + 1) * TC, G::NV + 1, err);
    }
  }
  __syncthreads();
  for (int k = tid; k < G::NV; k += NT) {
    const int lr = k / TC, lc = k - (k / TC) * TC;
    if (lr >= rn || lc >= cn) continue;
    const int root = find_s(lp, k, G::NV + 1);
    const int rr = root / TC, rc = root - (root / TC) * TC;
    d->parent[(size_t)(r0 + lr) * d->Ws + (c0 + lc)] = (r0 + rr) * d->Ws + (c0 + rc);
  }
}

// ---------------------------------------------------------------------------
// k_tile: decode + mesh + normals + edge mask + tile-local components
// ---------------------------------------------------------------------------
template <int TR, int TC>
__global__ void __launch_bounds__(NT) k_tile(const __grid_constant__ KArgs a) {
  using G = Geo<TR, TC>;
  extern __shared__ __align__(16) unsigned char smem[];
  float4* hx = reinterpret_cast<float4*>(smem + G::off_hx);
  float4* hn = reinterpret_cast<float4*>(smem + G::off_hn);
  int* lp = reinterpret_cast<int*>(smem + G::off_lp);
  uint8_t* hm = smem + G::off_hm;
  uint8_t* tb = smem + G::off_tb;
  const int tid = threadIdx.x;

  for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
    int lt;
    const ScanDesc* d = tile_desc(a, t, lt);
    const int H = d->H, W = d->W, Ws = d->Ws, s = d->s;
    const int tr = lt / d->tiles_c, tc = lt - (lt / d->tiles_c) * d->tiles_c;
    const int r0 = tr * TR, c0 = tc * TC;
    const int rn = min(TR, H - r0), cn = min(TC, Ws - c0);
    const float rmin = d->r_min, rmax = d->r_max;

    // 1. stage x, y, z, r of the tile and its halo (absent positions: r = -1)
    for (int k = tid; k < G::NH; k += NT) {
      const int hr = k / G::HC, hc = k - (k / G::HC) * G::HC;
      const int i = r0 - 1 + hr;
      int j = c0 - 1 + hc;
      float4 v = make_float4(0.f, 0.f, 0.f, -1.f);
      if (d->wrap) j = ((j % Ws) + Ws) % Ws;
      if (i >= 0 && i < H && j >= 0 && j < Ws) {
        const int row = d->order[i];
        if ((unsigned)row < (unsigned)H) {
          const size_t o = (size_t)row * W + (size_t)j * s;
          if (d->xyzr) {
            v = __ldg(d->xyzr + o);
          } else {
            const float r = __ldg(d->range + o);
            const float2 tg = d->trig[i];
            float sp, cp;
            sincosf(fmaf((float)(j * s), d->daz, d->az0), &sp, &cp);
            const float rc = r * tg.y;
            v = make_float4(rc * cp, rc * sp, r * tg.x, r);
          }
        }
      }
      hx[k] = v;
    }
    __syncthreads();

    // 2. mesh bits on the halo (Sec. 2, mesh construction): R, D, G joins
    //    between points in range and not across a depth jump
    for (int k = tid; k < G::NH; k += NT) {
      const int hr = k / G::HC, hc = k - (k / G::HC) * G::HC;
      const float rp = hx[k].w;
      uint8_t bits = 0;
      if (in_range(rp, rmin, rmax)) {
        bits = B_VALID;
        if (hc + 1 < G::HC) {
          const float rq = hx[k + 1].w;
          if (in_range(rq, rmin, rmax) && !jump_cut(rp, rq, d->jump_h)) bits |= B_R;
        }
        if (hr + 1 < G::HR) {
          const float rq = hx[k + G::HC].w;
          if (in_range(rq, rmin, rmax) && !jump_cut(rp, rq, d->jump_v)) bits |= B_D;
          if (hc + 1 < G::HC) {
            const float rg = hx[k + G::HC + 1].w;
            if (in_range(rg, rmin, rmax) && !jump_cut(rp, rg, d->jump_v)) bits |= B_G;
          }
        }
      }
      hm[k] = bits;
    }
    __syncthreads();

    // 3. normals of the tile plus one ring below and one column right
    for (int k = tid; k < G::NN; k += NT) {
      const int nr = k / G::NC, nc = k - (k / G::NC) * G::NC;
      hn[k] = vertex_normal<G::HC>(hx, hm, (nr + 1) * G::HC + (nc + 1), d->nsign);
    }
    __syncthreads();

    // 4. homogeneity mask of the tile's R, D, G edges; write mesh byte + normal
    for (int k = tid; k < G::NV; k += NT) {
      const int lr = k / TC, lc = k - (k / TC) * TC;
      uint8_t bits = 0;
      if (lr < rn && lc < cn) {
        bits = hm[(lr + 1) * G::HC + (lc + 1)];
        const float4 n = hn[lr * G::NC + lc];
        if (n.w != 0.f) bits |= B_HASN;
        if ((bits & B_R) && homog(n, hn[lr * G::NC + lc + 1], d)) bits |= B_HR;
        if ((bits & B_D) && homog(n, hn[(lr + 1) * G::NC + lc], d)) bits |= B_HD;
        if ((bits & B_G) && homog(n, hn[(lr + 1) * G::NC + lc + 1], d)) bits |= B_HG;
        const size_t v = (size_t)(r0 + lr) * Ws + (c0 + lc);
        d->mb[v] = bits;
        float* o = d->nrm + 3 * v;
        o[0] = n.x;
        o[1] = n.y;
        o[2] = n.z;
      }
      tb[k] = bits;
    }
    __syncthreads();

    // 5. tile-local components (Algorithm 1 restricted to the tile)
    local_components<TR, TC>(d, r0, c0, rn, cn, tb, lp, a.err);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// k_tile_ccl: tile-local components from a given mesh byte array
// ---------------------------------------------------------------------------
template <int TR, int TC>
__global__ void __launch_bounds__(NT) k_tile_ccl(const __grid_constant__ KArgs a) {
  using G = Geo<TR, TC>;
  __shared__ int lp[G::NV];
  __shared__ uint8_t tb[G::NV];
  const int tid = threadIdx.x;
  for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
    int lt;
    const ScanDesc* d = tile_desc(a, t, lt);
    const int tr = lt / d->tiles_c, tc = lt - (lt / d->tiles_c) * d->tiles_c;
    const int r0 = tr * TR, c0 = tc * TC;
    const int rn = min(TR, d->H - r0), cn = min(TC, d->Ws - c0);
    for (int k = tid; k < G::NV; k += NT) {
      const int lr = k / TC, lc = k - (k / TC) * TC;
      tb[k] = (lr < rn && lc < cn) ? d->mb[(size_t)(r0 + lr) * d->Ws + (c0 + lc)] : 0;
    }
    __syncthreads();
    local_components<TR, TC>(d, r0, c0, rn, cn, tb, lp, a.err);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// k_merge: join components across tile borders and the 360 deg seam
// ---------------------------------------------------------------------------
template <int TR, int TC>
__global__ void __launch_bounds__(NT) k_merge(const __grid_constant__ KArgs a) {
  const int tid = threadIdx.x;
  for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
    int lt;
    const ScanDesc* d = tile_desc(a, t, lt);
    const int Ws = d->Ws;
    const int tr = lt / d->tiles_c, tc = lt - (lt / d->tiles_c) * d->tiles_c;
    const int r0 = tr * TR, c0 = tc * TC;
    const int rn = min(TR, d->H - r0), cn = min(TC, Ws - c0);
    const int limit = d->H * Ws + 1;
    // border vertices: the last row of the tile, then the last column above it
    const int nb = cn + rn - 1;
    for (int k = tid; k < nb; k += NT) {
      int lr, lc;
      if (k < cn) {
        lr = rn - 1;
        lc = k;
      } else {
        lr = k - cn;
        lc = cn - 1;
      }
      const int i = r0 + lr, j = c0 + lc;
      const int v = i * Ws + j;
      const uint8_t bits = d->mb[v];
      if (!(bits & (B_HR | B_HD | B_HG))) continue;
      // bits that point off the grid (possible in a caller-given mask) are ignored
      const bool has_right = (j + 1 < Ws) || d->wrap;
      const bool has_down = i + 1 < d->H;
      const int jn = (j + 1 == Ws) ? 0 : j + 1;
      const bool jn_in = jn >= c0 && jn < c0 + cn;
      const bool in_next_row = (i + 1) < r0 + rn;
      if ((bits & B_HR) && has_right && !jn_in) union_g(d->parent, v, i * Ws + jn, limit, a.err);
      if ((bits & B_HD) && has_down && !in_next_row) union_g(d->parent, v, (i + 1) * Ws + j, limit, a.err);
      if ((bits & B_HG) && has_down && has_right && !(in_next_row && jn_in))
        union_g(d->parent, v, (i + 1) * Ws + jn, limit, a.err);
    }
  }
}

// ---------------------------------------------------------------------------
// k_flatten: labels, back-fill, segment count
// ---------------------------------------------------------------------------
__device__ __forceinline__ int32_t vertex_label(const ScanDesc* d, int i, int j, int limit) {
  const int v = i * d->Ws + j;
  if (!(d->mb[v] & B_VALID)) return -1;
  const int g = find_g(d->parent, v, limit);
  const int gi = g / d->Ws, gj = g - (g / d->Ws) * d->Ws;
  return gi * d->W + gj * d->s;
}

template <int TR, int TC>
__global__ void __launch_bounds__(NT) k_flatten(const __grid_constant__ KArgs a) {
  const int tid = threadIdx.x;
  for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
    int lt;
    const ScanDesc* d = tile_desc(a, t, lt);
    const int W = d->W, Ws = d->Ws, s = d->s;
    const int tr = lt / d->tiles_c, tc = lt - (lt / d->tiles_c) * d->tiles_c;
    const int r0 = tr * TR, c0 = tc * TC;
    const int rn = min(TR, d->H - r0), cn = min(TC, Ws - c0);
    const int cbeg = c0 * s, cend = min((c0 + cn) * s, W);
    const int ncols = cend - cbeg;
    const int limit = d->H * Ws + 1;
    const int npts = rn * ncols;
    // whole warps iterate together so the warp-wide count reduction is safe
    const int nround = (npts + NT - 1) / NT;
    for (int rnd = 0; rnd < nround; ++rnd) {
      const int k = rnd * NT + tid;
      int root = 0;
      if (k < npts) {
        const int lr = k / ncols, cc = k - (k / ncols) * ncols;
        const int i = r0 + lr, c = cbeg + cc;
        const int j = c / s, rem = c - j * s;
        int32_t lab;
        if (rem == 0) {
          const int v = i * Ws + j;
          if (d->mb[v] & B_VALID) {
            const int g = find_g(d->parent, v, limit);
            root = (g == v);
            const int gi = g / Ws, gj = g - gi * Ws;
            lab = gi * W + gj * s;
          } else {
            lab = -1;
          }
        } else {
          bool ok;
          if (d->valid) {
            ok = d->valid[(size_t)i * W + c] != 0;
          } else {
            const int row = d->order[i];
            float r = -1.f;
            if ((unsigned)row < (unsigned)d->H) {
              const size_t o = (size_t)row * W + c;
              r = d->xyzr ? __ldg(&d->xyzr[o].w) : __ldg(d->range + o);
            }
            ok = in_range(r, d->r_min, d->r_max);
          }
          if (!ok) {
            lab = -1;
          } else {
            const int32_t lo = vertex_label(d, i, j, limit);
            const int dlo = rem;
            int32_t hi = -1;
            int dhi = 0;
            bool have_hi = false;
            if (j + 1 < Ws) {
              hi = vertex_label(d, i, j + 1, limit);
              dhi = (j + 1) * s - c;
              have_hi = true;
            } else if (d->wrap) {
              hi = vertex_label(d, i, 0, limit);
              dhi = W - c;
              have_hi = true;
            }
            int32_t first = lo, second = have_hi ? hi : -1;
            if (have_hi && dhi < dlo) {
              first = hi;
              second = lo;
            }
            lab = first != -1 ? first : second;
          }
        }
        d->labels[(size_t)i * W + c] = lab;
      }
      const int cnt = __reduce_add_sync(0xffffffffu, root);
      if ((tid & 31) == 0 && cnt) atomicAdd(d->nseg, cnt);
    }
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <int TR, int TC>
static cudaError_t set_attrs() {
  return cudaFuncSetAttribute(k_tile<TR, TC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)Geo<TR, TC>::bytes);
}

cudaError_t prepare_kernels() {
  cudaError_t e;
  if ((e = set_attrs<8, 128>()) != cudaSuccess) return e;
  if ((e = set_attrs<4, 256>()) != cudaSuccess) return e;
  if ((e = set_attrs<16, 64>()) != cudaSuccess) return e;
  if ((e = set_attrs<2, 512>()) != cudaSuccess) return e;
  if ((e = set_attrs<8, 64>()) != cudaSuccess) return e;
  return cudaSuccess;
}

cudaError_t launch_prep(const KArgs& a, cudaStream_t st) {
  const int n = a.scans ? a.nscans : 1;
  k_prep<<<n, NT, 0, st>>>(a);
  return cudaGetLastError();
}

#define LSG_DISPATCH(tile, FN, ...)                       \
  switch (tile) {                                         \
    case LSG_TILE_4x256: return FN<4, 256>(__VA_ARGS__);  \
    case LSG_TILE_16x64: return FN<16, 64>(__VA_ARGS__);  \
    case LSG_TILE_2x512: return FN<2, 512>(__VA_ARGS__);  \
    case LSG_TILE_8x64: return FN<8, 64>(__VA_ARGS__);    \
    default: return FN<8, 128>(__VA_ARGS__);             \
  }

template <int TR, int TC>
static cudaError_t run_tile(const KArgs& a, cudaStream_t st) {
  k_tile<TR, TC><<<a.ntiles, NT, Geo<TR, TC>::bytes, st>>>(a);
  return cudaGetLastError();
}
template <int TR, int TC>
static cudaError_t run_tile_ccl(const KArgs& a, cudaStream_t st) {
  k_tile_ccl<TR, TC><<<a.ntiles, NT, 0, st>>>(a);
  return cudaGetLastError();
}
template <int TR, int TC>
static cudaError_t run_merge(const KArgs& a, cudaStream_t st) {
  k_merge<TR, TC><<<a.ntiles, NT, 0, st>>>(a);
  return cudaGetLastError();
}
template <int TR, int TC>
static cudaError_t run_flatten(const KArgs& a, cudaStream_t st) {
  k_flatten<TR, TC><<<a.ntiles, NT, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_tile(int tile, const KArgs& a, cudaStream_t st) { LSG_DISPATCH(tile, run_tile, a, st) }
cudaError_t launch_tile_ccl(int tile, const KArgs& a, cudaStream_t st) {
  LSG_DISPATCH(tile, run_tile_ccl, a, st)
}
cudaError_t launch_merge(int tile, const KArgs& a, cudaStream_t st) { LSG_DISPATCH(tile, run_merge, a, st) }
cudaError_t launch_flatten(int tile, const KArgs& a, cudaStream_t st) {
  LSG_DISPATCH(tile, run_flatten, a, st)
}

}  // namespace lsg
