// lsg_kernels.cu - CUDA kernels (sm_103a) of the Lidar surface-segmentation path.
//
// Mukherjee et al., "Fast Geometric Surface based Segmentation of Point Cloud
// from Lidar Data" (PReMI 2019), Sec. 2 and Algorithm 1.  One pass over a scan
// (or a batch of scans) is four launches:
//
//   k_prep     ring order by elevation (rank counting), sin/cos of the sorted
//              elevations, segment counter reset.               [Sec. 2, point model]
//   k_tile     one CTA per tile of TR rows x (29*NW) columns of mesh vertices.
//              The CTA stages x,y,z,r of the tile plus a halo (one ring above,
//              two below, one column left, two right) in shared memory.  Each
//              warp then sweeps a strip of 32 columns (29 of them its own)
//              down the rows, holding a three-row window in registers and
//              taking the neighbouring columns from the adjacent lanes with
//              warp shuffles: mesh bits and edge vectors of each row, the
//              weighted normal of the row above, the homogeneity mask of the
//              row above that.  Every edge vector and length is computed once
//              and reused by both endpoints.  The tile's components follow:
//              horizontal runs from a warp ballot, vertical joins with an
//              atomicMin union-find in shared memory (only where a run meets a
//              new run above), then joins across strips.  Writes the mesh byte,
//              the normal, and each vertex's tile-local root (16 bits).
//                                          [Sec. 2 mesh, normals; Algorithm 1]
//   k_merge    joins tile-local components across tile borders and the 360 deg
//              seam with a lock-free atomicMin union-find over the roots.
//   k_flatten  label = smallest full-resolution index of the component,
//              back-fill of non-sampled points, segment count with warp
//              reductions.                                [Algorithm 1; Sec. 2 end]
//
// Labels are exact: every union hooks the larger root under the smaller, so
// each component's root is its smallest vertex index whatever the thread
// order, and a tile-local root is the smallest index of its tile component.
#include <cuda_runtime.h>
#include <limits.h>
#include <stdint.h>

#include "lsg_internal.h"

namespace lsg {

constexpr uint8_t B_R = LSG_BIT_R, B_D = LSG_BIT_D, B_G = LSG_BIT_G;
constexpr uint8_t B_HR = LSG_BIT_HR, B_HD = LSG_BIT_HD, B_HG = LSG_BIT_HG;
constexpr uint8_t B_VALID = LSG_BIT_VALID, B_HASN = LSG_BIT_HASN;
constexpr unsigned FULL = 0xffffffffu;
constexpr int SO = 29;  // output columns per warp strip (lanes 1..29)
constexpr uint16_t NO_ROOT = 0xFFFF;  // tile-local root of a vertex out of range

// Row pitch of the tile-root array: Ws rounded up to 8 entries (16 bytes), so
// that a tile's rows can be read with aligned vector loads.
__host__ __device__ __forceinline__ int root_pitch(int Ws) { return (Ws + 7) & ~7; }

TileShape tile_shape(int tile) {
  switch (tile) {
    case LSG_TILE_32x116: return {32, 116};
    case LSG_TILE_32x232: return {32, 232};
    case LSG_TILE_64x116: return {64, 116};
    case LSG_TILE_64x232: return {64, 232};
    case LSG_TILE_16x116:
    default: return {16, 116};
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
  const float d = fabsf(__fsub_rn(rp, rq));
  return d > __fmul_rn(tau, fminf(rp, rq));
}

// Length of a vector via the hardware reciprocal square root (about 2 ulp).
__device__ __forceinline__ float vlen(float x, float y, float z) {
  const float q = fmaf(x, x, fmaf(y, y, z * z));
  return q > 0.f ? q * rsqrtf(q) : 0.f;
}

// One weighted triangle term of the normal sum (Sec. 2, normal estimation):
// w (a x b) with w = 1 / (|a| + |b|), added only when the triangle exists.
// The sweep zeroes the coordinates of points out of range, so every spoke is
// finite and a missing triangle's term is removed by a zero weight.
__device__ __forceinline__ void tri_term(float ax, float ay, float az, float la, float bx, float by, float bz,
                                         float lb, bool exists, float& sx, float& sy, float& sz) {
  const float w = exists ? __fdividef(1.0f, la + lb) : 0.f;  // hardware reciprocal, <= 2 ulp
  sx = fmaf(w, ay * bz - az * by, sx);
  sy = fmaf(w, az * bx - ax * bz, sy);
  sz = fmaf(w, ax * by - ay * bx, sz);
}

// Homogeneity predicate of Algorithm 1 between two vertices' normals
// (w = 1 when the vertex has a normal).
// Branch-free: both forms are evaluated and the predicate selects one.
__device__ __forceinline__ bool homog(const float4 u, const float4 v, bool angle_pred, float cos_t, float cx,
                                      float cy, float cz) {
  const bool both = (u.w != 0.f) & (v.w != 0.f);
  const bool by_angle = fmaf(u.x, v.x, fmaf(u.y, v.y, u.z * v.z)) > cos_t;
  const bool by_comp = (fabsf(u.x - v.x) < cx) & (fabsf(u.y - v.y) < cy) & (fabsf(u.z - v.z) < cz);
  return both & (angle_pred ? by_angle : by_comp);
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
      const int t = a;
      a = b;
      b = t;
    }
    const int old = atomicMin(P + b, a);
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

// find with path halving: each visited node is re-pointed at its grandparent.
// The store only shortens a path to an ancestor (P[x] <= x still holds), so it
// is safe next to concurrent atomicMin links.
__device__ __forceinline__ int find_halve(int32_t* P, int x, int limit) {
  int p = __ldcg(P + x);
  while (p != x && limit-- > 0) {
    const int gp = __ldcg(P + p);
    if (gp != p) __stcg(P + x, gp);
    x = gp;
    p = __ldcg(P + x);
  }
  return x;
}

__device__ void union_g(int32_t* P, int a, int b, int limit, int32_t* err) {
  for (int it = 0; it < limit; ++it) {
    a = find_halve(P, a, limit);
    b = find_halve(P, b, limit);
    if (a == b) return;
    if (a > b) {
      const int t = a;
      a = b;
      b = t;
    }
    const int old = atomicMin(P + b, a);
    if (old == b) return;
    b = old;
  }
  atomicOr(err, DERR_TIMEOUT);
}

// ---------------------------------------------------------------------------
// k_prep: ring order (Sec. 2: rings counted from the topmost sensor down)
// ---------------------------------------------------------------------------
constexpr int NT_PREP = 256;

// One scan's ring order by rank counting (se: shared scratch of
// LSG_MAX_RINGS floats; NTB threads).
template <int NTB>
__device__ __forceinline__ void prep_body(const ScanDesc* d, float* se, int32_t* err) {
  const int H = d->H;
  for (int k = threadIdx.x; k < H; k += NTB) {
    se[k] = d->elev[k];
    d->order[k] = -1;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < H; k += NTB) {
    const float e = se[k];
    if (e != e) atomicOr(err, DERR_NAN_ELEV);
    int rank = 0;
    for (int m = 0; m < H; ++m) {
      const float em = se[m];
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

__global__ void __launch_bounds__(NT_PREP) k_prep(const __grid_constant__ KArgs a) {
  __shared__ float se[LSG_MAX_RINGS];
  prep_body<NT_PREP>(a.scans ? a.scans + blockIdx.x : &a.one, se, a.err);
}

// ---------------------------------------------------------------------------
// tile geometry
// ---------------------------------------------------------------------------
constexpr int RING = 8;  // rows each lane keeps in flight (cp.async depth)

template <int TR, int NW>
struct Geo {
  static constexpr int NT = NW * 32;
  static constexpr int TC = NW * SO;             // output columns of a tile
  static constexpr int HR = TR + 3;              // rows read: r0-1 .. r0+TR+1
  static constexpr int NV = TR * TC;
  static constexpr size_t off_ring = 0;          // per-warp row rings [NW][RING+1][32] float4
  static constexpr size_t off_lp = off_ring + sizeof(float4) * NW * (RING + 1) * 32;  // tile union-find
  static constexpr size_t off_tb = off_lp + sizeof(int) * NV;  // tile mesh bytes
  static constexpr size_t off_rows = off_tb + ((NV + 15) / 16) * 16;  // long long [HR] input row offsets
  static constexpr size_t bytes = off_rows + sizeof(long long) * HR;
  static constexpr size_t ccl_bytes = sizeof(int) * NV + ((NV + 15) / 16) * 16;
};

// Issue the asynchronous copy of one point into the lane's ring slot (x,y,z,r
// input), or store the decoded / absent value directly.  ro = offset of the
// input row (ring order * W), or -1 when the row is outside the scan.
__device__ __forceinline__ void fetch_point(float4* slot, const float4* __restrict__ xyzr,
                                            const float* __restrict__ range, const float2* __restrict__ trig,
                                            int i, long long ro, bool colok, size_t coff, float sp, float cp) {
  if (colok && ro >= 0) {
    const size_t o = (size_t)ro + coff;
    if (xyzr) {
      const unsigned dst = (unsigned)__cvta_generic_to_shared(slot);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(xyzr + o) : "memory");
    } else {
      const float r = __ldg(range + o);
      const float2 te = __ldg(trig + i);
      const float rc = r * te.y;
      *slot = make_float4(rc * cp, rc * sp, r * te.x, r);
    }
    return;
  }
  *slot = make_float4(0.f, 0.f, 0.f, -1.f);
}

// Everything of a descriptor the tile kernels use, in registers.
struct Loc {
  int H, W, Ws, s, wrap, tiles_c;
  int r0, c0, rn, cn;
};

__device__ __forceinline__ Loc make_loc(const ScanDesc* d, int lt, int TR, int TC) {
  Loc L;
  L.H = d->H;
  L.W = d->W;
  L.Ws = d->Ws;
  L.s = d->s;
  L.wrap = d->wrap;
  L.tiles_c = d->tiles_c;
  const int tr = lt / L.tiles_c, tc = lt - tr * L.tiles_c;
  L.r0 = tr * TR;
  L.c0 = tc * TC;
  L.rn = min(TR, L.H - L.r0);
  L.cn = min(TC, L.Ws - L.c0);
  return L;
}

template <int TR, int NW>
__device__ __forceinline__ void tile_cross_and_roots(const Loc& L, const uint8_t* __restrict__ tb, int* lp,
                                                     uint16_t* __restrict__ lroot, int32_t* __restrict__ parent,
                                                     int32_t* err);

// Tile components of the tile bytes tb[TR][TC] (mesh + homogeneity bits of
// the tile's own vertices): horizontal runs from a ballot, vertical joins in a
// shared-memory union-find, then joins across strips and the seam.  Writes
// every vertex's tile-local root to lroot and marks each root in parent.
template <int TR, int NW>
__device__ __forceinline__ void tile_components(const Loc& L, const uint8_t* __restrict__ tb, int* lp,
                                uint16_t* __restrict__ lroot, int32_t* __restrict__ parent,
                                int32_t* err) {
  using G = Geo<TR, NW>;
  constexpr int TC = G::TC;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int lcw = w * SO + lane - 1;  // this lane's tile column
  const bool act = lane >= 1 && lane <= SO && lcw < L.cn;

  // C1: each warp walks its strip row by row
  uint8_t bprev = 0;
  for (int lr = 0; lr < L.rn; ++lr) {
    const uint8_t b = act ? tb[lr * TC + lcw] : 0;
    const bool hr_in = act && lane < SO && lcw + 1 < L.cn && (b & B_HR);
    const unsigned B = __ballot_sync(FULL, hr_in);
    const unsigned brk = ~B & ((1u << lane) - 1u);  // lanes left of me whose R edge breaks the run
    const int start = 32 - __clz(brk);              // first lane of my run (>= 1)
    const int v = lr * TC + lcw;
    if (act) lp[v] = lr * TC + (w * SO + start - 1);
    __syncwarp();
    if (act && lr > 0) {
      const uint8_t bu = bprev;
      const uint8_t bul = lane >= 2 ? tb[(lr - 1) * TC + lcw - 1] : 0;
      const uint8_t bl = lane >= 2 ? tb[lr * TC + lcw - 1] : 0;
      // D edge (lr-1, c) - (lr, c); implied when the left lane's D edge and
      // both rows' R edges already join the same vertices
      if (bu & B_HD) {
        const bool implied = (bul & B_HD) && (bul & B_HR) && (bl & B_HR);
        if (!implied) union_s(lp, v, v - TC, G::NV + 1, err);
      }
      // G edge (lr-1, c-1) - (lr, c)
      if (bul & B_HG) {
        const bool implied = (bul & B_HD) && (bl & B_HR);
        if (!implied) union_s(lp, v, v - TC - 1, G::NV + 1, err);
      }
    }
    __syncwarp();
    bprev = b;
  }
  __syncthreads();
  tile_cross_and_roots<TR, NW>(L, tb, lp, lroot, parent, err);
}

// C2: edges across strip borders, and the seam of a tile spanning the ring;
// C3: every vertex's tile-local root (vertices out of range: NO_ROOT), roots
// marked in the global union-find.
template <int TR, int NW>
__device__ __forceinline__ void tile_cross_and_roots(const Loc& L, const uint8_t* __restrict__ tb, int* lp,
                                                     uint16_t* __restrict__ lroot, int32_t* __restrict__ parent,
                                                     int32_t* err) {
  using G = Geo<TR, NW>;
  constexpr int TC = G::TC;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const bool full_ring = L.wrap && L.c0 == 0 && L.cn == L.Ws;
  for (int idx = threadIdx.x; idx < L.rn * NW; idx += G::NT) {
    const int lr = idx / NW, b = idx - (idx / NW) * NW;
    int ac = -1, bc = -1;
    if (b < NW - 1) {
      ac = b * SO + SO - 1;
      bc = ac + 1;
      if (bc >= L.cn) ac = -1;
    }
    if (b == NW - 1 && full_ring) {
      ac = L.cn - 1;
      bc = 0;
    }
    if (ac < 0) continue;
    const uint8_t bits = tb[lr * TC + ac];
    if (bits & B_HR) union_s(lp, lr * TC + ac, lr * TC + bc, G::NV + 1, err);
    if ((bits & B_HG) && lr + 1 < L.rn) union_s(lp, lr * TC + ac, (lr + 1) * TC + bc, G::NV + 1, err);
  }
  __syncthreads();

  // C3: roots (vertices out of range: 0xFFFF)
  for (int lr = w; lr < L.rn; lr += NW) {
    for (int lc = lane; lc < L.cn; lc += 32) {
      const int v = lr * TC + lc;
      const size_t gv = (size_t)(L.r0 + lr) * L.Ws + (L.c0 + lc);
      const size_t gr = (size_t)(L.r0 + lr) * root_pitch(L.Ws) + (L.c0 + lc);
      if (!(tb[v] & B_VALID)) {
        lroot[gr] = NO_ROOT;
        continue;
      }
      const int r = find_s(lp, v, G::NV + 1);
      lroot[gr] = (uint16_t)r;
      if (r == v) parent[gv] = (int32_t)gv;
    }
  }
}

// ---------------------------------------------------------------------------
// k_tile: decode + mesh + normals + edge mask + tile components
// ---------------------------------------------------------------------------
// One tile of one scan: decode + mesh + normals + edge mask + tile
// components (smem: Geo<TR,NW>::bytes of dynamic shared memory).
template <int TR, int NW>
__device__ __forceinline__ void tile_body(const ScanDesc* d, int lt, unsigned char* smem, int32_t* err) {
  using G = Geo<TR, NW>;
  constexpr int TC = G::TC;
  int* lp = reinterpret_cast<int*>(smem + G::off_lp);
  uint8_t* tb = smem + G::off_tb;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float4* ring = reinterpret_cast<float4*>(smem + G::off_ring) + (size_t)w * (RING + 1) * 32 + lane;
  const Loc L = make_loc(d, lt, TR, TC);
  const float4* __restrict__ xyzr = d->xyzr;
  const float* __restrict__ range = d->range;
  const int32_t* __restrict__ order = d->order;
  const float2* __restrict__ trig = d->trig;
  const float rmin = d->r_min, rmax = d->r_max, jh = d->jump_h, jv = d->jump_v;
  // offsets of the input rows the tile reads (ring order applied once)
  long long* rows_s = reinterpret_cast<long long*>(smem + G::off_rows);
  for (int k = threadIdx.x; k < L.rn + 3; k += G::NT) {
    const int i = L.r0 - 1 + k;
    long long ro = -1;
    if (i >= 0 && i < L.H) {
      const int row = __ldg(order + i);
      if ((unsigned)row < (unsigned)L.H) ro = (long long)row * L.W;
    }
    rows_s[k] = ro;
  }
  __syncthreads();

  // The sweep: warp w owns tile columns w*29-1 .. w*29+30 (one per lane),
  // of which lanes 1..29 are its output columns.  Each lane streams its
  // column's rows from global memory into its own ring of shared-memory
  // slots with cp.async, RING rows ahead of use (coalesced 16-byte copies
  // across the warp; a lane only reads slots it filled, so no barrier).  At
  // step hr it holds scan row r0-1+hr and completes: the R edge of that row,
  // the D and G edges of the row above, the normal of the row above that
  // (Sec. 2, normal estimation) and the homogeneity mask of the row above
  // that (Algorithm 1 predicate).
  {
    const int col = w * SO + lane;  // tile column + 1
    const int lc = col - 1;         // tile column
    const bool out_col = lane >= 1 && lane <= SO && lc < L.cn;
    int j = L.c0 + lc;              // scan column of this lane
    if (L.wrap) {
      if (j < 0) j += L.Ws;
      else if (j >= L.Ws) j -= L.Ws;
      if (j >= L.Ws) j %= L.Ws;
    }
    const bool colok = j >= 0 && j < L.Ws;
    const size_t coff = (size_t)(colok ? j : 0) * L.s;
    float sp = 0.f, cp = 1.f;
    if (!xyzr && colok) sincosf(fmaf((float)(j * L.s), d->daz, d->az0), &sp, &cp);
    const float nsign = d->nsign, cos_t = d->cos_t;
    const float cx = d->comp_x, cy = d->comp_y, cz = d->comp_z;
    const bool angle_pred = d->pred == LSG_PRED_ANGLE;
    uint8_t* __restrict__ mb_out = d->mb;
    float* __restrict__ nrm_out = d->nrm;

    float4 Pp = make_float4(0.f, 0.f, 0.f, -1.f);           // row k-1
    float eRx_p = 0.f, eRy_p = 0.f, eRz_p = 0.f, LR_p = 0.f;  // R edge of row k-1
    float eDx_pp = 0.f, eDy_pp = 0.f, eDz_pp = 0.f, LD_pp = 0.f;  // D edge of row k-2
    float eGx_ppL = 0.f, eGy_ppL = 0.f, eGz_ppL = 0.f, LG_ppL = 0.f;  // G edge of row k-2, left lane
    uint32_t m_pp = 0, m_p = 0;                                // mesh bits of rows k-2, k-1
    float4 n_pp = make_float4(0.f, 0.f, 0.f, 0.f);             // normal of row k-2
    const int rbase = L.r0 - 1;
    const int nsteps = L.rn + 3;
    size_t vout = (size_t)L.r0 * L.Ws + (size_t)(L.c0 + lc);  // output vertex of tile row 0
#pragma unroll
    for (int q = 0; q < RING; ++q) {
      if (q < nsteps) fetch_point(ring + q * 32, xyzr, range, trig, rbase + q, rows_s[q], colok, coff, sp, cp);
      asm volatile("cp.async.commit_group;\n" ::: "memory");
    }

    for (int hr = 0; hr < nsteps; ++hr) {
      // row hr has landed once at most RING-1 newer groups are pending
      asm volatile("cp.async.wait_group %0;\n" ::"n"(RING - 1) : "memory");
      float4 P = ring[(hr % (RING + 1)) * 32];
      // refill: the slot of row hr+RING was last read one step ago
      if (hr + RING < nsteps)
        fetch_point(ring + ((hr + RING) % (RING + 1)) * 32, xyzr, range, trig, rbase + hr + RING,
                    rows_s[hr + RING], colok, coff, sp, cp);
      asm volatile("cp.async.commit_group;\n" ::: "memory");
      if (!in_range(P.w, rmin, rmax)) P = make_float4(0.f, 0.f, 0.f, P.w);  // finite spokes only
      float4 Pr;
      Pr.x = __shfl_down_sync(FULL, P.x, 1);
      Pr.y = __shfl_down_sync(FULL, P.y, 1);
      Pr.z = __shfl_down_sync(FULL, P.z, 1);
      Pr.w = __shfl_down_sync(FULL, P.w, 1);
      const bool vP = in_range(P.w, rmin, rmax);
      const bool vPr = lane < 31 && in_range(Pr.w, rmin, rmax);
      // R edge of row k
      const bool Rk = vP && vPr && !jump_cut(P.w, Pr.w, jh);
      const float eRx = Pr.x - P.x, eRy = Pr.y - P.y, eRz = Pr.z - P.z;
      const float LR = vlen(eRx, eRy, eRz);
      // D and G edges of row k-1
      const bool vPp = in_range(Pp.w, rmin, rmax);
      const bool Dk1 = vPp && vP && !jump_cut(Pp.w, P.w, jv);
      const bool Gk1 = vPp && vPr && !jump_cut(Pp.w, Pr.w, jv);
      const float eDx = P.x - Pp.x, eDy = P.y - Pp.y, eDz = P.z - Pp.z;
      const float eGx = Pr.x - Pp.x, eGy = Pr.y - Pp.y, eGz = Pr.z - Pp.z;
      const float LD = vlen(eDx, eDy, eDz), LG = vlen(eGx, eGy, eGz);
      m_p |= (Dk1 ? B_D : 0u) | (Gk1 ? B_G : 0u);
      const uint32_t m_k = (Rk ? B_R : 0u) | (vP ? B_VALID : 0u);
      // neighbours' mesh bits (byte 0: row k-2, byte 1: row k-1, byte 2: row k)
      const uint32_t word = m_pp | (m_p << 8) | (m_k << 16);
      const uint32_t up = __shfl_up_sync(FULL, word, 1);
      const uint32_t dn = __shfl_down_sync(FULL, word, 1);
      const float eRxL = __shfl_up_sync(FULL, eRx_p, 1);
      const float eRyL = __shfl_up_sync(FULL, eRy_p, 1);
      const float eRzL = __shfl_up_sync(FULL, eRz_p, 1);
      const float LRL = __shfl_up_sync(FULL, LR_p, 1);

      // normal of row k-1, vertex p (spokes in the paper's order A..F):
      // A = eD, B = eG, C = eR(k-1), D = -eD(k-2), E = -eG(k-2, left),
      // F = -eR(k-1, left); triangle (p, q, q') counts when its 3 edges exist
      float4 n_p = make_float4(0.f, 0.f, 0.f, 0.f);
      {
        const uint32_t upp = up & 0xff, upl = (up >> 8) & 0xff, dnl = (dn >> 8) & 0xff;
        const bool sA = Dk1, sB = Gk1, sC = (m_p & B_R) != 0, sD = (m_pp & B_D) != 0;
        const bool sE = (upp & B_G) != 0, sF = (upl & B_R) != 0;
        float sx = 0.f, sy = 0.f, sz = 0.f;
        tri_term(eDx, eDy, eDz, LD, eGx, eGy, eGz, LG, sA && sB && Rk, sx, sy, sz);
        tri_term(eGx, eGy, eGz, LG, eRx_p, eRy_p, eRz_p, LR_p, sB && sC && (dnl & B_D), sx, sy, sz);
        tri_term(eRx_p, eRy_p, eRz_p, LR_p, -eDx_pp, -eDy_pp, -eDz_pp, LD_pp, sC && sD && (m_pp & B_G), sx, sy,
                 sz);
        tri_term(-eDx_pp, -eDy_pp, -eDz_pp, LD_pp, -eGx_ppL, -eGy_ppL, -eGz_ppL, LG_ppL,
                 sD && sE && (upp & B_R), sx, sy, sz);
        tri_term(-eGx_ppL, -eGy_ppL, -eGz_ppL, LG_ppL, -eRxL, -eRyL, -eRzL, LRL, sE && sF && (upp & B_D), sx, sy,
                 sz);
        tri_term(-eRxL, -eRyL, -eRzL, LRL, eDx, eDy, eDz, LD, sF && sA && (upl & B_G), sx, sy, sz);
        const float q2 = fmaf(sx, sx, fmaf(sy, sy, sz * sz));
        // q2 > 0 only when some triangle counted (absent terms are exact zeros)
        if ((m_p & B_VALID) && q2 > 0.f && q2 < 3.0e38f) {
          const float f = nsign * rsqrtf(q2);
          n_p = make_float4(sx * f, sy * f, sz * f, 1.f);
        }
      }

      // homogeneity mask and outputs of row k-2
      if (hr >= 3) {
        const float4 nr_pp = make_float4(__shfl_down_sync(FULL, n_pp.x, 1), __shfl_down_sync(FULL, n_pp.y, 1),
                                         __shfl_down_sync(FULL, n_pp.z, 1), __shfl_down_sync(FULL, n_pp.w, 1));
        const float4 nr_p = make_float4(__shfl_down_sync(FULL, n_p.x, 1), __shfl_down_sync(FULL, n_p.y, 1),
                                        __shfl_down_sync(FULL, n_p.z, 1), __shfl_down_sync(FULL, n_p.w, 1));
        const int lr = hr - 3;
        uint32_t bits = m_pp | (n_pp.w != 0.f ? B_HASN : 0u);
        bits |= ((m_pp & B_R) && homog(n_pp, nr_pp, angle_pred, cos_t, cx, cy, cz)) ? B_HR : 0u;
        bits |= ((m_pp & B_D) && homog(n_pp, n_p, angle_pred, cos_t, cx, cy, cz)) ? B_HD : 0u;
        bits |= ((m_pp & B_G) && homog(n_pp, nr_p, angle_pred, cos_t, cx, cy, cz)) ? B_HG : 0u;
        if (out_col && lr < L.rn) {
          const size_t v = vout;
          mb_out[v] = (uint8_t)bits;
          nrm_out[3 * v + 0] = n_pp.x;
          nrm_out[3 * v + 1] = n_pp.y;
          nrm_out[3 * v + 2] = n_pp.z;
          tb[lr * TC + lc] = (uint8_t)bits;
        }
        vout += L.Ws;
      }

      // rotate the window
      const float gxL = __shfl_up_sync(FULL, eGx, 1), gyL = __shfl_up_sync(FULL, eGy, 1);
      const float gzL = __shfl_up_sync(FULL, eGz, 1), gLL = __shfl_up_sync(FULL, LG, 1);
      m_pp = m_p;
      m_p = m_k;
      eDx_pp = eDx;
      eDy_pp = eDy;
      eDz_pp = eDz;
      LD_pp = LD;
      eGx_ppL = gxL;
      eGy_ppL = gyL;
      eGz_ppL = gzL;
      LG_ppL = gLL;
      eRx_p = eRx;
      eRy_p = eRy;
      eRz_p = eRz;
      LR_p = LR;
      n_pp = n_p;
      Pp = P;
    }
  }
  __syncthreads();

  // tile components (Algorithm 1 restricted to the tile)
  tile_components<TR, NW>(L, tb, lp, d->lroot, d->parent, err);
}

template <int TR, int NW>
__global__ void __launch_bounds__(NW * 32, 24 / NW) k_tile(const __grid_constant__ KArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
    int lt;
    const ScanDesc* d = tile_desc(a, t, lt);
    tile_body<TR, NW>(d, lt, smem, a.err);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// k_tile_ccl: tile components of a given mesh byte array
// ---------------------------------------------------------------------------
template <int TR, int NW>
__global__ void __launch_bounds__(NW * 32) k_tile_ccl(const __grid_constant__ KArgs a) {
  using G = Geo<TR, NW>;
  constexpr int TC = G::TC;
  extern __shared__ __align__(16) unsigned char smem[];
  int* lp = reinterpret_cast<int*>(smem);
  uint8_t* tb = smem + sizeof(int) * G::NV;
  for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
    int lt;
    const ScanDesc* d = tile_desc(a, t, lt);
    const Loc L = make_loc(d, lt, TR, TC);
    for (int k = threadIdx.x; k < G::NV; k += G::NT) {
      const int lr = k / TC, lc = k - (k / TC) * TC;
      tb[k] = (lr < L.rn && lc < L.cn) ? d->mb[(size_t)(L.r0 + lr) * L.Ws + (L.c0 + lc)] : 0;
    }
    __syncthreads();
    tile_components<TR, NW>(L, tb, lp, d->lroot, d->parent, a.err);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// global roots
// ---------------------------------------------------------------------------
// Scan-local index of the tile-local root of vertex (i, j).
template <int TR, int TC>
__device__ __forceinline__ int tile_root(const uint16_t* __restrict__ lroot, int Ws, int i, int j) {
  const int r = lroot[(size_t)i * root_pitch(Ws) + j];
  const int rr = r / TC, rc = r - (r / TC) * TC;
  return ((i / TR) * TR + rr) * Ws + (j / TC) * TC + rc;
}

// ---------------------------------------------------------------------------
// k_merge: join components across tile borders and the 360 deg seam
// ---------------------------------------------------------------------------
constexpr int NT_MERGE = 128;

// Border unions of one tile (NTB threads).
template <int TR, int NW, int NTB>
__device__ __forceinline__ void merge_body(const ScanDesc* d, int lt, int32_t* err) {
  constexpr int TC = NW * SO;
  const Loc L = make_loc(d, lt, TR, TC);
  const uint8_t* __restrict__ mb = d->mb;
  const uint16_t* __restrict__ lroot = d->lroot;
  int32_t* parent = d->parent;
  const int limit = L.H * L.Ws + 1;
  const bool full_ring = L.wrap && L.c0 == 0 && L.cn == L.Ws;
  // border vertices: the last row of the tile, then the last column above it
  const int nb = L.cn + L.rn - 1;
  for (int k = threadIdx.x; k < nb; k += NTB) {
    int lr, lc;
    if (k < L.cn) {
      lr = L.rn - 1;
      lc = k;
    } else {
      lr = k - L.cn;
      lc = L.cn - 1;
    }
    const int i = L.r0 + lr, j = L.c0 + lc;
    const uint8_t bits = mb[(size_t)i * L.Ws + j];
    if (!(bits & (B_HR | B_HD | B_HG))) continue;
    // bits pointing off the grid (possible in a caller-given mask) are ignored
    const bool has_right = (j + 1 < L.Ws) || L.wrap;
    const bool has_down = i + 1 < L.H;
    const int jn = (j + 1 == L.Ws) ? 0 : j + 1;
    const bool jn_in = (lc + 1 < L.cn) || full_ring;
    const bool down_in = lr + 1 < L.rn;
    const bool hr_out = (bits & B_HR) && has_right && !jn_in;
    const bool hd_out = (bits & B_HD) && has_down && !down_in;
    const bool hg_out = (bits & B_HG) && has_down && has_right && !(down_in && jn_in);
    if (!(hr_out || hd_out || hg_out)) continue;
    const size_t LP = root_pitch(L.Ws);
    if (lroot[(size_t)i * LP + j] == NO_ROOT) continue;
    // along the bottom border, a D edge whose two tile roots equal those of
    // the left neighbour's D edge adds nothing
    if (hd_out && !hr_out && !hg_out && k > 0 && k < L.cn) {
      const uint8_t bl = mb[(size_t)i * L.Ws + j - 1];
      if ((bl & B_HD) && lroot[(size_t)i * LP + j - 1] == lroot[(size_t)i * LP + j] &&
          lroot[(size_t)(i + 1) * LP + j - 1] == lroot[(size_t)(i + 1) * LP + j])
        continue;
    }
    const int rp = tile_root<TR, TC>(lroot, L.Ws, i, j);
    if (hr_out && lroot[(size_t)i * LP + jn] != NO_ROOT)
      union_g(parent, rp, tile_root<TR, TC>(lroot, L.Ws, i, jn), limit, err);
    if (hd_out && lroot[(size_t)(i + 1) * LP + j] != NO_ROOT)
      union_g(parent, rp, tile_root<TR, TC>(lroot, L.Ws, i + 1, j), limit, err);
    if (hg_out && lroot[(size_t)(i + 1) * LP + jn] != NO_ROOT)
      union_g(parent, rp, tile_root<TR, TC>(lroot, L.Ws, i + 1, jn), limit, err);
  }
}

template <int TR, int NW>
__global__ void __launch_bounds__(NT_MERGE) k_merge(const __grid_constant__ KArgs a) {
  for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
    int lt;
    const ScanDesc* d = tile_desc(a, t, lt);
    merge_body<TR, NW, NT_MERGE>(d, lt, a.err);
  }
}

// ---------------------------------------------------------------------------
// k_flatten: labels, back-fill, segment count
// ---------------------------------------------------------------------------
constexpr int NT_FLAT = 256;

// Root of a chain in the (now read-only) global union-find: cached loads.
__device__ __forceinline__ int find_ro(const int32_t* __restrict__ P, int x, int limit) {
  int p = __ldg(P + x);
  while (p != x && limit-- > 0) {
    x = p;
    p = __ldg(P + x);
  }
  return x;
}

// Label of any vertex of the scan (used for the back-fill neighbour that lies
// in the next tile).
template <int TR, int TC>
__device__ __forceinline__ int32_t vertex_label_global(const uint16_t* __restrict__ lroot,
                                                       const int32_t* __restrict__ parent, int Ws, int W,
                                                       int s, int i, int j, int limit) {
  if (lroot[(size_t)i * root_pitch(Ws) + j] == NO_ROOT) return -1;
  const int g = find_ro(parent, tile_root<TR, TC>(lroot, Ws, i, j), limit);
  const int gi = g / Ws, gj = g - gi * Ws;
  return gi * W + gj * s;
}

// Label of a point between sampled columns (Sec. 2, last paragraph): the
// nearer of the two bracketing sampled columns on its ring, ties to the
// earlier, the other when the nearer is unlabelled.
__device__ __forceinline__ int32_t backfill(int32_t lo, int dlo, int32_t hi, int dhi, bool have_hi) {
  int32_t first = lo, second = have_hi ? hi : -1;
  if (have_hi && dhi < dlo) {
    first = hi;
    second = lo;
  }
  return first != -1 ? first : second;
}

// Per tile: (1) stage the tile's 16-bit local roots in shared memory,
// (2) resolve every local root once to its global root and label (and count
// the global roots), (3) write every point's label, back-filling the points
// between sampled columns.  Loops are two-dimensional (warps over rows,
// lanes over columns): no integer division per point.
template <int TR, int NW>
struct FlatGeo {
  static constexpr int TC = NW * SO, NV = TR * TC;
  static constexpr size_t off_lr = 0;                                      // uint16 [NV] tile roots
  static constexpr size_t off_lab = ((sizeof(uint16_t) * NV + 15) / 16) * 16;  // int32 [NV] root labels
  static constexpr size_t off_list = off_lab + sizeof(int32_t) * NV;       // uint16 [NV] list of roots
  static constexpr size_t bytes = off_list + ((sizeof(uint16_t) * NV + 15) / 16) * 16;
};

// Labels of one tile (NTB threads; fsm: FlatGeo<TR,NW>::bytes of dynamic
// shared memory; nlist: a shared counter).
template <int TR, int NW, int NTB>
__device__ __forceinline__ void flatten_body(const ScanDesc* d, int lt, unsigned char* fsm, int& nlist) {
  using FG = FlatGeo<TR, NW>;
  constexpr int TC = FG::TC, NWF = NTB / 32;
  uint16_t* lr_s = reinterpret_cast<uint16_t*>(fsm + FG::off_lr);
  int32_t* lab_s = reinterpret_cast<int32_t*>(fsm + FG::off_lab);
  uint16_t* list_s = reinterpret_cast<uint16_t*>(fsm + FG::off_list);
  const int tid = threadIdx.x, lane = tid & 31, wf = tid >> 5;
  const Loc L = make_loc(d, lt, TR, TC);
  const int W = L.W, Ws = L.Ws, s = L.s;
  const uint16_t* __restrict__ lroot = d->lroot;
  const int32_t* __restrict__ parent = d->parent;
  int32_t* __restrict__ labels = d->labels;
  const int limit = L.H * Ws + 1;
  if (tid == 0) nlist = 0;
  // (1) the tile's roots, four at a time (rows are 8-byte aligned: the
  //     pitch is a multiple of 8 and TC a multiple of 4)
  const int nq = (L.cn + 3) >> 2;
  for (int lr = wf; lr < L.rn; lr += NWF) {
    const uint2* src = reinterpret_cast<const uint2*>(lroot + (size_t)(L.r0 + lr) * root_pitch(Ws) + L.c0);
    uint2* dst = reinterpret_cast<uint2*>(lr_s + lr * TC);
#pragma unroll 2
    for (int q = lane; q < nq; q += 32) dst[q] = __ldg(src + q);
  }
  __syncthreads();
  // (2) list the tile-local roots, then resolve each to its global root,
  //     four chains per thread at a time
  for (int lr = wf; lr < L.rn; lr += NWF) {
    for (int lc0 = 0; lc0 < L.cn; lc0 += 32) {
      const int lc = lc0 + lane;
      const int v = lr * TC + lc;
      const bool is_root = lc < L.cn && lr_s[v] == v;
      const unsigned m = __ballot_sync(FULL, is_root);
      int base = 0;
      if (lane == 0 && m) base = atomicAdd(&nlist, __popc(m));
      base = __shfl_sync(FULL, base, 0);
      if (is_root) list_s[base + __popc(m & ((1u << lane) - 1u))] = (uint16_t)v;
    }
  }
  __syncthreads();
  int nroots = 0;
  const int nl = nlist;
  for (int k0 = tid; k0 < nl; k0 += 4 * NTB) {
    int x[4], gv[4];
    bool live[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int k = k0 + q * NTB;
      live[q] = k < nl;
      const int v = live[q] ? list_s[k] : 0;
      gv[q] = (L.r0 + v / TC) * Ws + L.c0 + v % TC;
      x[q] = gv[q];
    }
    // walk the four chains together (independent loads in flight)
    for (int it = 0; it < limit; ++it) {
      bool more = false;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (!live[q]) continue;
        const int p = __ldg(parent + x[q]);
        if (p != x[q]) {
          x[q] = p;
          more = true;
        }
      }
      if (!more) break;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (!live[q]) continue;
      const int g = x[q];
      nroots += (g == gv[q]);
      const int gi = g / Ws, gj = g - gi * Ws;
      lab_s[list_s[k0 + q * NTB]] = gi * W + gj * s;
    }
  }
  const int cnt = __reduce_add_sync(FULL, nroots);
  if (lane == 0 && cnt) atomicAdd(d->nseg, cnt);
  __syncthreads();
  if (s == 1) {
    for (int lr = wf; lr < L.rn; lr += NWF) {
      int32_t* dst = labels + (size_t)(L.r0 + lr) * W + L.c0;
#pragma unroll 4
      for (int lc = lane; lc < L.cn; lc += 32) {
        const uint16_t r = lr_s[lr * TC + lc];
        dst[lc] = r == NO_ROOT ? -1 : lab_s[r];
      }
    }
  } else {
    for (int lr = wf; lr < L.rn; lr += NWF) {
      const int i = L.r0 + lr;
      const int row = d->order[i];
      for (int lc = lane; lc < L.cn; lc += 32) {
        const int j = L.c0 + lc;
        const uint16_t rl = lr_s[lr * TC + lc];
        const int32_t lo = rl == NO_ROOT ? -1 : lab_s[rl];
        labels[(size_t)i * W + (size_t)j * s] = lo;
        // the s-1 points after column j*s
        int jh = -1, cnext = 0;
        if (j + 1 < Ws) {
          jh = j + 1;
          cnext = (j + 1) * s;
        } else if (L.wrap) {
          jh = 0;
          cnext = W;
        }
        int32_t hi = -1;
        if (jh >= 0) {
          if (jh >= L.c0 && jh < L.c0 + L.cn) {
            const uint16_t rh = lr_s[lr * TC + (jh - L.c0)];
            hi = rh == NO_ROOT ? -1 : lab_s[rh];
          } else {
            hi = vertex_label_global<TR, TC>(lroot, parent, Ws, W, s, i, jh, limit);
          }
        }
        const int cend = min((j + 1) * s, W);
        for (int c = j * s + 1; c < cend; ++c) {
          bool ok;
          if (d->valid) {
            ok = d->valid[(size_t)i * W + c] != 0;
          } else {
            float r = -1.f;
            if ((unsigned)row < (unsigned)L.H) {
              const size_t o = (size_t)row * W + c;
              r = d->xyzr ? __ldg(&d->xyzr[o].w) : __ldg(d->range + o);
            }
            ok = in_range(r, d->r_min, d->r_max);
          }
          labels[(size_t)i * W + c] = ok ? backfill(lo, c - j * s, hi, cnext - c, jh >= 0) : -1;
        }
      }
    }
  }
}

template <int TR, int NW>
__global__ void __launch_bounds__(NT_FLAT) k_flatten(const __grid_constant__ KArgs a) {
  extern __shared__ __align__(16) unsigned char fsm[];
  __shared__ int nlist;
  for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
    int lt;
    const ScanDesc* d = tile_desc(a, t, lt);
    flatten_body<TR, NW, NT_FLAT>(d, lt, fsm, nlist);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// k_fused: the whole batched pass in one persistent launch
// ---------------------------------------------------------------------------
// Waits (one thread) until *cnt reaches need; gives up after about a second,
// recording a timeout in the error word instead of hanging.
__device__ __forceinline__ void wait_count(const int32_t* cnt, int need, int32_t* err) {
  for (unsigned it = 0;; ++it) {
    if (*reinterpret_cast<const volatile int32_t*>(cnt) >= need) break;
    if (it > (1u << 23)) {
      atomicOr(err, DERR_TIMEOUT);
      break;
    }
    __nanosleep(128);
  }
  __threadfence();
}

template <int TR, int NW>
struct FusedGeo {
  static constexpr size_t a = Geo<TR, NW>::bytes, b = FlatGeo<TR, NW>::bytes, c = sizeof(float) * LSG_MAX_RINGS;
  static constexpr size_t ab = a > b ? a : b;
  static constexpr size_t bytes = ab > c ? ab : c;
};

// Every CTA takes the next item of the schedule (one atomic per item), waits
// for the items it depends on (the scan's ring order for a tile, all the
// scan's tiles for a border merge, all its merges for a labels item), runs
// it, and counts it done.  Items only wait on items taken earlier, which are
// held by running CTAs, so the pass cannot deadlock whatever the number of
// CTAs that fit on the GPU.
template <int TR, int NW>
__global__ void __launch_bounds__(NW * 32) k_fused(const __grid_constant__ FusedArgs f) {
  constexpr int NTB = NW * 32;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int item_s;
  __shared__ int nlist;
  int32_t* next = f.counters;
  int32_t* doneP = f.counters + 1;
  int32_t* doneA = doneP + f.nscans;
  int32_t* doneB = doneA + f.nscans;
  for (;;) {
    if (threadIdx.x == 0) item_s = atomicAdd(next, 1);
    __syncthreads();
    const int it = item_s;
    __syncthreads();
    if (it >= f.nitems) break;
    const int2 wi = f.items[it];
    const int ph = wi.x >> 28, b = wi.x & 0x0fffffff, lt = wi.y;
    const ScanDesc* d = f.scans + b;
    if (threadIdx.x == 0 && ph != PH_PREP) {
      const int32_t* cnt = ph == PH_TILE ? doneP + b : (ph == PH_MERGE ? doneA + b : doneB + b);
      wait_count(cnt, ph == PH_TILE ? 1 : d->tiles_r * d->tiles_c, f.err);
    }
    __syncthreads();
    if (ph == PH_PREP) prep_body<NTB>(d, reinterpret_cast<float*>(smem), f.err);
    else if (ph == PH_TILE) tile_body<TR, NW>(d, lt, smem, f.err);
    else if (ph == PH_MERGE) merge_body<TR, NW, NTB>(d, lt, f.err);
    else flatten_body<TR, NW, NTB>(d, lt, smem, nlist);
    __syncthreads();
    if (threadIdx.x == 0 && ph != PH_FLAT) {
      __threadfence();  // this CTA's writes before the count that releases them
      atomicAdd(ph == PH_PREP ? doneP + b : (ph == PH_TILE ? doneA + b : doneB + b), 1);
    }
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <int TR, int NW>
static cudaError_t set_attrs() {
  cudaError_t e = cudaFuncSetAttribute(k_tile<TR, NW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)Geo<TR, NW>::bytes);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_flatten<TR, NW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)FlatGeo<TR, NW>::bytes);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_fused<TR, NW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)FusedGeo<TR, NW>::bytes);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_tile_ccl<TR, NW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)Geo<TR, NW>::ccl_bytes);
}

cudaError_t prepare_kernels() {
  cudaError_t e;
  if ((e = set_attrs<16, 4>()) != cudaSuccess) return e;
  if ((e = set_attrs<32, 4>()) != cudaSuccess) return e;
  if ((e = set_attrs<32, 8>()) != cudaSuccess) return e;
  if ((e = set_attrs<64, 4>()) != cudaSuccess) return e;
  if ((e = set_attrs<64, 8>()) != cudaSuccess) return e;
  return cudaSuccess;
}

cudaError_t launch_prep(const KArgs& a, cudaStream_t st) {
  const int n = a.scans ? a.nscans : 1;
  k_prep<<<n, NT_PREP, 0, st>>>(a);
  return cudaGetLastError();
}

#define LSG_DISPATCH(tile, FN, ...)                       \
  switch (tile) {                                         \
    case LSG_TILE_32x116: return FN<32, 4>(__VA_ARGS__);  \
    case LSG_TILE_32x232: return FN<32, 8>(__VA_ARGS__);  \
    case LSG_TILE_64x116: return FN<64, 4>(__VA_ARGS__);  \
    case LSG_TILE_64x232: return FN<64, 8>(__VA_ARGS__);  \
    default: return FN<16, 4>(__VA_ARGS__);               \
  }

template <int TR, int NW>
static cudaError_t run_tile(const KArgs& a, cudaStream_t st) {
  k_tile<TR, NW><<<a.ntiles, NW * 32, Geo<TR, NW>::bytes, st>>>(a);
  return cudaGetLastError();
}
template <int TR, int NW>
static cudaError_t run_tile_ccl(const KArgs& a, cudaStream_t st) {
  k_tile_ccl<TR, NW><<<a.ntiles, NW * 32, Geo<TR, NW>::ccl_bytes, st>>>(a);
  return cudaGetLastError();
}
template <int TR, int NW>
static cudaError_t run_merge(const KArgs& a, cudaStream_t st) {
  k_merge<TR, NW><<<a.ntiles, NT_MERGE, 0, st>>>(a);
  return cudaGetLastError();
}
template <int TR, int NW>
static cudaError_t run_flatten(const KArgs& a, cudaStream_t st) {
  k_flatten<TR, NW><<<a.ntiles, NT_FLAT, FlatGeo<TR, NW>::bytes, st>>>(a);
  return cudaGetLastError();
}

template <int TR, int NW>
static cudaError_t run_fused(const FusedArgs& f, cudaStream_t st) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fused<TR, NW>, NW * 32, FusedGeo<TR, NW>::bytes);
  if (e != cudaSuccess) return e;
  const int grid = max(1, min(sms * max(per_sm, 1), f.nitems));
  k_fused<TR, NW><<<grid, NW * 32, FusedGeo<TR, NW>::bytes, st>>>(f);
  return cudaGetLastError();
}

cudaError_t launch_fused(int tile, const FusedArgs& f, cudaStream_t st) { LSG_DISPATCH(tile, run_fused, f, st) }

cudaError_t launch_tile(int tile, const KArgs& a, cudaStream_t st) { LSG_DISPATCH(tile, run_tile, a, st) }
cudaError_t launch_tile_ccl(int tile, const KArgs& a, cudaStream_t st) {
  LSG_DISPATCH(tile, run_tile_ccl, a, st)
}
cudaError_t launch_merge(int tile, const KArgs& a, cudaStream_t st) { LSG_DISPATCH(tile, run_merge, a, st) }
cudaError_t launch_flatten(int tile, const KArgs& a, cudaStream_t st) {
  LSG_DISPATCH(tile, run_flatten, a, st)
}

}  // namespace lsg
