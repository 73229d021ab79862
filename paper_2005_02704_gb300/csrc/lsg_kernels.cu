// lsg_kernels.cu - CUDA kernels (sm_103a) of the Lidar surface-segmentation path.
//
// Mukherjee et al., "Fast Geometric Surface based Segmentation of Point Cloud
// from Lidar Data" (PReMI 2019), Sec. 2 and Algorithm 1.  One pass over a
// batch of scans is four launches (a single scan of at most kFuseMaxRings
// rings: three, its tile kernel doing k_prep's work for the rows it reads):
//
//   k_prep     ring order by elevation (rank counting), sin/cos of the sorted
//              elevations, segment counter reset.               [Sec. 2, point model]
//   k_tile     one CTA per tile of TR rows x (60*NW) columns of mesh vertices.
//              Each warp sweeps a strip of 64 columns (60 of them its own, two
//              per lane) down the rows: every lane streams its two columns'
//              x,y,z,r rows into shared-memory ring slots with cp.async a few
//              rows ahead, holds a three-row window in registers, and takes
//              the neighbouring columns from the adjacent lanes with warp
//              shuffles.  The geometry runs on packed binary32 pairs (both
//              columns in one instruction): mesh bits and edge vectors of
//              each row, the weighted normal of the row above, the
//              homogeneity mask of the row above that.  Every edge vector and
//              length is computed once and reused by both endpoints.  The
//              tile's components follow: horizontal runs from two warp
//              ballots, vertical joins with an atomicMin union-find over the
//              runs' first vertices in shared memory (only where the column to
//              the left does not already join the same two vertices), then
//              joins across strips.  Writes the mesh byte, the normal, and each
//              vertex's tile-local root (16 bits).
//                                          [Sec. 2 mesh, normals; Algorithm 1]
//   k_merge    joins tile-local components across tile borders and the 360 deg
//              seam with a lock-free atomicMin union-find over the roots.
//   k_flatten  label = smallest full-resolution index of the component,
//              back-fill of non-sampled points, segment count with warp
//              reductions (k_flatten1: the same for launches whose scans all
//              have s = 1, where every point is a vertex).
//                                                         [Algorithm 1; Sec. 2 end]
//
// Labels are exact: every union hooks the larger root under the smaller, so
// each component's root is its smallest vertex index whatever the thread
// order, and a tile-local root is the smallest index of its tile component.
#include <cuda_runtime.h>
#include <float.h>
#include <limits.h>
#include <stdint.h>

#include "lsg_internal.h"

namespace lsg {

constexpr uint8_t B_R = LSG_BIT_R, B_D = LSG_BIT_D, B_G = LSG_BIT_G;
constexpr uint8_t B_HR = LSG_BIT_HR, B_HD = LSG_BIT_HD, B_HG = LSG_BIT_HG;
static_assert(B_HR == B_R << 3 && B_HD == B_D << 3 && B_HG == B_G << 3,
              "a homogeneous bit is its edge bit three places up");
constexpr uint8_t B_VALID = LSG_BIT_VALID, B_HASN = LSG_BIT_HASN;
constexpr unsigned FULL = 0xffffffffu;
constexpr int SO = 60;  // output columns per warp strip (lanes 1..30, two columns each)
constexpr uint16_t NO_ROOT = 0xFFFF;  // tile-local root of a vertex out of range

// Row pitch of the tile-root array: Ws rounded up to 8 entries (16 bytes), so
// that a tile's rows can be read with aligned vector loads.
__host__ __device__ __forceinline__ int root_pitch(int Ws) { return (Ws + 7) & ~7; }

__host__ __device__ constexpr size_t align16(size_t x) { return (x + 15) / 16 * 16; }

TileShape tile_shape(int tile) {
  switch (tile) {
    case LSG_TILE_32x120: return {32, 120};
    case LSG_TILE_32x240: return {32, 240};
    case LSG_TILE_32x480: return {32, 480};
    case LSG_TILE_64x240: return {64, 240};
    case LSG_TILE_16x120: return {16, 120};
    case LSG_TILE_8x120: return {8, 120};
    case LSG_TILE_4x120: return {4, 120};
    case LSG_TILE_2x120: return {2, 120};
    case LSG_TILE_16x240:
    default: return {16, 240};
  }
}

int pick_tile(const int* H, const int* Ws, int n, int sms) {
  static const int order[7] = {LSG_TILE_32x120, LSG_TILE_32x240, LSG_TILE_16x240, LSG_TILE_16x120,
                               LSG_TILE_8x120,  LSG_TILE_4x120,  LSG_TILE_2x120};
  int best = order[0];
  long long best_n = -1;
  for (int k = 0; k < 7; ++k) {
    const TileShape ts = tile_shape(order[k]);
    long long nt = 0;
    for (int b = 0; b < n; ++b)
      if (H[b] > 0 && Ws[b] > 0) nt += (long long)((H[b] + ts.rows - 1) / ts.rows) * ((Ws[b] + ts.cols - 1) / ts.cols);
    if (nt >= 4LL * sms) return order[k];
    if (nt > best_n) {
      best_n = nt;
      best = order[k];
    }
  }
  return best;
}

// ---------------------------------------------------------------------------
// small device helpers
// ---------------------------------------------------------------------------
// Programmatic dependent launch: a kernel launched with the programmatic
// stream serialization attribute may be scheduled while the kernel before it
// in the stream is still running.  dep_wait blocks until that kernel has
// completed and its memory writes are visible (it returns at once for a
// kernel launched without the attribute); every kernel calls it before it
// reads anything.  dep_release lets the next kernel be scheduled now (it
// still waits in its own dep_wait).
__device__ __forceinline__ void dep_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void dep_release() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }

// Load of data another kernel wrote (CO = false: the read-only data path,
// for data that does not change while the kernel runs) or that an earlier
// work item of the same persistent launch wrote (CO = true: ld.global.cg,
// which reads L2, where the producer's writes are visible once its release
// count has been observed).
template <bool CO, typename T>
__device__ __forceinline__ T ld_in(const T* p) {
  if constexpr (CO) return __ldcg(p);
  else return __ldg(p);
}

__device__ __forceinline__ bool in_range(float r, float rmin, float rmax) {
  return rmin < r && r <= rmax;
}

__device__ __forceinline__ const ScanDesc* tile_desc(const KArgs& a, int t, int& lt) {
  if (a.scans) {
    const int tg = t + a.tile_base;
    const ScanDesc* d = a.scans + a.tile_scan[tg];
    lt = tg - d->tile0;
    return d;
  }
  lt = a.tile_list ? a.tile_list[t] : t;
  return &a.one;
}

// Union-find on shared memory.  P[x] <= x always holds, so the forest has no
// cycles and the root of every tree is its smallest index.  Finds halve
// paths: each visited node is re-pointed at its grandparent; the store only
// shortens a path to an ancestor (P[x] <= x still holds), so it is safe next
// to concurrent atomicMin links.

// Roots of a (when fa) and b (when fb) once every union is done (the forest
// no longer changes): plain loads without path halving, the two chains
// walked together so that their loads overlap; 0 for a chain not asked for.
__device__ __forceinline__ void find_done2_sh(const int* P, bool fa, int a, bool fb, int b, int limit, int& ra,
                                              int& rb) {
  int pa = fa ? P[a] : a, pb = fb ? P[b] : b;
  while ((pa != a || pb != b) && limit-- > 0) {
    if (pa != a) {
      a = pa;
      pa = P[a];
    }
    if (pb != b) {
      b = pb;
      pb = P[b];
    }
  }
  ra = fa ? a : 0;
  rb = fb ? b : 0;
}

// Joins the sets of a and b.  The two finds advance together, one
// path-halving step of each per round, so that their shared-memory loads
// are in flight at the same time.
__device__ void union_sh(int* P, int a, int b, int limit, int32_t* err) {
  volatile int* V = P;
  for (int it = 0; it < limit; ++it) {
    int pa = V[a], pb = V[b];
    for (int st = 0; (pa != a || pb != b) && st < limit; ++st) {
      const int ga = pa != a ? V[pa] : a;
      const int gb = pb != b ? V[pb] : b;
      if (pa != a) {
        if (ga != pa) V[a] = ga;
        a = ga;
      }
      if (pb != b) {
        if (gb != pb) V[b] = gb;
        b = gb;
      }
      pa = V[a];
      pb = V[b];
    }
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

// Joins the sets of a and b in the global union-find (same invariant, path
// halving and interleaved finds as union_sh; loads bypass L1 with
// ld.global.cg so they see the atomics, which resolve in L2): the two finds'
// L2 round trips overlap.
__device__ void union_g(int32_t* P, int a, int b, int limit, int32_t* err) {
  for (int it = 0; it < limit; ++it) {
    int pa = __ldcg(P + a), pb = __ldcg(P + b);
    for (int st = 0; (pa != a || pb != b) && st < limit; ++st) {
      const int ga = pa != a ? __ldcg(P + pa) : a;
      const int gb = pb != b ? __ldcg(P + pb) : b;
      if (pa != a) {
        if (ga != pa) __stcg(P + a, ga);
        a = ga;
      }
      if (pb != b) {
        if (gb != pb) __stcg(P + b, gb);
        b = gb;
      }
      pa = __ldcg(P + a);
      pb = __ldcg(P + b);
    }
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
  if (H == 0 || d->W == 0) {  // no points: nothing but the count (elevations unread)
    if (threadIdx.x == 0) *d->nseg = 0;
    return;
  }
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
  dep_wait();
  dep_release();
  prep_body<NT_PREP>(a.scans ? a.scans + blockIdx.x : &a.one, se, a.err);
}

// ---------------------------------------------------------------------------
// tile geometry
// ---------------------------------------------------------------------------
constexpr int RING = 4;  // row slots per lane and point (RING - 1 rows in flight)
constexpr int QCAP = 256;  // pending tile unions per warp (flushed before it can overflow)

template <int TR, int NW>
struct Geo {
  static constexpr int NT = NW * 32;
  static constexpr int TC = NW * SO;             // output columns of a tile
  static constexpr int HR = TR + 3;              // rows read: r0-1 .. r0+TR+1
  static constexpr int NV = TR * TC;
  // The sweep's per-warp row rings [NW][RING][2][32] float4 and, once the
  // sweep is over, the tile union-find int[NV] share the first region.
  static constexpr size_t ring_bytes = sizeof(float4) * NW * RING * 64;
  static constexpr size_t lp_bytes = sizeof(int) * NV;
  static constexpr size_t off_ring = 0;
  static constexpr size_t off_lp = 0;
  static constexpr size_t off_tb = ((ring_bytes > lp_bytes ? ring_bytes : lp_bytes) + 15) / 16 * 16;
  // input row offsets long long [HR + RING - 1] (the last RING - 1 entries:
  // rows past the sweep, never read), then float2 [HR] sin, cos
  static constexpr size_t off_rows = off_tb + ((NV + 15) / 16) * 16;
  static constexpr size_t off_trig = off_rows + ((sizeof(long long) * (HR + RING - 1) + 15) / 16) * 16;
  static constexpr size_t off_q = off_trig + ((sizeof(float2) * HR + 15) / 16) * 16;  // uint32 [NW][QCAP]
  // queue uint32 [NW][QCAP], then the run starts of every strip row uint16 [NW][TR][32]
  static constexpr size_t q_bytes = sizeof(uint32_t) * NW * QCAP + sizeof(uint16_t) * NW * TR * 32;
  static constexpr size_t bytes = off_q + q_bytes;
  static constexpr size_t ccl_bytes = lp_bytes + ((NV + 15) / 16) * 16 + q_bytes;  // k_tile_ccl: lp, tb, queue
};

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Issue the asynchronous copy of one point into a ring slot: x,y,z,r
// (16 bytes), or the range alone (4 bytes, into the slot's r; the sweep
// decodes x,y,z when it reads the slot).  ro = offset of the input row (ring
// order * W), or -1 when the row is outside the scan (or past the sweep);
// then, and for a column outside the scan, the copy reads nothing and fills
// the slot with zeros: an absent point (r = 0 is out of range, r_min >= 0).
// No branch: the copy's source size is 0 or the full size.
__device__ __forceinline__ void fetch_point(float4* slot, const float4* __restrict__ xyzr,
                                            const float* __restrict__ range, long long ro, bool colok,
                                            unsigned coff) {
  const bool ok = colok && ro >= 0;
  const size_t o = ok ? (size_t)ro + coff : 0;
  const unsigned dst = (unsigned)__cvta_generic_to_shared(slot);
  if (xyzr)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(xyzr + o), "r"(ok ? 16u : 0u)
                 : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(dst + 12u), "l"(range + o), "r"(ok ? 4u : 0u)
                 : "memory");
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

// Sampled column j taken around the ring (wrap only: Ws >= 3).
__device__ __forceinline__ int wrap_col(int j, int Ws) {
  if (j < 0) j += Ws;
  else if (j >= Ws) j -= Ws;
  if (j < 0 || j >= Ws) j = ((j % Ws) + Ws) % Ws;
  return j;
}

// ---------------------------------------------------------------------------
// packed binary32 arithmetic: a lane's two columns in one instruction
// (.x: the lane's first column, .y: its second)
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// a - b rounded once (b * -1 is exact), as a binary32 subtraction
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

// Hardware approximations (PTX rsqrt.approx / rcp.approx, flush-to-zero):
// relative error below 2^-22 and 1 ulp respectively.
__device__ __forceinline__ float rsq_approx(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Lengths of two vectors: q * rsqrt(q + 1e-37) + 1e-30.  The offsets leave
// every length above 1e-23 unchanged, keep the reciprocal square root finite
// for a zero vector (whose length comes out as 1e-30) and keep a sum of two
// lengths nonzero, so the reciprocal weights below stay finite.
__device__ __forceinline__ float2 len2(float2 x, float2 y, float2 z) {
  const float2 q = fma2(x, x, fma2(y, y, mul2(z, z)));
  const float2 qg = add2(q, make_float2(1e-37f, 1e-37f));
  return fma2(q, make_float2(rsq_approx(qg.x), rsq_approx(qg.y)), make_float2(1e-30f, 1e-30f));
}

// Depth-jump cut of two edges: |r_p - r_q| > tau * min(r_p, r_q) in
// binary32, round to nearest, never contracted (reproducible decisions).
__device__ __forceinline__ void jump_cut2(float2 rp, float2 rq, float2 tau, bool& ca, bool& cb) {
  const float2 dd = sub2(rp, rq);
  const float2 t = mul2(tau, make_float2(fminf(rp.x, rq.x), fminf(rp.y, rq.y)));
  ca = fabsf(dd.x) > t.x;
  cb = fabsf(dd.y) > t.y;
}

// Cross product a x b of two pairs of vectors.
__device__ __forceinline__ void cross2(float2 ax, float2 ay, float2 az, float2 bx, float2 by, float2 bz, float2& cx,
                                       float2& cy, float2& cz) {
  cx = fma2(ay, bz, mul2(neg2(az), by));
  cy = fma2(az, bx, mul2(neg2(ax), bz));
  cz = fma2(ax, by, mul2(neg2(ay), bx));
}

// Weight of a triangle at one of its vertices (Sec. 2, normal estimation):
// 1 / (|a| + |b|) for the vertex's two spokes a, b along the triangle's
// edges, times the triangle's existence (exactly 0 or 1).  Points out of
// range have zero coordinates, so every spoke is finite and a missing
// triangle's term is an exact zero.
__device__ __forceinline__ float2 weight2(float2 la, float2 lb, float2 ex) {
  const float2 l = add2(la, lb);
  return mul2(make_float2(rcp_approx(l.x), rcp_approx(l.y)), ex);
}

// Homogeneity predicate of Algorithm 1 for two vertex pairs.  A vertex
// without a normal carries NaN components, which fail either comparison.
template <bool ANGLE>
__device__ __forceinline__ void homog2(float2 ux, float2 uy, float2 uz, float2 vx, float2 vy, float2 vz, float cos_t,
                                       float cx, float cy, float cz, bool& ha, bool& hb) {
  if (ANGLE) {
    const float2 dt = fma2(ux, vx, fma2(uy, vy, mul2(uz, vz)));
    ha = dt.x > cos_t;
    hb = dt.y > cos_t;
  } else {
    const float2 ex = sub2(ux, vx), ey = sub2(uy, vy), ez = sub2(uz, vz);
    ha = (fabsf(ex.x) < cx) & (fabsf(ey.x) < cy) & (fabsf(ez.x) < cz);
    hb = (fabsf(ex.y) < cx) & (fabsf(ey.y) < cy) & (fabsf(ez.y) < cz);
  }
}

__device__ __forceinline__ float2 left_of(float2 v) {
  return make_float2(__shfl_up_sync(FULL, v.y, 1), v.x);
}
__device__ __forceinline__ float2 right_of(float2 v) {
  return make_float2(v.y, __shfl_down_sync(FULL, v.x, 1));
}

// ---------------------------------------------------------------------------
// k_tile: decode + mesh + normals + edge mask + tile components
// ---------------------------------------------------------------------------
// The sweep of one tile.  Warp w owns tile columns w*60-2 .. w*60+61, two
// per lane (lane l: columns w*60+2l-2 and w*60+2l-1); lanes 1..30 hold its
// 60 output columns, lanes 0 and 31 the halo.  Each lane streams its two
// columns' rows into its own shared-memory ring slots with cp.async, RING-1
// rows ahead of use (coalesced 16-byte copies; a lane reads only slots it
// filled, so no barrier).  At step hr it holds scan row k = r0-1+hr and
// completes: the R edges of row k and the D and G edges of row k-1; the
// normals of row k-1 (Sec. 2, normal estimation), whose three terms
// through row k-2 were summed one step earlier; the three terms of row k's
// normals through row k-1; and the homogeneity mask and outputs of row k-2
// (Algorithm 1 predicate).
//
// Spokes of a vertex p in the paper's order: A (down), B (down-right),
// C (right), D (up), E (up-left), F (left).  With d, g, r the D, G and R
// edge vectors leaving a vertex and gl, f the G and R edges arriving at it,
// the six terms are  A x B = d x g,  B x C = g x r,  F x A = d x f  (below p)
// and  C x D = d' x r,  D x E = d' x gl',  E x F = gl' x f  (above p, with
// d', gl' the edges from the row above): reversed spokes are folded into the
// operand order.  A triangle (p, q, q') counts when its three edges exist.
template <int TR, int NW, bool ANGLE, bool XYZR>
__device__ __forceinline__ void tile_sweep(const ScanDesc* __restrict__ d, const Loc& L, unsigned char* smem) {
  using G = Geo<TR, NW>;
  constexpr int TC = G::TC;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float4* ring = reinterpret_cast<float4*>(smem + G::off_ring) + (size_t)w * (RING * 64) + lane;
  const long long* rows_s = reinterpret_cast<const long long*>(smem + G::off_rows);
  const float2* trig_s = reinterpret_cast<const float2*>(smem + G::off_trig);
  uint8_t* tb = smem + G::off_tb;
  const float4* __restrict__ xyzr = d->xyzr;
  const float* __restrict__ range = d->range;
  const float rmin = d->r_min, rmax = d->r_max;
  // loop-invariant descriptor fields, read once
  const float jump_h = d->jump_h, jump_v = d->jump_v, nsign = d->nsign;
  const float cos_t = ANGLE ? d->cos_t : 0.f, ccx = ANGLE ? 0.f : d->comp_x, ccy = ANGLE ? 0.f : d->comp_y,
              ccz = ANGLE ? 0.f : d->comp_z;

  const int lcA = w * SO + 2 * lane - 2;  // tile column of the lane's first point
  int jA = L.c0 + lcA, jB = jA + 1;       // scan columns
  if (L.wrap) {
    jA = wrap_col(jA, L.Ws);
    jB = wrap_col(jB, L.Ws);
  }
  const bool okA = jA >= 0 && jA < L.Ws, okB = jB >= 0 && jB < L.Ws;
  const unsigned offA = (unsigned)(okA ? jA : 0) * (unsigned)L.s, offB = (unsigned)(okB ? jB : 0) * (unsigned)L.s;
  float spA = 0.f, cpA = 1.f, spB = 0.f, cpB = 1.f;
  if (!XYZR) {
    if (okA) sincosf(fmaf((float)(jA * L.s), d->daz, d->az0), &spA, &cpA);
    if (okB) sincosf(fmaf((float)(jB * L.s), d->daz, d->az0), &spB, &cpB);
  }
  const bool strip = lane >= 1 && lane <= SO / 2;  // holds two of the strip's columns
  const bool outA = strip && lcA < L.cn;            // first column is an output
  const bool outB = strip && lcA + 1 < L.cn;        // second column is an output
  const int nsteps = L.rn + 3;  // rows r0-1 .. r0+rn+1
  unsigned vout = (unsigned)L.r0 * (unsigned)L.Ws + (unsigned)(L.c0 + lcA);  // output vertex, tile row 0
  // the output arrays' bases in registers (read through d every row, they
  // would be reloaded after each store, which might alias the descriptor)
  uint8_t* const mb_out = d->mb;
  float* const nrm_out = d->nrm;

  auto fetch = [&](int q, int k) {
    const long long ro = rows_s[k];
    float4* sl = ring + (q & (RING - 1)) * 64;
    fetch_point(sl, XYZR ? xyzr : nullptr, range, ro, okA, offA);
    fetch_point(sl + 32, XYZR ? xyzr : nullptr, range, ro, okB, offB);
  };
#pragma unroll
  for (int q = 0; q < RING - 1; ++q) {
    if (q < nsteps) fetch(q, q);
    cp_async_commit();
  }

  const float2 Z2 = make_float2(0.f, 0.f);
  const float QNAN = __int_as_float(0x7fc00000);
  float2 ppx = Z2, ppy = Z2, ppz = Z2, ppr = Z2;  // row k-1 (zeroed out of range)
  float2 rx1 = Z2, ry1 = Z2, rz1 = Z2, lr1 = Z2;                        // R edges of row k-1
  float2 er1 = Z2;                                                      // their existence (0 / 1)
  float2 ux = Z2, uy = Z2, uz = Z2;                // row k-1's normal sums: the terms above it
  float2 nx2 = make_float2(QNAN, QNAN), ny2 = nx2, nz2 = nx2;  // normals of row k-2 (NaN: none)
  uint32_t m2 = 0;   // mesh bytes of row k-2 (first | second << 8)
  uint32_t win = 0;  // mesh bytes: row k-1 in bits 0-15, row k in bits 16-31

  for (int hr = 0; hr < nsteps; ++hr) {
    // row hr has landed once at most RING-2 newer groups are pending
    cp_async_wait<RING - 2>();
    const int slot = hr & (RING - 1);
    float4 PA = ring[slot * 64], PB = ring[slot * 64 + 32];
    if (!XYZR) {  // range-only input: x,y,z from the ring's elevation and the column's azimuth
      const float2 te = trig_s[hr];
      const float rcA = PA.w * te.y, rcB = PB.w * te.y;
      PA = make_float4(rcA * cpA, rcA * spA, PA.w * te.x, PA.w);
      PB = make_float4(rcB * cpB, rcB * spB, PB.w * te.x, PB.w);
    }
    // refill the slot read one step ago with row hr+RING-1
    fetch(hr + RING - 1, hr + RING - 1);  // past the sweep: an absent row, nothing read
    cp_async_commit();

    const bool vA = in_range(PA.w, rmin, rmax), vB = in_range(PB.w, rmin, rmax);
    const float2 px = make_float2(vA ? PA.x : 0.f, vB ? PB.x : 0.f);
    const float2 py = make_float2(vA ? PA.y : 0.f, vB ? PB.y : 0.f);
    const float2 pz = make_float2(vA ? PA.z : 0.f, vB ? PB.z : 0.f);
    const float2 pr = make_float2(PA.w, PB.w);
    // right neighbours: the lane's second point and the next lane's first
    const float2 qx = right_of(px), qy = right_of(py), qz = right_of(pz), qr = right_of(pr);
    const bool vN = in_range(qr.y, rmin, rmax);
    // R edges of row k
    const float2 ex = sub2(qx, px), ey = sub2(qy, py), ez = sub2(qz, pz);
    const float2 le = len2(ex, ey, ez);
    const float2 jh = make_float2(jump_h, jump_h), jv = make_float2(jump_v, jump_v);
    bool cA, cB;
    jump_cut2(pr, qr, jh, cA, cB);
    const bool RA = vA && vB && !cA, RB = vB && vN && !cB;
    // D and G edges of row k-1
    const bool vpA = win & B_VALID, vpB = (win >> 8) & B_VALID;
    const float2 dx = sub2(px, ppx), dy = sub2(py, ppy), dz = sub2(pz, ppz);
    const float2 gx = sub2(qx, ppx), gy = sub2(qy, ppy), gz = sub2(qz, ppz);
    const float2 ld = len2(dx, dy, dz), lg = len2(gx, gy, gz);
    bool dA, dB, gA, gB;
    jump_cut2(ppr, pr, jv, dA, dB);
    jump_cut2(ppr, qr, jv, gA, gB);
    const bool DA = vpA && vA && !dA, DB = vpB && vB && !dB;
    const bool GA = vpA && vB && !gA, GB = vpB && vN && !gB;
    win |= ((DA ? B_D : 0u) | (GA ? B_G : 0u)) | (((DB ? B_D : 0u) | (GB ? B_G : 0u)) << 8) |
           ((((RA ? B_R : 0u) | (vA ? B_VALID : 0u)) | (((RB ? B_R : 0u) | (vB ? B_VALID : 0u)) << 8)) << 16);
    // triangle existence as exact 0 / 1 products: the lower (d, g, r) and
    // upper (g, r above, d to the right) triangles of each column's quad
    // between rows k-1 and k
    const float2 eD = make_float2(DA ? 1.f : 0.f, DB ? 1.f : 0.f);
    const float2 eG = make_float2(GA ? 1.f : 0.f, GB ? 1.f : 0.f);
    const float2 eR = make_float2(RA ? 1.f : 0.f, RB ? 1.f : 0.f);
    const float2 tLo = mul2(mul2(eD, eG), eR);
    const float2 tUp = mul2(mul2(eG, er1), right_of(eD));
    // Each triangle's cross product once, shared by its three vertices (the
    // spokes' cross products of the paper's six terms are the same vector
    // for every corner of a triangle): lower (p, q, q') = (k-1 c, k c,
    // k c+1): d x r; upper (p, q', p') = (k-1 c, k c+1, k-1 c+1): d' x r1,
    // with d' the D edge of the column to the right.  The two edges at the
    // right angle are the shortest, so the product's rounding error is no
    // larger than that of any corner's own two spokes.
    const float2 drx = right_of(dx), dry = right_of(dy), drz = right_of(dz), ldr = right_of(ld);
    float2 lox, loy, loz, upx, upy, upz;
    cross2(dx, dy, dz, ex, ey, ez, lox, loy, loz);
    cross2(drx, dry, drz, rx1, ry1, rz1, upx, upy, upz);
    // the weights at each corner: 1 / (sum of the corner's two spokes)
    const float2 wLp = weight2(ld, lg, tLo), wLq = weight2(ld, le, tLo), wLr = weight2(lg, le, tLo);
    const float2 wUp = weight2(lg, lr1, tUp), wUr = weight2(lr1, ldr, tUp), wUq = weight2(ldr, lg, tUp);

    // normals of row k-1: its own quads' lower and upper triangles, and the
    // upper triangle of the quad to its left (corner p', one lane over)
    float2 sx = fma2(wLp, lox, fma2(wUp, upx, ux));
    float2 sy = fma2(wLp, loy, fma2(wUp, upy, uy));
    float2 sz = fma2(wLp, loz, fma2(wUp, upz, uz));
    sx = add2(sx, left_of(mul2(wUr, upx)));
    sy = add2(sy, left_of(mul2(wUr, upy)));
    sz = add2(sz, left_of(mul2(wUr, upz)));
    const float2 q2 = fma2(sx, sx, fma2(sy, sy, mul2(sz, sz)));
    // a sum shorter than 2^-63 counts as no normal (as does a zero sum, which
    // is what a vertex out of range has: none of its triangles exists)
    const bool hA = q2.x >= FLT_MIN && q2.x < 3.0e38f;
    const bool hB = q2.y >= FLT_MIN && q2.y < 3.0e38f;
    const float2 fn = make_float2(hA ? nsign * rsq_approx(q2.x) : QNAN, hB ? nsign * rsq_approx(q2.y) : QNAN);
    const float2 nx1 = mul2(sx, fn), ny1 = mul2(sy, fn), nz1 = mul2(sz, fn);
    const uint32_t m1 = (win & 0xffffu) | (hA ? (uint32_t)B_HASN : 0u) | (hB ? (uint32_t)B_HASN << 8 : 0u);

    // normals of row k, the terms through row k-1: its own quads' lower
    // triangles (corner q), and the lower and upper triangles of the quad to
    // its left (corner q', one lane over)
    ux = fma2(wLq, lox, left_of(fma2(wLr, lox, mul2(wUq, upx))));
    uy = fma2(wLq, loy, left_of(fma2(wLr, loy, mul2(wUq, upy))));
    uz = fma2(wLq, loz, left_of(fma2(wLr, loz, mul2(wUq, upz))));

    // homogeneity mask and outputs of row k-2
    if (hr >= 3) {
      const float2 nRx = right_of(nx2), nRy = right_of(ny2), nRz = right_of(nz2);
      const float2 nGx = right_of(nx1), nGy = right_of(ny1), nGz = right_of(nz1);
      bool hRA, hRB, hDA, hDB, hGA, hGB;
      homog2<ANGLE>(nx2, ny2, nz2, nRx, nRy, nRz, cos_t, ccx, ccy, ccz, hRA, hRB);
      homog2<ANGLE>(nx2, ny2, nz2, nx1, ny1, nz1, cos_t, ccx, ccy, ccz, hDA, hDB);
      homog2<ANGLE>(nx2, ny2, nz2, nGx, nGy, nGz, cos_t, ccx, ccy, ccz, hGA, hGB);
      // an edge bit (R, D, G: bits 0-2 of each byte) moves up three places to
      // its homogeneous bit (HR, HD, HG) where the predicate holds
      const uint32_t hm = (hRA ? 1u : 0u) | (hDA ? 2u : 0u) | (hGA ? 4u : 0u) | (hRB ? 0x100u : 0u) |
                          (hDB ? 0x200u : 0u) | (hGB ? 0x400u : 0u);
      const uint32_t m2h = m2 | ((m2 & hm) << 3);
      const uint32_t m2A = m2 & 0xffu, m2B = m2 >> 8;
      const uint32_t bA = m2h & 0xffu, bB = m2h >> 8;
      const int lr = hr - 3;  // < L.rn: the sweep ends at row r0 + rn + 1
      {
        if (strip)
          *reinterpret_cast<uint16_t*>(tb + lr * TC + lcA) =
              (uint16_t)((outA ? bA : 0u) | (outB ? bB << 8 : 0u));
        if (outA) {
          const bool hasA = m2A & B_HASN, hasB = m2B & B_HASN;
          const float oxA = hasA ? nx2.x : 0.f, oyA = hasA ? ny2.x : 0.f, ozA = hasA ? nz2.x : 0.f;
          const float oxB = hasB ? nx2.y : 0.f, oyB = hasB ? ny2.y : 0.f, ozB = hasB ? nz2.y : 0.f;
          uint8_t* mp = mb_out + vout;
          float* np = nrm_out + 3 * (size_t)vout;
          if (outB && ((reinterpret_cast<uintptr_t>(mp) & 1) == 0)) {
            *reinterpret_cast<uint16_t*>(mp) = (uint16_t)(bA | (bB << 8));
          } else {
            mp[0] = (uint8_t)bA;
            if (outB) mp[1] = (uint8_t)bB;
          }
          if (outB && ((reinterpret_cast<uintptr_t>(np) & 7) == 0)) {
            float2* np2 = reinterpret_cast<float2*>(np);
            np2[0] = make_float2(oxA, oyA);
            np2[1] = make_float2(ozA, oxB);
            np2[2] = make_float2(oyB, ozB);
          } else {
            np[0] = oxA;
            np[1] = oyA;
            np[2] = ozA;
            if (outB) {
              np[3] = oxB;
              np[4] = oyB;
              np[5] = ozB;
            }
          }
        }
      }
      vout += (unsigned)L.Ws;
    }

    // rotate the window
    win >>= 16;
    m2 = m1;
    ppx = px;
    ppy = py;
    ppz = pz;
    ppr = pr;
    rx1 = ex;
    ry1 = ey;
    rz1 = ez;
    lr1 = le;
    er1 = eR;
    nx2 = nx1;
    ny2 = ny1;
    nz2 = nz1;
  }
  cp_async_wait_all();
}

// ---------------------------------------------------------------------------
// tile components (Algorithm 1 restricted to the tile)
// ---------------------------------------------------------------------------
// Runs of a strip row.  Lanes 1..30 hold the strip's columns in pairs
// (strip position 2*lane: the first, 2*lane+1: the second); linkA / linkB
// are the homogeneous R edges first -> second and second -> next lane's
// first.  Gives the strip positions of the first vertex of the runs that
// hold the lane's two columns.
__device__ __forceinline__ void run_starts(bool linkA, bool linkB, int lane, int& posA, int& posB) {
  const unsigned LA = __ballot_sync(FULL, linkA), LB = __ballot_sync(FULL, linkB);
  // lanes below this one that a run does not pass through (lane 0 never links)
  const unsigned brk = (~(LA & LB) & ((1u << lane) - 1u)) | 1u;
  const int m = 31 - __clz(brk);
  posA = ((LB >> m) & 1u) ? 2 * m + 1 : 2 * m + 2;
  posB = linkA ? posA : 2 * lane + 1;
}

template <int TR, int NW>
__device__ __forceinline__ void tile_cross_and_roots(const Loc& L, const uint8_t* __restrict__ tb, int* lp,
                                                     const uint32_t* q, uint16_t* __restrict__ lroot,
                                                     int32_t* __restrict__ parent, int32_t* err);

// Tile components of the tile bytes tb[TR][TC] (mesh + homogeneity bits of
// the tile's own vertices; zero outside the tile).  C1: each warp walks its
// strip row by row; the horizontal runs come from two ballots, and only a
// run's first vertex (plus the strip's and the tile's last column) enters
// the shared-memory union-find.  A vertical edge is joined unless the
// column to its left already joins the same two vertices (its D edge and
// the two R edges, or its D edge and the lower R edge for a G edge).  Then
// C2 / C3 (below).  Writes every vertex's tile-local root to lroot and marks
// each root in parent.
// Performs a warp's queued unions (pairs of tile-local indices), one per
// lane at a time, then empties the queue.
__device__ __forceinline__ void flush_unions(int* lp, const uint32_t* wq, int n, int limit, int32_t* err) {
  __syncwarp();
  for (int j = (int)(threadIdx.x & 31); j < n; j += 32) {
    const uint32_t pr = wq[j];
    union_sh(lp, (int)(pr & 0xffffu), (int)(pr >> 16), limit, err);
  }
  __syncwarp();
}

// Appends the pairs (a, b) of the lanes with f set to the warp's queue.
__device__ __forceinline__ void queue_union(uint32_t* wq, int& qn, bool f, int a, int b) {
  const unsigned m = __ballot_sync(FULL, f);
  if (f) wq[qn + __popc(m & ((1u << (threadIdx.x & 31)) - 1u))] = (uint32_t)a | ((uint32_t)b << 16);
  qn += __popc(m);
}

// Tile components of the tile bytes tb[TR][TC] (mesh + homogeneity bits of
// the tile's own vertices; zero outside the tile).  C1: each warp walks its
// strip row by row; the horizontal runs come from two ballots, and only a
// run's first vertex (plus the strip's and the tile's last column) enters
// the shared-memory union-find.  A vertical edge is joined unless the
// column to its left already joins the same two vertices (its D edge and
// the two R edges, or its D edge and the lower R edge for a G edge; a G
// edge is also implied by the upper R edge and the column's own D edge:
// every D edge is joined, by a union or through the column to its left, so
// the implications form no cycle); the joins wait in a per-warp queue and
// run 32 at a time.  The rows' run starts are kept for C3.  Then C2 / C3
// (below).  Writes every vertex's tile-local root to lroot and marks each
// root in parent.
template <int TR, int NW>
__device__ __forceinline__ void tile_components(const Loc& L, const uint8_t* __restrict__ tb, int* lp, uint32_t* q,
                                                uint16_t* __restrict__ lroot, int32_t* __restrict__ parent,
                                                int32_t* err) {
  using G = Geo<TR, NW>;
  constexpr int TC = G::TC;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int lcA = w * SO + 2 * lane - 2;       // tile column of the lane's first column
  const int base = w * SO - 2;                 // tile column of strip position 0
  const bool act = lane >= 1 && lane <= SO / 2;
  const bool lead = lane == 0 && w > 0;        // reads the previous strip's last column
  uint32_t* wq = q + w * QCAP;
  uint16_t* rs = reinterpret_cast<uint16_t*>(q + NW * QCAP) + w * TR * 32;  // this strip's run starts
  int qn = 0;                                  // queued unions (warp-uniform)
  uint32_t prev = 0;                           // previous row's bytes of the lane's columns
  int psA = 0, psB = 0;                        // previous row's run starts (tile-linear)
#pragma unroll 2  // consecutive rows' independent work overlaps
  for (int lr = 0; lr < L.rn; ++lr) {
    uint32_t cur = 0;
    if (act) cur = *reinterpret_cast<const uint16_t*>(tb + lr * TC + lcA);
    else if (lead) cur = (uint32_t)tb[lr * TC + lcA + 1] << 8;
    const uint32_t bA = cur & 0xffu, bB = cur >> 8;
    const bool linkA = act && (bA & B_HR) && lcA + 1 < L.cn;
    const bool linkB = act && lane < SO / 2 && (bB & B_HR) && lcA + 2 < L.cn;
    int posA, posB;
    run_starts(linkA, linkB, lane, posA, posB);
    rs[lr * 32 + lane] = (uint16_t)(posA | (posB << 8));
    const int vA = lr * TC + lcA;
    const int sA = lr * TC + base + posA, sB = lr * TC + base + posB;
    if (act) {
      if (posA == 2 * lane || lcA == L.cn - 1) lp[vA] = sA;
      if (posB == 2 * lane + 1 || lane == SO / 2 || lcA + 1 == L.cn - 1) lp[vA + 1] = sB;
    }
    const uint32_t up = __shfl_up_sync(FULL, cur | (prev << 16), 1);
    const int upsB = __shfl_up_sync(FULL, psB, 1);
    // both columns at once, byte 0 the first and byte 1 the second: P the
    // column's previous row, Lp and Lc its left neighbour's previous and this
    // row (the first column's left: the previous lane's second column, or
    // the previous strip's last column for lane 1, whose G edge is a C2
    // edge; the second column's left: the first).  Shifted right by 3, 4 or
    // 5 places, a byte's HR, HD or HG bit lands in the byte's bit 0.
    const uint32_t P = prev;
    const uint32_t Lp = (up >> 24) | ((prev & 0xffu) << 8), Lc = ((up >> 8) & 0xffu) | ((cur & 0xffu) << 8);
    const uint32_t gate = (act && lr > 0) ? 0x0101u : 0u;
    const uint32_t fD = (P >> 4) & ~((Lp >> 4) & (Lp >> 3) & (Lc >> 3)) & gate;
    const uint32_t fG = (Lp >> 5) & ~(((Lp >> 4) & (Lc >> 3)) | ((Lp >> 3) & (P >> 4))) & gate &
                        (lane > 1 ? 0x0101u : 0x0100u);
    const bool fDA = fD & 1u, fGA = fG & 1u, fDB = (fD >> 8) & 1u, fGB = (fG >> 8) & 1u;
    queue_union(wq, qn, fDA, sA, psA);
    queue_union(wq, qn, fGA, sA, upsB);
    queue_union(wq, qn, fDB, sB, psB);
    queue_union(wq, qn, fGB, sB, psA);
    if (qn > QCAP - 4 * 32) {
      flush_unions(lp, wq, qn, G::NV + 1, err);
      qn = 0;
    }
    prev = cur;
    psA = sA;
    psB = sB;
  }
  flush_unions(lp, wq, qn, G::NV + 1, err);
  __syncthreads();
  tile_cross_and_roots<TR, NW>(L, tb, lp, q, lroot, parent, err);
}

// C2: edges across strip borders, and the seam of a tile spanning the ring
// (from a strip's or the tile's last column, both kept in the union-find, to
// a strip's first column or column 0, both run starts); C3: every vertex's
// tile-local root (vertices out of range: NO_ROOT) from its run's first
// vertex, roots marked in the global union-find.
template <int TR, int NW>
__device__ __forceinline__ void tile_cross_and_roots(const Loc& L, const uint8_t* __restrict__ tb, int* lp,
                                                     const uint32_t* q, uint16_t* __restrict__ lroot,
                                                     int32_t* __restrict__ parent, int32_t* err) {
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
    if (bits & B_HR) union_sh(lp, lr * TC + ac, lr * TC + bc, G::NV + 1, err);
    if ((bits & B_HG) && lr + 1 < L.rn) union_sh(lp, lr * TC + ac, (lr + 1) * TC + bc, G::NV + 1, err);
  }
  __syncthreads();

  // C3: each warp over its strip's rows
  const int lcA = w * SO + 2 * lane - 2;
  const bool act = lane >= 1 && lane <= SO / 2;
  const size_t pitch = root_pitch(L.Ws);
  const uint16_t* rs = reinterpret_cast<const uint16_t*>(q + NW * QCAP) + w * TR * 32;  // C1's run starts
#pragma unroll 2  // consecutive rows' independent work overlaps
  for (int lr = 0; lr < L.rn; ++lr) {
    const uint32_t cur = act ? *reinterpret_cast<const uint16_t*>(tb + lr * TC + lcA) : 0u;
    const uint32_t bA = cur & 0xffu, bB = cur >> 8;
    const uint32_t ps = rs[lr * 32 + lane];
    const int posA = (int)(ps & 0xffu), posB = (int)(ps >> 8);
    const int vA = lr * TC + lcA;
    int rA = 0, rB = 0;
    find_done2_sh(lp, act && posA == 2 * lane, vA, act && posB == 2 * lane + 1, vA + 1, G::NV + 1, rA, rB);
    const uint32_t pub = (uint32_t)rA | ((uint32_t)rB << 16);
    const uint32_t gA = __shfl_sync(FULL, pub, posA >> 1), gB = __shfl_sync(FULL, pub, posB >> 1);
    if (act && lcA < L.cn) {
      const uint32_t RA = (posA & 1) ? (gA >> 16) : (gA & 0xffffu);
      const uint32_t RB = (posB & 1) ? (gB >> 16) : (gB & 0xffffu);
      const bool valA = bA & B_VALID, valB = bB & B_VALID;
      const size_t gi = (size_t)(L.r0 + lr);
      *reinterpret_cast<uint32_t*>(lroot + gi * pitch + (L.c0 + lcA)) =
          (valA ? RA : (uint32_t)NO_ROOT) | ((valB ? RB : (uint32_t)NO_ROOT) << 16);
      const size_t gv = gi * L.Ws + (L.c0 + lcA);
      if (valA && RA == (uint32_t)vA) parent[gv] = (int32_t)gv;
      if (valB && RB == (uint32_t)(vA + 1)) parent[gv + 1] = (int32_t)(gv + 1);
    }
  }
}

// The row table of tile_body for a single scan launched without k_prep
// (KArgs::fuse_prep, H <= kFuseMaxRings): the tile finds the input rows of
// the sorted rings it reads (r0-1 .. r0+rn+1; elevations descending, ties by
// input row, as k_prep's rank count orders them).  Elevations that fall
// strictly along the input rows give the identity order, strictly rising
// ones its reverse; otherwise every ring's rank is counted, and a NaN
// elevation is flagged.  Tiles of the first tile column also store the ring
// order of their own rows (read by the back-fill at s > 1), and tile 0
// clears the segment count.  The elevations sit in the sweep's row slots,
// idle until the sweep starts.
template <int TR, int NW>
__device__ __forceinline__ void tile_rows_fused(const ScanDesc* d, const Loc& L, int lt, unsigned char* smem,
                                                int32_t* err) {
  using G = Geo<TR, NW>;
  static_assert(G::ring_bytes >= sizeof(float) * kFuseMaxRings, "elevations fit in the row slots");
  long long* rows_s = reinterpret_cast<long long*>(smem + G::off_rows);
  float2* trig_s = reinterpret_cast<float2*>(smem + G::off_trig);
  float* se = reinterpret_cast<float*>(smem + G::off_ring);
  const int H = L.H, nk = L.rn + 3;
  bool desc = true, asc = true;
  for (int k = threadIdx.x; k < H; k += G::NT) {
    const float e = __ldg(d->elev + k);
    se[k] = e;
    if (k + 1 < H) {
      const float f = __ldg(d->elev + k + 1);
      desc = desc && e > f;
      asc = asc && e < f;
    }
  }
  for (int k = threadIdx.x; k < nk + RING - 1; k += G::NT) {
    rows_s[k] = -1;  // absent unless a ring of the scan lands there
    if (k < nk) trig_s[k] = make_float2(0.f, 1.f);
  }
  desc = __syncthreads_and(desc);
  asc = __syncthreads_and(asc);
  auto place = [&](int q, int i) {  // input row q is sorted ring i
    const int k = i - (L.r0 - 1);
    if (k < 0 || k >= nk) return;
    rows_s[k] = (long long)q * L.W;
    if (!d->xyzr) {
      float sn, cs;
      sincosf(se[q], &sn, &cs);
      trig_s[k] = make_float2(sn, cs);
    }
    if (L.c0 == 0 && k >= 1 && k <= L.rn) d->order[i] = q;
  };
  if (desc || asc) {
    for (int k = threadIdx.x; k < nk; k += G::NT) {
      const int i = L.r0 - 1 + k;
      if (i >= 0 && i < H) place(desc ? i : H - 1 - i, i);
    }
  } else {
    for (int q = threadIdx.x; q < H; q += G::NT) {
      const float e = se[q];
      if (e != e) atomicOr(err, DERR_NAN_ELEV);
      int rank = 0;
      for (int m = 0; m < H; ++m) {
        const float em = se[m];
        rank += (em > e) || (em == e && m < q);
      }
      if (rank < H) place(q, rank);
    }
  }
  if (lt == 0 && threadIdx.x == 0) *d->nseg = 0;
}

// One tile of one scan: decode + mesh + normals + edge mask + tile
// components (smem: Geo<TR,NW>::bytes of dynamic shared memory).  FUSE: the
// ring order comes from tile_rows_fused instead of k_prep.
template <int TR, int NW, bool CO = false, bool FUSE = false>
__device__ __forceinline__ void tile_body(const ScanDesc* d, int lt, unsigned char* smem, int32_t* err) {
  using G = Geo<TR, NW>;
  const Loc L = make_loc(d, lt, TR, G::TC);
  // offsets of the input rows the tile reads (ring order applied once) and,
  // for range-only input, their elevations' sine and cosine
  long long* rows_s = reinterpret_cast<long long*>(smem + G::off_rows);
  float2* trig_s = reinterpret_cast<float2*>(smem + G::off_trig);
  if constexpr (FUSE) {
    tile_rows_fused<TR, NW>(d, L, lt, smem, err);
  } else {
    for (int k = threadIdx.x; k < L.rn + 3 + RING - 1; k += G::NT) {
      const int i = L.r0 - 1 + k;
      long long ro = -1;
      float2 te = make_float2(0.f, 1.f);
      if (i >= 0 && i < L.H && k < L.rn + 3) {
        const int row = ld_in<CO>(d->order + i);
        if ((unsigned)row < (unsigned)L.H) ro = (long long)row * L.W;
        if (!d->xyzr) te = ld_in<CO>(d->trig + i);
      }
      rows_s[k] = ro;
      if (k < L.rn + 3) trig_s[k] = te;  // trig_s has the sweep's rows only
    }
  }
  __syncthreads();
  const bool angle = d->pred == LSG_PRED_ANGLE;
  if (d->xyzr) {
    if (angle) tile_sweep<TR, NW, true, true>(d, L, smem);
    else tile_sweep<TR, NW, false, true>(d, L, smem);
  } else {
    if (angle) tile_sweep<TR, NW, true, false>(d, L, smem);
    else tile_sweep<TR, NW, false, false>(d, L, smem);
  }
  __syncthreads();
  tile_components<TR, NW>(L, smem + G::off_tb, reinterpret_cast<int*>(smem + G::off_lp),
                          reinterpret_cast<uint32_t*>(smem + G::off_q), d->lroot, d->parent, err);
}

// FUSE: a single scan launched without k_prep (KArgs::fuse_prep).
template <int TR, int NW, bool FUSE = false>
__global__ void __launch_bounds__(NW * 32, 16 / NW) k_tile(const __grid_constant__ KArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  dep_wait();
  dep_release();
  for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
    int lt;
    const ScanDesc* d = tile_desc(a, t, lt);
    tile_body<TR, NW, false, FUSE>(d, lt, smem, a.err);
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
  dep_wait();
  dep_release();
  int* lp = reinterpret_cast<int*>(smem);
  uint8_t* tb = smem + G::lp_bytes;
  uint32_t* q = reinterpret_cast<uint32_t*>(smem + G::lp_bytes + ((G::NV + 15) / 16) * 16);
  for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
    int lt;
    const ScanDesc* d = tile_desc(a, t, lt);
    const Loc L = make_loc(d, lt, TR, TC);
    for (int k = threadIdx.x; k < G::NV; k += G::NT) {
      const int lr = k / TC, lc = k - (k / TC) * TC;
      tb[k] = (lr < L.rn && lc < L.cn) ? d->mb[(size_t)(L.r0 + lr) * L.Ws + (L.c0 + lc)] : 0;
    }
    __syncthreads();
    tile_components<TR, NW>(L, tb, lp, q, d->lroot, d->parent, a.err);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// global roots
// ---------------------------------------------------------------------------
// Scan-local index of the tile-local root of vertex (i, j).
template <int TR, int TC, bool CO = false>
__device__ __forceinline__ int tile_root(const uint16_t* lroot, int Ws, int i, int j) {
  const int r = ld_in<CO>(lroot + (size_t)i * root_pitch(Ws) + j);
  const int rr = r / TC, rc = r - (r / TC) * TC;
  return ((i / TR) * TR + rr) * Ws + (j / TC) * TC + rc;
}

// ---------------------------------------------------------------------------
// k_merge: join components across tile borders and the 360 deg seam
// ---------------------------------------------------------------------------
// threads of k_merge: one per border vertex of a tile (the last row and the
// last column), rounded up to whole warps
template <int TR, int NW>
__host__ __device__ constexpr int nt_merge() {
  return ((NW * SO + TR - 1 + 31) / 32) * 32;
}

// Border unions of one tile (NTB threads, all of them calling).  Each lane
// takes one border vertex and forms the pairs of tile roots its outgoing
// homogeneous edges join, as (smaller, larger) scan-local indices.  Along a
// border most pairs repeat (a component crossing it joins the same two tile
// roots at every column), so each warp issues every distinct pair once.
template <int TR, int NW, int NTB, bool CO = false>
__device__ __forceinline__ void merge_body(const ScanDesc* d, int lt, int32_t* err) {
  static_assert(NTB % 32 == 0, "whole warps");
  constexpr int TC = NW * SO;
  constexpr uint64_t NONE = ~0ull;
  const Loc L = make_loc(d, lt, TR, TC);
  const uint8_t* mb = d->mb;
  const uint16_t* lroot = d->lroot;
  int32_t* parent = d->parent;
  const int limit = L.H * L.Ws + 1;
  const bool full_ring = L.wrap && L.c0 == 0 && L.cn == L.Ws;
  const size_t LP = root_pitch(L.Ws);
  const int lane = threadIdx.x & 31;
  __shared__ uint64_t pairs_s[NTB / 32][96];  // each warp's distinct pairs (three per lane at most)
  uint64_t* wk = pairs_s[threadIdx.x >> 5];
  // border vertices: the last row of the tile, then the last column above it
  const int nb = L.cn + L.rn - 1;
  for (int k0 = 0; k0 < nb; k0 += NTB) {  // trip count uniform over the block
    const int k = k0 + (int)threadIdx.x;
    uint64_t key[3] = {NONE, NONE, NONE};
    if (k < nb) {
      int lr, lc;
      if (k < L.cn) {
        lr = L.rn - 1;
        lc = k;
      } else {
        lr = k - L.cn;
        lc = L.cn - 1;
      }
      const int i = L.r0 + lr, j = L.c0 + lc;
      const uint8_t bits = ld_in<CO>(mb + (size_t)i * L.Ws + j);
      // bits pointing off the grid (possible in a caller-given mask) are ignored
      const bool has_right = (j + 1 < L.Ws) || L.wrap;
      const bool has_down = i + 1 < L.H;
      const int jn = (j + 1 == L.Ws) ? 0 : j + 1;
      const bool jn_in = (lc + 1 < L.cn) || full_ring;
      const bool down_in = lr + 1 < L.rn;
      const bool hr_out = (bits & B_HR) && has_right && !jn_in;
      const bool hd_out = (bits & B_HD) && has_down && !down_in;
      const bool hg_out = (bits & B_HG) && has_down && has_right && !(down_in && jn_in);
      if ((hr_out || hd_out || hg_out) && ld_in<CO>(lroot + (size_t)i * LP + j) != NO_ROOT) {
        const int rp = tile_root<TR, TC, CO>(lroot, L.Ws, i, j);
        auto pair = [rp](int rq) {
          const uint32_t lo = (uint32_t)min(rp, rq), hi = (uint32_t)max(rp, rq);
          return ((uint64_t)lo << 32) | hi;
        };
        if (hr_out && ld_in<CO>(lroot + (size_t)i * LP + jn) != NO_ROOT)
          key[0] = pair(tile_root<TR, TC, CO>(lroot, L.Ws, i, jn));
        if (hd_out && ld_in<CO>(lroot + (size_t)(i + 1) * LP + j) != NO_ROOT)
          key[1] = pair(tile_root<TR, TC, CO>(lroot, L.Ws, i + 1, j));
        if (hg_out && ld_in<CO>(lroot + (size_t)(i + 1) * LP + jn) != NO_ROOT)
          key[2] = pair(tile_root<TR, TC, CO>(lroot, L.Ws, i + 1, jn));
        if (key[1] == key[0]) key[1] = NONE;
        if (key[2] == key[0] || key[2] == key[1]) key[2] = NONE;
      }
    }
    // a diagonal pair often repeats the next lane's down pair (bottom row)
    // or right pair (right column): that lane's entry joins it
    const uint64_t nd = __shfl_down_sync(FULL, key[1], 1), nr = __shfl_down_sync(FULL, key[0], 1);
    if (lane < 31 && (key[2] == nd || key[2] == nr)) key[2] = NONE;
    // the first lane of each group of equal pairs lists its pair, then the
    // warp's list is deduplicated once more and joined one pair per lane
    // (the unions of different pairs run side by side, not one edge kind
    // after another)
    int nk = 0;
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      const unsigned same = __match_any_sync(FULL, key[e]);
      const bool lead = key[e] != NONE && lane == __ffs(same) - 1;
      const unsigned m = __ballot_sync(FULL, lead);
      if (lead) wk[nk + __popc(m & ((1u << lane) - 1u))] = key[e];
      nk += __popc(m);
    }
    __syncwarp();
    for (int k0 = 0; k0 < nk; k0 += 32) {
      const uint64_t kk = k0 + lane < nk ? wk[k0 + lane] : NONE;
      const unsigned same = __match_any_sync(FULL, kk);
      if (kk != NONE && lane == __ffs(same) - 1)
        union_g(parent, (int)(kk >> 32), (int)(kk & 0xffffffffu), limit, err);
    }
    __syncwarp();
  }
}

template <int TR, int NW>
__global__ void __launch_bounds__(nt_merge<TR, NW>()) k_merge(const __grid_constant__ KArgs a) {
  dep_wait();
  dep_release();
  for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
    int lt;
    const ScanDesc* d = tile_desc(a, t, lt);
    merge_body<TR, NW, nt_merge<TR, NW>()>(d, lt, a.err);
  }
}

// ---------------------------------------------------------------------------
// k_flatten: labels, back-fill, segment count
// ---------------------------------------------------------------------------
constexpr int NT_FLAT = 128;

// Root of a chain in the (now read-only) global union-find.
template <bool CO>
__device__ __forceinline__ int find_ro(const int32_t* P, int x, int limit) {
  int p = ld_in<CO>(P + x);
  while (p != x && limit-- > 0) {
    x = p;
    p = ld_in<CO>(P + x);
  }
  return x;
}

// Label of any vertex of the scan (used for the back-fill neighbour that lies
// in the next tile).
template <int TR, int TC, bool CO>
__device__ __forceinline__ int32_t vertex_label_global(const uint16_t* lroot, const int32_t* parent, int Ws, int W,
                                                       int s, int i, int j, int limit) {
  if (ld_in<CO>(lroot + (size_t)i * root_pitch(Ws) + j) == NO_ROOT) return -1;
  const int g = find_ro<CO>(parent, tile_root<TR, TC, CO>(lroot, Ws, i, j), limit);
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

// Per tile: (1) stage the tile's 16-bit local roots in shared memory four
// at a time and list the tile-local roots, (2) resolve every local root
// once to its global root and label (and count the global roots), (3) write
// every point's label, back-filling the points between sampled columns.
template <int TR, int NW>
struct FlatGeo {
  static constexpr int TC = NW * SO, NV = TR * TC;
  static constexpr int NQ = TC / 4;                                         // root quads per tile row
  static constexpr size_t off_lab = 0;                                      // int32 [NV] root labels
  static constexpr size_t off_lr = align16(sizeof(int32_t) * NV);          // uint16 [NV] tile roots
  static constexpr size_t off_list = off_lr + align16(sizeof(uint16_t) * NV);  // uint16 [NV] list of roots
  static constexpr size_t bytes = off_list + align16(sizeof(uint16_t) * NV);
  // launches whose scans all have s = 1 use the root labels alone
  static constexpr size_t s1_bytes = align16(sizeof(int32_t) * NV);
};

__device__ __forceinline__ int32_t root_label(const int32_t* lab_s, uint32_t r) {
  return r == NO_ROOT ? -1 : lab_s[r];
}

// Labels of one tile at s = 1, where every point is a mesh vertex: (1) each
// thread takes quads of the tile's local roots and resolves the global root
// of every entry that is a tile root itself (up to four union-find chains in
// flight), storing its label (the root's index) in lab_s; (2) after one
// barrier, each thread writes the labels of the same quads as 16-byte
// stores, every entry taking its tile root's label.
template <int TR, int NW, int NTB, bool CO>
__device__ __forceinline__ void flatten_s1(const ScanDesc* d, const Loc& L, int32_t* lab_s) {
  constexpr int TC = NW * SO;
  const int tid = threadIdx.x, lane = tid & 31;
  const int Ws = L.Ws;
  const uint16_t* lroot = d->lroot;
  const int32_t* parent = d->parent;
  int32_t* __restrict__ labels = d->labels;
  const int limit = L.H * Ws + 1;
  const size_t pitch = root_pitch(Ws);
  const int nq = (L.cn + 3) >> 2, nquad = L.rn * nq;  // quads holding at least one column of the tile
  auto quad_ptr = [&](int lr, int q) {
    return reinterpret_cast<const uint2*>(lroot + (size_t)(L.r0 + lr) * pitch + L.c0) + q;
  };
  int nroots = 0;
  // the quad's four union-find entries are loaded with its roots, so that a
  // root that no border join moved needs no second round trip (entries of
  // vertices that are not roots are read and dropped; a row's last quad
  // reads at most three entries past the scan's parent array, into the
  // scan's own tile-root array, which follows it in the workspace)
  const bool vec = (Ws & 3) == 0;  // the quads' entries are 16-byte aligned
  for (int k = tid; k < nquad; k += NTB) {
    const int lr = k / nq, q = k - lr * nq;
    const int g0 = (L.r0 + lr) * Ws + L.c0 + 4 * q;  // scan index of the quad's first vertex
    const uint2 r4 = ld_in<CO>(quad_ptr(lr, q));
    int p[4];
    if (vec) {
      const int4 p4 = ld_in<CO>(reinterpret_cast<const int4*>(parent + g0));
      p[0] = p4.x;
      p[1] = p4.y;
      p[2] = p4.z;
      p[3] = p4.w;
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j) p[j] = 4 * q + j < L.cn ? ld_in<CO>(parent + g0 + j) : g0 + j;
    }
    const int v0 = lr * TC + 4 * q;
    const uint32_t e[4] = {r4.x & 0xffffu, r4.x >> 16, r4.y & 0xffffu, r4.y >> 16};
    int x[4];
    bool root[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      // entries past the tile's last column belong to the next tile or the
      // row padding
      root[j] = e[j] == (uint32_t)(v0 + j) && 4 * q + j < L.cn;
      x[j] = root[j] ? p[j] : g0 + j;  // the first step of the chain, already loaded
    }
    // the chains of the roots that a border join moved
    bool walk[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) walk[j] = root[j] && x[j] != g0 + j;
    for (int it = 0; it < limit && (walk[0] || walk[1] || walk[2] || walk[3]); ++it) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if (!walk[j]) continue;
        const int pp = ld_in<CO>(parent + x[j]);
        if (pp != x[j]) x[j] = pp;
        else walk[j] = false;
      }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (!root[j]) continue;
      nroots += x[j] == g0 + j;
      lab_s[v0 + j] = x[j];  // s = 1: the point index is the vertex index
    }
  }
  const int cnt = __reduce_add_sync(FULL, nroots);
  if (lane == 0 && cnt) atomicAdd(d->nseg, cnt);
  __syncthreads();
  for (int k = tid; k < nquad; k += NTB) {
    const int lr = k / nq, q = k - lr * nq;
    const uint2 r4 = ld_in<CO>(quad_ptr(lr, q));
    const int lc = 4 * q;
    // entries past the tile's last column (the next tile's, or the row
    // padding, which nothing writes) are never used as indices
    const int lim = L.cn - lc;
    const uint32_t e0 = r4.x & 0xffffu, e1 = lim > 1 ? (r4.x >> 16) : (uint32_t)NO_ROOT;
    const uint32_t e2 = lim > 2 ? (r4.y & 0xffffu) : (uint32_t)NO_ROOT;
    const uint32_t e3 = lim > 3 ? (r4.y >> 16) : (uint32_t)NO_ROOT;
    const int4 o = make_int4(root_label(lab_s, e0), root_label(lab_s, e1), root_label(lab_s, e2),
                             root_label(lab_s, e3));
    int32_t* dst = labels + (size_t)(L.r0 + lr) * L.W + L.c0 + lc;
    if (lc + 4 <= L.cn && (reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
      *reinterpret_cast<int4*>(dst) = o;
    } else {
      dst[0] = o.x;
      if (lc + 1 < L.cn) dst[1] = o.y;
      if (lc + 2 < L.cn) dst[2] = o.z;
      if (lc + 3 < L.cn) dst[3] = o.w;
    }
  }
}

// Labels of one tile (NTB threads; fsm: FlatGeo<TR,NW>::bytes of dynamic
// shared memory; nlist: a shared counter).
template <int TR, int NW, int NTB, bool CO = false>
__device__ __forceinline__ void flatten_body(const ScanDesc* d, int lt, unsigned char* fsm, int& nlist,
                                             bool s1_smem = false, int32_t* err = nullptr) {
  using FG = FlatGeo<TR, NW>;
  constexpr int TC = FG::TC, NQ = FG::NQ, NWF = NTB / 32;
  static_assert(TC % 4 == 0, "tile rows are read as quads of roots");
  uint16_t* lr_s = reinterpret_cast<uint16_t*>(fsm + FG::off_lr);
  int32_t* lab_s = reinterpret_cast<int32_t*>(fsm + FG::off_lab);
  uint16_t* list_s = reinterpret_cast<uint16_t*>(fsm + FG::off_list);
  const int tid = threadIdx.x, lane = tid & 31, wf = tid >> 5;
  const Loc L = make_loc(d, lt, TR, TC);
  if (L.s == 1) {
    flatten_s1<TR, NW, NTB, CO>(d, L, lab_s);
    return;
  }
  if (s1_smem) {  // launched with the s = 1 shared memory only: refuse the scan
    if (threadIdx.x == 0 && err) atomicOr(err, DERR_LAUNCH);
    return;
  }
  const int W = L.W, Ws = L.Ws, s = L.s;
  const uint16_t* lroot = d->lroot;
  const int32_t* parent = d->parent;
  int32_t* __restrict__ labels = d->labels;
  const int limit = L.H * Ws + 1;
  if (tid == 0) nlist = 0;
  __syncthreads();
  // (1) the tile's roots, four at a time (rows are 8-byte aligned: the pitch
  //     is a multiple of 8 and TC a multiple of 4); the roots among them are
  //     appended to the list (one atomic per warp and pass)
  const int nquad = L.rn * NQ, nq = (L.cn + 3) >> 2;
  for (int k0 = 0; k0 < nquad; k0 += NTB) {
    const int k = k0 + tid;
    const int lr = k / NQ, q = k - (k / NQ) * NQ;
    const int v0 = lr * TC + 4 * q;
    uint32_t m = 0;  // which of the four are roots
    if (k < nquad) {
      uint2 r4 = make_uint2(0xFFFFFFFFu, 0xFFFFFFFFu);
      if (q < nq) r4 = ld_in<CO>(reinterpret_cast<const uint2*>(lroot + (size_t)(L.r0 + lr) * root_pitch(Ws) + L.c0) + q);
      // entries past the tile's last column (the next tile's, or the row
      // padding, which nothing writes) are staged as NO_ROOT
      const int lim = L.cn - 4 * q;  // columns of the quad inside the tile
      if (lim < 4) {
        if (lim <= 0) {
          r4 = make_uint2(0xFFFFFFFFu, 0xFFFFFFFFu);
        } else if (lim == 1) {
          r4.x |= 0xFFFF0000u;
          r4.y = 0xFFFFFFFFu;
        } else if (lim == 2) {
          r4.y = 0xFFFFFFFFu;
        } else {
          r4.y |= 0xFFFF0000u;
        }
      }
      *reinterpret_cast<uint2*>(lr_s + v0) = r4;
      m = ((r4.x & 0xffffu) == (uint32_t)v0) | (((r4.x >> 16) == (uint32_t)(v0 + 1)) << 1) |
          (((r4.y & 0xffffu) == (uint32_t)(v0 + 2)) << 2) | (((r4.y >> 16) == (uint32_t)(v0 + 3)) << 3);
    }
    const int c = __popc(m);
    int incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(FULL, incl, o);
      if (lane >= o) incl += t;
    }
    int base = 0;
    if (lane == 31 && incl) base = atomicAdd(&nlist, incl);
    base = __shfl_sync(FULL, base, 31);
    int pos = base + incl - c;
    while (m) {
      const int j = __ffs(m) - 1;
      list_s[pos++] = (uint16_t)(v0 + j);
      m &= m - 1;
    }
  }
  __syncthreads();
  // (2) resolve each listed root to its global root, four chains per thread
  //     at a time (independent loads in flight)
  int nroots = 0;
  const int nl = nlist;
  auto scan_index = [&](int v) { return (L.r0 + v / TC) * Ws + L.c0 + v % TC; };
  for (int k0 = tid; k0 < nl; k0 += 4 * NTB) {
    int x[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int k = k0 + q * NTB;
      x[q] = scan_index(k < nl ? list_s[k] : 0);
    }
    for (int it = 0; it < limit; ++it) {
      bool more = false;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (k0 + q * NTB >= nl) continue;
        const int p = ld_in<CO>(parent + x[q]);
        if (p != x[q]) {
          x[q] = p;
          more = true;
        }
      }
      if (!more) break;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int k = k0 + q * NTB;
      if (k >= nl) continue;
      const int v = list_s[k], g = x[q];
      nroots += (g == scan_index(v));
      int lab = g;  // s = 1: W = Ws, so the point index is the vertex index
      if (s != 1) {
        const int gi = g / Ws, gj = g - gi * Ws;
        lab = gi * W + gj * s;
      }
      lab_s[v] = lab;
    }
  }
  const int cnt = __reduce_add_sync(FULL, nroots);
  if (lane == 0 && cnt) atomicAdd(d->nseg, cnt);
  __syncthreads();
  // (3) labels
  if (s == 1) {
    for (int k = tid; k < nquad; k += NTB) {
      const int lr = k / NQ, q = k - (k / NQ) * NQ;
      const int lc = 4 * q;
      if (lc >= L.cn) continue;
      const uint2 r4 = *reinterpret_cast<const uint2*>(lr_s + lr * TC + lc);
      const int4 o = make_int4(root_label(lab_s, r4.x & 0xffffu), root_label(lab_s, r4.x >> 16),
                               root_label(lab_s, r4.y & 0xffffu), root_label(lab_s, r4.y >> 16));
      int32_t* dst = labels + (size_t)(L.r0 + lr) * W + L.c0 + lc;
      if (lc + 4 <= L.cn && (reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
        *reinterpret_cast<int4*>(dst) = o;
      } else {
        dst[0] = o.x;
        if (lc + 1 < L.cn) dst[1] = o.y;
        if (lc + 2 < L.cn) dst[2] = o.z;
        if (lc + 3 < L.cn) dst[3] = o.w;
      }
    }
  } else {
    for (int lr = wf; lr < L.rn; lr += NWF) {
      const int i = L.r0 + lr;
      const int row = ld_in<CO>(d->order + i);
      for (int lc = lane; lc < L.cn; lc += 32) {
        const int j = L.c0 + lc;
        const int32_t lo = root_label(lab_s, lr_s[lr * TC + lc]);
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
            hi = root_label(lab_s, lr_s[lr * TC + (jh - L.c0)]);
          } else {
            hi = vertex_label_global<TR, TC, CO>(lroot, parent, Ws, W, s, i, jh, limit);
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

// CTAs of k_flatten per SM: as many as the shared memory of an s = 1 launch
// holds, at most twelve of 128 threads (the phases wait on loads, so resident
// tiles hide each other's latency; twelve leaves 40 registers a thread, and a
// CTA fits in what one tile-kernel CTA frees, so that the label work of one
// scan group interleaves with the tile work of the next).
template <int TR, int NW>
constexpr int flat_min_blocks() {
  constexpr int n = (int)((220u * 1024u) / FlatGeo<TR, NW>::s1_bytes);
  return n < 1 ? 1 : (n > 12 ? 12 : n);
}

template <int TR, int NW>
__global__ void __launch_bounds__(NT_FLAT, (flat_min_blocks<TR, NW>())) k_flatten(const __grid_constant__ KArgs a) {
  extern __shared__ __align__(16) unsigned char fsm[];
  __shared__ int nlist;
  dep_wait();
  for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
    int lt;
    const ScanDesc* d = tile_desc(a, t, lt);
    flatten_body<TR, NW, NT_FLAT>(d, lt, fsm, nlist, a.s1_only != 0, a.err);
    __syncthreads();
  }
}

// Labels of a launch whose scans all have s = 1: the register-resident pass
// alone, compiled without the general back-fill path, whose state made the
// shared kernel spill more at the same register budget.  A scan with s > 1
// is refused through the error word (its labels stay unwritten).
template <int TR, int NW>
__global__ void __launch_bounds__(NT_FLAT, (flat_min_blocks<TR, NW>())) k_flatten1(const __grid_constant__ KArgs a) {
  extern __shared__ __align__(16) unsigned char fsm[];
  dep_wait();
  for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
    int lt;
    const ScanDesc* d = tile_desc(a, t, lt);
    const Loc L = make_loc(d, lt, TR, NW * SO);
    if (L.s == 1)
      flatten_s1<TR, NW, NT_FLAT, false>(d, L, reinterpret_cast<int32_t*>(fsm + FlatGeo<TR, NW>::off_lab));
    else if (threadIdx.x == 0)
      atomicOr(a.err, DERR_LAUNCH);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// k_fused: the whole batched pass in one persistent launch
// ---------------------------------------------------------------------------
// Waits (one thread) until *cnt reaches need; gives up after about a second,
// recording a timeout in the error word instead of hanging.
__device__ __forceinline__ void wait_count(const int32_t* cnt, int need, int32_t* err,
                                           unsigned limit = 1u << 23) {
  for (unsigned it = 0;; ++it) {
    if (*reinterpret_cast<const volatile int32_t*>(cnt) >= need) break;
    if (it > limit) {
      atomicOr(err, DERR_TIMEOUT);
      break;
    }
    __nanosleep(128);
  }
  __threadfence();
}

// Self-test of the bounded wait: one thread waits for a counter that nothing
// increments, gives up after `limit` polls and flags the timeout.
__global__ void k_wait_probe(const int32_t* cnt, int32_t* err, unsigned limit) {
  if (threadIdx.x == 0 && blockIdx.x == 0) wait_count(cnt, 1, err, limit);
}

template <int TR, int NW>
struct FusedGeo {
  static constexpr size_t a = Geo<TR, NW>::bytes, b = FlatGeo<TR, NW>::bytes, c = sizeof(float) * LSG_MAX_RINGS;
  static constexpr size_t b1 = FlatGeo<TR, NW>::s1_bytes;
  static constexpr size_t ab = a > b ? a : b, ab1 = a > b1 ? a : b1;
  static constexpr size_t bytes = ab > c ? ab : c;
  // plans whose scans all have s = 1: the labels items need the root labels only
  static constexpr size_t s1_bytes = ab1 > c ? ab1 : c;
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
    else if (ph == PH_TILE) tile_body<TR, NW, true>(d, lt, smem, f.err);
    else if (ph == PH_MERGE) merge_body<TR, NW, NTB, true>(d, lt, f.err);
    else flatten_body<TR, NW, NTB, true>(d, lt, smem, nlist, f.s1_only != 0, f.err);
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
  e = cudaFuncSetAttribute(k_tile<TR, NW, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Geo<TR, NW>::bytes);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_flatten<TR, NW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)FlatGeo<TR, NW>::bytes);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_flatten1<TR, NW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)FlatGeo<TR, NW>::s1_bytes);
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
  if ((e = set_attrs<32, 2>()) != cudaSuccess) return e;
  if ((e = set_attrs<32, 4>()) != cudaSuccess) return e;
  if ((e = set_attrs<32, 8>()) != cudaSuccess) return e;
  if ((e = set_attrs<64, 4>()) != cudaSuccess) return e;
  if ((e = set_attrs<16, 2>()) != cudaSuccess) return e;
  if ((e = set_attrs<8, 2>()) != cudaSuccess) return e;
  if ((e = set_attrs<4, 2>()) != cudaSuccess) return e;
  if ((e = set_attrs<2, 2>()) != cudaSuccess) return e;
  return cudaSuccess;
}

// Launch of a kernel taking KArgs; with pdl, as a programmatic dependent of
// the kernel before it in the stream (see dep_wait).
template <typename K>
static cudaError_t launch_k(K kern, int grid, int block, size_t smem, cudaStream_t st, bool pdl, const KArgs& a) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = pdl ? at : nullptr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, a);
}

cudaError_t launch_wait_probe(const int32_t* cnt, int32_t* err, unsigned limit, cudaStream_t st) {
  k_wait_probe<<<1, 32, 0, st>>>(cnt, err, limit);
  return cudaGetLastError();
}

cudaError_t launch_prep(const KArgs& a, cudaStream_t st) {
  const int n = a.scans ? a.nscans : 1;
  k_prep<<<n, NT_PREP, 0, st>>>(a);
  return cudaGetLastError();
}

#define LSG_DISPATCH(tile, FN, ...)                       \
  switch (tile) {                                         \
    case LSG_TILE_32x120: return FN<32, 2>(__VA_ARGS__);  \
    case LSG_TILE_32x240: return FN<32, 4>(__VA_ARGS__);  \
    case LSG_TILE_32x480: return FN<32, 8>(__VA_ARGS__);  \
    case LSG_TILE_64x240: return FN<64, 4>(__VA_ARGS__);  \
    case LSG_TILE_16x120: return FN<16, 2>(__VA_ARGS__);  \
    case LSG_TILE_8x120: return FN<8, 2>(__VA_ARGS__);    \
    case LSG_TILE_4x120: return FN<4, 2>(__VA_ARGS__);    \
    case LSG_TILE_2x120: return FN<2, 2>(__VA_ARGS__);    \
    default: return FN<16, 4>(__VA_ARGS__);               \
  }

template <int TR, int NW>
static cudaError_t run_tile(const KArgs& a, cudaStream_t st, bool pdl) {
  if (a.fuse_prep) return launch_k(k_tile<TR, NW, true>, a.ntiles, NW * 32, Geo<TR, NW>::bytes, st, pdl, a);
  return launch_k(k_tile<TR, NW>, a.ntiles, NW * 32, Geo<TR, NW>::bytes, st, pdl, a);
}
template <int TR, int NW>
static cudaError_t run_tile_ccl(const KArgs& a, cudaStream_t st, bool pdl) {
  return launch_k(k_tile_ccl<TR, NW>, a.ntiles, NW * 32, Geo<TR, NW>::ccl_bytes, st, pdl, a);
}
template <int TR, int NW>
static cudaError_t run_merge(const KArgs& a, cudaStream_t st, bool pdl) {
  return launch_k(k_merge<TR, NW>, a.ntiles, nt_merge<TR, NW>(), 0, st, pdl, a);
}
template <int TR, int NW>
static cudaError_t run_flatten(const KArgs& a, cudaStream_t st, bool pdl) {
  if (a.s1_only) return launch_k(k_flatten1<TR, NW>, a.ntiles, NT_FLAT, FlatGeo<TR, NW>::s1_bytes, st, pdl, a);
  return launch_k(k_flatten<TR, NW>, a.ntiles, NT_FLAT, FlatGeo<TR, NW>::bytes, st, pdl, a);
}

template <int TR, int NW>
static cudaError_t run_fused(const FusedArgs& f, cudaStream_t st) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t smem = f.s1_only ? FusedGeo<TR, NW>::s1_bytes : FusedGeo<TR, NW>::bytes;
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fused<TR, NW>, NW * 32, smem);
  if (e != cudaSuccess) return e;
  const int grid = max(1, min(sms * max(per_sm, 1), f.nitems));
  k_fused<TR, NW><<<grid, NW * 32, smem, st>>>(f);
  return cudaGetLastError();
}

cudaError_t launch_fused(int tile, const FusedArgs& f, cudaStream_t st) { LSG_DISPATCH(tile, run_fused, f, st) }

cudaError_t launch_tile(int tile, const KArgs& a, cudaStream_t st, bool pdl) {
  LSG_DISPATCH(tile, run_tile, a, st, pdl)
}
cudaError_t launch_tile_ccl(int tile, const KArgs& a, cudaStream_t st, bool pdl) {
  LSG_DISPATCH(tile, run_tile_ccl, a, st, pdl)
}
cudaError_t launch_merge(int tile, const KArgs& a, cudaStream_t st, bool pdl) {
  LSG_DISPATCH(tile, run_merge, a, st, pdl)
}
cudaError_t launch_flatten(int tile, const KArgs& a, cudaStream_t st, bool pdl) {
  LSG_DISPATCH(tile, run_flatten, a, st, pdl)
}

}  // namespace lsg
