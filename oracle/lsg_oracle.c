/*
 * lsg_oracle.c - plain, slow, obviously correct CPU oracle (FP64).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline arm may load this code.  It shares nothing with the
 * CUDA path (no headers, no helpers, no tables); the two meet only through the
 * seeded scans of the input generator and through documented output formats.
 *
 * It computes what Mukherjee et al., "Fast Geometric Surface based
 * Segmentation of Point Cloud from Lidar Data" (PReMI 2019) define, step by
 * step, in the paper's order:
 *
 *   Sec. 2, point model     a scan is P = {p(theta, phi, r)}; rings are counted
 *                           from the topmost sensor down, columns from the
 *                           first shot of the spin; azimuth sub-sampling keeps
 *                           every s-th shot.
 *   Sec. 2, mesh            p(i,j) joins (i+1,j), (i+1,j+1), (i,j+1); the last
 *                           ring joins only horizontally; the last column wraps
 *                           to the first (cylinder); a join needs both ranges in
 *                           the sensor's range.
 *   Sec. 2, normals         spokes A..F taken anticlockwise, cross products of
 *                           consecutive spokes, weighted by 1/(|V_k|+|V_k+1|),
 *                           averaged.
 *   Sec. 2, Algorithm 1     label propagation over mesh neighbours whose normal
 *                           components differ by less than (I, J, K).
 *   Sec. 2, last paragraph  non-sampled points take the label of the nearest
 *                           labelled point along the sweep.
 *
 * Readings where the paper is silent (each is listed with its reason in the
 * project's design notes):
 *   - ring order: sort by elevation, descending; ties by input row.
 *   - validity: r_min < r <= r_max, r = 0 is a dropout.
 *   - depth-jump cut: edge (p,q) is cut when |r_p - r_q| > tau * min(r_p, r_q),
 *     tau = jump_rel_h for horizontal edges and jump_rel_v for the others.
 *     This decides an integer from floats, so it is evaluated in IEEE binary32
 *     (round to nearest, no contraction), the precision the GPU path uses.
 *   - wrap needs at least 3 sampled columns (a cylinder of 2 columns would
 *     join the same pair twice).
 *   - a triangle (p, q_k, q_k+1) contributes to the normal of p only when all
 *     three of its edges are in the mesh.
 *   - orientation: n = -sign(dphi) * sum, which faces the sensor for surfaces
 *     seen from the front when rings run top to bottom.
 *   - angle predicate (the benchmark workloads' form): homogeneous when both
 *     normals exist and angle(n_p, n_q) < theta_t; component predicate (the
 *     paper's form): |dx| < I, |dy| < J, |dz| < K.
 *   - labels: every valid sampled point is a mesh vertex; its label is the
 *     smallest full-resolution linear index i*W + c in its component.
 *
 * Byte layout of the per-vertex mesh byte (also the GPU's output format):
 *   bit 0 R edge (i,j)-(i,j+1)    bit 3 R edge homogeneous
 *   bit 1 D edge (i,j)-(i+1,j)    bit 4 D edge homogeneous
 *   bit 2 G edge (i,j)-(i+1,j+1)  bit 5 G edge homogeneous
 *   bit 6 vertex valid            bit 7 vertex has a normal
 *
 * Parity pins: every function here is checked against closed forms, brute
 * force or invariants in the oracle test-suite (plane and box scenes, tiny
 * grids against a breadth-first search, Algorithm 1 against the component
 * labelling, decimation and shift invariance, hand-worked fixtures).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OB_R 0x01
#define OB_D 0x02
#define OB_G 0x04
#define OB_HR 0x08
#define OB_HD 0x10
#define OB_HG 0x20
#define OB_VALID 0x40
#define OB_HASN 0x80

#define OPRED_ANGLE 0
#define OPRED_COMPONENT 1

/* ------------------------------------------------------------------------ */
/* Step 1: decode (Sec. 2 point model)                                       */
/* ------------------------------------------------------------------------ */

/* order[i] = input row of the i-th ring counted from the top.
 * Plain insertion sort by (elevation descending, input row ascending). */
int oracle_ring_order(int H, const float* elev, int* order) {
  for (int k = 0; k < H; ++k) {
    if (elev[k] != elev[k]) return -1; /* NaN elevation */
    order[k] = k;
  }
  for (int a = 1; a < H; ++a) {
    int cur = order[a];
    int b = a - 1;
    while (b >= 0 && (elev[order[b]] < elev[cur] ||
                      (elev[order[b]] == elev[cur] && order[b] > cur))) {
      order[b + 1] = order[b];
      --b;
    }
    order[b + 1] = cur;
  }
  return 0;
}

/* Sorted-grid copy of the scan at full resolution: rs[i*W+c] = range,
 * xyz[3*(i*W+c)] in double, valid[i*W+c] = r_min < r <= r_max.
 * xyzr != NULL: take the given float xyz.  Otherwise range-only decode:
 * (r cos(theta) cos(phi), r cos(theta) sin(phi), r sin(theta)) in double with
 * phi = phi0 + c * dphi (Sec. 2: p(theta, phi, r)). */
int oracle_decode(int H, int W, const int* order, const float* elev, float az0, float daz,
                  const float* xyzr, const float* range, float r_min, float r_max,
                  float* rs, double* xyz, unsigned char* valid) {
  for (int i = 0; i < H; ++i) {
    int row = order[i];
    double th = (double)elev[row];
    for (int c = 0; c < W; ++c) {
      size_t src = (size_t)row * W + c, dst = (size_t)i * W + c;
      float r = xyzr ? xyzr[4 * src + 3] : range[src];
      rs[dst] = r;
      valid[dst] = (r_min < r && r <= r_max) ? 1 : 0;
      if (xyzr) {
        xyz[3 * dst + 0] = (double)xyzr[4 * src + 0];
        xyz[3 * dst + 1] = (double)xyzr[4 * src + 1];
        xyz[3 * dst + 2] = (double)xyzr[4 * src + 2];
      } else {
        double phi = (double)az0 + (double)c * (double)daz;
        double rd = (double)r;
        xyz[3 * dst + 0] = rd * cos(th) * cos(phi);
        xyz[3 * dst + 1] = rd * cos(th) * sin(phi);
        xyz[3 * dst + 2] = rd * sin(th);
      }
    }
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Step 2: mesh (Sec. 2 mesh construction)                                   */
/* ------------------------------------------------------------------------ */

static int o_wrap_eff(int wrap, int Ws) { return (wrap && Ws >= 3) ? 1 : 0; }

/* Depth-jump cut, decided in binary32 (see header). */
static int o_cut(float rp, float rq, float tau) {
  volatile float d = rp - rq;
  float ad = d < 0.0f ? -d : d;
  float m = rp < rq ? rp : rq;
  volatile float t = tau * m;
  return ad > t;
}

/* Mesh bits (bits 0-2) and the valid bit (bit 6) for every sampled vertex
 * (i, j), column c = j*s, Ws = ceil(W/s). */
int oracle_mesh(int H, int W, int s, int wrap, const float* rs, const unsigned char* valid,
                float jump_h, float jump_v, unsigned char* mb) {
  int Ws = (W + s - 1) / s;
  int wr = o_wrap_eff(wrap, Ws);
  for (int i = 0; i < H; ++i) {
    for (int j = 0; j < Ws; ++j) {
      size_t p = (size_t)i * W + (size_t)j * s;
      unsigned char b = 0;
      if (valid[p]) b |= OB_VALID;
      int jn = j + 1;
      int has_right = (jn < Ws) || wr;
      if (jn >= Ws) jn = 0;
      size_t pr = (size_t)i * W + (size_t)jn * s;
      /* R: (i,j) - (i,j+1) */
      if (has_right && valid[p] && valid[pr] && !o_cut(rs[p], rs[pr], jump_h)) b |= OB_R;
      if (i + 1 < H) {
        size_t pd = (size_t)(i + 1) * W + (size_t)j * s;
        size_t pg = (size_t)(i + 1) * W + (size_t)jn * s;
        /* D: (i,j) - (i+1,j) */
        if (valid[p] && valid[pd] && !o_cut(rs[p], rs[pd], jump_v)) b |= OB_D;
        /* G: (i,j) - (i+1,j+1) */
        if (has_right && valid[p] && valid[pg] && !o_cut(rs[p], rs[pg], jump_v)) b |= OB_G;
      }
      mb[(size_t)i * Ws + j] = b;
    }
  }
  return 0;
}

/* Is there a mesh edge between sampled vertices (i1,j1) and (i2,j2)?
 * Looks the pair up among the three forward edges of either endpoint. */
static int o_edge(const unsigned char* mb, int H, int Ws, int wr, int i1, int j1, int i2, int j2,
                  int want_homog) {
  for (int pass = 0; pass < 2; ++pass) {
    int a_i = pass ? i2 : i1, a_j = pass ? j2 : j1;
    int b_i = pass ? i1 : i2, b_j = pass ? j1 : j2;
    if (a_i < 0 || a_i >= H || b_i < 0 || b_i >= H) return 0;
    int jn = a_j + 1;
    int ok_right = (jn < Ws) || wr;
    if (jn >= Ws) jn = 0;
    unsigned char bits = mb[(size_t)a_i * Ws + a_j];
    if (b_i == a_i && ok_right && b_j == jn)
      return want_homog ? ((bits & OB_HR) != 0) : ((bits & OB_R) != 0);
    if (b_i == a_i + 1 && b_j == a_j)
      return want_homog ? ((bits & OB_HD) != 0) : ((bits & OB_D) != 0);
    if (b_i == a_i + 1 && ok_right && b_j == jn)
      return want_homog ? ((bits & OB_HG) != 0) : ((bits & OB_G) != 0);
  }
  return 0;
}

/* The six neighbours of (i,j) in the paper's anticlockwise order:
 * A=(i+1,j) B=(i+1,j+1) C=(i,j+1) D=(i-1,j) E=(i-1,j-1) F=(i,j-1).
 * Columns wrap when the mesh wraps; out[k] = {i, j} or {-1,-1}. */
static void o_spokes(int H, int Ws, int wr, int i, int j, int out[6][2]) {
  static const int di[6] = {+1, +1, 0, -1, -1, 0};
  static const int dj[6] = {0, +1, +1, 0, -1, -1};
  for (int k = 0; k < 6; ++k) {
    int ii = i + di[k], jj = j + dj[k];
    if (wr) jj = (jj + Ws) % Ws;
    if (ii < 0 || ii >= H || jj < 0 || jj >= Ws) {
      out[k][0] = out[k][1] = -1;
    } else {
      out[k][0] = ii;
      out[k][1] = jj;
    }
  }
}

/* The paper's map M: for each vertex, its mesh neighbours in the order
 * A..F (Sec. 2).  nbr[6*v + k] = vertex index or -1; cnt[v] = |v|. */
int oracle_neighbours(int H, int W, int s, int wrap, const unsigned char* mb, int* nbr, int* cnt) {
  int Ws = (W + s - 1) / s;
  int wr = o_wrap_eff(wrap, Ws);
  for (int i = 0; i < H; ++i)
    for (int j = 0; j < Ws; ++j) {
      int sp[6][2];
      o_spokes(H, Ws, wr, i, j, sp);
      int n = 0;
      size_t v = (size_t)i * Ws + j;
      for (int k = 0; k < 6; ++k) {
        int e = sp[k][0] >= 0 && o_edge(mb, H, Ws, wr, i, j, sp[k][0], sp[k][1], 0);
        nbr[6 * v + k] = e ? sp[k][0] * Ws + sp[k][1] : -1;
        n += e;
      }
      cnt[v] = n;
    }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Step 3: normals (Sec. 2 normal estimation)                                */
/* ------------------------------------------------------------------------ */

/* For each vertex: n = -sign(dphi) * sum_k w_k (V_k x V_k+1) / |...| over the
 * incident triangles (p, q_k, q_k+1), k = AB, BC, CD, DE, EF, FA, whose three
 * edges exist; w_k = 1 / (|V_k| + |V_k+1|), V_k = q_k - p.
 * normal[3v] = unit normal or 0; bit 7 of mb set when it exists.
 * kappa[v] (optional) = sum_k w_k |V_k| |V_k+1| / |sum_k w_k V_k x V_k+1|,
 * the condition number of the weighted sum; snorm[v] (optional) =
 * |sum_k w_k V_k x V_k+1|; ntri[v] (optional) = number of counted triangles.
 * These three only serve the tolerance tests. */
int oracle_normals(int H, int W, int s, int wrap, float daz, const double* xyz, unsigned char* mb,
                   double* normal, double* kappa, double* snorm, int32_t* ntri_out) {
  int Ws = (W + s - 1) / s;
  int wr = o_wrap_eff(wrap, Ws);
  double sgn = daz < 0.0f ? -1.0 : 1.0;
  for (int i = 0; i < H; ++i)
    for (int j = 0; j < Ws; ++j) {
      size_t v = (size_t)i * Ws + j;
      size_t p = (size_t)i * W + (size_t)j * s;
      normal[3 * v] = normal[3 * v + 1] = normal[3 * v + 2] = 0.0;
      if (kappa) kappa[v] = INFINITY;
      if (snorm) snorm[v] = 0.0;
      if (ntri_out) ntri_out[v] = 0;
      mb[v] &= (unsigned char)~OB_HASN;
      if (!(mb[v] & OB_VALID)) continue;
      int sp[6][2];
      o_spokes(H, Ws, wr, i, j, sp);
      double sum[3] = {0, 0, 0};
      double mag = 0.0;
      int ntri = 0;
      for (int k = 0; k < 6; ++k) {
        int k1 = (k + 1) % 6;
        if (sp[k][0] < 0 || sp[k1][0] < 0) continue;
        if (!o_edge(mb, H, Ws, wr, i, j, sp[k][0], sp[k][1], 0)) continue;
        if (!o_edge(mb, H, Ws, wr, i, j, sp[k1][0], sp[k1][1], 0)) continue;
        if (!o_edge(mb, H, Ws, wr, sp[k][0], sp[k][1], sp[k1][0], sp[k1][1], 0)) continue;
        size_t qa = (size_t)sp[k][0] * W + (size_t)sp[k][1] * s;
        size_t qb = (size_t)sp[k1][0] * W + (size_t)sp[k1][1] * s;
        double a[3], b[3];
        for (int t = 0; t < 3; ++t) {
          a[t] = xyz[3 * qa + t] - xyz[3 * p + t];
          b[t] = xyz[3 * qb + t] - xyz[3 * p + t];
        }
        double la = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
        double lb = sqrt(b[0] * b[0] + b[1] * b[1] + b[2] * b[2]);
        double w = 1.0 / (la + lb);
        double cr[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
        for (int t = 0; t < 3; ++t) sum[t] += w * cr[t];
        mag += w * la * lb;
        ++ntri;
      }
      if (ntri_out) ntri_out[v] = ntri;
      if (ntri == 0) continue;
      double len = sqrt(sum[0] * sum[0] + sum[1] * sum[1] + sum[2] * sum[2]);
      if (snorm) snorm[v] = len;
      if (!(len > 0.0)) continue;
      for (int t = 0; t < 3; ++t) normal[3 * v + t] = -sgn * sum[t] / len;
      if (kappa) kappa[v] = mag / len;
      mb[v] |= OB_HASN;
    }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Step 4: homogeneity of each mesh edge (Algorithm 1 predicate)             */
/* ------------------------------------------------------------------------ */

/* Angle between unit normals, atan2(|a x b|, a . b), in [0, pi]. */
double oracle_angle(const double* a, const double* b) {
  double cx = a[1] * b[2] - a[2] * b[1];
  double cy = a[2] * b[0] - a[0] * b[2];
  double cz = a[0] * b[1] - a[1] * b[0];
  double dt = a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
  return atan2(sqrt(cx * cx + cy * cy + cz * cz), dt);
}

/* Sets bits 3-5 for each existing edge whose endpoints both have normals and
 * satisfy the predicate.  margin[3v+e] (optional) = the signed distance of the
 * edge from the threshold: theta_t - angle (angle mode) or the smallest of
 * I-|dx|, J-|dy|, K-|dz| (component mode); NAN for edges that do not exist or
 * lack a normal. */
int oracle_edge_mask(int H, int W, int s, int wrap, int pred, double angle_t, const double* comp,
                     const double* normal, unsigned char* mb, double* margin) {
  int Ws = (W + s - 1) / s;
  int wr = o_wrap_eff(wrap, Ws);
  for (int i = 0; i < H; ++i)
    for (int j = 0; j < Ws; ++j) {
      size_t v = (size_t)i * Ws + j;
      mb[v] &= (unsigned char)~(OB_HR | OB_HD | OB_HG);
      int jn = j + 1 < Ws ? j + 1 : 0;
      int nb[3][2] = {{i, jn}, {i + 1, j}, {i + 1, jn}};
      const unsigned char ebit[3] = {OB_R, OB_D, OB_G};
      const unsigned char hbit[3] = {OB_HR, OB_HD, OB_HG};
      for (int e = 0; e < 3; ++e) {
        if (margin) margin[3 * v + e] = NAN;
        if (!(mb[v] & ebit[e])) continue;
        size_t u = (size_t)nb[e][0] * Ws + nb[e][1];
        if (!(mb[v] & OB_HASN) || !(mb[u] & OB_HASN)) continue;
        const double* np = normal + 3 * v;
        const double* nq = normal + 3 * u;
        double m;
        int ok;
        if (pred == OPRED_ANGLE) {
          double ang = oracle_angle(np, nq);
          m = angle_t - ang;
          ok = ang < angle_t;
        } else {
          double dx = fabs(np[0] - nq[0]), dy = fabs(np[1] - nq[1]), dz = fabs(np[2] - nq[2]);
          ok = dx < comp[0] && dy < comp[1] && dz < comp[2];
          m = comp[0] - dx;
          if (comp[1] - dy < m) m = comp[1] - dy;
          if (comp[2] - dz < m) m = comp[2] - dz;
        }
        if (margin) margin[3 * v + e] = m;
        if (ok) mb[v] |= hbit[e];
      }
      (void)wr;
    }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Step 5: labels                                                            */
/* ------------------------------------------------------------------------ */

/* Components of (valid vertices, homogeneous edges) by breadth-first search,
 * visiting seeds in increasing vertex index so that each component's first
 * vertex is its smallest.  vlabel[v] = i*W + j*s of that first vertex for
 * valid vertices, -1 otherwise.  Returns the number of components. */
int oracle_components(int H, int W, int s, int wrap, const unsigned char* mb, int32_t* vlabel) {
  int Ws = (W + s - 1) / s;
  int wr = o_wrap_eff(wrap, Ws);
  size_t Nv = (size_t)H * Ws;
  int* queue = (int*)malloc(sizeof(int) * (Nv ? Nv : 1));
  if (!queue) return -1;
  for (size_t v = 0; v < Nv; ++v) vlabel[v] = -1;
  int ncomp = 0;
  for (size_t seed = 0; seed < Nv; ++seed) {
    if (!(mb[seed] & OB_VALID) || vlabel[seed] != -1) continue;
    int si = (int)(seed / Ws), sj = (int)(seed % Ws);
    int32_t lab = si * W + sj * s;
    size_t head = 0, tail = 0;
    queue[tail++] = (int)seed;
    vlabel[seed] = lab;
    while (head < tail) {
      int v = queue[head++];
      int i = v / Ws, j = v % Ws;
      int sp[6][2];
      o_spokes(H, Ws, wr, i, j, sp);
      for (int k = 0; k < 6; ++k) {
        if (sp[k][0] < 0) continue;
        if (!o_edge(mb, H, Ws, wr, i, j, sp[k][0], sp[k][1], 1)) continue;
        int u = sp[k][0] * Ws + sp[k][1];
        if (vlabel[u] == -1) {
          vlabel[u] = lab;
          queue[tail++] = u;
        }
      }
    }
    ++ncomp;
  }
  free(queue);
  return ncomp;
}

/* Algorithm 1 as the paper states it: for each point (in vertex order) with
 * label 0, give it the next label and flood its mesh neighbours through a
 * stack, pushing a neighbour when it is unlabelled and the predicate holds
 * between the popped point and that neighbour.  The predicate is read from
 * the homogeneity bits computed by oracle_edge_mask.  Labels are 1, 2, ... in
 * order of discovery; 0 stays for points outside P (invalid).
 * Returns the number of labels. */
int oracle_algorithm1(int H, int W, int s, int wrap, const unsigned char* mb, int32_t* L) {
  int Ws = (W + s - 1) / s;
  int wr = o_wrap_eff(wrap, Ws);
  size_t Nv = (size_t)H * Ws;
  /* a point is pushed at most once, so Nv slots suffice */
  int* stack = (int*)malloc(sizeof(int) * (Nv ? Nv : 1));
  if (!stack) return -1;
  for (size_t v = 0; v < Nv; ++v) L[v] = 0;
  int label = 1;
  for (size_t p0 = 0; p0 < Nv; ++p0) {
    if (!(mb[p0] & OB_VALID)) continue; /* not a point of P */
    if (L[p0] != 0) continue;
    L[p0] = label;
    size_t top = 0;
    stack[top++] = (int)p0;
    while (top > 0) {
      int p = stack[--top];
      int i = p / Ws, j = p % Ws;
      int sp[6][2];
      o_spokes(H, Ws, wr, i, j, sp);
      for (int k = 0; k < 6; ++k) {
        if (sp[k][0] < 0) continue;
        if (!o_edge(mb, H, Ws, wr, i, j, sp[k][0], sp[k][1], 0)) continue; /* q in v(p) */
        int q = sp[k][0] * Ws + sp[k][1];
        if (L[q] != 0) continue;
        if (!o_edge(mb, H, Ws, wr, i, j, sp[k][0], sp[k][1], 1)) continue; /* predicate */
        L[q] = label;
        stack[top++] = q;
      }
    }
    ++label;
  }
  free(stack);
  return label - 1;
}

/* ------------------------------------------------------------------------ */
/* Step 6: back-fill of non-sampled points (Sec. 2, last paragraph)          */
/* ------------------------------------------------------------------------ */

/* labels[i*W + c] for every full-resolution point.  Sampled columns take the
 * vertex label.  A valid non-sampled point takes the label of the nearer of
 * the two sampled columns that bracket it on its ring (ties to the earlier
 * one); when that one is unlabelled it takes the other; the column after the
 * last sampled one is column 0 when the mesh wraps, absent otherwise.
 * Invalid points get -1. */
int oracle_backfill(int H, int W, int s, int wrap, const unsigned char* valid,
                    const int32_t* vlabel, int32_t* labels) {
  int Ws = (W + s - 1) / s;
  int wr = o_wrap_eff(wrap, Ws);
  for (int i = 0; i < H; ++i)
    for (int c = 0; c < W; ++c) {
      size_t o = (size_t)i * W + c;
      if (!valid[o]) { labels[o] = -1; continue; }
      int jl = c / s;
      if (c % s == 0) { labels[o] = vlabel[(size_t)i * Ws + jl]; continue; }
      int32_t lo = vlabel[(size_t)i * Ws + jl];
      int dlo = c - jl * s;
      int32_t hi = -1;
      int dhi = 0, have_hi = 0;
      if (jl + 1 < Ws) {
        hi = vlabel[(size_t)i * Ws + jl + 1];
        dhi = (jl + 1) * s - c;
        have_hi = 1;
      } else if (wr) {
        hi = vlabel[(size_t)i * Ws + 0];
        dhi = W - c;
        have_hi = 1;
      }
      int32_t first = lo, second = have_hi ? hi : -1;
      if (have_hi && dhi < dlo) { first = hi; second = lo; }
      labels[o] = first != -1 ? first : second;
    }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Whole path                                                                */
/* ------------------------------------------------------------------------ */

/* One scan through every step.  Outputs (caller-allocated):
 *   order[H], mb[H*Ws], normal[3*H*Ws] (double), labels[H*W], *nseg;
 *   optional: kappa[H*Ws], margin[3*H*Ws], vlabel[H*Ws], snorm[H*Ws], ntri[H*Ws].
 * Returns 0, or a negative code on bad input. */
int oracle_segment(int H, int W, const float* elev, float az0, float daz, const float* xyzr,
                   const float* range, int s, float r_min, float r_max, float jump_h, float jump_v,
                   int pred, double angle_t, const double* comp, int wrap, int* order,
                   unsigned char* mb, double* normal, int32_t* labels, int32_t* nseg,
                   double* kappa, double* margin, int32_t* vlabel_out, double* snorm,
                   int32_t* ntri) {
  if (H < 0 || W < 0 || s < 1) return -1;
  if (H == 0 || W == 0) { *nseg = 0; return 0; }
  int Ws = (W + s - 1) / s;
  size_t N = (size_t)H * W, Nv = (size_t)H * Ws;
  float* rs = (float*)malloc(sizeof(float) * N);
  double* xyz = (double*)malloc(sizeof(double) * 3 * N);
  unsigned char* valid = (unsigned char*)malloc(N);
  int32_t* vlabel = vlabel_out ? vlabel_out : (int32_t*)malloc(sizeof(int32_t) * Nv);
  int rc = 0;
  if (!rs || !xyz || !valid || !vlabel) { rc = -2; goto done; }
  if (oracle_ring_order(H, elev, order)) { rc = -3; goto done; }
  oracle_decode(H, W, order, elev, az0, daz, xyzr, range, r_min, r_max, rs, xyz, valid);
  oracle_mesh(H, W, s, wrap, rs, valid, jump_h, jump_v, mb);
  oracle_normals(H, W, s, wrap, daz, xyz, mb, normal, kappa, snorm, ntri);
  oracle_edge_mask(H, W, s, wrap, pred, angle_t, comp, normal, mb, margin);
  *nseg = oracle_components(H, W, s, wrap, mb, vlabel);
  oracle_backfill(H, W, s, wrap, valid, vlabel, labels);
done:
  free(rs);
  free(xyz);
  free(valid);
  if (!vlabel_out) free(vlabel);
  return rc;
}

/* Labels from a given mesh byte array (the edge mask is taken as given) and
 * the per-point validity; the parity hook's counterpart. */
int oracle_label_from_mask(int H, int W, int s, int wrap, const unsigned char* mb,
                           const unsigned char* valid, int32_t* labels, int32_t* nseg) {
  int Ws = (W + s - 1) / s;
  size_t Nv = (size_t)H * Ws;
  int32_t* vlabel = (int32_t*)malloc(sizeof(int32_t) * (Nv ? Nv : 1));
  if (!vlabel) return -2;
  int n = oracle_components(H, W, s, wrap, mb, vlabel);
  oracle_backfill(H, W, s, wrap, valid, vlabel, labels);
  *nseg = n;
  free(vlabel);
  return n < 0 ? -2 : 0;
}

/* ------------------------------------------------------------------------ */
/* Post-processing: segment sizes and small-segment removal                  */
/* (Sec. 2, last paragraph: segments with too few points may be eliminated)  */
/* ------------------------------------------------------------------------ */

/* labels_in[H*W]: labels as produced by the path (-1 or the segment's
 * smallest point index).  sizes[H*W]: number of points carrying each label
 * (0 for indices that are not labels).  nsum[3*H*W] (optional): sum of the
 * unit normals of the segment's mesh vertices that have one (vertex (i, j)
 * carries labels_in[i*W + j*s]).  labels_out: labels_in with every segment of
 * fewer than min_points points set to -1.  Returns the number of segments
 * kept. */
int oracle_segment_stats(int H, int W, int s, const int32_t* labels_in, const double* normal,
                         const unsigned char* mb, int min_points, int32_t* labels_out, int32_t* sizes,
                         double* nsum) {
  size_t N = (size_t)H * W;
  int Ws = (W + s - 1) / s;
  for (size_t p = 0; p < N; ++p) sizes[p] = 0;
  if (nsum)
    for (size_t p = 0; p < 3 * N; ++p) nsum[p] = 0.0;
  for (size_t p = 0; p < N; ++p)
    if (labels_in[p] >= 0) sizes[labels_in[p]] += 1;
  if (nsum && normal && mb)
    for (int i = 0; i < H; ++i)
      for (int j = 0; j < Ws; ++j) {
        size_t v = (size_t)i * Ws + j;
        int32_t lab = labels_in[(size_t)i * W + (size_t)j * s];
        if (lab < 0 || !(mb[v] & OB_HASN)) continue;
        for (int t = 0; t < 3; ++t) nsum[3 * (size_t)lab + t] += normal[3 * v + t];
      }
  int kept = 0;
  for (size_t p = 0; p < N; ++p) {
    int32_t lab = labels_in[p];
    labels_out[p] = (lab >= 0 && sizes[lab] >= min_points) ? lab : -1;
    if (lab >= 0 && (size_t)lab == p && sizes[lab] >= min_points) ++kept;
  }
  return kept;
}
