// lsg_api.cu - the C ABI declared in include/lsg.h: contexts, argument
// checks, workspace, the single-scan and batched passes, graph capture and
// the tile-shape autotuner.  Host code only; the kernels are in lsg_kernels.cu.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "lsg_internal.h"

using namespace lsg;

// Pinned staging buffer for the descriptor tables of lsg_batch_launch; the
// event marks when the device copy out of it has run.
struct DynStage {
  void* host = nullptr;
  void* dev = nullptr;
  size_t cap = 0;
  cudaEvent_t copied = nullptr;
};

struct lsg_ctx {
  int device = 0;
  size_t budget = 0;        // 0 = unlimited
  size_t used = 0;          // bytes currently held (context workspace + plans)
  void* ws = nullptr;       // single-scan / dynamic-batch workspace
  size_t ws_bytes = 0;
  int32_t* d_err = nullptr; // sticky device error word
  int tile = LSG_TILE_AUTO;  // or a fixed shape (lsg_set_tile)
  int sms = 1;              // streaming multiprocessors of the device
  DynStage stage[2];        // alternated by successive lsg_batch_launch calls
  int next_stage = 0;
};

struct lsg_plan {
  lsg_ctx* ctx = nullptr;
  int tile = LSG_TILE_32x240;
  int n = 0;
  std::vector<ScanDesc> host_desc;  // tile fields filled per tile shape
  ScanDesc* d_desc = nullptr;
  int32_t* d_tile_scan = nullptr;
  int32_t ntiles = 0;
  void* ws = nullptr;               // order + trig + parent of every scan
  size_t bytes = 0;                 // everything this plan holds
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};  // phase boundaries
  int fused = 1;                    // one persistent launch (1) or four phased launches (0)
  int2* d_items = nullptr;          // fused schedule
  int32_t nitems = 0;
  int32_t* d_counters = nullptr;    // [1 + 3n] fused progress counters
  int launches = 0;                 // kernel launches in one replay of the graph
  // host-buffer plans (lsg_batch_plan_io): the scans' device buffers and host
  // buffers, and the number of chunks the copies and passes are cut into
  int chunks = 0;                   // 0: device-resident plan
  std::vector<lsg_scan> dev_in;     // device inputs of each scan
  std::vector<lsg_out> dev_out;     // device outputs of each scan
  std::vector<lsg_host_io> io;      // host buffers of each scan
  size_t h2d_bytes = 0, d2h_bytes = 0;  // host transfers of one run
};

namespace {

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

lsg_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return LSG_OK;
  if (e == cudaErrorMemoryAllocation) return LSG_E_OOM;
  return LSG_E_CUDA;
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace

namespace lsg {

// Validates one scan's shape and parameters; fills Ws.
lsg_status check_scan(const lsg_scan* sc, const lsg_params* p, const lsg_out* o, int* Ws_out) {
  if (!sc || !p || !o) return LSG_E_ARG;
  if (sc->rings < 0 || sc->cols < 0) return LSG_E_SHAPE;
  if (sc->rings > LSG_MAX_RINGS || sc->cols > LSG_MAX_COLS) return LSG_E_SHAPE;
  if ((int64_t)sc->rings * sc->cols > (int64_t)LSG_MAX_POINTS) return LSG_E_SHAPE;
  if (p->subsample < 1) return LSG_E_ARG;
  if (!(p->r_min >= 0.f) || !(p->r_max > p->r_min)) return LSG_E_ARG;
  if (!(p->jump_rel_h >= 0.f) || !(p->jump_rel_v >= 0.f)) return LSG_E_ARG;
  if (p->predicate == LSG_PRED_ANGLE) {
    if (!(p->angle_rad > 0.f) || !(p->angle_rad < 3.14159265f)) return LSG_E_ARG;
  } else if (p->predicate == LSG_PRED_COMPONENT) {
    for (int k = 0; k < 3; ++k)
      if (!(p->comp[k] > 0.f)) return LSG_E_ARG;
  } else {
    return LSG_E_ARG;
  }
  if (!isfinite(sc->azimuth0) || !isfinite(sc->azimuth_step)) return LSG_E_ARG;
  const int Ws = sc->cols > 0 ? (sc->cols + p->subsample - 1) / p->subsample : 0;
  *Ws_out = Ws;
  if (sc->rings == 0 || sc->cols == 0) {
    if (!o->nseg) return LSG_E_ARG;
    return LSG_OK;
  }
  if (!sc->elevation) return LSG_E_ARG;
  if (!sc->xyzr && !sc->range) return LSG_E_ARG;
  if (sc->xyzr && ((uintptr_t)sc->xyzr & 15u)) return LSG_E_ARG;
  if (!o->meshbits || !o->normals || !o->labels || !o->nseg) return LSG_E_ARG;
  return LSG_OK;
}

// Fills the shape/parameter fields of a descriptor (pointers to the
// workspace are set by the caller).
ScanDesc make_desc(const lsg_scan* sc, const lsg_params* p, const lsg_out* o, int Ws) {
  ScanDesc d;
  memset(&d, 0, sizeof(d));
  d.xyzr = reinterpret_cast<const float4*>(sc->xyzr);
  d.range = sc->range;
  d.elev = sc->elevation;
  d.valid = nullptr;
  d.mb = o->meshbits;
  d.nrm = o->normals;
  d.labels = o->labels;
  d.nseg = o->nseg;
  d.H = sc->rings;
  d.W = sc->cols;
  d.Ws = Ws;
  d.s = p->subsample;
  d.wrap = (p->wrap && Ws >= 3) ? 1 : 0;
  d.az0 = sc->azimuth0;
  d.daz = sc->azimuth_step;
  d.r_min = p->r_min;
  d.r_max = p->r_max;
  d.jump_h = p->jump_rel_h;
  d.jump_v = p->jump_rel_v;
  d.pred = p->predicate;
  d.cos_t = (float)cos((double)p->angle_rad);
  d.comp_x = p->comp[0];
  d.comp_y = p->comp[1];
  d.comp_z = p->comp[2];
  d.nsign = sc->azimuth_step < 0.f ? 1.f : -1.f;
  return d;
}

void set_tiles(ScanDesc& d, int tile, int tile0) {
  const TileShape ts = tile_shape(tile);
  d.tiles_r = (d.H + ts.rows - 1) / ts.rows;
  d.tiles_c = (d.Ws + ts.cols - 1) / ts.cols;
  d.tile0 = tile0;
}

}  // namespace lsg

namespace {

// tile-root rows are padded to a multiple of 8 entries (see root_pitch)
size_t scan_ws_bytes(int H, int Ws) {
  const size_t lp = (size_t)((Ws + 7) & ~7);
  return align_up(sizeof(int32_t) * H, 256) + align_up(sizeof(float2) * H, 256) +
         align_up(sizeof(int32_t) * (size_t)H * Ws, 256) + align_up(sizeof(uint16_t) * (size_t)H * lp, 256);
}

void carve_ws(ScanDesc& d, char* base) {
  d.order = reinterpret_cast<int32_t*>(base);
  base += align_up(sizeof(int32_t) * d.H, 256);
  d.trig = reinterpret_cast<float2*>(base);
  base += align_up(sizeof(float2) * d.H, 256);
  d.parent = reinterpret_cast<int32_t*>(base);
  base += align_up(sizeof(int32_t) * (size_t)d.H * d.Ws, 256);
  d.lroot = reinterpret_cast<uint16_t*>(base);
}

lsg_status reserve(lsg_ctx* ctx, size_t need) {
  if (need <= ctx->ws_bytes) return LSG_OK;
  const size_t grow = align_up(need, 1 << 20);
  if (ctx->budget && ctx->used - ctx->ws_bytes + grow > ctx->budget) return LSG_E_BUDGET;
  if (ctx->ws) {
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_status(e);
    cudaFree(ctx->ws);
    ctx->used -= ctx->ws_bytes;
    ctx->ws = nullptr;
    ctx->ws_bytes = 0;
  }
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, grow);
  if (e != cudaSuccess) return cuda_status(e);
  ctx->ws = p;
  ctx->ws_bytes = grow;
  ctx->used += grow;
  return LSG_OK;
}

// The context's tile shape for a call over scans of (rings, sampled columns).
int ctx_tile(const lsg_ctx* ctx, const int* H, const int* Ws, int n) {
  return ctx->tile >= 0 ? ctx->tile : pick_tile(H, Ws, n, ctx->sms);
}

lsg_status run_pass(KArgs a, int tile, bool geometry, cudaStream_t st) {
  a.s1_only = a.one.s == 1;
  cudaError_t e = cudaSuccess;
  if (geometry && a.one.H <= kFuseMaxRings) {
    // no k_prep: each tile finds the ring order of the rows it reads
    a.fuse_prep = 1;
    e = launch_tile(tile, a, st, false);
  } else {
    // the kernels after k_prep start while their predecessor drains
    e = launch_prep(a, st);
    if (e == cudaSuccess) e = geometry ? launch_tile(tile, a, st, true) : launch_tile_ccl(tile, a, st, true);
  }
  if (e == cudaSuccess) e = launch_merge(tile, a, st, true);
  if (e == cudaSuccess) e = launch_flatten(tile, a, st, true);
  return cuda_status(e);
}

}  // namespace

extern "C" {

void lsg_default_params(lsg_params* p) {
  if (!p) return;
  p->subsample = 1;
  p->r_min = 0.f;
  p->r_max = 100.f;
  p->jump_rel_h = 0.10f;
  p->jump_rel_v = 1.0f;
  p->predicate = LSG_PRED_ANGLE;
  p->angle_rad = (float)(10.0 * 3.14159265358979323846 / 180.0);
  p->comp[0] = p->comp[1] = p->comp[2] = 0.2f;
  p->wrap = 1;
}

const char* lsg_status_str(lsg_status s) {
  switch (s) {
    case LSG_OK: return "ok";
    case LSG_E_ARG: return "invalid argument";
    case LSG_E_SHAPE: return "invalid scan shape";
    case LSG_E_OOM: return "device allocation failed";
    case LSG_E_BUDGET: return "memory budget exceeded";
    case LSG_E_CUDA: return "CUDA runtime error";
    case LSG_E_TIMEOUT: return "bounded device wait ran out";
    case LSG_E_DEVICE: return "device flagged bad input";
  }
  return "unknown status";
}

lsg_status lsg_create(int device, size_t mem_budget_bytes, lsg_ctx** out) {
  if (!out) return LSG_E_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return LSG_E_ARG;
  DeviceGuard g(device);
  cudaError_t e = prepare_kernels();
  if (e != cudaSuccess) return cuda_status(e);
  lsg_ctx* c = new (std::nothrow) lsg_ctx();
  if (!c) return LSG_E_OOM;
  c->device = device;
  c->budget = mem_budget_bytes;
  if (cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || c->sms < 1)
    c->sms = 1;
  e = cudaMalloc(&c->d_err, 256);
  if (e != cudaSuccess) {
    delete c;
    return cuda_status(e);
  }
  c->used = 256;
  e = cudaMemset(c->d_err, 0, sizeof(int32_t));
  if (e != cudaSuccess) {
    cudaFree(c->d_err);
    delete c;
    return cuda_status(e);
  }
  *out = c;
  return LSG_OK;
}

lsg_status lsg_destroy(lsg_ctx* ctx) {
  if (!ctx) return LSG_E_ARG;
  DeviceGuard g(ctx->device);
  cudaDeviceSynchronize();
  if (ctx->ws) cudaFree(ctx->ws);
  if (ctx->d_err) cudaFree(ctx->d_err);
  for (DynStage& st : ctx->stage) {
    if (st.host) cudaFreeHost(st.host);
    if (st.dev) cudaFree(st.dev);
    if (st.copied) cudaEventDestroy(st.copied);
  }
  delete ctx;
  return LSG_OK;
}

size_t lsg_memory_used(const lsg_ctx* ctx) { return ctx ? ctx->used : 0; }

lsg_status lsg_set_tile(lsg_ctx* ctx, int tile) {
  if (!ctx) return LSG_E_ARG;
  if (tile != LSG_TILE_AUTO && (tile < 0 || tile >= LSG_TILE_COUNT)) return LSG_E_ARG;
  ctx->tile = tile;
  return LSG_OK;
}

lsg_status lsg_segment(lsg_ctx* ctx, const lsg_scan* scan, const lsg_params* params,
                       const lsg_out* out, lsg_stream stream) {
  if (!ctx) return LSG_E_ARG;
  int Ws = 0;
  lsg_status st = check_scan(scan, params, out, &Ws);
  if (st != LSG_OK) return st;
  DeviceGuard g(ctx->device);
  cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
  if (scan->rings == 0 || scan->cols == 0)
    return cuda_status(cudaMemsetAsync(out->nseg, 0, sizeof(int32_t), cs));
  st = reserve(ctx, scan_ws_bytes(scan->rings, Ws));
  if (st != LSG_OK) return st;
  const int tile = ctx_tile(ctx, &scan->rings, &Ws, 1);
  KArgs a;
  memset(&a, 0, sizeof(a));
  a.one = make_desc(scan, params, out, Ws);
  set_tiles(a.one, tile, 0);
  carve_ws(a.one, static_cast<char*>(ctx->ws));
  a.ntiles = a.one.tiles_r * a.one.tiles_c;
  a.nscans = 1;
  a.err = ctx->d_err;
  return run_pass(a, tile, true, cs);
}

lsg_status lsg_label_from_mask(lsg_ctx* ctx, int32_t H, int32_t W, int32_t s, int32_t wrap,
                               const uint8_t* meshbits, const uint8_t* valid, int32_t* labels,
                               int32_t* nseg, lsg_stream stream) {
  if (!ctx || !nseg) return LSG_E_ARG;
  if (H < 0 || W < 0 || H > LSG_MAX_RINGS || W > LSG_MAX_COLS) return LSG_E_SHAPE;
  if ((int64_t)H * W > (int64_t)LSG_MAX_POINTS) return LSG_E_SHAPE;
  if (s < 1) return LSG_E_ARG;
  DeviceGuard g(ctx->device);
  cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
  if (H == 0 || W == 0) return cuda_status(cudaMemsetAsync(nseg, 0, sizeof(int32_t), cs));
  if (!meshbits || !labels || (s > 1 && !valid)) return LSG_E_ARG;
  const int Ws = (W + s - 1) / s;
  lsg_status st = reserve(ctx, scan_ws_bytes(H, Ws));
  if (st != LSG_OK) return st;
  KArgs a;
  memset(&a, 0, sizeof(a));
  ScanDesc& d = a.one;
  d.H = H;
  d.W = W;
  d.Ws = Ws;
  d.s = s;
  d.wrap = (wrap && Ws >= 3) ? 1 : 0;
  d.mb = const_cast<uint8_t*>(meshbits);
  d.valid = valid;
  d.labels = labels;
  d.nseg = nseg;
  const int tile = ctx_tile(ctx, &H, &Ws, 1);
  set_tiles(d, tile, 0);
  carve_ws(d, static_cast<char*>(ctx->ws));
  a.ntiles = d.tiles_r * d.tiles_c;
  a.nscans = 1;
  a.err = ctx->d_err;
  a.s1_only = s == 1;
  // no elevations: the ring order is the identity and only nseg is reset
  cudaError_t e = cudaMemsetAsync(nseg, 0, sizeof(int32_t), cs);
  if (e == cudaSuccess) e = launch_tile_ccl(tile, a, cs);
  if (e == cudaSuccess) e = launch_merge(tile, a, cs, true);
  if (e == cudaSuccess) e = launch_flatten(tile, a, cs, true);
  return cuda_status(e);
}

lsg_status lsg_selftest_wait_timeout(lsg_ctx* ctx) {
  if (!ctx) return LSG_E_ARG;
  DeviceGuard g(ctx->device);
  int32_t* cnt = nullptr;
  cudaError_t e = cudaMalloc(&cnt, sizeof(int32_t));
  if (e != cudaSuccess) return cuda_status(e);
  e = cudaMemset(cnt, 0, sizeof(int32_t));
  if (e == cudaSuccess) e = launch_wait_probe(cnt, ctx->d_err, 4096u, nullptr);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  cudaFree(cnt);
  if (e != cudaSuccess) return cuda_status(e);
  const lsg_status st = lsg_get_error(ctx);
  if (st == LSG_E_TIMEOUT) return LSG_OK;
  return st == LSG_OK ? LSG_E_DEVICE : st;
}

lsg_status lsg_get_error(lsg_ctx* ctx) {
  if (!ctx) return LSG_E_ARG;
  DeviceGuard g(ctx->device);
  int32_t v = 0;
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_status(e);
  e = cudaMemcpy(&v, ctx->d_err, sizeof(v), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_status(e);
  cudaMemset(ctx->d_err, 0, sizeof(int32_t));
  if (v & DERR_TIMEOUT) return LSG_E_TIMEOUT;
  if (v) return LSG_E_DEVICE;
  return LSG_OK;
}

// ---------------------------------------------------------------------------
// dynamic batch (a different set of scans on every call)
// ---------------------------------------------------------------------------
static lsg_status grow_stage(lsg_ctx* ctx, DynStage& sg, size_t need) {
  if (sg.cap >= need) return LSG_OK;
  const size_t cap = align_up(need * 2, 1 << 16);
  if (ctx->budget && ctx->used - sg.cap + cap > ctx->budget) return LSG_E_BUDGET;
  if (sg.copied) {
    cudaError_t e = cudaEventSynchronize(sg.copied);
    if (e != cudaSuccess) return cuda_status(e);
  }
  if (sg.host) cudaFreeHost(sg.host);
  if (sg.dev) cudaFree(sg.dev);
  ctx->used -= sg.cap;
  sg.host = sg.dev = nullptr;
  sg.cap = 0;
  cudaError_t e;
  if ((e = cudaMallocHost(&sg.host, cap)) != cudaSuccess) return cuda_status(e);
  if ((e = cudaMalloc(&sg.dev, cap)) != cudaSuccess) return cuda_status(e);
  sg.cap = cap;
  ctx->used += cap;
  return LSG_OK;
}

lsg_status lsg_reserve(lsg_ctx* ctx, size_t workspace_bytes, int32_t max_scans, int32_t max_tiles) {
  if (!ctx || max_scans < 0 || max_tiles < 0) return LSG_E_ARG;
  DeviceGuard g(ctx->device);
  lsg_status st = reserve(ctx, workspace_bytes > 0 ? workspace_bytes : 256);
  const size_t need = align_up(sizeof(ScanDesc) * (size_t)max_scans, 256) + sizeof(int32_t) * (size_t)max_tiles;
  for (int k = 0; k < 2 && st == LSG_OK; ++k) st = grow_stage(ctx, ctx->stage[k], need);
  return st;
}

static lsg_status batch_launch(lsg_ctx* ctx, int32_t n, const lsg_scan* scans, const lsg_params* params,
                               const lsg_out* outs, const lsg_host_io* io, lsg_stream stream);

lsg_status lsg_batch_launch(lsg_ctx* ctx, int32_t n, const lsg_scan* scans, const lsg_params* params,
                            const lsg_out* outs, lsg_stream stream) {
  return batch_launch(ctx, n, scans, params, outs, nullptr, stream);
}

lsg_status lsg_batch_launch_io(lsg_ctx* ctx, int32_t n, const lsg_scan* scans, const lsg_params* params,
                               const lsg_out* outs, const lsg_host_io* io, lsg_stream stream) {
  if (!io) return LSG_E_ARG;
  return batch_launch(ctx, n, scans, params, outs, io, stream);
}

// Host -> device copies of one scan's inputs (x,y,z,r or ranges, and the
// elevations) from its host buffers.
static cudaError_t copy_in(const lsg_scan& sc, const lsg_host_io& io, cudaStream_t cs) {
  const size_t pts = (size_t)sc.rings * sc.cols;
  if (!pts) return cudaSuccess;
  cudaError_t e = sc.xyzr ? cudaMemcpyAsync(const_cast<float*>(sc.xyzr), io.xyzr, pts * 16, cudaMemcpyHostToDevice, cs)
                          : cudaMemcpyAsync(const_cast<float*>(sc.range), io.xyzr, pts * 4, cudaMemcpyHostToDevice, cs);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(const_cast<float*>(sc.elevation), io.elevation, sizeof(float) * sc.rings,
                        cudaMemcpyHostToDevice, cs);
  return e;
}

// Device -> host copies of the results io lists.
static cudaError_t copy_out(const lsg_scan& sc, int Ws, const lsg_out& o, const lsg_host_io& io, cudaStream_t cs) {
  const size_t pts = (size_t)sc.rings * sc.cols, nv = (size_t)sc.rings * Ws;
  cudaError_t e = cudaSuccess;
  if (io.nseg) e = cudaMemcpyAsync(io.nseg, o.nseg, sizeof(int32_t), cudaMemcpyDeviceToHost, cs);
  if (e == cudaSuccess && io.labels && pts) e = cudaMemcpyAsync(io.labels, o.labels, pts * 4, cudaMemcpyDeviceToHost, cs);
  if (e == cudaSuccess && io.meshbits && nv) e = cudaMemcpyAsync(io.meshbits, o.meshbits, nv, cudaMemcpyDeviceToHost, cs);
  if (e == cudaSuccess && io.normals && nv)
    e = cudaMemcpyAsync(io.normals, o.normals, nv * 12, cudaMemcpyDeviceToHost, cs);
  return e;
}

// A batch of one: the single-scan pass (descriptor passed by value, kernels
// as programmatic dependents), with the host copies when io is given.
static lsg_status launch_one(lsg_ctx* ctx, const lsg_scan* sc, const lsg_params* p, const lsg_out* o,
                             const lsg_host_io* io, int Ws, int tile, lsg_stream stream) {
  DeviceGuard g(ctx->device);
  cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
  if (io) {
    if (sc->rings > 0 && sc->cols > 0 && (!io->xyzr || !io->elevation)) return LSG_E_ARG;
    const cudaError_t e = copy_in(*sc, *io, cs);
    if (e != cudaSuccess) return cuda_status(e);
  }
  lsg_status st = LSG_OK;
  if (sc->rings == 0 || sc->cols == 0) {
    st = cuda_status(cudaMemsetAsync(o->nseg, 0, sizeof(int32_t), cs));
  } else {
    st = reserve(ctx, scan_ws_bytes(sc->rings, Ws));
    if (st != LSG_OK) return st;
    KArgs a;
    memset(&a, 0, sizeof(a));
    a.one = make_desc(sc, p, o, Ws);
    set_tiles(a.one, tile, 0);
    carve_ws(a.one, static_cast<char*>(ctx->ws));
    a.ntiles = a.one.tiles_r * a.one.tiles_c;
    a.nscans = 1;
    a.err = ctx->d_err;
    st = run_pass(a, tile, true, cs);
  }
  if (st == LSG_OK && io) st = cuda_status(copy_out(*sc, Ws, *o, *io, cs));
  return st;
}

static lsg_status batch_launch(lsg_ctx* ctx, int32_t n, const lsg_scan* scans, const lsg_params* params,
                               const lsg_out* outs, const lsg_host_io* io, lsg_stream stream) {
  if (!ctx || n < 1 || !scans || !params || !outs) return LSG_E_ARG;
  std::vector<int> Ws(n), Hs(n);
  size_t ws_total = 0;
  int64_t ntiles = 0;
  for (int b = 0; b < n; ++b) {
    lsg_status st = check_scan(&scans[b], &params[b], &outs[b], &Ws[b]);
    if (st != LSG_OK) return st;
    ws_total += scan_ws_bytes(scans[b].rings, Ws[b]);
    Hs[b] = scans[b].cols > 0 ? scans[b].rings : 0;
  }
  const int tile = ctx_tile(ctx, Hs.data(), Ws.data(), n);
  if (n == 1) return launch_one(ctx, scans, params, outs, io, Ws[0], tile, stream);
  const TileShape ts = tile_shape(tile);
  for (int b = 0; b < n; ++b)
    if (Hs[b] > 0 && Ws[b] > 0)
      ntiles += (int64_t)((Hs[b] + ts.rows - 1) / ts.rows) * ((Ws[b] + ts.cols - 1) / ts.cols);
  if (ntiles > INT32_MAX) return LSG_E_SHAPE;
  DeviceGuard g(ctx->device);
  cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
  lsg_status st = reserve(ctx, ws_total > 0 ? ws_total : 256);
  if (st != LSG_OK) return st;
  // descriptor table + tile table in one staging buffer
  const size_t desc_bytes = align_up(sizeof(ScanDesc) * n, 256);
  const size_t need = desc_bytes + sizeof(int32_t) * (size_t)(ntiles > 0 ? ntiles : 1);
  DynStage& sg = ctx->stage[ctx->next_stage];
  ctx->next_stage ^= 1;
  cudaError_t e = cudaSuccess;
  if (sg.copied) e = cudaEventSynchronize(sg.copied);  // the previous copy out of it is done
  if (e != cudaSuccess) return cuda_status(e);
  st = grow_stage(ctx, sg, need);
  if (st != LSG_OK) return st;
  if (!sg.copied && (e = cudaEventCreateWithFlags(&sg.copied, cudaEventDisableTiming)) != cudaSuccess)
    return cuda_status(e);
  if (io) {
    // inputs host -> device, on the same stream ahead of the pass
    for (int b = 0; b < n; ++b)
      if (scans[b].rings > 0 && scans[b].cols > 0 && (!io[b].xyzr || !io[b].elevation)) return LSG_E_ARG;
    for (int b = 0; b < n && e == cudaSuccess; ++b) e = copy_in(scans[b], io[b], cs);
    if (e != cudaSuccess) return cuda_status(e);
  }
  ScanDesc* hd = static_cast<ScanDesc*>(sg.host);
  int32_t* htile = reinterpret_cast<int32_t*>(static_cast<char*>(sg.host) + desc_bytes);
  char* base = static_cast<char*>(ctx->ws);
  int32_t t0 = 0;
  for (int b = 0; b < n; ++b) {
    ScanDesc d = make_desc(&scans[b], &params[b], &outs[b], Ws[b]);
    carve_ws(d, base);
    base += scan_ws_bytes(d.H, d.Ws);
    set_tiles(d, tile, t0);
    const int nt = (d.H && d.W) ? d.tiles_r * d.tiles_c : 0;
    for (int k = 0; k < nt; ++k) htile[t0 + k] = b;
    t0 += nt;
    hd[b] = d;
  }
  e = cudaMemcpyAsync(sg.dev, sg.host, desc_bytes + sizeof(int32_t) * (size_t)t0, cudaMemcpyHostToDevice, cs);
  if (e == cudaSuccess) e = cudaEventRecord(sg.copied, cs);
  if (e != cudaSuccess) return cuda_status(e);
  KArgs a;
  memset(&a, 0, sizeof(a));
  a.scans = static_cast<const ScanDesc*>(sg.dev);
  a.tile_scan = reinterpret_cast<const int32_t*>(static_cast<char*>(sg.dev) + desc_bytes);
  a.ntiles = t0;
  a.nscans = n;
  a.err = ctx->d_err;
  a.s1_only = 1;
  for (int b = 0; b < n; ++b)
    if (params[b].subsample != 1) a.s1_only = 0;
  e = launch_prep(a, cs);
  if (e == cudaSuccess && t0 > 0) e = launch_tile(tile, a, cs, true);
  if (e == cudaSuccess && t0 > 0) e = launch_merge(tile, a, cs, true);
  if (e == cudaSuccess && t0 > 0) e = launch_flatten(tile, a, cs, true);
  if (io) {
    // results device -> host, behind the pass
    for (int b = 0; b < n && e == cudaSuccess; ++b) e = copy_out(scans[b], Ws[b], outs[b], io[b], cs);
  }
  return cuda_status(e);
}

// ---------------------------------------------------------------------------
// batched path
// ---------------------------------------------------------------------------
static lsg_status plan_layout(lsg_plan* pl, int tile) {
  // tile fields of every descriptor + the tile -> scan table, on the host
  std::vector<int32_t> ts;
  int32_t t0 = 0;
  for (int b = 0; b < pl->n; ++b) {
    ScanDesc& d = pl->host_desc[b];
    set_tiles(d, tile, t0);
    const int nt = (d.H && d.W) ? d.tiles_r * d.tiles_c : 0;
    for (int k = 0; k < nt; ++k) ts.push_back(b);
    t0 += nt;
  }
  pl->ntiles = t0;
  if (pl->d_tile_scan) cudaFree(pl->d_tile_scan);
  pl->d_tile_scan = nullptr;
  cudaError_t e = cudaSuccess;
  if (t0 > 0) {
    e = cudaMalloc(&pl->d_tile_scan, sizeof(int32_t) * t0);
    if (e == cudaSuccess)
      e = cudaMemcpy(pl->d_tile_scan, ts.data(), sizeof(int32_t) * t0, cudaMemcpyHostToDevice);
  }
  // fused schedule: every scan's ring order first, then the tiles of all
  // scans in order, with a scan's border merges placed LAG items after its
  // last tile and its labels LAG items after its last merge.  LAG exceeds the
  // number of CTAs that run at once, so an item rarely finds its inputs
  // unfinished, while a scan's labels still follow its tiles closely enough
  // for their data to be in L2.
  const size_t LAG = 2048;
  std::vector<int2> items;
  items.reserve(pl->n + 3 * (size_t)t0);
  for (int b = 0; b < pl->n; ++b) items.push_back(make_int2(PH_PREP << 28 | b, 0));
  struct Due {
    size_t at;
    int ph, b;
  };
  std::vector<Due> due;  // FIFO, `at` non-decreasing per phase
  size_t head = 0;
  auto tiles_of = [&](int b) {
    const ScanDesc& d = pl->host_desc[b];
    return (d.H && d.W) ? d.tiles_r * d.tiles_c : 0;
  };
  auto emit_due = [&](bool all) {
    while (head < due.size() && (all || due[head].at <= items.size())) {
      const Due x = due[head++];
      for (int k = 0; k < tiles_of(x.b); ++k) items.push_back(make_int2(x.ph << 28 | x.b, k));
      if (x.ph == PH_MERGE) due.push_back(Due{items.size() + LAG, PH_FLAT, x.b});
    }
  };
  for (int b = 0; b < pl->n; ++b) {
    for (int k = 0; k < tiles_of(b); ++k) {
      emit_due(false);
      items.push_back(make_int2(PH_TILE << 28 | b, k));
    }
    if (tiles_of(b) > 0) due.push_back(Due{items.size() + LAG, PH_MERGE, b});
  }
  emit_due(true);
  pl->nitems = (int32_t)items.size();
  if (pl->d_items) cudaFree(pl->d_items);
  pl->d_items = nullptr;
  if (e == cudaSuccess) e = cudaMalloc(&pl->d_items, sizeof(int2) * items.size());
  if (e == cudaSuccess)
    e = cudaMemcpy(pl->d_items, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !pl->d_counters) e = cudaMalloc(&pl->d_counters, sizeof(int32_t) * (1 + 3 * (size_t)pl->n));
  if (e == cudaSuccess)
    e = cudaMemcpy(pl->d_desc, pl->host_desc.data(), sizeof(ScanDesc) * pl->n, cudaMemcpyHostToDevice);
  pl->tile = tile;
  return cuda_status(e);
}

// Scan groups of the overlapped schedule.
constexpr int kGroups = 4;

namespace {

// One host<->device copy of a run; consecutive copies whose source and
// destination both continue the previous one are merged.
struct Copy {
  char* dst;
  const char* src;
  size_t bytes;
};

void add_copy(std::vector<Copy>& v, void* dst, const void* src, size_t bytes) {
  if (!bytes || !dst || !src) return;
  char* d = static_cast<char*>(dst);
  const char* s = static_cast<const char*>(src);
  if (!v.empty() && v.back().dst + v.back().bytes == d && v.back().src + v.back().bytes == s) {
    v.back().bytes += bytes;
    return;
  }
  v.push_back(Copy{d, s, bytes});
}

cudaError_t issue(const std::vector<Copy>& v, cudaMemcpyKind kind, cudaStream_t st, size_t& total) {
  for (const Copy& c : v) {
    const cudaError_t e = cudaMemcpyAsync(c.dst, c.src, c.bytes, kind, st);
    if (e != cudaSuccess) return e;
    total += c.bytes;
  }
  return cudaSuccess;
}

// Chunk boundaries: runs of consecutive scans whose point counts grow by
// kChunkGrowth from one chunk to the next.  The outputs cannot start back
// before the first chunk's inputs have landed and its pass has run, so a
// small first chunk starts the device -> host direction early; the growth
// stays below the ratio at which a chunk's inputs would take longer to land
// than the chunk before it takes to go back (the outputs are 17 bytes a
// point against 16 in, and the link is slower that way), so the outputs
// never wait once started.
constexpr double kChunkGrowth = 1.1;

std::vector<int> chunk_bounds(const lsg_plan* pl) {
  std::vector<int64_t> pts(pl->n + 1, 0);
  for (int b = 0; b < pl->n; ++b) pts[b + 1] = pts[b] + (int64_t)pl->dev_in[b].rings * pl->dev_in[b].cols;
  const int C = std::max(1, std::min(pl->chunks, pl->n));
  std::vector<double> share(C + 1, 0.0);  // cumulative share of the points after c chunks
  for (int c = 0; c < C; ++c) share[c + 1] = share[c] + std::pow(kChunkGrowth, c);
  std::vector<int> bounds{0};
  for (int c = 1; c < C; ++c) {
    const int64_t target = (int64_t)((double)pts[pl->n] * (share[c] / share[C]));
    int b = (int)(std::lower_bound(pts.begin(), pts.end(), target) - pts.begin());
    b = std::max(bounds.back() + 1, std::min(b, pl->n - (C - c)));
    bounds.push_back(b);
  }
  bounds.push_back(pl->n);
  return bounds;
}

}  // namespace

// Do the plan's scans [b0, b1) all have s = 1?
static int plan_s1_only(const lsg_plan* pl, int b0, int b1) {
  for (int b = b0; b < b1; ++b)
    if (pl->host_desc[b].s != 1) return 0;
  return 1;
}

// Capture of a host-buffer plan: per chunk of scans, the inputs go host ->
// device on one branch, the chunk's pass (ring order, tiles, border joins,
// labels) runs on a second once they have landed, and its outputs go device
// -> host on a third once the pass is done, so that the copies of the
// neighbouring chunks, in both directions, run under each chunk's pass.  The
// small copies (elevations in, segment counts out) go once for the whole
// batch, ahead of the first chunk and after the last: every copy in the graph
// costs a few microseconds of its own.
static cudaError_t capture_io(lsg_plan* pl, cudaStream_t cs, int& launches) {
  cudaStream_t s_in = nullptr, s_run = nullptr, s_out = nullptr;
  std::vector<cudaEvent_t> evs;
  auto new_event = [&](cudaEvent_t* ev) {
    const cudaError_t e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    if (e == cudaSuccess) evs.push_back(*ev);
    return e;
  };
  cudaError_t e = cudaStreamCreateWithFlags(&s_in, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s_run, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s_out, cudaStreamNonBlocking);
  cudaEvent_t fork = nullptr;
  if (e == cudaSuccess) e = new_event(&fork);
  if (e == cudaSuccess) e = cudaEventRecord(fork, cs);
  for (cudaStream_t st : {s_in, s_run, s_out})
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, fork, 0);
  const std::vector<int> bounds = chunk_bounds(pl);
  size_t h2d = 0, d2h = 0;
  launches = 0;
  std::vector<Copy> elev_all, cnt_all;
  for (int b = 0; b < pl->n; ++b) {
    const ScanDesc& d = pl->host_desc[b];
    if (d.H > 0 && d.W > 0)
      add_copy(elev_all, const_cast<float*>(pl->dev_in[b].elevation), pl->io[b].elevation, sizeof(float) * d.H);
    add_copy(cnt_all, pl->io[b].nseg, pl->dev_out[b].nseg, sizeof(int32_t));
  }
  if (e == cudaSuccess) e = issue(elev_all, cudaMemcpyHostToDevice, s_in, h2d);
  for (size_t c = 0; c + 1 < bounds.size() && e == cudaSuccess; ++c) {
    const int b0 = bounds[c], b1 = bounds[c + 1];
    std::vector<Copy> in, lab, mb, nrm;
    for (int b = b0; b < b1; ++b) {
      const lsg_scan& sc = pl->dev_in[b];
      const lsg_host_io& io = pl->io[b];
      const ScanDesc& d = pl->host_desc[b];
      const size_t pts = (size_t)d.H * d.W, nv = (size_t)d.H * d.Ws;
      if (pts) {
        if (sc.xyzr) add_copy(in, const_cast<float*>(sc.xyzr), io.xyzr, pts * 16);
        else add_copy(in, const_cast<float*>(sc.range), io.xyzr, pts * 4);
        add_copy(lab, io.labels, pl->dev_out[b].labels, pts * 4);
        add_copy(mb, io.meshbits, pl->dev_out[b].meshbits, nv);
        add_copy(nrm, io.normals, pl->dev_out[b].normals, nv * 12);
      }
    }
    cudaEvent_t ev_in = nullptr, ev_run = nullptr;
    if (e == cudaSuccess) e = new_event(&ev_in);
    if (e == cudaSuccess) e = new_event(&ev_run);
    if (e == cudaSuccess) e = issue(in, cudaMemcpyHostToDevice, s_in, h2d);
    if (e == cudaSuccess) e = cudaEventRecord(ev_in, s_in);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s_run, ev_in, 0);
    // the chunk's pass: ring order over its scans, then its tiles
    KArgs a;
    memset(&a, 0, sizeof(a));
    a.scans = pl->d_desc + b0;
    a.nscans = b1 - b0;
    a.err = pl->ctx->d_err;
    a.s1_only = plan_s1_only(pl, b0, b1);
    if (e == cudaSuccess) e = launch_prep(a, s_run);
    ++launches;
    const int32_t t0 = pl->host_desc[b0].tile0, t1 = b1 < pl->n ? pl->host_desc[b1].tile0 : pl->ntiles;
    if (t1 > t0) {
      a.scans = pl->d_desc;
      a.tile_scan = pl->d_tile_scan;
      a.nscans = pl->n;
      a.tile_base = t0;
      a.ntiles = t1 - t0;
      if (e == cudaSuccess) e = launch_tile(pl->tile, a, s_run);
      if (e == cudaSuccess) e = launch_merge(pl->tile, a, s_run);
      if (e == cudaSuccess) e = launch_flatten(pl->tile, a, s_run);
      launches += 3;
    }
    if (e == cudaSuccess) e = cudaEventRecord(ev_run, s_run);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s_out, ev_run, 0);
    if (e == cudaSuccess) e = issue(lab, cudaMemcpyDeviceToHost, s_out, d2h);
    if (e == cudaSuccess) e = issue(mb, cudaMemcpyDeviceToHost, s_out, d2h);
    if (e == cudaSuccess) e = issue(nrm, cudaMemcpyDeviceToHost, s_out, d2h);
  }
  if (e == cudaSuccess) e = issue(cnt_all, cudaMemcpyDeviceToHost, s_out, d2h);
  for (cudaStream_t st : {s_in, s_run, s_out}) {
    cudaEvent_t join = nullptr;
    if (e == cudaSuccess) e = new_event(&join);
    if (e == cudaSuccess) e = cudaEventRecord(join, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, join, 0);
  }
  pl->h2d_bytes = h2d;
  pl->d2h_bytes = d2h;
  for (cudaEvent_t ev : evs) cudaEventDestroy(ev);
  for (cudaStream_t st : {s_in, s_run, s_out})
    if (st) cudaStreamDestroy(st);
  return e;
}

static lsg_status plan_capture(lsg_plan* pl) {
  if (pl->exec) cudaGraphExecDestroy(pl->exec);
  if (pl->graph) cudaGraphDestroy(pl->graph);
  pl->exec = nullptr;
  pl->graph = nullptr;
  cudaStream_t cs;
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_status(e);
  KArgs a;
  memset(&a, 0, sizeof(a));
  a.scans = pl->d_desc;
  a.tile_scan = pl->d_tile_scan;
  a.ntiles = pl->ntiles;
  a.nscans = pl->n;
  a.err = pl->ctx->d_err;
  a.s1_only = plan_s1_only(pl, 0, pl->n);
  for (int k = 0; k < 5 && e == cudaSuccess; ++k)
    if (!pl->ev[k]) e = cudaEventCreate(&pl->ev[k]);
  // side streams and fork / join events of the grouped schedule
  cudaStream_t side[kGroups] = {};
  cudaEvent_t fork[kGroups] = {}, join[kGroups] = {};
  bool joined[kGroups] = {};
  if (pl->fused == 2) {
    for (int g = 0; g < kGroups && e == cudaSuccess; ++g) {
      e = cudaStreamCreateWithFlags(&side[g], cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&fork[g], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&join[g], cudaEventDisableTiming);
    }
  }
  if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  lsg_status st = LSG_OK;
  int launches = 0;
  if (e == cudaSuccess) {
    // scans with no points only get their counter cleared (by k_prep, which
    // runs one block per scan); the tile kernels see only non-empty scans.
    // Event-record nodes between the phases give per-kernel device times.
    cudaError_t le = cudaEventRecordWithFlags(pl->ev[0], cs, cudaEventRecordExternal);
    if (pl->chunks > 0) {
      // host-buffer plan: the copies and passes of every chunk; the phase
      // events give the whole run's time
      if (le == cudaSuccess) le = capture_io(pl, cs, launches);
      for (int k = 1; k < 5 && le == cudaSuccess; ++k)
        le = cudaEventRecordWithFlags(pl->ev[k], cs, cudaEventRecordExternal);
    } else if (pl->fused == 2) {
      // scan groups of about equal tile counts, each a chain of the tile,
      // merge and label kernels on its own branch of the graph: as one
      // group's tiles finish, its latency-bound merge and labels run beside
      // the other groups' tile work
      if (le == cudaSuccess) le = launch_prep(a, cs);
      launches = 1;
      if (le == cudaSuccess) le = cudaEventRecordWithFlags(pl->ev[1], cs, cudaEventRecordExternal);
      if (le == cudaSuccess) le = cudaEventRecord(fork[0], cs);
      int b0 = 0;
      for (int g = 0; g < kGroups && le == cudaSuccess; ++g) {
        const int32_t t0 = pl->host_desc[b0].tile0;
        const int32_t target = (int32_t)(((int64_t)pl->ntiles * (g + 1)) / kGroups);
        int b1 = b0;
        while (b1 < pl->n && (pl->host_desc[b1].tile0 < target || b1 == b0)) ++b1;
        if (g == kGroups - 1) b1 = pl->n;
        const int32_t t1 = b1 < pl->n ? pl->host_desc[b1].tile0 : pl->ntiles;
        b0 = b1;
        if (t1 <= t0) continue;
        KArgs ag = a;
        ag.tile_base = t0;
        ag.ntiles = t1 - t0;
        joined[g] = true;
        le = cudaStreamWaitEvent(side[g], fork[0], 0);
        if (le == cudaSuccess) le = launch_tile(pl->tile, ag, side[g]);
        if (le == cudaSuccess) le = launch_merge(pl->tile, ag, side[g]);
        if (le == cudaSuccess) le = launch_flatten(pl->tile, ag, side[g]);
        launches += 3;
        if (le == cudaSuccess) le = cudaEventRecord(join[g], side[g]);
        if (b0 >= pl->n) break;
      }
      for (int g = 0; g < kGroups && le == cudaSuccess; ++g)
        if (joined[g]) le = cudaStreamWaitEvent(cs, join[g], 0);
      if (le == cudaSuccess) le = cudaEventRecordWithFlags(pl->ev[2], cs, cudaEventRecordExternal);
      if (le == cudaSuccess) le = cudaEventRecordWithFlags(pl->ev[3], cs, cudaEventRecordExternal);
      if (le == cudaSuccess) le = cudaEventRecordWithFlags(pl->ev[4], cs, cudaEventRecordExternal);
    } else if (pl->fused) {
      // counters reset, then the single persistent launch
      FusedArgs f;
      f.scans = pl->d_desc;
      f.items = pl->d_items;
      f.nitems = pl->nitems;
      f.nscans = pl->n;
      f.counters = pl->d_counters;
      f.err = pl->ctx->d_err;
      f.s1_only = plan_s1_only(pl, 0, pl->n);
      if (le == cudaSuccess) le = cudaMemsetAsync(pl->d_counters, 0, sizeof(int32_t) * (1 + 3 * (size_t)pl->n), cs);
      if (le == cudaSuccess) le = cudaEventRecordWithFlags(pl->ev[1], cs, cudaEventRecordExternal);
      if (le == cudaSuccess) le = launch_fused(pl->tile, f, cs);
      launches = 1;
      if (le == cudaSuccess) le = cudaEventRecordWithFlags(pl->ev[2], cs, cudaEventRecordExternal);
      if (le == cudaSuccess) le = cudaEventRecordWithFlags(pl->ev[3], cs, cudaEventRecordExternal);
      if (le == cudaSuccess) le = cudaEventRecordWithFlags(pl->ev[4], cs, cudaEventRecordExternal);
    } else {
      if (le == cudaSuccess) le = launch_prep(a, cs);
      if (le == cudaSuccess) le = cudaEventRecordWithFlags(pl->ev[1], cs, cudaEventRecordExternal);
      if (le == cudaSuccess && pl->ntiles > 0) le = launch_tile(pl->tile, a, cs);
      if (le == cudaSuccess) le = cudaEventRecordWithFlags(pl->ev[2], cs, cudaEventRecordExternal);
      if (le == cudaSuccess && pl->ntiles > 0) le = launch_merge(pl->tile, a, cs);
      if (le == cudaSuccess) le = cudaEventRecordWithFlags(pl->ev[3], cs, cudaEventRecordExternal);
      if (le == cudaSuccess && pl->ntiles > 0) le = launch_flatten(pl->tile, a, cs);
      if (le == cudaSuccess) le = cudaEventRecordWithFlags(pl->ev[4], cs, cudaEventRecordExternal);
      launches = pl->ntiles > 0 ? 4 : 1;
    }
    e = cudaStreamEndCapture(cs, &pl->graph);
    if (le != cudaSuccess) e = le;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&pl->exec, pl->graph, 0);
  st = cuda_status(e);
  pl->launches = st == LSG_OK ? launches : 0;
  for (int g = 0; g < kGroups; ++g) {
    if (side[g]) cudaStreamDestroy(side[g]);
    if (fork[g]) cudaEventDestroy(fork[g]);
    if (join[g]) cudaEventDestroy(join[g]);
  }
  cudaStreamDestroy(cs);
  return st;
}

static lsg_status plan_create(lsg_ctx* ctx, int32_t n, const lsg_scan* scans, const lsg_params* params,
                              const lsg_out* outs, const lsg_host_io* io, int32_t chunks, int tile, lsg_plan** plan) {
  if (!ctx || !plan || n < 1 || !scans || !params || !outs) return LSG_E_ARG;
  *plan = nullptr;
  if (tile == LSG_TILE_AUTO) tile = ctx->tile;
  if (tile != LSG_TILE_AUTO && (tile < 0 || tile >= LSG_TILE_COUNT)) return LSG_E_ARG;
  std::vector<int> Ws(n), Hs(n);
  size_t ws_total = 0;
  for (int b = 0; b < n; ++b) {
    lsg_status st = check_scan(&scans[b], &params[b], &outs[b], &Ws[b]);
    if (st != LSG_OK) return st;
    ws_total += scan_ws_bytes(scans[b].rings, Ws[b]);
    Hs[b] = scans[b].cols > 0 ? scans[b].rings : 0;
  }
  if (tile == LSG_TILE_AUTO) tile = pick_tile(Hs.data(), Ws.data(), n, ctx->sms);
  // bound on the tile table over every tile shape (at least 2 rows x 120 columns)
  size_t tiles_max = 0;
  for (int b = 0; b < n; ++b)
    tiles_max += (size_t)(scans[b].rings / 2 + 1) * (Ws[b] / 120 + 1);
  // workspace, descriptors, tile table, fused schedule (scan + 3 items per tile) and counters
  const size_t bytes = ws_total + align_up(sizeof(ScanDesc) * n, 256) + sizeof(int32_t) * tiles_max +
                       sizeof(int2) * (n + 3 * tiles_max) + sizeof(int32_t) * (1 + 3 * (size_t)n);
  if (ctx->budget && ctx->used + bytes > ctx->budget) return LSG_E_BUDGET;
  DeviceGuard g(ctx->device);
  lsg_plan* pl = new (std::nothrow) lsg_plan();
  if (!pl) return LSG_E_OOM;
  pl->ctx = ctx;
  pl->n = n;
  pl->host_desc.resize(n);
  cudaError_t e = cudaMalloc(&pl->ws, ws_total > 0 ? ws_total : 256);
  if (e == cudaSuccess) e = cudaMalloc(&pl->d_desc, sizeof(ScanDesc) * n);
  if (e != cudaSuccess) {
    if (pl->ws) cudaFree(pl->ws);
    delete pl;
    return cuda_status(e);
  }
  char* base = static_cast<char*>(pl->ws);
  for (int b = 0; b < n; ++b) {
    ScanDesc d = make_desc(&scans[b], &params[b], &outs[b], Ws[b]);
    carve_ws(d, base);
    base += scan_ws_bytes(d.H, d.Ws);
    pl->host_desc[b] = d;
  }
  pl->bytes = bytes;
  ctx->used += bytes;
  if (io) {
    pl->chunks = chunks;
    pl->fused = 0;
    pl->dev_in.assign(scans, scans + n);
    pl->dev_out.assign(outs, outs + n);
    pl->io.assign(io, io + n);
  }
  lsg_status st = plan_layout(pl, tile);
  if (st == LSG_OK) st = plan_capture(pl);
  if (st != LSG_OK) {
    lsg_plan_destroy(pl);
    return st;
  }
  *plan = pl;
  return LSG_OK;
}

lsg_status lsg_batch_plan(lsg_ctx* ctx, int32_t n, const lsg_scan* scans, const lsg_params* params,
                          const lsg_out* outs, int tile, lsg_plan** plan) {
  return plan_create(ctx, n, scans, params, outs, nullptr, 0, tile, plan);
}

// Host memory the copies of a host-buffer plan may use: page-locked (or
// registered) memory, so that they run asynchronously inside the graph.
static bool pinned_host(const void* p) {
  if (!p) return true;  // optional outputs may be absent
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeHost;
}

lsg_status lsg_batch_plan_io(lsg_ctx* ctx, int32_t n, const lsg_scan* scans, const lsg_params* params,
                             const lsg_out* outs, const lsg_host_io* io, int32_t chunks, int tile, lsg_plan** plan) {
  if (!ctx || !plan || !io || n < 1 || !scans || chunks < 1) return LSG_E_ARG;
  *plan = nullptr;
  DeviceGuard g(ctx->device);
  for (int b = 0; b < n; ++b) {
    const bool empty = scans[b].rings == 0 || scans[b].cols == 0;
    if (!empty && (!io[b].xyzr || !io[b].elevation)) return LSG_E_ARG;
    if (!pinned_host(io[b].xyzr) || !pinned_host(io[b].elevation) || !pinned_host(io[b].labels) ||
        !pinned_host(io[b].nseg) || !pinned_host(io[b].meshbits) || !pinned_host(io[b].normals))
      return LSG_E_ARG;
  }
  return plan_create(ctx, n, scans, params, outs, io, chunks, tile, plan);
}

lsg_status lsg_plan_io_bytes(const lsg_plan* plan, size_t* h2d, size_t* d2h) {
  if (!plan || plan->chunks == 0) return LSG_E_ARG;
  if (h2d) *h2d = plan->h2d_bytes;
  if (d2h) *d2h = plan->d2h_bytes;
  return LSG_OK;
}

lsg_status lsg_batch_run(lsg_plan* plan, lsg_stream stream) {
  if (!plan || !plan->exec) return LSG_E_ARG;
  DeviceGuard g(plan->ctx->device);
  return cuda_status(cudaGraphLaunch(plan->exec, reinterpret_cast<cudaStream_t>(stream)));
}

int lsg_plan_tile(const lsg_plan* plan) { return plan ? plan->tile : -1; }

lsg_status lsg_plan_set_fused(lsg_plan* plan, int fused) {
  if (!plan) return LSG_E_ARG;
  if (plan->chunks > 0 && fused != 0) return LSG_E_ARG;  // host-buffer plans run phased chunks
  DeviceGuard g(plan->ctx->device);
  plan->fused = (fused == 1 || fused == 2) ? fused : 0;
  return plan_capture(plan);
}

lsg_status lsg_plan_phase_times(lsg_plan* plan, float* ms) {
  if (!plan || !ms || !plan->ev[4]) return LSG_E_ARG;
  DeviceGuard g(plan->ctx->device);
  cudaError_t e = cudaEventSynchronize(plan->ev[4]);
  for (int k = 0; k < 4 && e == cudaSuccess; ++k) e = cudaEventElapsedTime(&ms[k], plan->ev[k], plan->ev[k + 1]);
  return cuda_status(e);
}

lsg_status lsg_autotune(lsg_plan* plan, int reps, lsg_stream stream, int* best_tile, float* best_ms) {
  if (!plan || reps < 1) return LSG_E_ARG;
  DeviceGuard g(plan->ctx->device);
  cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return LSG_E_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return LSG_E_CUDA;
  }
  int best = plan->tile, best_fused = plan->fused;
  float best_t = INFINITY;
  lsg_status st = LSG_OK;
  // every tile shape under every schedule (one persistent launch, four
  // launches, scan groups on overlapping branches)
  for (int fused = plan->chunks > 0 ? 0 : 2; fused >= 0 && st == LSG_OK; --fused) {
    for (int t = 0; t < LSG_TILE_COUNT && st == LSG_OK; ++t) {
      plan->fused = fused;
      st = plan_layout(plan, t);
      if (st == LSG_OK) st = plan_capture(plan);
      if (st != LSG_OK) break;
      cudaGraphLaunch(plan->exec, cs);  // warm-up
      cudaEventRecord(e0, cs);
      for (int r = 0; r < reps; ++r) cudaGraphLaunch(plan->exec, cs);
      cudaEventRecord(e1, cs);
      cudaError_t e = cudaEventSynchronize(e1);
      if (e != cudaSuccess) {
        st = cuda_status(e);
        break;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      ms /= reps;
      if (ms < best_t) {
        best_t = ms;
        best = t;
        best_fused = fused;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  plan->fused = best_fused;
  if (st == LSG_OK) st = plan_layout(plan, best);
  if (st == LSG_OK) st = plan_capture(plan);
  if (best_tile) *best_tile = best;
  if (best_ms) *best_ms = best_t;
  return st;
}

int lsg_plan_fused(const lsg_plan* plan) { return plan ? plan->fused : -1; }

int lsg_plan_launches(const lsg_plan* plan) { return plan ? plan->launches : -1; }

lsg_status lsg_plan_destroy(lsg_plan* plan) {
  if (!plan) return LSG_E_ARG;
  DeviceGuard g(plan->ctx->device);
  cudaDeviceSynchronize();
  if (plan->exec) cudaGraphExecDestroy(plan->exec);
  if (plan->graph) cudaGraphDestroy(plan->graph);
  for (int k = 0; k < 5; ++k)
    if (plan->ev[k]) cudaEventDestroy(plan->ev[k]);
  if (plan->d_tile_scan) cudaFree(plan->d_tile_scan);
  if (plan->d_items) cudaFree(plan->d_items);
  if (plan->d_counters) cudaFree(plan->d_counters);
  if (plan->d_desc) cudaFree(plan->d_desc);
  if (plan->ws) cudaFree(plan->ws);
  plan->ctx->used -= plan->bytes;
  delete plan;
  return LSG_OK;
}


// ---------------------------------------------------------------------------
// streaming: one revolution segmented while its columns arrive
// ---------------------------------------------------------------------------
}  // extern "C"

struct lsg_spin {
  lsg_ctx* ctx = nullptr;
  int tile = 0;
  KArgs a;                    // a.one: the scan, with this spin's own workspace
  void* ws = nullptr;         // workspace, then the tile lists
  size_t bytes = 0;
  int32_t* d_cols = nullptr;  // [tiles_c][tiles_r] local tile indices by tile column: 1, 2, .., last, 0
  int cols_seen = 0;          // full-resolution columns in place
  int done_to = 1;            // tile columns [1, done_to) computed (column 0 waits for the seam)
  int merged_to = 1;          // tile columns [1, merged_to) joined to their right neighbours
  int finished = 0;
};

namespace {

// Launches k_tile or k_merge over the tile columns at positions [q0, q1) of
// the spin's column order (1, 2, .., last, 0); pdl as for launch_tile.
cudaError_t spin_launch(const lsg_spin* sp, bool merge, int q0, int q1, cudaStream_t cs, bool pdl = false) {
  if (q1 <= q0) return cudaSuccess;
  KArgs a = sp->a;
  a.tile_list = sp->d_cols + (size_t)q0 * a.one.tiles_r;
  a.ntiles = (q1 - q0) * a.one.tiles_r;
  return merge ? launch_merge(sp->tile, a, cs, pdl) : launch_tile(sp->tile, a, cs, pdl);
}

}  // namespace

extern "C" {

lsg_status lsg_spin_begin(lsg_ctx* ctx, const lsg_scan* scan, const lsg_params* params, const lsg_out* out,
                          lsg_spin** spin, lsg_stream stream) {
  if (!ctx || !spin) return LSG_E_ARG;
  *spin = nullptr;
  int Ws = 0;
  lsg_status st = check_scan(scan, params, out, &Ws);
  if (st != LSG_OK) return st;
  DeviceGuard g(ctx->device);
  cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
  lsg_spin* sp = new (std::nothrow) lsg_spin();
  if (!sp) return LSG_E_OOM;
  sp->ctx = ctx;
  sp->tile = ctx_tile(ctx, &scan->rings, &Ws, 1);
  memset(&sp->a, 0, sizeof(sp->a));
  sp->a.one = make_desc(scan, params, out, Ws);
  set_tiles(sp->a.one, sp->tile, 0);
  sp->a.nscans = 1;
  sp->a.err = ctx->d_err;
  sp->a.s1_only = params->subsample == 1;
  ScanDesc& d = sp->a.one;
  if (scan->rings == 0 || scan->cols == 0) {
    const cudaError_t e = cudaMemsetAsync(out->nseg, 0, sizeof(int32_t), cs);
    if (e != cudaSuccess) {
      delete sp;
      return cuda_status(e);
    }
    *spin = sp;
    return LSG_OK;
  }
  const size_t wsb = align_up(scan_ws_bytes(d.H, Ws), 256);
  const size_t ntiles = (size_t)d.tiles_r * d.tiles_c;
  const size_t bytes = wsb + sizeof(int32_t) * ntiles;
  if (ctx->budget && ctx->used + bytes > ctx->budget) {
    delete sp;
    return LSG_E_BUDGET;
  }
  cudaError_t e = cudaMalloc(&sp->ws, bytes);
  if (e != cudaSuccess) {
    delete sp;
    return cuda_status(e);
  }
  sp->bytes = bytes;
  ctx->used += bytes;
  carve_ws(d, static_cast<char*>(sp->ws));
  sp->d_cols = reinterpret_cast<int32_t*>(static_cast<char*>(sp->ws) + wsb);
  std::vector<int32_t> cols(ntiles);
  for (int q = 0; q < d.tiles_c; ++q) {
    const int tc = (q + 1) % d.tiles_c;  // position q holds tile column q+1; the last position column 0
    for (int tr = 0; tr < d.tiles_r; ++tr) cols[(size_t)q * d.tiles_r + tr] = tr * d.tiles_c + tc;
  }
  e = cudaMemcpy(sp->d_cols, cols.data(), sizeof(int32_t) * ntiles, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = launch_prep(sp->a, cs);
  if (e != cudaSuccess) {
    lsg_spin_destroy(sp);
    return cuda_status(e);
  }
  *spin = sp;
  return LSG_OK;
}

lsg_status lsg_spin_push(lsg_spin* sp, int32_t cols_ready, lsg_stream stream) {
  if (!sp || sp->finished) return LSG_E_ARG;
  const ScanDesc& d = sp->a.one;
  if (cols_ready < sp->cols_seen || cols_ready > d.W) return LSG_E_ARG;
  sp->cols_seen = cols_ready;
  if (d.H == 0 || d.W == 0) return LSG_OK;
  DeviceGuard g(sp->ctx->device);
  cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
  const int TC = tile_shape(sp->tile).cols;
  const int jr = (cols_ready + d.s - 1) / d.s;  // sampled columns in place
  // tile column t needs its sampled columns and two to the right (the last
  // one: the first two, around the seam, or none)
  int t_end = sp->done_to;
  while (t_end < d.tiles_c && jr >= std::min((t_end + 1) * TC + 2, d.Ws)) ++t_end;
  cudaError_t e = spin_launch(sp, false, sp->done_to - 1, t_end - 1, cs);
  if (e != cudaSuccess) return cuda_status(e);
  sp->done_to = std::max(sp->done_to, t_end);
  // tile column t joins its right neighbour once both are computed; the last
  // column (right neighbour across the seam: column 0) waits for the finish
  const int m_end = std::min(sp->done_to - 1, d.tiles_c - 1);
  e = spin_launch(sp, true, sp->merged_to - 1, m_end - 1, cs);
  if (e != cudaSuccess) return cuda_status(e);
  sp->merged_to = std::max(sp->merged_to, m_end);
  return LSG_OK;
}

lsg_status lsg_spin_finish(lsg_spin* sp, lsg_stream stream) {
  if (!sp || sp->finished) return LSG_E_ARG;
  sp->finished = 1;
  const ScanDesc& d = sp->a.one;
  sp->cols_seen = d.W;
  if (d.H == 0 || d.W == 0) return LSG_OK;
  DeviceGuard g(sp->ctx->device);
  cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
  // the remaining tile columns and column 0 (the tail of the column
  // order), then their joins, then labels: three launches, each non-empty
  // (pushes never reach column 0 or its join), the last two as programmatic
  // dependents of the one before
  cudaError_t e = spin_launch(sp, false, sp->done_to - 1, d.tiles_c, cs);
  if (e == cudaSuccess) e = spin_launch(sp, true, sp->merged_to - 1, d.tiles_c, cs, true);
  sp->done_to = sp->merged_to = d.tiles_c;
  if (e == cudaSuccess) {
    KArgs a = sp->a;
    a.tile_list = nullptr;
    a.ntiles = d.tiles_r * d.tiles_c;
    e = launch_flatten(sp->tile, a, cs, true);
  }
  return cuda_status(e);
}

lsg_status lsg_spin_destroy(lsg_spin* sp) {
  if (!sp) return LSG_E_ARG;
  if (sp->ws) {
    DeviceGuard g(sp->ctx->device);
    cudaDeviceSynchronize();
    cudaFree(sp->ws);
    sp->ctx->used -= sp->bytes;
  }
  delete sp;
  return LSG_OK;
}

}  // extern "C"
