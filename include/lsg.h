/*
 * lsg.h - C ABI of the GB300 Lidar surface-segmentation library (liblsg.so).
 *
 * The library implements the data-parallel path of Mukherjee, Das, Ghosh,
 * Chowdhury and Saha, "Fast Geometric Surface based Segmentation of Point
 * Cloud from Lidar Data" (PReMI 2019): one spinning-Lidar scan, organised as
 * rings x shots, goes in; the mesh, the per-vertex normals and the segment
 * label of every point come out.  Every step runs in CUDA kernels for sm_103a.
 *
 * Conventions shared by all calls
 * --------------------------------
 * - Pointers documented as "device" must point to memory of the context's
 *   device.  The caller allocates and owns every input and output buffer;
 *   the library owns only its workspace (inside the context or the plan).
 * - Calls are asynchronous and ordered on the given stream (a cudaStream_t
 *   passed as void*, NULL = the legacy default stream).  Outputs are valid
 *   once that stream has synchronised.  Argument and shape errors are
 *   returned synchronously and launch nothing.  Errors detected on the device
 *   (a NaN elevation, a bounded wait that ran out) are recorded in a sticky
 *   error word of the context, read by lsg_get_error.
 * - A context must not be used from two host threads, or on two streams, at
 *   the same time: its workspace is shared by its calls.
 * - Nothing throws across this ABI.
 *
 * Grid convention (Sec. 2, mesh construction): ring i counts from the
 * topmost sensor down (rings are sorted by elevation, descending, ties by
 * input row); column c counts shots from the first of the spin; with
 * sub-sampling s the mesh vertices are the columns c = j*s, j < Ws =
 * ceil(W/s).  All outputs are indexed in this sorted ring order.
 */
#ifndef LSG_H
#define LSG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lsg_ctx lsg_ctx;
typedef struct lsg_plan lsg_plan;
typedef struct lsg_spin lsg_spin;
typedef void* lsg_stream; /* cudaStream_t */

typedef enum {
  LSG_OK = 0,
  LSG_E_ARG = 1,     /* bad pointer or parameter value */
  LSG_E_SHAPE = 2,   /* negative or too large rings / columns */
  LSG_E_OOM = 3,     /* device allocation failed */
  LSG_E_BUDGET = 4,  /* workspace would exceed the context's memory budget */
  LSG_E_CUDA = 5,    /* a CUDA runtime call failed */
  LSG_E_TIMEOUT = 6, /* a bounded device-side wait ran out */
  LSG_E_DEVICE = 7   /* the device flagged bad input data (e.g. NaN elevation) */
} lsg_status;

/* Homogeneity predicate (Algorithm 1). */
enum {
  LSG_PRED_ANGLE = 0,    /* angle(n_p, n_q) < angle_rad */
  LSG_PRED_COMPONENT = 1 /* |dx| < comp[0], |dy| < comp[1], |dz| < comp[2] */
};

/* Bits of the per-vertex mesh byte (output meshbits). */
#define LSG_BIT_R 0x01     /* mesh edge (i,j)-(i,j+1)   (column wraps)   */
#define LSG_BIT_D 0x02     /* mesh edge (i,j)-(i+1,j)                    */
#define LSG_BIT_G 0x04     /* mesh edge (i,j)-(i+1,j+1) (column wraps)   */
#define LSG_BIT_HR 0x08    /* edge R is homogeneous                      */
#define LSG_BIT_HD 0x10    /* edge D is homogeneous                      */
#define LSG_BIT_HG 0x20    /* edge G is homogeneous                      */
#define LSG_BIT_VALID 0x40 /* the vertex is a point of the scan (in range) */
#define LSG_BIT_HASN 0x80  /* the vertex has a normal                    */

/* Upper limits of one scan. */
#define LSG_MAX_RINGS 4096
#define LSG_MAX_COLS (1 << 20)
#define LSG_MAX_POINTS (1 << 28)

/*
 * One scan.  Sec. 2: P = {p(theta, phi, r)}, theta the fixed elevation of a
 * sensor, phi the azimuth of the shot, r the measured range.
 *   rings, cols     H >= 0 sensors, W >= 0 shots per revolution.
 *   elevation       device float[H], radians, any order (the library sorts).
 *   azimuth0, azimuth_step
 *                   phi_c = azimuth0 + c * azimuth_step (radians; the sign of
 *                   the step is the spin direction).
 *   xyzr            device float[H][W][4] = x, y, z, range per shot, rows in
 *                   the order of `elevation`; 16-byte aligned.  Or NULL:
 *   range           device float[H][W] ranges; x, y, z are then decoded as
 *                   r (cos theta cos phi, cos theta sin phi, sin theta).
 * A range r is a point of the scan when r_min < r <= r_max (r = 0 marks a
 * dropout).
 */
typedef struct {
  int32_t rings;
  int32_t cols;
  const float* elevation;
  float azimuth0;
  float azimuth_step;
  const float* xyzr;
  const float* range;
} lsg_scan;

/*
 * Parameters (lsg_default_params fills the defaults given in brackets).
 *   subsample   s >= 1, keep every s-th shot as a mesh vertex [1] (Sec. 2).
 *   r_min, r_max  validity window, 0 <= r_min < r_max [0, 100].
 *   jump_rel_h, jump_rel_v  depth-jump cut: a mesh edge (p,q) is dropped when
 *               |r_p - r_q| > tau * min(r_p, r_q), tau = jump_rel_h for the
 *               R edge and jump_rel_v for D and G [0.10, 1.0]; +inf disables.
 *               Evaluated in IEEE binary32 round-to-nearest.
 *   predicate   LSG_PRED_ANGLE or LSG_PRED_COMPONENT [ANGLE].
 *   angle_rad   angle threshold in (0, pi) [10 deg].
 *   comp        (I, J, K) > 0 of the component predicate [0.2, 0.2, 0.2]
 *               (the paper's setting, Sec. 3).
 *   wrap        1 = join the last column to the first (full 360 deg spin,
 *               Sec. 2), 0 = open sweep [1].  Wrapping needs Ws >= 3 and is
 *               ignored below that.
 */
typedef struct {
  int32_t subsample;
  float r_min;
  float r_max;
  float jump_rel_h;
  float jump_rel_v;
  int32_t predicate;
  float angle_rad;
  float comp[3];
  int32_t wrap;
} lsg_params;

/*
 * Outputs of one scan (device, caller-owned; every pointer required).
 *   meshbits  uint8[H][Ws]   mesh and homogeneity bits (LSG_BIT_*)
 *   normals   float[H][Ws][3] unit normal facing the sensor (0 if none):
 *             n = -sign(azimuth_step) * sum_k w_k V_k x V_k+1 / |...|, over
 *             the incident triangles (p, q_k, q_k+1) whose three edges are in
 *             the mesh, spokes V_k = q_k - p in the order (i+1,j), (i+1,j+1),
 *             (i,j+1), (i-1,j), (i-1,j-1), (i,j-1), w_k = 1/(|V_k|+|V_k+1|)
 *             (Sec. 2, normal estimation).
 *   labels    int32[H][W]    segment label of every point: the smallest
 *             i*W + c over the points of its segment; -1 for points out of
 *             range.  Non-sampled points take the label of the nearer
 *             bracketing sampled column on their ring (ties to the earlier,
 *             falling back to the other when the nearer is unlabelled)
 *             (Sec. 2, last paragraph; Algorithm 1).
 *   nseg      int32[1]       number of segments.
 */
typedef struct {
  uint8_t* meshbits;
  float* normals;
  int32_t* labels;
  int32_t* nseg;
} lsg_out;

/* Tile shapes of the fused kernels: rows x columns of mesh vertices per CTA.
 * Each warp of a CTA sweeps a strip of 60 columns (two per lane) down the
 * tile's rows, so the widths are multiples of 60 (2 warps: 120, 4 warps:
 * 240, 8 warps: 480).  LSG_TILE_AUTO: each call picks the shape from its
 * work (see lsg_set_tile). */
enum {
  LSG_TILE_AUTO = -1,
  LSG_TILE_16x240 = 0,
  LSG_TILE_32x120 = 1,
  LSG_TILE_32x240 = 2,
  LSG_TILE_32x480 = 3,
  LSG_TILE_64x240 = 4,
  LSG_TILE_16x120 = 5,
  LSG_TILE_8x120 = 6,
  LSG_TILE_4x120 = 7,
  LSG_TILE_2x120 = 8,
  LSG_TILE_COUNT = 9
};

/* Fills *p with the defaults listed above. */
void lsg_default_params(lsg_params* p);

/* Human-readable name of a status code (static string). */
const char* lsg_status_str(lsg_status s);

/* Creates a context on CUDA device `device` whose workspace may use at most
 * mem_budget_bytes of device memory (0 = no limit).  *out receives the
 * context; destroy it with lsg_destroy. */
lsg_status lsg_create(int device, size_t mem_budget_bytes, lsg_ctx** out);

/* Frees the context and its workspace (synchronises the device first). */
lsg_status lsg_destroy(lsg_ctx* ctx);

/* Selects the tile shape of the context's calls (lsg_segment,
 * lsg_label_from_mask, lsg_batch_launch, lsg_spin_begin, and lsg_batch_plan
 * given LSG_TILE_AUTO).  LSG_TILE_AUTO (the default) lets each call pick from
 * its work: the first of 32x120, 32x240, 16x240, 16x120, 8x120, 4x120,
 * 2x120 that gives at least four tiles per SM, else the one that gives the
 * most tiles (small scans fill the GPU with small tiles of short row sweeps,
 * large batches keep the efficient ones). */
lsg_status lsg_set_tile(lsg_ctx* ctx, int tile);

/*
 * Segments one scan (Sec. 2: meshing, normal estimation, Algorithm 1,
 * back-fill): decode -> mesh -> normals -> edge mask -> connected components
 * -> back-fill.  The workspace (ring order and sin/cos per ring, union-find
 * parents and tile-local roots: 12*H + 6*H*Ws bytes) is allocated in the
 * context on first need.
 */
lsg_status lsg_segment(lsg_ctx* ctx, const lsg_scan* scan, const lsg_params* params,
                       const lsg_out* out, lsg_stream stream);

/*
 * Labels from a given mesh byte array (the edge mask is taken as given):
 * the components and back-fill steps of lsg_segment alone (Algorithm 1 and
 * Sec. 2, last paragraph).  Used to check labelling exactly against another
 * implementation's mask.
 *   H, W, s, wrap  grid as in lsg_segment (wrap needs Ws >= 3).
 *   meshbits       device uint8[H][Ws], sorted ring order; only the
 *                  homogeneity bits and the valid bit are read.
 *   valid          device uint8[H][W] (1 = point in range), sorted ring
 *                  order; may be NULL when s == 1.
 *   labels, nseg   device outputs as in lsg_out.
 */
lsg_status lsg_label_from_mask(lsg_ctx* ctx, int32_t H, int32_t W, int32_t s, int32_t wrap,
                               const uint8_t* meshbits, const uint8_t* valid, int32_t* labels,
                               int32_t* nseg, lsg_stream stream);

/*
 * Batched path: many scans of uneven shape in one pass.  The plan fixes the
 * scans' device pointers, shapes and parameters, allocates the workspace for
 * all of them (within the context's budget) and captures the pass in a CUDA
 * graph; lsg_batch_run replays it.  Rewrite the inputs in place between
 * replays to process new data of the same shapes.
 *   n          number of scans (>= 1)
 *   scans[n], params[n], outs[n]  as for lsg_segment (host arrays, copied)
 *   tile       LSG_TILE_* shape, or LSG_TILE_AUTO: the context's shape if
 *              lsg_set_tile fixed one, else the per-call choice described
 *              at lsg_set_tile over the whole batch; lsg_autotune may
 *              replace it later.
 */
lsg_status lsg_batch_plan(lsg_ctx* ctx, int32_t n, const lsg_scan* scans, const lsg_params* params,
                          const lsg_out* outs, int tile, lsg_plan** plan);

/* Device bytes the context holds now (workspace, descriptor staging, error
 * word, and the plans and spins made from it); 0 for NULL. */
size_t lsg_memory_used(const lsg_ctx* ctx);

/*
 * Dynamic batch: one pass over n scans whose set changes from call to call
 * (the serving path).  Same semantics and outputs as n lsg_segment calls, in
 * four launches (a batch of one: as lsg_segment, three launches when the scan
 * has at most 256 rings); the scans' descriptors go to the device through a pinned
 * staging buffer of the context (two of them, alternated; a call waits until
 * the copy out of the buffer it reuses has run).  The workspace of all n scans
 * comes from the context, so one context serves one stream at a time.  A
 * batch of one runs as lsg_segment does (descriptor by value, no staging).
 */
lsg_status lsg_batch_launch(lsg_ctx* ctx, int32_t n, const lsg_scan* scans, const lsg_params* params,
                            const lsg_out* outs, lsg_stream stream);

/* Host buffers of one scan for lsg_batch_launch_io and lsg_batch_plan_io
 * (pinned memory lets the copies run asynchronously; any NULL output is
 * skipped). */
typedef struct {
  const float* xyzr;      /* host input in the scan's form: [H][W][4] x,y,z,r
                             (lsg_scan.xyzr set), or [H][W] ranges (lsg_scan.range
                             set) */
  const float* elevation; /* host [H] input */
  int32_t* labels;        /* host [H][W] result, or NULL */
  int32_t* nseg;          /* host [1] result, or NULL */
  uint8_t* meshbits;      /* host [H][Ws] result, or NULL */
  float* normals;         /* host [H][Ws][3] result, or NULL */
} lsg_host_io;

/*
 * lsg_batch_launch with the host transfers of the serving path in the same
 * call, all ordered on `stream`: every scan's input (x,y,z,r, or ranges for
 * a range-only scan) and elevations are copied from io[b] into the device
 * buffers scans[b].xyzr (or .range) and scans[b].elevation (which must be
 * writable device memory), then the pass runs, then the results listed in
 * io[b] are copied back.
 */
lsg_status lsg_batch_launch_io(lsg_ctx* ctx, int32_t n, const lsg_scan* scans, const lsg_params* params,
                               const lsg_out* outs, const lsg_host_io* io, lsg_stream stream);

/* Pre-sizes a context so that later calls with at most max_scans scans,
 * max_tiles tiles and workspace_bytes of workspace allocate nothing (the
 * workspace of a scan is 12*H + 6*H*Ws bytes, rounded up to 256 per array). */
lsg_status lsg_reserve(lsg_ctx* ctx, size_t workspace_bytes, int32_t max_scans, int32_t max_tiles);

/* Replays the plan's graph on `stream`. */
lsg_status lsg_batch_run(lsg_plan* plan, lsg_stream stream);

/* Times every tile shape under the three schedules (see lsg_plan_set_fused)
 * on the plan (reps replays each, CUDA events on
 * `stream`), keeps the fastest and re-captures the graph.  *best_tile and
 * *best_ms (either may be NULL) receive the choice and its time per pass;
 * lsg_plan_fused tells the schedule chosen. */
lsg_status lsg_autotune(lsg_plan* plan, int reps, lsg_stream stream, int* best_tile, float* best_ms);

/* Tile shape the plan currently uses. */
int lsg_plan_tile(const lsg_plan* plan);

/* Chooses how the plan's pass runs (the schedule):
 *   1 (the default) one persistent launch that walks a list of work items
 *     (each scan's ring order, then per tile: geometry and tile components,
 *     border merge, labels), each item waiting (bounded) only on items
 *     listed before it;
 *   0 four phased launches (ring order, tiles, merges, labels);
 *   2 the ring order, then the scans in four groups of about equal tile
 *     counts, each group's tile, merge and label launches on its own branch
 *     of the graph, so a group's merges and labels overlap the tile work of
 *     the groups still running.
 * Any other value means 0.  Outputs are identical.  Re-captures the graph. */
lsg_status lsg_plan_set_fused(lsg_plan* plan, int fused);

/* The plan's schedule (0, 1 or 2, see lsg_plan_set_fused). */
int lsg_plan_fused(const lsg_plan* plan);

/* Kernel launches in one lsg_batch_run of the plan as captured now (phased:
 * 4, fused: 1, grouped: 1 + 3 per scan group; 1 when no scan has points);
 * -1 for a null plan. */
int lsg_plan_launches(const lsg_plan* plan);

/* Device time of each phase of the plan's last replay, in milliseconds.
 * Phased plans: ms[0] ring order, ms[1] tile kernel (decode, mesh, normals,
 * edge mask, tile-local components), ms[2] border merge, ms[3] labels and
 * back-fill.  Fused plans: ms[0] counter reset, ms[1] the persistent launch
 * (the whole pass), ms[2] = ms[3] = 0.  Grouped plans (schedule 2): ms[0] ring
 * order, ms[1] the grouped branches (the rest of the pass), ms[2] = ms[3] =
 * 0.  Measured by CUDA events recorded inside the graph; waits for the
 * replay to finish. */
lsg_status lsg_plan_phase_times(lsg_plan* plan, float* ms);

/* Frees the plan (synchronises the device first). */
lsg_status lsg_plan_destroy(lsg_plan* plan);

/*
 * Batched path from and to host memory (the problem of Sec. 2 end to end: a
 * scan with its ring elevations goes in, the mesh, normals and labels come
 * out).  Like lsg_batch_plan, plus the host transfers in the captured graph:
 * the batch is cut into `chunks` runs of consecutive scans whose point
 * counts grow by a factor 1.1 from one run to the next (a small first run
 * starts the copies back early); for each, the inputs io[b].xyzr and
 * io[b].elevation are copied into the device buffers scans[b] (x,y,z,r or
 * ranges, by the scan's form, and the elevations, all of which must be
 * writable device memory),
 * the chunk's pass runs once they have landed, and the chunk's outputs are
 * copied into io[b].labels, .nseg, .meshbits and .normals (NULL ones
 * skipped) once its pass is done; the copies of neighbouring chunks, in both
 * directions, run under each chunk's pass.  The elevations of every scan go
 * in ahead of the first chunk and the segment counts come back after the
 * last.  Consecutive scans whose host and device buffers are contiguous
 * share one copy.  lsg_batch_run replays the whole sequence; the host
 * outputs are complete once the stream has synchronised, and the host inputs
 * may be rewritten after that.
 *   io[n]      host buffers of every scan: page-locked memory (cudaHostAlloc
 *              or cudaHostRegister), else LSG_E_ARG; not copied, must
 *              outlive the plan.
 *   chunks     >= 1 (at most n are used).
 *   tile       as for lsg_batch_plan.
 * The plan runs the phased kernels per chunk; lsg_plan_set_fused accepts
 * only 0 for it, lsg_autotune tries the tile shapes, and
 * lsg_plan_phase_times gives the whole run in ms[0].
 */
lsg_status lsg_batch_plan_io(lsg_ctx* ctx, int32_t n, const lsg_scan* scans, const lsg_params* params,
                             const lsg_out* outs, const lsg_host_io* io, int32_t chunks, int tile,
                             lsg_plan** plan);

/* Bytes one run of a host-buffer plan copies host -> device (*h2d) and
 * device -> host (*d2h); LSG_E_ARG for a device-resident plan. */
lsg_status lsg_plan_io_bytes(const lsg_plan* plan, size_t* h2d, size_t* d2h);

/* Reads and clears the context's sticky device error word (synchronises the
 * device).  LSG_OK when no device-side error was recorded. */
lsg_status lsg_get_error(lsg_ctx* ctx);

/* Self-test of failure detection, without a fault: a kernel runs the
 * persistent schedule's bounded wait on a device counter that nothing
 * increments, gives up after about 4096 polls (about a millisecond) and
 * records a timeout in the context's error word.  Returns LSG_OK when
 * lsg_get_error then reports LSG_E_TIMEOUT (which it clears, so the context
 * stays usable), LSG_E_DEVICE when it reports something else or nothing, and
 * a CUDA or allocation status on failure.  Synchronises the device; any
 * error word recorded before the call is read and cleared with it. */
lsg_status lsg_selftest_wait_timeout(lsg_ctx* ctx);

/*
 * Per-segment statistics and small-segment removal: the optional
 * post-processing of Sec. 2 (last paragraph), which eliminates segments with
 * too few points.  Runs on the outputs of lsg_segment, in place.
 *   H, W, s       grid of the scan (as in lsg_segment)
 *   min_points    segments of fewer points become -1 (0 keeps every segment)
 *   labels        device int32[H][W], in/out
 *   sizes         device int32[H*W], out: sizes[L] = number of points whose
 *                 label was L before removal (0 where L is not a label)
 *   nsum          device float[H*W][3], out, or NULL: nsum[L] = sum of the
 *                 unit normals of the segment's vertices that have one (its
 *                 direction is the segment's mean normal); float atomics, so
 *                 the summation order (last bits) varies from run to run
 *   normals, meshbits  lsg_segment's outputs (read only when nsum != NULL)
 *   nseg          device int32[1], out: number of segments kept
 */
lsg_status lsg_segment_stats(lsg_ctx* ctx, int32_t H, int32_t W, int32_t s, int32_t min_points,
                             int32_t* labels, const float* normals, const uint8_t* meshbits, int32_t* sizes,
                             float* nsum, int32_t* nseg, lsg_stream stream);

/* ---- Streaming: one revolution segmented while its columns arrive ----
 *
 * The paper builds the mesh while the sensor spins (Sec. 2, meshing; Fig. 1:
 * the first stage can run with the scanning).  These calls do the per-tile
 * work of lsg_segment column by column as the revolution arrives, so that
 * after the last column only the first tile column (whose left neighbours
 * are the revolution's last columns, across the seam), the joins that touch
 * it and the labels remain.  The outputs equal lsg_segment's bit for bit.
 *
 * lsg_spin_begin   scan, params, out as for lsg_segment; the elevations must
 *                  be in place, the x,y,z,r (or range) columns may still be
 *                  arriving.  Allocates the spin's own workspace (counted
 *                  against the context's budget: LSG_E_BUDGET) with the
 *                  context's tile shape, computes the ring order and zeroes
 *                  *nseg on `stream`.  *spin receives the handle.
 * lsg_spin_push    columns [0, cols_ready) of the scan's input (full
 *                  resolution, in firing order) are in place in device
 *                  memory, ordered before this call on `stream` (e.g. by
 *                  copies on it).  Launches the tiles whose columns, and the
 *                  two sampled columns to their right, are all in place, and
 *                  the joins between computed tile columns.  cols_ready must
 *                  not decrease and not exceed cols (LSG_E_ARG).
 * lsg_spin_finish  the whole revolution is in place: computes the rest; the
 *                  outputs are valid once `stream` reaches this point.
 *                  LSG_E_ARG if already finished.
 * lsg_spin_destroy frees the spin (synchronises the device).
 * Calls on one spin must be ordered on one stream; pushes after the finish
 * return LSG_E_ARG. */
lsg_status lsg_spin_begin(lsg_ctx* ctx, const lsg_scan* scan, const lsg_params* params, const lsg_out* out,
                          lsg_spin** spin, lsg_stream stream);
lsg_status lsg_spin_push(lsg_spin* spin, int32_t cols_ready, lsg_stream stream);
lsg_status lsg_spin_finish(lsg_spin* spin, lsg_stream stream);
lsg_status lsg_spin_destroy(lsg_spin* spin);

/* Largest scan (rings x sampled columns) lsg_segment_noalloc accepts. */
#define LSG_NOALLOC_MAX_VERTICES (1 << 20)

/*
 * lsg_segment without any device allocation (the paper has no counterpart:
 * this is a deployment variant of lsg_segment).
 *
 * For callers that cannot call cudaMalloc: a sensor thread with a hard
 * latency budget (cudaMalloc / cudaFree can synchronise the device and take
 * driver-wide locks) or a host framework that owns all device memory and
 * forbids side allocations.  The caller still allocates and owns the inputs
 * and outputs; the workspace is one fixed device array inside the library
 * (about 6.3 MB on every device that loads the library, held until the
 * process exits).
 *
 *   scan, params, out  as for lsg_segment; uses the current CUDA device and
 *                      the default tile shape.  Outputs equal lsg_segment's.
 *   returns LSG_E_SHAPE when rings * ceil(cols/subsample) exceeds
 *   LSG_NOALLOC_MAX_VERTICES (nothing is launched), LSG_E_ARG / LSG_E_SHAPE
 *   as lsg_segment for bad arguments, LSG_E_CUDA if a launch fails.
 *
 * Every call looks up the array's device address on the current device (a
 * host-side lookup; the first call on a device also sets the kernels'
 * shared-memory attributes).  Every call shares the one array and leaves its
 * contents behind, so calls whose work overlaps on the GPU (different
 * streams, or different host threads, without ordering between them) race
 * and corrupt each other's results: order them on one stream.  Device-side
 * flags (a NaN elevation) are not returned by this call; it clears them at
 * its start, and lsg_noalloc_get_error reads them.
 */
lsg_status lsg_segment_noalloc(const lsg_scan* scan, const lsg_params* params, const lsg_out* out,
                               lsg_stream stream);

/*
 * The device flags of the allocation-free passes (the paper has no
 * counterpart).  Waits for `stream`, reads the flags the last
 * lsg_segment_noalloc call on the current device raised, clears them, and
 * returns LSG_OK (none), LSG_E_DEVICE (bad input seen on the device, e.g. a
 * NaN elevation, whose outputs are then unspecified), LSG_E_TIMEOUT (a
 * bounded union-find loop ran out) or LSG_E_CUDA.  Allocates nothing; call it
 * on the stream of the pass it checks.
 */
lsg_status lsg_noalloc_get_error(lsg_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* LSG_H */
