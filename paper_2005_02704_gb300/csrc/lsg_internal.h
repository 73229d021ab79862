// lsg_internal.h - descriptors and kernel launchers shared by the library's
// translation units (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lsg.h"  // include/ is on the include path

namespace lsg {

// Everything one kernel needs to know about one scan.  Built on the host,
// passed by value (single scan) or in a device table (batched pass).
struct ScanDesc {
  // inputs
  const float4* xyzr;   // [H][W] (input ring order) or null
  const float* range;   // [H][W] when xyzr is null
  const float* elev;    // [H]
  const uint8_t* valid; // [H][W] sorted order; label-from-mask path only
  // outputs
  uint8_t* mb;          // [H][Ws]
  float* nrm;           // [H][Ws][3]
  int32_t* labels;      // [H][W]
  int32_t* nseg;        // [1]
  // workspace
  int32_t* order;       // [H]   sorted ring -> input row
  float2* trig;         // [H]   (sin, cos) of the sorted ring's elevation
  int32_t* parent;      // [H*Ws] union-find over scan-local vertex indices
                        //        (only entries of tile-local roots are used)
  uint16_t* lroot;      // [H*Ws] each vertex's tile-local root (tile-local index)
  // shape
  int32_t H, W, Ws, s, wrap;  // wrap already reduced to (wrap && Ws >= 3)
  int32_t tiles_r, tiles_c, tile0;
  // parameters
  float az0, daz, r_min, r_max, jump_h, jump_v;
  float cos_t, comp_x, comp_y, comp_z, nsign;
  int32_t pred;
};

struct KArgs {
  const ScanDesc* scans;     // device table, or null: use `one`
  const int32_t* tile_scan;  // device [ntiles] tile -> scan (batched), or null
  const int32_t* tile_list;  // device [ntiles] local tile indices of `one`, or null: all of its tiles
  int32_t ntiles;
  int32_t tile_base;         // batched: first entry of tile_scan this launch covers
  int32_t nscans;
  int32_t* err;              // device error word
  int32_t s1_only;           // 1: every scan of the launch has s = 1 (the label
                             // kernel then needs less shared memory)
  int32_t fuse_prep;         // 1: single scan, no k_prep before the tile kernel:
                             // each tile finds the ring order of the rows it reads
                             // (at most kFuseMaxRings rings)
  ScanDesc one;
};

// Rings of a single scan up to which the tile kernel finds the ring order
// itself (its elevations fit in the tile's idle row slots).
constexpr int kFuseMaxRings = 256;

// The persistent fused pass: one launch that walks a schedule of work items
// (ring order of a scan, then its tiles, border merges and labels), each item
// waiting only on items scheduled before it.
enum : int32_t { PH_PREP = 0, PH_TILE = 1, PH_MERGE = 2, PH_FLAT = 3 };

struct FusedArgs {
  const ScanDesc* scans;  // device table
  const int2* items;      // [nitems] (phase << 28 | scan, local tile)
  int32_t nitems;
  int32_t nscans;
  int32_t* counters;      // [0] next item, then per scan: rings done, tiles done, merges done
  int32_t* err;
  int32_t s1_only;        // 1: every scan has s = 1 (less shared memory per CTA)
};

// Device error codes (sticky, OR-ed into *err).
enum : int32_t { DERR_NAN_ELEV = 1, DERR_TIMEOUT = 2, DERR_LAUNCH = 4 };

struct TileShape {
  int rows, cols;
};
TileShape tile_shape(int tile);

// Tile shape for a call whose scans are given by (rings, sampled columns):
// the first of 32x120, 32x240, 16x240, 16x120 that yields at least two
// tiles per SM, else the one that yields the most tiles.
int pick_tile(const int* H, const int* Ws, int n, int sms);

// Host helpers shared by the entry points (lsg_api.cu).
lsg_status check_scan(const lsg_scan* sc, const lsg_params* p, const lsg_out* o, int* Ws_out);
ScanDesc make_desc(const lsg_scan* sc, const lsg_params* p, const lsg_out* o, int Ws);
void set_tiles(ScanDesc& d, int tile, int tile0);

// Kernel launchers (lsg_kernels.cu).  All return the launch error.
cudaError_t launch_prep(const KArgs& a, cudaStream_t st);
// pdl: launch as a programmatic dependent of the previous kernel in the
// stream (which must be one of these kernels or k_prep of the same pass), so
// its CTAs are scheduled while that kernel drains.  Not for graph capture.
cudaError_t launch_tile(int tile, const KArgs& a, cudaStream_t st, bool pdl = false);
cudaError_t launch_tile_ccl(int tile, const KArgs& a, cudaStream_t st, bool pdl = false);
cudaError_t launch_merge(int tile, const KArgs& a, cudaStream_t st, bool pdl = false);
cudaError_t launch_flatten(int tile, const KArgs& a, cudaStream_t st, bool pdl = false);
cudaError_t launch_fused(int tile, const FusedArgs& f, cudaStream_t st);
// The persistent schedule's bounded wait on a counter nothing increments
// (cnt: a zeroed device int), giving up after `limit` polls.
cudaError_t launch_wait_probe(const int32_t* cnt, int32_t* err, unsigned limit, cudaStream_t st);
cudaError_t prepare_kernels();  // one-time function attributes

}  // namespace lsg
