// lsg_noalloc.cu - lsg_segment_noalloc: the single-scan pass of lsg_segment
// for callers that must not allocate device memory.
//
// Who needs it: a sensor driver thread with a hard latency budget cannot
// afford cudaMalloc/cudaFree on its path (they can synchronise the whole
// device and take driver-wide locks, so their cost is unbounded), and some
// host frameworks hand out every byte of device memory themselves and forbid
// side allocations by their plug-ins.  Such callers can still own their input
// and output buffers but cannot let the library grow a workspace.
//
// How: the workspace (ring order, per-ring sin/cos, union-find parents,
// tile-local roots and a device error word) lives in one file-scope __device__
// array of fixed size, created when the library is loaded on a device and
// held until the process exits.  Host code cannot use the array's name as a
// device address, so every call looks the address up with
// cudaGetSymbolAddress (on the current device; a host-side lookup that
// allocates nothing) and passes that pointer to the same kernels lsg_segment
// uses.  Looking it up on every call keeps the pointer right even after the
// device's primary context was torn down and recreated (the module, and with
// it the array, is then loaded anew).  No call allocates or frees anything.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <mutex>

#include "lsg_internal.h"

namespace {

// Layout of the fixed workspace (byte offsets, each 256-byte aligned).
constexpr size_t kOrderOff = 0;                                         // int32[LSG_MAX_RINGS]
constexpr size_t kTrigOff = kOrderOff + sizeof(int32_t) * LSG_MAX_RINGS;  // float2[LSG_MAX_RINGS]
constexpr size_t kErrOff = kTrigOff + sizeof(float2) * LSG_MAX_RINGS;     // int32 error word
constexpr size_t kParentOff = kErrOff + 256;                             // int32[max vertices]
constexpr size_t kRootOff = kParentOff + sizeof(int32_t) * (size_t)LSG_NOALLOC_MAX_VERTICES;  // uint16[max]
// tile-root rows are padded to 8 entries: at most 7 extra per ring
constexpr size_t kScratchBytes = kRootOff + sizeof(uint16_t) * ((size_t)LSG_NOALLOC_MAX_VERTICES + 8 * LSG_MAX_RINGS);
static_assert(kTrigOff % 256 == 0 && kErrOff % 256 == 0 && kParentOff % 256 == 0 && kRootOff % 256 == 0,
              "alignment");

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void* g_prepared_for[kMaxDevices] = {};  // the array's address when the kernel attributes were last set

}  // namespace

// The workspace itself: one copy on every device that loads the library.
static __device__ __align__(256) unsigned char g_lsg_scratch[kScratchBytes];

// Device address of g_lsg_scratch on the current device.  The kernels' shared
// memory attributes are set again whenever the address differs from the one
// seen when they were last set (a first call, or a module loaded anew).
static lsg_status scratch_for_current_device(char** base) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LSG_E_ARG;
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_lsg_scratch);
  if (e != cudaSuccess || p == nullptr) return LSG_E_CUDA;
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (g_prepared_for[dev] != p) {
    if (lsg::prepare_kernels() != cudaSuccess) return LSG_E_CUDA;
    g_prepared_for[dev] = p;
  }
  *base = static_cast<char*>(p);
  return LSG_OK;
}

extern "C" lsg_status lsg_segment_noalloc(const lsg_scan* scan, const lsg_params* params,
                                          const lsg_out* out, lsg_stream stream) {
  int Ws = 0;
  lsg_status st = lsg::check_scan(scan, params, out, &Ws);
  if (st != LSG_OK) return st;
  if ((int64_t)scan->rings * Ws > (int64_t)LSG_NOALLOC_MAX_VERTICES) return LSG_E_SHAPE;
  char* base = nullptr;
  st = scratch_for_current_device(&base);
  if (st != LSG_OK) return st;
  cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
  if (scan->rings == 0 || scan->cols == 0)
    return cudaMemsetAsync(out->nseg, 0, sizeof(int32_t), cs) == cudaSuccess ? LSG_OK : LSG_E_CUDA;

  lsg::KArgs a;
  memset(&a, 0, sizeof(a));
  a.one = lsg::make_desc(scan, params, out, Ws);
  lsg::set_tiles(a.one, LSG_TILE_16x240, 0);
  a.one.order = reinterpret_cast<int32_t*>(base + kOrderOff);
  a.one.trig = reinterpret_cast<float2*>(base + kTrigOff);
  a.one.parent = reinterpret_cast<int32_t*>(base + kParentOff);
  a.one.lroot = reinterpret_cast<uint16_t*>(base + kRootOff);
  a.ntiles = a.one.tiles_r * a.one.tiles_c;
  a.nscans = 1;
  a.err = reinterpret_cast<int32_t*>(base + kErrOff);
  a.s1_only = a.one.s == 1;
  // The error word accumulates flags with atomicOr, so it must start at zero;
  // everything else is fully written by the kernels before it is read.
  cudaError_t e = cudaMemsetAsync(a.err, 0, sizeof(int32_t), cs);
  if (e == cudaSuccess) e = lsg::launch_prep(a, cs);
  if (e == cudaSuccess) e = lsg::launch_tile(LSG_TILE_16x240, a, cs, true);
  if (e == cudaSuccess) e = lsg::launch_merge(LSG_TILE_16x240, a, cs, true);
  if (e == cudaSuccess) e = lsg::launch_flatten(LSG_TILE_16x240, a, cs, true);
  return e == cudaSuccess ? LSG_OK : LSG_E_CUDA;
}

// Reads and clears the device flags the last allocation-free passes on this
// device raised, in stream order; nothing is allocated.
extern "C" lsg_status lsg_noalloc_get_error(lsg_stream stream) {
  char* base = nullptr;
  lsg_status st = scratch_for_current_device(&base);
  if (st != LSG_OK) return st;
  cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
  int32_t v = 0;
  cudaError_t e = cudaMemcpyAsync(&v, base + kErrOff, sizeof(v), cudaMemcpyDeviceToHost, cs);
  if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
  if (e == cudaSuccess) e = cudaMemsetAsync(base + kErrOff, 0, sizeof(int32_t), cs);
  if (e != cudaSuccess) return LSG_E_CUDA;
  if (v & lsg::DERR_TIMEOUT) return LSG_E_TIMEOUT;
  return v ? LSG_E_DEVICE : LSG_OK;
}
