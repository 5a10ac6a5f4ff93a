// Allocation-free variant of the value scan (lqt_scan_value_noalloc).
//
// Some callers cannot allocate device memory while they run: a control loop
// whose memory budget is fixed at start-up, or a plugin hosted by an
// application that owns the device allocator.  They cannot provide the
// caller-owned workspace of lqt_scan_value either, so this entry point keeps
// the scan's scratch in one file-scope device array of fixed size instead.
//
// Rules of use (also stated in include/lqt.h):
//  - The array holds LQT_STATIC_SCRATCH_BYTES bytes on every device that loads
//    the library, until the process exits.  Problems whose scan needs more are
//    rejected with LQT_EWORKSPACE before anything is launched.
//  - Host code cannot use the array's name as a device address; the first call
//    on each device looks the address up with cudaGetSymbolAddress (with that
//    device current) and caches it.  Make that first call before any stream
//    capture.
//  - Every call uses the same array, so calls that overlap on the GPU (two
//    streams, two host threads) race and corrupt each other's results.  Every
//    byte the scan reads from the array is written earlier in the same call,
//    so nothing needs clearing between calls.
#include <mutex>

#include <cuda_runtime.h>

#include "lqt_internal.h"

namespace lqt {

static __device__ __align__(256) unsigned char g_static_scratch[LQT_STATIC_SCRATCH_BYTES];

static constexpr int kMaxDevices = 64;
static void* g_scratch_ptr[kMaxDevices];
static std::mutex g_scratch_mutex;

// Device address of g_static_scratch on the current device (looked up once per
// device).  Returns nullptr on failure.
static void* scratch_address() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (g_scratch_ptr[dev] == nullptr) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess) return nullptr;
    g_scratch_ptr[dev] = p;
  }
  return g_scratch_ptr[dev];
}

}  // namespace lqt

extern "C" lqt_status lqt_scan_value_noalloc(const lqt_problem* p, const lqt_elements* el, double* S, double* v,
                                             double* zeta, void* stream) {
  using namespace lqt;
  if (!p || !el || !el->A || !el->b || !el->C || !el->eta || !el->J || !S || !v) return LQT_EINVAL;
  const size_t need = lqt_workspace_size(p, LQT_WS_VALUE);
  if (need == 0) return LQT_EINVAL;
  if (need > (size_t)LQT_STATIC_SCRATCH_BYTES) return LQT_EWORKSPACE;
  void* ws = scratch_address();
  if (!ws) return LQT_ECUDA;
  return lqt_scan_value(p, el, S, v, zeta, ws, (size_t)LQT_STATIC_SCRATCH_BYTES, stream);
}
