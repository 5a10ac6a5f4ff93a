// Throughput probe of the FMA pipes (lqt_probe_fma_rate): the roofline
// denominators of the solver's kernels, measured on the device they run on.
//
// Each thread runs CH independent multiply-add chains x <- x a + b for `iters`
// rounds, so a warp always has CH independent FMA instructions to issue; with
// enough warps per SM the time is the pipe's issue rate.  Lanes at or above
// `active_lanes` of each warp skip the loop, which measures what a partially
// active warp instruction costs.
#include <cuda_runtime.h>

#include "lqt_internal.h"

namespace lqt {

template <typename T, int CH>
__global__ void fma_chains_kernel(T* out, int iters, T a, T b, int active_lanes) {
  T x[CH];
#pragma unroll
  for (int c = 0; c < CH; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
  if ((int)(threadIdx.x & 31) < active_lanes) {
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int c = 0; c < CH; ++c) x[c] = fma(x[c], a, b);
    }
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < CH; ++c) s += x[c];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace lqt

extern "C" lqt_status lqt_probe_fma_rate(int32_t precision, int32_t blocks, int32_t threads, int32_t iters,
                                         int32_t active_lanes, double* out, void* stream) {
  using namespace lqt;
  if (precision < 0 || precision > 1 || blocks < 1 || threads < 32 || threads > 1024 || threads % 32 != 0 ||
      iters < 1 || active_lanes < 1 || active_lanes > 32 || !out)
    return LQT_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  if (precision == 0)
    fma_chains_kernel<double, 8><<<blocks, threads, 0, st>>>(out, iters, 0.999999, 1e-7, active_lanes);
  else
    fma_chains_kernel<float, 8><<<blocks, threads, 0, st>>>((float*)out, iters, 0.999999f, 1e-7f, active_lanes);
  return cudaGetLastError() == cudaSuccess ? LQT_OK : LQT_ECUDA;
}
