// FP64 / FP32 pipe probe for the roofline denominators of the LQT kernels.
// Prints (1) FMA throughput of independent chains for several block sizes and
// (2) the cost of one warp-wide FP64 FMA instruction on one sub-partition with
// 1..32 active lanes.  Stand-alone: nvcc -gencode arch=compute_103a,code=sm_103a
// -O3 fp64_peak_probe.cu -o fp64_peak_probe && ./fp64_peak_probe
#include <cstdio>
#include <cuda_runtime.h>

template <typename T, int CH>
__global__ void fma_chains(T* out, int iters, T a, T b, int active_lanes) {
  T x[CH];
#pragma unroll
  for (int c = 0; c < CH; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
  if ((int)(threadIdx.x & 31) < active_lanes) {
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int c = 0; c < CH; ++c) x[c] = x[c] * a + b;
    }
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < CH; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T, int CH>
static float time_it(int blocks, int threads, int iters, int lanes) {
  T* out;
  cudaMalloc(&out, sizeof(T) * blocks * threads);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  fma_chains<T, CH><<<blocks, threads>>>(out, iters, (T)0.999999, (T)1e-7, lanes);
  cudaEventRecord(e0);
  fma_chains<T, CH><<<blocks, threads>>>(out, iters, (T)0.999999, (T)1e-7, lanes);
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  float ms;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaFree(out);
  return ms;
}

int main() {
  int sms, clk_khz;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
  cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, 0);
  printf("SMs %d, max SM clock %.0f MHz\n", sms, clk_khz / 1e3);
  const int threads_list[] = {32, 64, 128, 256, 512, 1024};
  for (int t : threads_list) {
    float ms = time_it<double, 8>(sms, t, 20000, 32);
    printf("DFMA  %4d threads/SM: %8.3f ms  %.3f TFLOP/s\n", t, ms, 2.0 * 8 * 20000.0 * sms * t / ms / 1e9);
  }
  for (int t : threads_list) {
    float ms = time_it<float, 8>(sms, t, 100000, 32);
    printf("FFMA  %4d threads/SM: %8.3f ms  %.3f TFLOP/s\n", t, ms, 2.0 * 8 * 100000.0 * sms * t / ms / 1e9);
  }
  const int lanes_list[] = {1, 4, 8, 32};
  for (int l : lanes_list) {
    float ms = time_it<double, 8>(1, 32, 5000, l);
    printf("one warp, %2d active lanes: %.1f ns per FP64 FMA instruction\n", l, ms * 1e6 / (8 * 5000.0));
  }
  return 0;
}
