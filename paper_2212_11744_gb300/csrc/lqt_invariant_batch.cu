// Batched kernels of the time-invariant element build (lqt_invariant.cu):
// one thread per boundary of the concatenation of a batch's problems.
#include <cuda_runtime.h>

#include "lqt_device.cuh"
#include "lqt_internal.h"
#include "lqt_invariant.cuh"

namespace lqt {

// Batches: one thread per boundary of the concatenation (terminal elements as
// in the general batched build: Hf = identity).
template <int N, int M>
__global__ void __launch_bounds__(128) inv_batch_build_kernel(BatchDev bd, const double* tables, ElemPtrs out) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= bd.total) return;
  const int32_t b = batch_find(bd.off, bd.B, g);
  const BatchProb& P = bd.probs[b];
  const int64_t j = g - P.off;
  if (j < P.T) {
    inv_element<N, M>(P.cf, P.t, j, bd.K, tables + (int64_t)b * inv_table_doubles(N, M, bd.K), out, g);
    return;
  }
  double eta[N];
  double z = 0.0;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    double e = 0.0;
    if (P.rf)
      for (int l = 0; l < N; ++l) e = fma(P.Xf[i * N + l], P.rf[l], e);
    eta[i] = e;
    if (P.rf) z = fma(P.rf[i], e, z);
  }
  for (int e = 0; e < N * N; ++e) {
    const int i = e / N, c = e % N;
    out.A[g * N * N + e] = 0.0;
    out.C[g * N * N + e] = 0.0;
    out.J[g * N * N + e] = 0.5 * (P.Xf[i * N + c] + P.Xf[c * N + i]);
  }
#pragma unroll
  for (int i = 0; i < N; ++i) {
    out.b[g * N + i] = 0.0;
    out.eta[g * N + i] = eta[i];
  }
  if (out.zeta) out.zeta[g] = 0.5 * z;
}

// n = 64: one warp per boundary of the concatenation.
__global__ void __launch_bounds__(32) inv_batch_build_warp_kernel(BatchDev bd, const double* tables, ElemPtrs out) {
  constexpr int N = 64, M = 16;
  extern __shared__ double sm[];
  const int lane = threadIdx.x;
  for (int64_t g = blockIdx.x; g < bd.total; g += gridDim.x) {
    const int32_t b = batch_find(bd.off, bd.B, g);
    const BatchProb& P = bd.probs[b];
    const int64_t j = g - P.off;
    if (j < P.T) {
      inv_element_warp<N, M>(lane, P.cf, P.t, j, bd.K, tables + (int64_t)b * inv_table_doubles(N, M, bd.K), out, g,
                             sm);
      continue;
    }
    // terminal element (Hf = identity): J = sym(Xf), eta = Xf rf, zeta = rf'Xf rf / 2
    double zt = 0.0;
    for (int i = lane; i < N; i += 32) {
      double e = 0.0;
      if (P.rf)
        for (int l = 0; l < N; ++l) e = fma(P.Xf[i * N + l], P.rf[l], e);
      out.eta[g * N + i] = e;
      out.b[g * N + i] = 0.0;
      if (P.rf) zt = fma(P.rf[i], e, zt);
    }
    for (int o = 16; o > 0; o >>= 1) zt += __shfl_xor_sync(0xffffffffu, zt, o);
    for (int e = lane; e < N * N; e += 32) {
      const int i = e / N, c = e % N;
      out.A[g * N * N + e] = 0.0;
      out.C[g * N * N + e] = 0.0;
      out.J[g * N * N + e] = 0.5 * (P.Xf[i * N + c] + P.Xf[c * N + i]);
    }
    if (lane == 0 && out.zeta) out.zeta[g] = 0.5 * zt;
    __syncwarp();
  }
}

void launch_inv_batch_build_warp(const BatchDev& bd, const double* tables, const ElemPtrs& out, cudaStream_t st) {
  const size_t smem = (4 * (2 * 64 + 1) + 16) * sizeof(double);
  const int64_t grid = bd.total < 152 * 32 ? bd.total : 152 * 32;
  inv_batch_build_warp_kernel<<<(unsigned)grid, 32, smem, st>>>(bd, tables, out);
  count_launch();
}

template <int N, int M>
void launch_inv_batch_build(const BatchDev& bd, const double* tables, const ElemPtrs& out, cudaStream_t st) {
  inv_batch_build_kernel<N, M><<<(unsigned)((bd.total + 127) / 128), 128, 0, st>>>(bd, tables, out);
  count_launch();
}

template void launch_inv_batch_build<1, 1>(const BatchDev&, const double*, const ElemPtrs&, cudaStream_t);
template void launch_inv_batch_build<2, 1>(const BatchDev&, const double*, const ElemPtrs&, cudaStream_t);
template void launch_inv_batch_build<2, 2>(const BatchDev&, const double*, const ElemPtrs&, cudaStream_t);
template void launch_inv_batch_build<3, 1>(const BatchDev&, const double*, const ElemPtrs&, cudaStream_t);
template void launch_inv_batch_build<3, 2>(const BatchDev&, const double*, const ElemPtrs&, cudaStream_t);
template void launch_inv_batch_build<3, 4>(const BatchDev&, const double*, const ElemPtrs&, cudaStream_t);
template void launch_inv_batch_build<4, 1>(const BatchDev&, const double*, const ElemPtrs&, cudaStream_t);
template void launch_inv_batch_build<4, 2>(const BatchDev&, const double*, const ElemPtrs&, cudaStream_t);
template void launch_inv_batch_build<4, 4>(const BatchDev&, const double*, const ElemPtrs&, cudaStream_t);
template void launch_inv_batch_build<8, 1>(const BatchDev&, const double*, const ElemPtrs&, cudaStream_t);
template void launch_inv_batch_build<8, 2>(const BatchDev&, const double*, const ElemPtrs&, cudaStream_t);
template void launch_inv_batch_build<8, 4>(const BatchDev&, const double*, const ElemPtrs&, cudaStream_t);
template void launch_inv_batch_build<8, 8>(const BatchDev&, const double*, const ElemPtrs&, cudaStream_t);
template void launch_inv_batch_build<16, 8>(const BatchDev&, const double*, const ElemPtrs&, cudaStream_t);

}  // namespace lqt
