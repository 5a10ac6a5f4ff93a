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
