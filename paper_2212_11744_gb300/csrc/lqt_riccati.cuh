// Riccati-form right-hand sides shared by the sequential sweep (lqt_seq.cu)
// and the within-block densification (lqt_dense.cu): the ODEs of S, v, zeta
// (Sec. II-B, eq. LQT_differential_S_v, plus the zeta equation) in t, and the
// closed-loop state ODE (eq. optimal_trajectory_ODE_LQT with eq.
// LQT_optimal_control), written with the factor B = Lt Lt^T.
#pragma once

#include "lqt_device.cuh"

namespace lqt {

template <int N>
struct RicState {
  double S[Dim<N>::NS];
  double v[N];
  double zeta;
};

template <int N>
__host__ __device__ constexpr int ric_doubles() {
  return Dim<N>::NS + N + 1;
}

// dS/dt = -(SF)^T - SF - Q + (S Lt)(S Lt)^T
// dv/dt = -q + S c - F^T v + (S Lt)(Lt^T v)
// dz/dt = -rho/2 + |Lt^T v|^2 / 2 + v^T c
template <int N, int M>
__device__ __forceinline__ void riccati_rhs(const RicState<N>& y, const double* __restrict__ F,
                                            const double* __restrict__ c, const double* __restrict__ Lt,
                                            const double* __restrict__ Q, const double* __restrict__ qr,
                                            RicState<N>& k) {
  double SL[N * M], w[M], SF[N * N];
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int a = 0; a < M; ++a) {
      double s = 0.0;
#pragma unroll
      for (int l = 0; l < N; ++l) s = fma(y.S[sidx<N>(i, l)], Lt[l * M + a], s);
      SL[i * M + a] = s;
    }
#pragma unroll
  for (int a = 0; a < M; ++a) {
    double s = 0.0;
#pragma unroll
    for (int l = 0; l < N; ++l) s = fma(Lt[l * M + a], y.v[l], s);
    w[a] = s;
  }
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = 0; j < N; ++j) {
      double s = 0.0;
#pragma unroll
      for (int l = 0; l < N; ++l) s = fma(y.S[sidx<N>(i, l)], F[l * N + j], s);
      SF[i * N + j] = s;
    }
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = i; j < N; ++j) {
      double s = -Q[i * N + j] - SF[i * N + j] - SF[j * N + i];
#pragma unroll
      for (int a = 0; a < M; ++a) s = fma(SL[i * M + a], SL[j * M + a], s);
      k.S[sidx<N>(i, j)] = s;
    }
  double z = -0.5 * qr[N];
#pragma unroll
  for (int a = 0; a < M; ++a) z = fma(0.5 * w[a], w[a], z);
#pragma unroll
  for (int i = 0; i < N; ++i) {
    double s = -qr[i];
    if (c) {
#pragma unroll
      for (int l = 0; l < N; ++l) s = fma(y.S[sidx<N>(i, l)], c[l], s);
    }
#pragma unroll
    for (int l = 0; l < N; ++l) s = fma(-F[l * N + i], y.v[l], s);
#pragma unroll
    for (int a = 0; a < M; ++a) s = fma(SL[i * M + a], w[a], s);
    k.v[i] = s;
    if (c) z = fma(y.v[i], c[i], z);
  }
  k.zeta = z;
}

// dx/dt = F x - Lt Lt^T (S x - v) + c
template <int N, int M>
__device__ __forceinline__ void closed_loop_rhs(const double* __restrict__ S, const double* __restrict__ v,
                                                const double* __restrict__ x, const double* __restrict__ F,
                                                const double* __restrict__ c, const double* __restrict__ Lt,
                                                double* __restrict__ dx) {
  double e[N], w[M];
#pragma unroll
  for (int i = 0; i < N; ++i) {
    double s = -v[i];
#pragma unroll
    for (int l = 0; l < N; ++l) s = fma(S[sidx<N>(i, l)], x[l], s);
    e[i] = s;
  }
#pragma unroll
  for (int a = 0; a < M; ++a) {
    double s = 0.0;
#pragma unroll
    for (int l = 0; l < N; ++l) s = fma(Lt[l * M + a], e[l], s);
    w[a] = s;
  }
#pragma unroll
  for (int i = 0; i < N; ++i) {
    double s = c ? c[i] : 0.0;
#pragma unroll
    for (int l = 0; l < N; ++l) s = fma(F[i * N + l], x[l], s);
#pragma unroll
    for (int a = 0; a < M; ++a) s = fma(-Lt[i * M + a], w[a], s);
    dx[i] = s;
  }
}

template <int N>
__device__ __forceinline__ void ric_axpy(RicState<N>& y, const RicState<N>& base, double s, const RicState<N>& k) {
#pragma unroll
  for (int i = 0; i < Dim<N>::NS; ++i) y.S[i] = fma(s, k.S[i], base.S[i]);
#pragma unroll
  for (int i = 0; i < N; ++i) y.v[i] = fma(s, k.v[i], base.v[i]);
  y.zeta = fma(s, k.zeta, base.zeta);
}

}  // namespace lqt
