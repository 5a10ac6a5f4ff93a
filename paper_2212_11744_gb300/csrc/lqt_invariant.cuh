// Device parts of the time-invariant element build shared by the
// single-problem (lqt_invariant.cu) and batched (lqt_invariant_batch.cu)
// kernels: the table layout and the per-sub-interval (b, eta, zeta)
// integration.  The method is described in lqt_invariant.cu.
#pragma once

#include <cfloat>

#include <cuda_runtime.h>

#include "lqt_device.cuh"
#include "lqt_internal.h"

namespace lqt {

constexpr int kInvMaxN = 16;
constexpr int kInvMaxM = 8;

// Table of one problem, in doubles: for RK4 step i (0..K-1) and stage st
// (0..3, in evaluation order), AL (n x M), P (n x M), A (n x n), J (n x n);
// then the element's A, C, J (full n x n each); then the integrator's own
// working buffers, kept here rather than in a thread's stack.
__host__ __device__ __forceinline__ int64_t inv_stage_doubles(int n, int M) { return 2 * n * M + 2 * n * n; }
__host__ __device__ __forceinline__ int64_t inv_work_doubles(int n, int M) {
  // four element records, AL, P, w, J F and n + 1 zeros (team integrator), which
  // also covers the thread integrator's four A, C, J triples
  return 4 * (3 * n * n + 2 * n + 1) + 2 * n * M + M + n * n + n + 1 + 8;
}
__host__ __device__ __forceinline__ int64_t inv_table_doubles(int n, int M, int K) {
  return 4 * (int64_t)K * inv_stage_doubles(n, M) + 3 * n * n + inv_work_doubles(n, M);
}

// ---------------------------------------------------------------------------
// the per-sub-interval (b, eta, zeta) integration
// ---------------------------------------------------------------------------

template <int N>
struct BEZ {
  double b[N], eta[N], zeta;
};

template <int N>
__device__ __forceinline__ void bez_axpy(BEZ<N>& y, const BEZ<N>& base, double s, const BEZ<N>& k) {
#pragma unroll
  for (int i = 0; i < N; ++i) {
    y.b[i] = fma(s, k.b[i], base.b[i]);
    y.eta[i] = fma(s, k.eta[i], base.eta[i]);
  }
  y.zeta = fma(s, k.zeta, base.zeta);
}

// db = -AL w - A c, deta = -q - F^T eta + J c + P w, dzeta = -rho/2 + |w|^2/2 +
// eta^T c with w = Lt^T eta and the stage's recorded AL, P, A, J.
template <int N, int M>
__device__ __forceinline__ void bez_rhs(const BEZ<N>& y, const double* __restrict__ rec, const double* __restrict__ F,
                                        const double* __restrict__ Lt, const double* __restrict__ c,
                                        const double* __restrict__ qr, BEZ<N>& k) {
  const double* AL = rec;
  const double* P = rec + N * M;
  const double* A = rec + 2 * N * M;
  const double* J = A + N * N;
  double w[M];
#pragma unroll
  for (int a = 0; a < M; ++a) {
    double s = 0.0;
#pragma unroll
    for (int l = 0; l < N; ++l) s = fma(Lt[l * M + a], y.eta[l], s);
    w[a] = s;
  }
  double z = -0.5 * qr[N];
#pragma unroll
  for (int a = 0; a < M; ++a) z = fma(0.5 * w[a], w[a], z);
#pragma unroll
  for (int i = 0; i < N; ++i) {
    double sb = 0.0, se = -qr[i];
#pragma unroll
    for (int a = 0; a < M; ++a) {
      sb = fma(-AL[i * M + a], w[a], sb);
      se = fma(P[i * M + a], w[a], se);
    }
#pragma unroll
    for (int l = 0; l < N; ++l) se = fma(-F[l * N + i], y.eta[l], se);
    if (c) {
#pragma unroll
      for (int l = 0; l < N; ++l) {
        sb = fma(-A[i * N + l], c[l], sb);
        se = fma(J[i * N + l], c[l], se);
      }
      z = fma(y.eta[i], c[i], z);
    }
    k.b[i] = sb;
    k.eta[i] = se;
  }
  k.zeta = z;
}

// Sub-interval j has the first one's length: equal to 1e-12 relative plus
// the rounding of the time points themselves (a linspace over [0, 100] with
// 2^20 sub-intervals has lengths that differ by ~1e-11 relative).
__device__ __forceinline__ bool same_length(const double* t, int64_t j) {
  const double h = t[j + 1] - t[j], h0 = t[1] - t[0];
  const double tol = 1e-12 * fabs(h0) + 8.0 * DBL_EPSILON * (fabs(t[j]) + fabs(t[j + 1]) + fabs(t[0]) + fabs(t[1]));
  return fabs(h - h0) <= tol;
}

// Element j of one problem into the public arrays at index g.
template <int N, int M>
__device__ __forceinline__ void inv_element(const Coefs& cf, const double* t, int64_t j, int32_t K,
                                            const double* __restrict__ table, const ElemPtrs& out, int64_t g) {
  const double h = (t[j + 1] - t[j]) / K;
  if (!same_length(t, j)) flag(kStatusNonUniform);
  constexpr int64_t SD = 2 * N * M + 2 * N * N;
  const double* F = cf.F.ptr;
  const double* Lt = cf.Lt.ptr;
  BEZ<N> y, yn, yt, k;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    y.b[i] = 0.0;
    y.eta[i] = 0.0;
  }
  y.zeta = 0.0;
  for (int32_t i = K - 1; i >= 0; --i) {
    const double* rec = table + 4 * (int64_t)i * SD;
    const int32_t ps[3] = {2 * i + 2, 2 * i + 1, 2 * i};
    const double *c[3], *qr[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      c[q] = cf.c.ptr ? cf.c.ptr + sample_index(cf.c.mode, j, ps[q], K) * N : nullptr;
      qr[q] = cf.qr.ptr + sample_index(cf.qr.mode, j, ps[q], K) * (N + 1);
    }
    bez_rhs<N, M>(y, rec, F, Lt, c[0], qr[0], k);
    bez_axpy(yn, y, -h / 6.0, k);
    bez_axpy(yt, y, -0.5 * h, k);
    bez_rhs<N, M>(yt, rec + SD, F, Lt, c[1], qr[1], k);
    bez_axpy(yn, yn, -h / 3.0, k);
    bez_axpy(yt, y, -0.5 * h, k);
    bez_rhs<N, M>(yt, rec + 2 * SD, F, Lt, c[1], qr[1], k);
    bez_axpy(yn, yn, -h / 3.0, k);
    bez_axpy(yt, y, -h, k);
    bez_rhs<N, M>(yt, rec + 3 * SD, F, Lt, c[2], qr[2], k);
    bez_axpy(y, yn, -h / 6.0, k);
  }
  const double* fin = table + 4 * (int64_t)K * SD;
  double* A = out.A + g * N * N;
  double* C = out.C + g * N * N;
  double* J = out.J + g * N * N;
  for (int e = 0; e < N * N; ++e) {
    A[e] = fin[e];
    C[e] = fin[N * N + e];
    J[e] = fin[2 * N * N + e];
  }
#pragma unroll
  for (int i = 0; i < N; ++i) {
    out.b[g * N + i] = y.b[i];
    out.eta[g * N + i] = y.eta[i];
  }
  if (out.zeta) out.zeta[g] = y.zeta;
}

// The same (b, eta, zeta) integration with one warp per sub-interval (n = 64:
// the stage matrices' rows spread over the lanes).  sm: 4 (2N+1) + M doubles.
template <int N, int M>
__device__ __forceinline__ void inv_element_warp(int lane, const Coefs& cf, const double* t, int64_t j, int32_t K,
                                                 const double* __restrict__ table, const ElemPtrs& out, int64_t g,
                                                 double* sm) {
  constexpr int V = 2 * N + 1;  // b, eta, zeta
  constexpr int64_t SD = 2 * N * M + 2 * N * N;
  double* y = sm;
  double* yn = y + V;
  double* yt = yn + V;
  double* k = yt + V;
  double* w = k + V;
  const double h = (t[j + 1] - t[j]) / K;
  if (lane == 0 && !same_length(t, j)) flag(kStatusNonUniform);
  const double* F = cf.F.ptr;
  const double* Lt = cf.Lt.ptr;
  for (int e = lane; e < V; e += 32) y[e] = 0.0;
  __syncwarp();
  // k = f(yy) at stage record rec with samples c, qr
  auto rhs = [&](const double* yy, const double* rec, const double* c, const double* qr) {
    const double* AL = rec;
    const double* P = rec + N * M;
    const double* A = rec + 2 * N * M;
    const double* J = A + N * N;
    const double* eta = yy + N;
    for (int a = lane; a < M; a += 32) {
      double s = 0.0;
      for (int l = 0; l < N; ++l) s = fma(Lt[l * M + a], eta[l], s);
      w[a] = s;
    }
    __syncwarp();
    for (int i = lane; i < N; i += 32) {
      double sb = 0.0, se = -qr[i];
      for (int a = 0; a < M; ++a) {
        sb = fma(-AL[i * M + a], w[a], sb);
        se = fma(P[i * M + a], w[a], se);
      }
      for (int l = 0; l < N; ++l) se = fma(-F[l * N + i], eta[l], se);
      if (c)
        for (int l = 0; l < N; ++l) {
          sb = fma(-A[i * N + l], c[l], sb);
          se = fma(J[i * N + l], c[l], se);
        }
      k[i] = sb;
      k[N + i] = se;
    }
    if (lane == 0) {
      double z = -0.5 * qr[N];
      for (int a = 0; a < M; ++a) z = fma(0.5 * w[a], w[a], z);
      if (c)
        for (int l = 0; l < N; ++l) z = fma(eta[l], c[l], z);
      k[2 * N] = z;
    }
    __syncwarp();
  };
  auto axpy = [&](double* o, const double* base, double sc) {
    for (int e = lane; e < V; e += 32) o[e] = fma(sc, k[e], base[e]);
    __syncwarp();
  };
  for (int32_t i = K - 1; i >= 0; --i) {
    const double* rec = table + 4 * (int64_t)i * SD;
    const int32_t ps[3] = {2 * i + 2, 2 * i + 1, 2 * i};
    const double *c[3], *qr[3];
    for (int q = 0; q < 3; ++q) {
      c[q] = cf.c.ptr ? cf.c.ptr + sample_index(cf.c.mode, j, ps[q], K) * N : nullptr;
      qr[q] = cf.qr.ptr + sample_index(cf.qr.mode, j, ps[q], K) * (N + 1);
    }
    rhs(y, rec, c[0], qr[0]);
    axpy(yn, y, -h / 6.0);
    axpy(yt, y, -0.5 * h);
    rhs(yt, rec + SD, c[1], qr[1]);
    axpy(yn, yn, -h / 3.0);
    axpy(yt, y, -0.5 * h);
    rhs(yt, rec + 2 * SD, c[1], qr[1]);
    axpy(yn, yn, -h / 3.0);
    axpy(yt, y, -h);
    rhs(yt, rec + 3 * SD, c[2], qr[2]);
    axpy(y, yn, -h / 6.0);
  }
  const double* fin = table + 4 * (int64_t)K * SD;
  for (int e = lane; e < N * N; e += 32) {
    out.A[g * N * N + e] = fin[e];
    out.C[g * N * N + e] = fin[N * N + e];
    out.J[g * N * N + e] = fin[2 * N * N + e];
  }
  for (int i = lane; i < N; i += 32) {
    out.b[g * N + i] = y[i];
    out.eta[g * N + i] = y[N + i];
  }
  if (lane == 0 && out.zeta) out.zeta[g] = y[2 * N];
  __syncwarp();
}

}  // namespace lqt
