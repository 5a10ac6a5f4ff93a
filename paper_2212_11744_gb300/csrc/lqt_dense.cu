// Within-block densification (lqt_densify): the optimal solution at every RK4
// sub-step t_j + i h_j, i = 0..K-1, of every sub-interval, from the solution at
// the sub-interval boundaries (Sec. IV-E: the trajectory inside a
// sub-interval; Sec. VI-A: the K-step fine grid).
//
// Every sub-interval j is independent (one thread each):
//   backward: K classical RK4 steps of the Riccati ODEs for S, v, zeta (Sec.
//     II-B, eq. LQT_differential_S_v) from the boundary values at t_{j+1}
//     down to t_j, with the same half-step coefficient samples as the element
//     build; the sub-step values y_i (i = 1..K-1) go straight to the outputs,
//     the Riccati right-hand side at each y_i (the Hermite slopes) stays in a
//     per-thread array;
//   forward: K - 1 RK4 steps of the closed-loop ODE (eq.
//     optimal_trajectory_ODE_LQT) from x_j, with S, v at the step midpoints
//     from the cubic Hermite interpolant y(t + h/2) = (y_i + y_{i+1})/2 +
//     h (y_i' - y_{i+1}')/8;
//   controls u = U^-1 L^T (v - S x) (eq. LQT_optimal_control) with the U, L
//     sample at each sub-step: the prepared gain Ku when L and U do not vary
//     within a sub-interval, else a Cholesky solve of that sub-step's U.
// At the boundaries (i = 0 and the final point) the outputs are the given
// boundary solution.
#include <cuda_runtime.h>

#include "lqt_device.cuh"
#include "lqt_internal.h"
#include "lqt_riccati.cuh"

namespace lqt {

constexpr int kDenseMaxK = 16;

struct DenseArgs {
  int64_t T;
  int32_t K, m;
  const double* t;
  Coefs cf;
  Coef L, U;  // raw samples: n x m and m x m
  const double *S, *v, *zeta, *x;  // boundary solution, [T+1]
  double *Sd, *vd, *zd, *xd, *ud;  // [T K + 1]
  int ku_exact;  // L and U constant within every sub-interval: cf.Ku holds U^-1 L^T for every sub-step
};

// u = U^-1 L^T e for one sample (U symmetric positive definite, m <= MM, the
// padded factor width).
template <int N, int MM>
__device__ __forceinline__ void control_from(const double* __restrict__ L, const double* __restrict__ U, int m,
                                             const double* e, double* __restrict__ u) {
  double R[MM * MM], w[MM];
  for (int a = 0; a < m; ++a) {
    double s = 0.0;
#pragma unroll
    for (int l = 0; l < N; ++l) s = fma(L[l * m + a], e[l], s);
    w[a] = s;
    for (int b = 0; b < m; ++b) R[a * MM + b] = U[a * m + b];
  }
  // Cholesky U = R R^T (lower triangle of R), then two triangular solves
  for (int k = 0; k < m; ++k) {
    double d = R[k * MM + k];
    for (int l = 0; l < k; ++l) d = fma(-R[k * MM + l], R[k * MM + l], d);
    d = sqrt(d);
    R[k * MM + k] = d;
    const double inv = 1.0 / d;
    for (int i = k + 1; i < m; ++i) {
      double s = R[i * MM + k];
      for (int l = 0; l < k; ++l) s = fma(-R[i * MM + l], R[k * MM + l], s);
      R[i * MM + k] = s * inv;
    }
  }
  for (int i = 0; i < m; ++i) {
    double s = w[i];
    for (int l = 0; l < i; ++l) s = fma(-R[i * MM + l], w[l], s);
    w[i] = s / R[i * MM + i];
  }
  for (int i = m - 1; i >= 0; --i) {
    double s = w[i];
    for (int l = i + 1; l < m; ++l) s = fma(-R[l * MM + i], w[l], s);
    w[i] = s / R[i * MM + i];
  }
  for (int a = 0; a < m; ++a) u[a] = w[a];
}

// Returns false if a value is not finite.
template <int N>
__device__ __forceinline__ bool store_values(const RicState<N>& y, double* S, double* v, double* z) {
  bool ok = isfinite(y.zeta);
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int l = 0; l < N; ++l) S[i * N + l] = y.S[sidx<N>(i, l)];
#pragma unroll
  for (int i = 0; i < Dim<N>::NS; ++i) ok = ok && isfinite(y.S[i]);
#pragma unroll
  for (int i = 0; i < N; ++i) {
    v[i] = y.v[i];
    ok = ok && isfinite(y.v[i]);
  }
  *z = y.zeta;
  return ok;
}

template <int N>
__device__ __forceinline__ void load_values(RicState<N>& y, const double* S, const double* v, const double* z) {
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int l = i; l < N; ++l) y.S[sidx<N>(i, l)] = S[i * N + l];
#pragma unroll
  for (int i = 0; i < N; ++i) y.v[i] = v[i];
  y.zeta = *z;
}

template <int N, int M>
__device__ __forceinline__ void control_at(const DenseArgs& a, int64_t j, int32_t p, const RicState<N>& y,
                                           const double* x, double* u) {
  double e[N];
#pragma unroll
  for (int i = 0; i < N; ++i) {
    double s = y.v[i];
#pragma unroll
    for (int l = 0; l < N; ++l) s = fma(-y.S[sidx<N>(i, l)], x[l], s);
    e[i] = s;
  }
  if (a.ku_exact) {
    // the prepared gain of the sub-interval (of the final boundary at p = 2K)
    const int64_t k = (p == 2 * a.K) ? j + 1 : j;
    const double* Kk = a.cf.Ku + (a.cf.Ku_per_boundary ? k * a.m * N : 0);
    for (int q = 0; q < a.m; ++q) {
      double s = 0.0;
#pragma unroll
      for (int l = 0; l < N; ++l) s = fma(Kk[q * N + l], e[l], s);
      u[q] = s;
    }
    return;
  }
  const double* L = a.L.ptr + sample_index(a.L.mode, j, p, a.K) * N * a.m;
  const double* U = a.U.ptr + sample_index(a.U.mode, j, p, a.K) * a.m * a.m;
  control_from<N, M>(L, U, a.m, e, u);
}

template <int N, int M>
__global__ void __launch_bounds__(128) densify_kernel(DenseArgs a) {
  constexpr int NS = Dim<N>::NS;
  const int32_t K = a.K;
  const Coefs& cf = a.cf;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < a.T; j += (int64_t)gridDim.x * blockDim.x) {
    const double h = (a.t[j + 1] - a.t[j]) / K;
    const int64_t g0 = j * K;
    RicState<N> D[kDenseMaxK + 1];
    RicState<N> y, yt, yn, k;
    bool ok = true;
    load_values<N>(y, a.S + (j + 1) * N * N, a.v + (j + 1) * N, a.zeta + j + 1);
    // backward K steps from t_{j+1}
    for (int32_t i = K - 1; i >= 0; --i) {
      const int32_t ps[3] = {2 * i + 2, 2 * i + 1, 2 * i};
      const double *F[3], *c[3], *Lt[3], *Q[3], *qr[3];
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        F[q] = cf.F.ptr + sample_index(cf.F.mode, j, ps[q], K) * N * N;
        c[q] = cf.c.ptr ? cf.c.ptr + sample_index(cf.c.mode, j, ps[q], K) * N : nullptr;
        Lt[q] = cf.Lt.ptr + sample_index(cf.Lt.mode, j, ps[q], K) * N * M;
        Q[q] = cf.Q.ptr + sample_index(cf.Q.mode, j, ps[q], K) * N * N;
        qr[q] = cf.qr.ptr + sample_index(cf.qr.mode, j, ps[q], K) * (N + 1);
      }
      riccati_rhs<N, M>(y, F[0], c[0], Lt[0], Q[0], qr[0], k);
      D[i + 1] = k;
      ric_axpy(yn, y, -h / 6.0, k);
      ric_axpy(yt, y, -0.5 * h, k);
      riccati_rhs<N, M>(yt, F[1], c[1], Lt[1], Q[1], qr[1], k);
      ric_axpy(yn, yn, -h / 3.0, k);
      ric_axpy(yt, y, -0.5 * h, k);
      riccati_rhs<N, M>(yt, F[1], c[1], Lt[1], Q[1], qr[1], k);
      ric_axpy(yn, yn, -h / 3.0, k);
      ric_axpy(yt, y, -h, k);
      riccati_rhs<N, M>(yt, F[2], c[2], Lt[2], Q[2], qr[2], k);
      ric_axpy(y, yn, -h / 6.0, k);
      if (i > 0) ok = store_values<N>(y, a.Sd + (g0 + i) * N * N, a.vd + (g0 + i) * N, a.zd + g0 + i) && ok;
    }
    // slope at t_j with block j's first sample; y now holds the re-integrated value at t_j
    {
      const double* F = cf.F.ptr + sample_index(cf.F.mode, j, 0, K) * N * N;
      const double* c = cf.c.ptr ? cf.c.ptr + sample_index(cf.c.mode, j, 0, K) * N : nullptr;
      const double* Lt = cf.Lt.ptr + sample_index(cf.Lt.mode, j, 0, K) * N * M;
      const double* Q = cf.Q.ptr + sample_index(cf.Q.mode, j, 0, K) * N * N;
      const double* qr = cf.qr.ptr + sample_index(cf.qr.mode, j, 0, K) * (N + 1);
      riccati_rhs<N, M>(y, F, c, Lt, Q, qr, D[0]);
    }
    // boundary point t_j: the given solution
    double x[N];
    {
      RicState<N> yb;
      load_values<N>(yb, a.S + j * N * N, a.v + j * N, a.zeta + j);
      store_values<N>(yb, a.Sd + g0 * N * N, a.vd + g0 * N, a.zd + g0);
#pragma unroll
      for (int i = 0; i < N; ++i) {
        x[i] = a.x[j * N + i];
        a.xd[g0 * N + i] = x[i];
      }
      if (a.ud) control_at<N, M>(a, j, 0, yb, x, a.ud + g0 * a.m);
    }
    // forward K - 1 steps from x_j
    RicState<N> y0 = y;
    for (int32_t i = 0; i + 1 < K; ++i) {
      RicState<N> y1, ym;
      load_values<N>(y1, a.Sd + (g0 + i + 1) * N * N, a.vd + (g0 + i + 1) * N, a.zd + g0 + i + 1);
      const RicState<N>& d0 = D[i];
      const RicState<N>& d1 = D[i + 1];
#pragma unroll
      for (int q = 0; q < NS; ++q) ym.S[q] = fma(0.125 * h, d0.S[q] - d1.S[q], 0.5 * (y0.S[q] + y1.S[q]));
#pragma unroll
      for (int q = 0; q < N; ++q) ym.v[q] = fma(0.125 * h, d0.v[q] - d1.v[q], 0.5 * (y0.v[q] + y1.v[q]));
      const int32_t ps[3] = {2 * i, 2 * i + 1, 2 * i + 2};
      const double *F[3], *c[3], *Lt[3];
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        F[q] = cf.F.ptr + sample_index(cf.F.mode, j, ps[q], K) * N * N;
        c[q] = cf.c.ptr ? cf.c.ptr + sample_index(cf.c.mode, j, ps[q], K) * N : nullptr;
        Lt[q] = cf.Lt.ptr + sample_index(cf.Lt.mode, j, ps[q], K) * N * M;
      }
      double kx[N], ax[N], xt[N];
      closed_loop_rhs<N, M>(y0.S, y0.v, x, F[0], c[0], Lt[0], kx);
#pragma unroll
      for (int q = 0; q < N; ++q) {
        ax[q] = fma(h / 6.0, kx[q], x[q]);
        xt[q] = fma(0.5 * h, kx[q], x[q]);
      }
      closed_loop_rhs<N, M>(ym.S, ym.v, xt, F[1], c[1], Lt[1], kx);
#pragma unroll
      for (int q = 0; q < N; ++q) {
        ax[q] = fma(h / 3.0, kx[q], ax[q]);
        xt[q] = fma(0.5 * h, kx[q], x[q]);
      }
      closed_loop_rhs<N, M>(ym.S, ym.v, xt, F[1], c[1], Lt[1], kx);
#pragma unroll
      for (int q = 0; q < N; ++q) {
        ax[q] = fma(h / 3.0, kx[q], ax[q]);
        xt[q] = fma(h, kx[q], x[q]);
      }
      closed_loop_rhs<N, M>(y1.S, y1.v, xt, F[2], c[2], Lt[2], kx);
#pragma unroll
      for (int q = 0; q < N; ++q) {
        x[q] = fma(h / 6.0, kx[q], ax[q]);
        a.xd[(g0 + i + 1) * N + q] = x[q];
        ok = ok && isfinite(x[q]);
      }
      if (a.ud) control_at<N, M>(a, j, 2 * (i + 1), y1, x, a.ud + (g0 + i + 1) * a.m);
      y0 = y1;
    }
    if (!ok) flag(kStatusNonFinite);
    // final point t_T
    if (j == a.T - 1) {
      const int64_t g = a.T * K;
      RicState<N> yb;
      load_values<N>(yb, a.S + a.T * N * N, a.v + a.T * N, a.zeta + a.T);
      store_values<N>(yb, a.Sd + g * N * N, a.vd + g * N, a.zd + g);
      double xT[N];
#pragma unroll
      for (int i = 0; i < N; ++i) {
        xT[i] = a.x[a.T * N + i];
        a.xd[g * N + i] = xT[i];
      }
      if (a.ud) control_at<N, M>(a, j, 2 * K, yb, xT, a.ud + g * a.m);
    }
  }
}

template <int N, int M>
static cudaError_t launch_dense_nm(const DenseArgs& a, cudaStream_t st) {
  constexpr int threads = 128;
  int64_t blocks = (a.T + threads - 1) / threads;
  if (blocks > 152 * 64) blocks = 152 * 64;
  densify_kernel<N, M><<<(unsigned)blocks, threads, 0, st>>>(a);
  count_launch();
  return cudaGetLastError();
}

template <int N>
static cudaError_t launch_dense_n(const DenseArgs& a, int M, cudaStream_t st) {
  switch (M) {
    case 1: return launch_dense_nm<N, 1>(a, st);
    case 2: if constexpr (N >= 2) return launch_dense_nm<N, 2>(a, st); else return cudaErrorInvalidValue;
    case 4: if constexpr (N >= 3) return launch_dense_nm<N, 4>(a, st); else return cudaErrorInvalidValue;
    case 8: if constexpr (N >= 8) return launch_dense_nm<N, 8>(a, st); else return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
  }
}

bool densify_supported(const lqt_problem& p) { return p.n <= 8 && p.K <= kDenseMaxK; }

cudaError_t launch_densify(const lqt_problem& p, const Layout& lay, const Coefs& cf, const double* S, const double* v,
                           const double* zeta, const double* x, double* Sd, double* vd, double* zd, double* xd,
                           double* ud, cudaStream_t st) {
  DenseArgs a;
  a.T = p.T; a.K = p.K; a.m = p.m; a.t = p.t; a.cf = cf;
  a.L = Coef{(const double*)p.L.ptr, p.L.mode};
  a.U = Coef{(const double*)p.U.ptr, p.U.mode};
  a.S = S; a.v = v; a.zeta = zeta; a.x = x;
  a.Sd = Sd; a.vd = vd; a.zd = zd; a.xd = xd; a.ud = ud;
  // Ku (prepared at the boundaries from sample (j, 0), or (T-1, 2K) at T) is
  // the gain of every sub-step when no coefficient of it varies per stage
  a.ku_exact = (p.L.mode != LQT_PER_STAGE && p.U.mode != LQT_PER_STAGE && cf.Ku != nullptr) ? 1 : 0;
  switch (p.n) {
    case 1: return launch_dense_n<1>(a, lay.M, st);
    case 2: return launch_dense_n<2>(a, lay.M, st);
    case 3: return launch_dense_n<3>(a, lay.M, st);
    case 4: return launch_dense_n<4>(a, lay.M, st);
    case 8: return launch_dense_n<8>(a, lay.M, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace lqt
