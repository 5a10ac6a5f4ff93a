// The sequential method of Sec. VI-A on ONE GPU thread: the comparison
// baseline for the parallel solver.  RK4 of the Riccati ODEs for S, v (Sec.
// II-B, eq. LQT_differential_S_v) and zeta backward over the K-step fine
// grid, then RK4 of the closed-loop ODE (eq. optimal_trajectory_ODE_LQT with
// eq. LQT_optimal_control) forward, with S, v at the step midpoints from the
// cubic Hermite interpolant of the backward solution.
#include <cuda_runtime.h>

#include "lqt_device.cuh"
#include "lqt_internal.h"
#include "lqt_riccati.cuh"

namespace lqt {

struct SeqArgs {
  int64_t T;
  int32_t K, m;
  const double* t;
  Coefs cf;
  const double* x0;
  const double *termJ, *termEta, *termZeta;  // terminal values S(t_T), v(t_T), zeta(t_T)
  double* grid;  // [(K T + 1)][ric_doubles]
  double *S, *v, *zeta, *x, *u, *cost;
};

template <int N, int M>
__global__ void sequential_kernel(SeqArgs a) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  constexpr int RD = ric_doubles<N>();
  constexpr int NS = Dim<N>::NS;
  const int32_t K = a.K;
  const int64_t T = a.T;
  const Coefs& cf = a.cf;
  RicState<N> y, yt, yn, k;
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = i; j < N; ++j) y.S[sidx<N>(i, j)] = a.termJ[i * N + j];
#pragma unroll
  for (int i = 0; i < N; ++i) y.v[i] = a.termEta[i];
  y.zeta = *a.termZeta;
  auto store = [&](int64_t idx, const RicState<N>& s) {
    double* g = a.grid + idx * RD;
#pragma unroll
    for (int i = 0; i < NS; ++i) g[i] = s.S[i];
#pragma unroll
    for (int i = 0; i < N; ++i) g[NS + i] = s.v[i];
    g[NS + N] = s.zeta;
  };
  auto load = [&](int64_t idx, RicState<N>& s) {
    const double* g = a.grid + idx * RD;
#pragma unroll
    for (int i = 0; i < NS; ++i) s.S[i] = g[i];
#pragma unroll
    for (int i = 0; i < N; ++i) s.v[i] = g[NS + i];
    s.zeta = g[NS + N];
  };
  store(K * T, y);
  for (int64_t j = T - 1; j >= 0; --j) {
    const double h = (a.t[j + 1] - a.t[j]) / K;
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
      store(j * K + i, y);
    }
  }
  // boundary outputs
  for (int64_t j = 0; j <= T; ++j) {
    RicState<N> s;
    load(j * K, s);
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
      for (int l = 0; l < N; ++l) a.S[j * N * N + i * N + l] = s.S[sidx<N>(i, l)];
#pragma unroll
    for (int i = 0; i < N; ++i) a.v[j * N + i] = s.v[i];
    if (a.zeta) a.zeta[j] = s.zeta;
  }
  // forward rollout
  double x[N];
#pragma unroll
  for (int i = 0; i < N; ++i) {
    x[i] = a.x0[i];
    a.x[i] = x[i];
  }
  for (int64_t j = 0; j < T; ++j) {
    const double h = (a.t[j + 1] - a.t[j]) / K;
    RicState<N> y0, y1, ym, d0, d1;
    load(j * K, y0);
    {
      const double* F = cf.F.ptr + sample_index(cf.F.mode, j, 0, K) * N * N;
      const double* c = cf.c.ptr ? cf.c.ptr + sample_index(cf.c.mode, j, 0, K) * N : nullptr;
      const double* Lt = cf.Lt.ptr + sample_index(cf.Lt.mode, j, 0, K) * N * M;
      const double* Q = cf.Q.ptr + sample_index(cf.Q.mode, j, 0, K) * N * N;
      const double* qr = cf.qr.ptr + sample_index(cf.qr.mode, j, 0, K) * (N + 1);
      riccati_rhs<N, M>(y0, F, c, Lt, Q, qr, d0);
    }
    for (int32_t i = 0; i < K; ++i) {
      load(j * K + i + 1, y1);
      const int32_t ps[3] = {2 * i, 2 * i + 1, 2 * i + 2};
      const double *F[3], *c[3], *Lt[3];
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        F[q] = cf.F.ptr + sample_index(cf.F.mode, j, ps[q], K) * N * N;
        c[q] = cf.c.ptr ? cf.c.ptr + sample_index(cf.c.mode, j, ps[q], K) * N : nullptr;
        Lt[q] = cf.Lt.ptr + sample_index(cf.Lt.mode, j, ps[q], K) * N * M;
      }
      {
        const double* Q = cf.Q.ptr + sample_index(cf.Q.mode, j, ps[2], K) * N * N;
        const double* qr = cf.qr.ptr + sample_index(cf.qr.mode, j, ps[2], K) * (N + 1);
        riccati_rhs<N, M>(y1, F[2], c[2], Lt[2], Q, qr, d1);
      }
      // Hermite midpoint y(t + h/2) = (y0 + y1)/2 + h (y0' - y1')/8
#pragma unroll
      for (int q = 0; q < NS; ++q) ym.S[q] = fma(0.125 * h, d0.S[q] - d1.S[q], 0.5 * (y0.S[q] + y1.S[q]));
#pragma unroll
      for (int q = 0; q < N; ++q) ym.v[q] = fma(0.125 * h, d0.v[q] - d1.v[q], 0.5 * (y0.v[q] + y1.v[q]));
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
      for (int q = 0; q < N; ++q) x[q] = fma(h / 6.0, kx[q], ax[q]);
      y0 = y1;
      d0 = d1;
    }
#pragma unroll
    for (int i = 0; i < N; ++i) a.x[(j + 1) * N + i] = x[i];
  }
  // controls u_k = Ku (v_k - S_k x_k) and the cost
  for (int64_t kb = 0; kb <= T; ++kb) {
    if (!a.u) break;
    const double* Sk = a.S + kb * N * N;
    const double* xk = a.x + kb * N;
    double e[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
      double s = a.v[kb * N + i];
#pragma unroll
      for (int l = 0; l < N; ++l) s = fma(-Sk[i * N + l], xk[l], s);
      e[i] = s;
    }
    const double* Kk = cf.Ku + (cf.Ku_per_boundary ? kb * a.m * N : 0);
    for (int q = 0; q < a.m; ++q) {
      double s = 0.0;
#pragma unroll
      for (int l = 0; l < N; ++l) s = fma(Kk[q * N + l], e[l], s);
      a.u[kb * a.m + q] = s;
    }
  }
  if (a.cost) {
    double c = a.zeta ? a.zeta[0] : 0.0;
#pragma unroll
    for (int i = 0; i < N; ++i) {
      double s = 0.0;
#pragma unroll
      for (int l = 0; l < N; ++l) s = fma(a.S[i * N + l], a.x0[l], s);
      c = fma(a.x0[i], fma(0.5, s, -a.v[i]), c);
    }
    *a.cost = c;
  }
}

size_t sequential_workspace_bytes(int32_t n, int64_t T, int32_t K) {
  const size_t rd = (size_t)n * (n + 1) / 2 + n + 1;
  // fine-grid solution + a terminal element (n x n J, eta, zeta and scratch)
  return ((size_t)K * T + 1) * rd * sizeof(double) + 4 * (size_t)n * n * sizeof(double) + 4096;
}

template <int N, int M>
static void launch_seq_nm(const SeqArgs& a, cudaStream_t st) {
  sequential_kernel<N, M><<<1, 32, 0, st>>>(a);
  count_launch();
}

template <int N>
static cudaError_t launch_seq_n(const SeqArgs& a, int M, cudaStream_t st) {
  switch (M) {
    case 1: launch_seq_nm<N, 1>(a, st); break;
    case 2: if constexpr (N >= 2) { launch_seq_nm<N, 2>(a, st); break; } else return cudaErrorInvalidValue;
    case 4: if constexpr (N >= 3) { launch_seq_nm<N, 4>(a, st); break; } else return cudaErrorInvalidValue;
    case 8: if constexpr (N >= 8) { launch_seq_nm<N, 8>(a, st); break; } else return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
  }
  return cudaSuccess;
}

// The terminal values S(t_T) = Hf'Xf Hf, v(t_T) = Hf'Xf rf, zeta(t_T) =
// rf'Xf rf / 2 come from the same kernel as the terminal element.
cudaError_t launch_sequential(const lqt_problem& p, const Layout& lay, const Coefs& cf, const double* x0, double* S,
                              double* v, double* zeta, double* x, double* u, double* cost, char* ws,
                              cudaStream_t st) {
  (void)lay;
  const int n = p.n;
  char* cur = ws;
  double* grid = (double*)cur;
  cur += ((size_t)p.K * p.T + 1) * ((size_t)n * (n + 1) / 2 + n + 1) * sizeof(double);
  cur = (char*)(((uintptr_t)cur + 255) & ~(uintptr_t)255);
  double* termJ = (double*)cur;
  double* termEta = termJ + n * n;
  double* termZeta = termEta + n;
  SeqArgs a;
  a.T = p.T; a.K = p.K; a.m = p.m; a.t = p.t; a.cf = cf; a.x0 = x0;
  a.termJ = termJ; a.termEta = termEta; a.termZeta = termZeta;
  a.grid = grid; a.S = S; a.v = v; a.zeta = zeta; a.x = x; a.u = u; a.cost = cost;
  cudaError_t e = launch_terminal_values(p, termJ, termEta, termZeta, st);
  if (e != cudaSuccess) return e;
  switch (n) {
    case 1: return launch_seq_n<1>(a, lay.M, st);
    case 2: return launch_seq_n<2>(a, lay.M, st);
    case 3: return launch_seq_n<3>(a, lay.M, st);
    case 4: return launch_seq_n<4>(a, lay.M, st);
    case 8: return launch_seq_n<8>(a, lay.M, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace lqt
