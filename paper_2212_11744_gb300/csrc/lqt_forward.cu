// Elements from the forward conditional HJB ODEs (Sec. IV-C, Theorem
// Forward_HJB_LQT), for Method 2 of the optimal-trajectory recovery (Sec. IV-E).
// One thread per sub-interval j (n <= 8; n = 16 and 64 run one team per
// element, build_forward_team_kernel in lqt_team.cu): K classical RK4 steps
// in tau from the boundary A = I, b = C = eta = J = 0, zeta = 0 at tau = t_j
// (eq. abcej_boundary) up to tau = t_{j+1}.  With Q = H^T X H, q = H^T X r,
// rho = r^T X r and B = L U^-1 L^T = Lt Lt^T:
//   dA/dtau    = F A - C Q A
//   db/dtau    = c + F b + C (q - Q b)
//   dC/dtau    = B + F C + (F C)^T - C Q C
//   deta/dtau  = A^T (q - Q b)
//   dJ/dtau    = A^T Q A
//   dzeta/dtau = rho/2 - b^T (q - Q b / 2)
// (the zeta equation is the state-free part of the forward conditional HJB,
// eq. forward_conditional_HJB, at x = 0 and z = b).
#include <cuda_runtime.h>

#include "lqt_device.cuh"
#include "lqt_internal.h"

namespace lqt {

template <int N, int M>
__device__ __forceinline__ void forward_rhs(const Elem<N>& y, const double* __restrict__ F,
                                            const double* __restrict__ c, const double* __restrict__ Lt,
                                            const double* __restrict__ Q, const double* __restrict__ qr,
                                            Elem<N>& k) {
  // QA = Q A, CQ = C Q, w = q - Q b
  double QA[N * N], CQ[N * N], w[N];
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = 0; j < N; ++j) {
      double s1 = 0.0, s2 = 0.0;
#pragma unroll
      for (int l = 0; l < N; ++l) {
        s1 = fma(Q[i * N + l], y.A[l * N + j], s1);
        s2 = fma(y.C[sidx<N>(i, l)], Q[l * N + j], s2);
      }
      QA[i * N + j] = s1;
      CQ[i * N + j] = s2;
    }
#pragma unroll
  for (int i = 0; i < N; ++i) {
    double s = qr[i];
#pragma unroll
    for (int l = 0; l < N; ++l) s = fma(-Q[i * N + l], y.b[l], s);
    w[i] = s;
  }
  // dA = F A - C (Q A)
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = 0; j < N; ++j) {
      double s = 0.0;
#pragma unroll
      for (int l = 0; l < N; ++l) {
        s = fma(F[i * N + l], y.A[l * N + j], s);
        s = fma(-y.C[sidx<N>(i, l)], QA[l * N + j], s);
      }
      k.A[i * N + j] = s;
    }
  // db = c + F b + C w
#pragma unroll
  for (int i = 0; i < N; ++i) {
    double s = c ? c[i] : 0.0;
#pragma unroll
    for (int l = 0; l < N; ++l) {
      s = fma(F[i * N + l], y.b[l], s);
      s = fma(y.C[sidx<N>(i, l)], w[l], s);
    }
    k.b[i] = s;
  }
  // dC = Lt Lt^T + F C + (F C)^T - (C Q) C   (upper triangle)
  double FC[N * N];
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = 0; j < N; ++j) {
      double s = 0.0;
#pragma unroll
      for (int l = 0; l < N; ++l) s = fma(F[i * N + l], y.C[sidx<N>(l, j)], s);
      FC[i * N + j] = s;
    }
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = i; j < N; ++j) {
      double s = FC[i * N + j] + FC[j * N + i];
#pragma unroll
      for (int a = 0; a < M; ++a) s = fma(Lt[i * M + a], Lt[j * M + a], s);
#pragma unroll
      for (int l = 0; l < N; ++l) s = fma(-CQ[i * N + l], y.C[sidx<N>(l, j)], s);
      k.C[sidx<N>(i, j)] = s;
    }
  // deta = A^T w ; dJ = A^T (Q A) (upper triangle)
#pragma unroll
  for (int i = 0; i < N; ++i) {
    double s = 0.0;
#pragma unroll
    for (int l = 0; l < N; ++l) s = fma(y.A[l * N + i], w[l], s);
    k.eta[i] = s;
  }
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = i; j < N; ++j) {
      double s = 0.0;
#pragma unroll
      for (int l = 0; l < N; ++l) s = fma(y.A[l * N + i], QA[l * N + j], s);
      k.J[sidx<N>(i, j)] = s;
    }
  // dzeta = rho/2 - b^T (q - Q b / 2) = rho/2 - b^T (w + q)/2
  double z = 0.5 * qr[N];
#pragma unroll
  for (int i = 0; i < N; ++i) z = fma(-0.5 * y.b[i], w[i] + qr[i], z);
  k.zeta = z;
}

template <int N>
__device__ __forceinline__ void faxpy(Elem<N>& y, const Elem<N>& base, double s, const Elem<N>& k) {
#pragma unroll
  for (int i = 0; i < N * N; ++i) y.A[i] = fma(s, k.A[i], base.A[i]);
#pragma unroll
  for (int i = 0; i < N; ++i) {
    y.b[i] = fma(s, k.b[i], base.b[i]);
    y.eta[i] = fma(s, k.eta[i], base.eta[i]);
  }
#pragma unroll
  for (int i = 0; i < Dim<N>::NS; ++i) {
    y.C[i] = fma(s, k.C[i], base.C[i]);
    y.J[i] = fma(s, k.J[i], base.J[i]);
  }
  y.zeta = fma(s, k.zeta, base.zeta);
}

struct ForwardArgs {
  int64_t T;
  int32_t K;
  const double* t;
  Coefs cf;
  ElemPtrs out;
};

template <int N, int M>
__global__ void __launch_bounds__(128) build_forward_kernel(ForwardArgs a) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= a.T) return;
  const Coefs& cf = a.cf;
  const int32_t K = a.K;
  const double h = (a.t[j + 1] - a.t[j]) / K;
  Elem<N> y, yn, yt, k;
#pragma unroll
  for (int i = 0; i < N * N; ++i) y.A[i] = (i % (N + 1) == 0) ? 1.0 : 0.0;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    y.b[i] = 0.0;
    y.eta[i] = 0.0;
  }
#pragma unroll
  for (int i = 0; i < Dim<N>::NS; ++i) {
    y.C[i] = 0.0;
    y.J[i] = 0.0;
  }
  y.zeta = 0.0;
  for (int32_t i = 0; i < K; ++i) {
    // stage times in half steps from t_j: 2i, 2i+1, 2i+1, 2i+2
    const int32_t ps[3] = {2 * i, 2 * i + 1, 2 * i + 2};
    const double *F[3], *c[3], *Lt[3], *Q[3], *qr[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      F[q] = cf.F.ptr + sample_index(cf.F.mode, j, ps[q], K) * N * N;
      c[q] = cf.c.ptr ? cf.c.ptr + sample_index(cf.c.mode, j, ps[q], K) * N : nullptr;
      Lt[q] = cf.Lt.ptr + sample_index(cf.Lt.mode, j, ps[q], K) * N * M;
      Q[q] = cf.Q.ptr + sample_index(cf.Q.mode, j, ps[q], K) * N * N;
      qr[q] = cf.qr.ptr + sample_index(cf.qr.mode, j, ps[q], K) * (N + 1);
    }
    forward_rhs<N, M>(y, F[0], c[0], Lt[0], Q[0], qr[0], k);
    faxpy(yn, y, h / 6.0, k);
    faxpy(yt, y, 0.5 * h, k);
    forward_rhs<N, M>(yt, F[1], c[1], Lt[1], Q[1], qr[1], k);
    faxpy(yn, yn, h / 3.0, k);
    faxpy(yt, y, 0.5 * h, k);
    forward_rhs<N, M>(yt, F[1], c[1], Lt[1], Q[1], qr[1], k);
    faxpy(yn, yn, h / 3.0, k);
    faxpy(yt, y, h, k);
    forward_rhs<N, M>(yt, F[2], c[2], Lt[2], Q[2], qr[2], k);
    faxpy(y, yn, h / 6.0, k);
  }
  store_public<N>(a.out, j, y);
}

template <int N, int M>
static cudaError_t launch_fwd_nm(const ForwardArgs& a, cudaStream_t st) {
  build_forward_kernel<N, M><<<(unsigned)((a.T + 127) / 128), 128, 0, st>>>(a);
  count_launch();
  return cudaGetLastError();
}

template <int N>
static cudaError_t launch_fwd_n(const ForwardArgs& a, int M, cudaStream_t st) {
  switch (M) {
    case 1: return launch_fwd_nm<N, 1>(a, st);
    case 2: if constexpr (N >= 2) return launch_fwd_nm<N, 2>(a, st); else return cudaErrorInvalidValue;
    case 4: if constexpr (N >= 3) return launch_fwd_nm<N, 4>(a, st); else return cudaErrorInvalidValue;
    case 8: if constexpr (N >= 8) return launch_fwd_nm<N, 8>(a, st); else return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_build_forward(const lqt_problem& p, const Layout& lay, const Coefs& cf, const ElemPtrs& out,
                                 cudaStream_t st, double* team_scratch) {
  ForwardArgs a{p.T, p.K, p.t, cf, out};
  switch (p.n) {
    case 1: return launch_fwd_n<1>(a, lay.M, st);
    case 2: return launch_fwd_n<2>(a, lay.M, st);
    case 3: return launch_fwd_n<3>(a, lay.M, st);
    case 4: return launch_fwd_n<4>(a, lay.M, st);
    case 8: return launch_fwd_n<8>(a, lay.M, st);
    case 16:
    case 64: return team_launch_build_forward(p, lay, cf, out, team_scratch, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace lqt
