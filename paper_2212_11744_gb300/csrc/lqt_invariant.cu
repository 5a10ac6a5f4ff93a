// Time-invariant specialisation of the element build.
//
// When F, L, U, X (and H) are constant and the sub-intervals have one length
// h K, the A, C, J parts of the backward conditional HJB ODEs (Sec. IV-B,
// Theorem Backward_HJB_LQT) do not involve b, eta, zeta, r or c:
//   dA/ds = A B J - A F,  dC/ds = -A B A^T,  dJ/ds = -Q - J F - F^T J + J B J,
// so every sub-interval's RK4 produces the same A, C, J and the same values of
// A and J at every RK4 stage (the paper's remark in Sec. VI-B: a time-invariant
// model has one conditional value function per block).  Only
//   db/ds = -A B eta - A c,  deta/ds = -q - F^T eta + J c + J B eta,
//   dzeta/ds = -rho/2 + eta^T B eta / 2 + eta^T c
// differ between sub-intervals, through the samples of r (q = H^T X r,
// rho = r^T X r) and c.  So one thread per problem integrates A, C, J once and
// records, for every RK4 step and stage, AL = A Lt, P = J Lt, A and J (B =
// Lt Lt^T); then one thread per sub-interval integrates (b, eta, zeta) with
// those recorded stage matrices -- O(K n M + K n^2) work per sub-interval
// instead of O(K n^3).  The RK4 steps are the same as the general build's, so
// the elements are the general build's up to rounding.
#include <cuda_runtime.h>

#include "lqt_device.cuh"
#include "lqt_internal.h"
#include "lqt_invariant.cuh"

namespace lqt {

size_t invariant_table_bytes(int n, int M, int K) { return (size_t)inv_table_doubles(n, M, K) * sizeof(double); }

// ---------------------------------------------------------------------------
// the shared A, C, J integration (one thread per problem, runtime n)
// ---------------------------------------------------------------------------

// An A, C, J triple (full n x n each) in global scratch.
struct ACJ {
  double *A, *C, *J;
};

// k = f(y) for the A, C, J equations; records the stage's AL, P, A, J at rec.
__device__ void acj_rhs_record(int n, int M, const ACJ& y, const double* F, const double* Lt, const double* Q,
                               const ACJ& k, double* rec) {
  double* AL = rec;
  double* P = rec + n * M;
  double* Ar = rec + 2 * n * M;
  double* Jr = Ar + n * n;
  for (int i = 0; i < n; ++i)
    for (int a = 0; a < M; ++a) {
      double s1 = 0.0, s2 = 0.0;
      for (int l = 0; l < n; ++l) {
        s1 = fma(y.A[i * n + l], Lt[l * M + a], s1);
        s2 = fma(y.J[i * n + l], Lt[l * M + a], s2);
      }
      AL[i * M + a] = s1;
      P[i * M + a] = s2;
    }
  for (int e = 0; e < n * n; ++e) {
    Ar[e] = y.A[e];
    Jr[e] = y.J[e];
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double a = 0.0, c = 0.0, jf = 0.0, fj = 0.0, pp = 0.0;
      for (int b = 0; b < M; ++b) {
        a = fma(AL[i * M + b], P[j * M + b], a);
        c = fma(-AL[i * M + b], AL[j * M + b], c);
        pp = fma(P[i * M + b], P[j * M + b], pp);
      }
      for (int l = 0; l < n; ++l) {
        a = fma(-y.A[i * n + l], F[l * n + j], a);
        jf = fma(y.J[i * n + l], F[l * n + j], jf);
        fj = fma(y.J[j * n + l], F[l * n + i], fj);
      }
      k.A[i * n + j] = a;
      k.C[i * n + j] = c;
      k.J[i * n + j] = -Q[i * n + j] - jf - fj + pp;
    }
}

__device__ void acj_axpy(int n, const ACJ& y, const ACJ& base, double s, const ACJ& k) {
  for (int e = 0; e < n * n; ++e) {
    y.A[e] = fma(s, k.A[e], base.A[e]);
    y.C[e] = fma(s, k.C[e], base.C[e]);
    y.J[e] = fma(s, k.J[e], base.J[e]);
  }
}

// K backward RK4 steps of A, C, J from (I, 0, 0), recording every stage.
__device__ void inv_master(int n, int M, int K, double h, const double* F, const double* Lt, const double* Q,
                           double* table) {
  const int64_t SD = inv_stage_doubles(n, M);
  double* fin = table + 4 * (int64_t)K * SD;
  double* w = fin + 3 * n * n;
  const int nn = n * n;
  const ACJ y{w, w + nn, w + 2 * nn}, yn{w + 3 * nn, w + 4 * nn, w + 5 * nn};
  const ACJ yt{w + 6 * nn, w + 7 * nn, w + 8 * nn}, k{w + 9 * nn, w + 10 * nn, w + 11 * nn};
  for (int e = 0; e < nn; ++e) {
    y.A[e] = (e % (n + 1) == 0) ? 1.0 : 0.0;
    y.C[e] = 0.0;
    y.J[e] = 0.0;
  }
  for (int i = K - 1; i >= 0; --i) {
    double* rec = table + 4 * (int64_t)i * SD;
    acj_rhs_record(n, M, y, F, Lt, Q, k, rec);
    acj_axpy(n, yn, y, -h / 6.0, k);
    acj_axpy(n, yt, y, -0.5 * h, k);
    acj_rhs_record(n, M, yt, F, Lt, Q, k, rec + SD);
    acj_axpy(n, yn, yn, -h / 3.0, k);
    acj_axpy(n, yt, y, -0.5 * h, k);
    acj_rhs_record(n, M, yt, F, Lt, Q, k, rec + 2 * SD);
    acj_axpy(n, yn, yn, -h / 3.0, k);
    acj_axpy(n, yt, y, -h, k);
    acj_rhs_record(n, M, yt, F, Lt, Q, k, rec + 3 * SD);
    acj_axpy(n, y, yn, -h / 6.0, k);
  }
  for (int e = 0; e < nn; ++e) {
    fin[e] = y.A[e];
    // C and J are symmetric; store their symmetric parts as the general build does
    const int i = e / n, j = e % n;
    fin[nn + e] = 0.5 * (y.C[i * n + j] + y.C[j * n + i]);
    fin[2 * nn + e] = 0.5 * (y.J[i * n + j] + y.J[j * n + i]);
  }
}

struct InvMasterArgs {
  int32_t n, M, K;
  int32_t B;  // problems (1 for a single problem)
  const BatchProb* probs;  // batch descriptors (null for a single problem)
  const double *t, *F, *Lt, *Q;  // single problem
  double* tables;  // B tables back to back
};

__global__ void inv_master_kernel(InvMasterArgs a) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= a.B) return;
  const double* t = a.probs ? a.probs[b].t : a.t;
  const double* F = a.probs ? a.probs[b].cf.F.ptr : a.F;
  const double* Lt = a.probs ? a.probs[b].cf.Lt.ptr : a.Lt;
  const double* Q = a.probs ? a.probs[b].cf.Q.ptr : a.Q;
  const double h = (t[1] - t[0]) / a.K;
  inv_master(a.n, a.M, a.K, h, F, Lt, Q, a.tables + (int64_t)b * inv_table_doubles(a.n, a.M, a.K));
}

struct InvBuildArgs {
  int64_t T;
  int32_t K;
  const double* t;
  Coefs cf;
  const double* table;
  ElemPtrs out;
};

template <int N, int M>
__global__ void __launch_bounds__(128) inv_build_kernel(InvBuildArgs a) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= a.T) return;
  inv_element<N, M>(a.cf, a.t, j, a.K, a.table, a.out, j);
}

// n = 64: one warp per sub-interval (inv_element_warp).
template <int N, int M>
__global__ void __launch_bounds__(32) inv_build_warp_kernel(InvBuildArgs a) {
  extern __shared__ double sm[];
  for (int64_t j = blockIdx.x; j < a.T; j += gridDim.x)
    inv_element_warp<N, M>(threadIdx.x, a.cf, a.t, j, a.K, a.table, a.out, j, sm);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

template <int N, int M>
static void inv_launch_nm(const InvBuildArgs* a, const BatchDev* bd, const double* tables, const ElemPtrs& out,
                          cudaStream_t st) {
  if (bd) {
    launch_inv_batch_build<N, M>(*bd, tables, out, st);
  } else {
    inv_build_kernel<N, M><<<(unsigned)((a->T + 127) / 128), 128, 0, st>>>(*a);
    count_launch();
  }
}

template <int N>
static cudaError_t inv_launch_n(int M, const InvBuildArgs* a, const BatchDev* bd, const double* tables,
                                const ElemPtrs& out, cudaStream_t st) {
  switch (M) {
    case 1: inv_launch_nm<N, 1>(a, bd, tables, out, st); break;
    case 2: if constexpr (N >= 2) { inv_launch_nm<N, 2>(a, bd, tables, out, st); break; } else return cudaErrorInvalidValue;
    case 4: if constexpr (N >= 3) { inv_launch_nm<N, 4>(a, bd, tables, out, st); break; } else return cudaErrorInvalidValue;
    case 8: if constexpr (N >= 8) { inv_launch_nm<N, 8>(a, bd, tables, out, st); break; } else return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

static cudaError_t inv_dispatch(int n, int M, const InvBuildArgs* a, const BatchDev* bd, const double* tables,
                                const ElemPtrs& out, cudaStream_t st) {
  switch (n) {
    case 1: return inv_launch_n<1>(M, a, bd, tables, out, st);
    case 2: return inv_launch_n<2>(M, a, bd, tables, out, st);
    case 3: return inv_launch_n<3>(M, a, bd, tables, out, st);
    case 4: return inv_launch_n<4>(M, a, bd, tables, out, st);
    case 8: return inv_launch_n<8>(M, a, bd, tables, out, st);
    case 16:
      if (M != 8) return cudaErrorInvalidValue;
      inv_launch_nm<16, 8>(a, bd, tables, out, st);
      return cudaGetLastError();
    default: return cudaErrorInvalidValue;
  }
}

// n = 16 is compiled for a factor width of 8 (m = 5..8), n = 64 for its fixed
// width 16.
bool invariant_supported(int n, int M) {
  return (n <= 8 && M <= kInvMaxM) || (n == 16 && M == 8) || (n == 64 && M == 16);
}

cudaError_t launch_build_invariant(const lqt_problem& p, const Layout& lay, const Coefs& cf, const ElemPtrs& out,
                                   double* table, cudaStream_t st) {
  InvBuildArgs a{p.T, p.K, p.t, cf, table, out};
  const int64_t td = inv_table_doubles(p.n, lay.M, p.K);
  cudaError_t e = cudaSuccess;
  if (p.n == 16) {
    launch_inv_master_team<16, 8>(p.K, 1, nullptr, p.t, cf, table, td, st);
    e = inv_dispatch(p.n, lay.M, &a, nullptr, table, out, st);
  } else if (p.n == 64) {
    launch_inv_master_team<64, 16>(p.K, 1, nullptr, p.t, cf, table, td, st);
    const size_t smem = (4 * (2 * 64 + 1) + 16) * sizeof(double);
    const int64_t grid = p.T < 152 * 32 ? p.T : 152 * 32;
    inv_build_warp_kernel<64, 16><<<(unsigned)grid, 32, smem, st>>>(a);
    count_launch();
    e = cudaGetLastError();
  } else {
    InvMasterArgs m{p.n, lay.M, p.K, 1, nullptr, p.t, cf.F.ptr, cf.Lt.ptr, cf.Q.ptr, table};
    inv_master_kernel<<<1, 32, 0, st>>>(m);
    count_launch();
    e = inv_dispatch(p.n, lay.M, &a, nullptr, table, out, st);
  }
  if (e != cudaSuccess) return e;
  return launch_terminal_element(p, out, st);
}

cudaError_t batch_build_invariant(const BatchDev& bd, const ElemPtrs& el, double* tables, cudaStream_t st) {
  const int64_t td = inv_table_doubles(bd.n, bd.M, bd.K);
  if (bd.n == 16) {
    launch_inv_master_team<16, 8>(bd.K, bd.B, bd.probs, nullptr, Coefs{}, tables, td, st);
  } else if (bd.n == 64) {
    launch_inv_master_team<64, 16>(bd.K, bd.B, bd.probs, nullptr, Coefs{}, tables, td, st);
    launch_inv_batch_build_warp(bd, tables, el, st);
    return cudaGetLastError();
  } else {
    InvMasterArgs m{bd.n, bd.M, bd.K, bd.B, bd.probs, nullptr, nullptr, nullptr, nullptr, tables};
    inv_master_kernel<<<(unsigned)((bd.B + 127) / 128), 128, 0, st>>>(m);
    count_launch();
  }
  return inv_dispatch(bd.n, bd.M, nullptr, &bd, tables, el, st);
}

}  // namespace lqt
