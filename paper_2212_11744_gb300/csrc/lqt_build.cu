// Stage (a): conditional value function elements of every sub-interval, one
// CUDA thread per sub-interval, state in registers (Sec. IV-B, Theorem
// Backward_HJB_LQT; boundary eq. abcej_boundary; terminal element Sec. IV-D,
// eq. LQT_final_initialisation).
//
// Also the coefficient preparation kernel: B = L U^-1 L^T is used only through
// a factor Lt = L R^-T (U = R R^T), so that A B J = (A Lt)(J Lt)^T,
// A B A^T = (A Lt)(A Lt)^T, J B J = (J Lt)(J Lt)^T and B eta = Lt (Lt^T eta);
// with m < n this cuts the FP64 work of every right-hand side.
#include <cuda_runtime.h>

#include "lqt_device.cuh"
#include "lqt_internal.h"

namespace lqt {

// ---------------------------------------------------------------------------
// coefficient preparation
// ---------------------------------------------------------------------------

struct PrepArgs {
  int32_t n, m, nr, K, M;
  int64_t T;
  Coef L, U, H, X, r;
  int32_t mode_Lt, mode_Q, mode_qr;
  int64_t cnt_Lt, cnt_Q, cnt_qr, cnt_Ku;
  double *Lt, *Q, *qr, *Ku;
};

// Index of the input sample that a derived sample s (of mode `dmode`) uses.
__device__ __forceinline__ int64_t input_index(int32_t imode, int32_t dmode, int64_t s, int32_t K, int64_t T) {
  if (imode == kConst) return 0;
  if (dmode == imode) return s;
  // dmode == kStageBlock: s = (2K+1) j + p
  const int64_t j = s / (2 * K + 1);
  const int32_t p = (int32_t)(s - j * (2 * K + 1));
  return sample_index(imode, j, p, K);
}

// Cholesky U = R R^T of the m x m sample (lower R, row-major), in place.
__device__ void cholesky_lower(double* R, int m) {
  for (int j = 0; j < m; ++j) {
    double d = R[j * m + j];
    for (int k = 0; k < j; ++k) d -= R[j * m + k] * R[j * m + k];
    if (!(d > 0.0)) flag(kStatusSingular);
    d = sqrt(d);
    R[j * m + j] = d;
    const double inv = 1.0 / d;
    for (int i = j + 1; i < m; ++i) {
      double s = R[i * m + j];
      for (int k = 0; k < j; ++k) s -= R[i * m + k] * R[j * m + k];
      R[i * m + j] = s * inv;
    }
    for (int i = 0; i < j; ++i) R[i * m + j] = 0.0;
  }
}

constexpr int kMaxM = 16;
constexpr int kMaxN = 64;

// One thread per derived sample; blockIdx.y selects the quantity (with two
// rows in the grid only Lt and Ku are made).
__global__ void prepare_kernel(PrepArgs a) {
  const int which = gridDim.y == 2 ? (blockIdx.y == 0 ? 0 : 3) : blockIdx.y;
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int n = a.n, m = a.m, nr = a.nr;
  if (which == 0) {  // Lt = L R^-T, zero-padded to M columns
    if (s >= a.cnt_Lt) return;
    const double* L = a.L.ptr + input_index(a.L.mode, a.mode_Lt, s, a.K, a.T) * n * m;
    const double* U = a.U.ptr + input_index(a.U.mode, a.mode_Lt, s, a.K, a.T) * m * m;
    double R[kMaxM * kMaxM];
    for (int i = 0; i < m * m; ++i) R[i] = U[i];
    cholesky_lower(R, m);
    double* out = a.Lt + s * n * a.M;
    for (int i = 0; i < n; ++i) {
      // solve Lt_i R^T = L_i  (forward substitution over columns)
      double row[kMaxM];
      for (int c = 0; c < m; ++c) {
        double v = L[i * m + c];
        for (int k = 0; k < c; ++k) v -= row[k] * R[c * m + k];
        row[c] = v / R[c * m + c];
      }
      for (int c = 0; c < a.M; ++c) out[i * a.M + c] = c < m ? row[c] : 0.0;
    }
  } else if (which == 1) {  // Q = H^T X H (full n x n, symmetrised); only when H is given
    if (s >= a.cnt_Q) return;
    const double* X = a.X.ptr + input_index(a.X.mode, a.mode_Q, s, a.K, a.T) * nr * nr;
    const double* H = a.H.ptr + input_index(a.H.mode, a.mode_Q, s, a.K, a.T) * nr * n;
    double* out = a.Q + s * (n * n);
    for (int i = 0; i < n; ++i)
      for (int j = i; j < n; ++j) {
        double vij = 0.0, vji = 0.0;
        for (int k = 0; k < nr; ++k)
          for (int l = 0; l < nr; ++l) {
            vij += H[k * n + i] * X[k * nr + l] * H[l * n + j];
            vji += H[k * n + j] * X[k * nr + l] * H[l * n + i];
          }
        out[i * n + j] = out[j * n + i] = 0.5 * (vij + vji);
      }
  } else if (which == 2) {  // qr = [H^T X r, r^T X r]
    if (s >= a.cnt_qr) return;
    const double* X = a.X.ptr + input_index(a.X.mode, a.mode_qr, s, a.K, a.T) * nr * nr;
    const double* H = a.H.ptr ? a.H.ptr + input_index(a.H.mode, a.mode_qr, s, a.K, a.T) * nr * n : nullptr;
    const double* r = a.r.ptr ? a.r.ptr + input_index(a.r.mode, a.mode_qr, s, a.K, a.T) * nr : nullptr;
    double* out = a.qr + s * (n + 1);
    double Xr[kMaxN];
    double rho = 0.0;
    for (int k = 0; k < nr; ++k) {
      double v = 0.0;
      if (r)
        for (int l = 0; l < nr; ++l) v += X[k * nr + l] * r[l];
      Xr[k] = v;
      if (r) rho += r[k] * v;
    }
    for (int i = 0; i < n; ++i) {
      double v;
      if (!H) {
        v = Xr[i];
      } else {
        v = 0.0;
        for (int k = 0; k < nr; ++k) v += H[k * n + i] * Xr[k];
      }
      out[i] = v;
    }
    out[n] = rho;
  } else {  // Ku = U^-1 L^T at the boundaries (solve U Ku = L^T)
    if (s >= a.cnt_Ku) return;
    // boundary k = s uses sample (j, p) = (k, 0), or (T-1, 2K) at k = T
    int64_t j = s < a.T ? s : a.T - 1;
    int32_t p = s < a.T ? 0 : 2 * a.K;
    if (a.cnt_Ku == 1) { j = 0; p = 0; }
    const double* L = a.L.ptr + sample_index(a.L.mode, j, p, a.K) * n * m;
    const double* U = a.U.ptr + sample_index(a.U.mode, j, p, a.K) * m * m;
    double R[kMaxM * kMaxM];
    for (int i = 0; i < m * m; ++i) R[i] = U[i];
    cholesky_lower(R, m);
    double* out = a.Ku + s * m * n;
    for (int col = 0; col < n; ++col) {
      double y[kMaxM];
      for (int i = 0; i < m; ++i) {  // R y = L^T[:, col]
        double v = L[col * m + i];
        for (int k = 0; k < i; ++k) v -= R[i * m + k] * y[k];
        y[i] = v / R[i * m + i];
      }
      for (int i = m - 1; i >= 0; --i) {  // R^T z = y
        double v = y[i];
        for (int k = i + 1; k < m; ++k) v -= R[k * m + i] * y[k];
        y[i] = v / R[i * m + i];
      }
      for (int i = 0; i < m; ++i) out[i * n + col] = y[i];
    }
  }
}

// q = X r, rho = r^T X r per sample when H is the identity (one thread per
// sample, loops unrolled for the compiled n).
template <int N>
__global__ void __launch_bounds__(256) qr_identity_kernel(const double* __restrict__ X, int32_t X_mode,
                                                          const double* __restrict__ r, int32_t r_mode, int32_t dmode,
                                                          int64_t cnt, int32_t K, int64_t T, double* __restrict__ qr) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= cnt) return;
  const double* Xs = X + input_index(X_mode, dmode, s, K, T) * N * N;
  double rr[N], q[N];
  if (r) {
    const double* rs = r + input_index(r_mode, dmode, s, K, T) * N;
#pragma unroll
    for (int i = 0; i < N; ++i) rr[i] = rs[i];
  } else {
#pragma unroll
    for (int i = 0; i < N; ++i) rr[i] = 0.0;
  }
  double rho = 0.0;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    double v = 0.0;
#pragma unroll
    for (int l = 0; l < N; ++l) v = fma(Xs[i * N + l], rr[l], v);
    q[i] = v;
    rho = fma(rr[i], v, rho);
  }
  double* out = qr + s * (N + 1);
#pragma unroll
  for (int i = 0; i < N; ++i) out[i] = q[i];
  out[N] = rho;
}

// The same with N consecutive threads per sample (N a power of two <= 32),
// thread i forming row i of X r: a warp reads 32 consecutive rows, so the
// stream of X samples (the largest input when X is sampled per half-step) is
// read in full 128-byte lines; rho is reduced over the N lanes.
template <int N, bool VEC>
__global__ void __launch_bounds__(256) qr_rows_kernel(const double* __restrict__ X, int32_t X_mode,
                                                      const double* __restrict__ r, int32_t r_mode, int32_t dmode,
                                                      int64_t cnt, int32_t K, int64_t T, double* __restrict__ qr) {
  static_assert(N >= 2 && N <= 32 && (N & (N - 1)) == 0, "rows kernel needs a power-of-two N <= 32");
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t s = tid / N;
  const int i = (int)(tid % N);
  const bool live = s < cnt;
  double q = 0.0, ri = 0.0;
  if (live) {
    const double* row = X + input_index(X_mode, dmode, s, K, T) * N * N + i * N;
    if (r) {
      const double* rs = r + input_index(r_mode, dmode, s, K, T) * N;
      if constexpr (VEC) {
        // X and r start on 16-byte boundaries (checked by the launcher) and N is
        // even, so every row and sample does: read them in pairs
        const double2* row2 = reinterpret_cast<const double2*>(row);
        const double2* rs2 = reinterpret_cast<const double2*>(rs);
#pragma unroll
        for (int l = 0; l < N / 2; ++l) {
          const double2 a = __ldg(row2 + l), b = __ldg(rs2 + l);
          q = fma(a.x, b.x, q);
          q = fma(a.y, b.y, q);
        }
      } else {
#pragma unroll
        for (int l = 0; l < N; ++l) q = fma(row[l], rs[l], q);
      }
      ri = rs[i];
    }
  }
  double rho = ri * q;
#pragma unroll
  for (int o = N / 2; o > 0; o >>= 1) rho += __shfl_xor_sync(0xffffffffu, rho, o);
  if (live) {
    qr[s * (N + 1) + i] = q;
    if (i == 0) qr[s * (N + 1) + N] = rho;
  }
}

template <int N>
static void launch_qr_identity(const PrepArgs& a, cudaStream_t st) {
  const int threads = 256;
  if constexpr (N >= 2 && N <= 32 && (N & (N - 1)) == 0) {
    const int64_t total = a.cnt_qr * N;
    const unsigned grid = (unsigned)((total + threads - 1) / threads);
    const bool vec = ((reinterpret_cast<uintptr_t>(a.X.ptr) | reinterpret_cast<uintptr_t>(a.r.ptr)) & 15u) == 0;
    if (vec)
      qr_rows_kernel<N, true><<<grid, threads, 0, st>>>(a.X.ptr, a.X.mode, a.r.ptr, a.r.mode, a.mode_qr, a.cnt_qr,
                                                         a.K, a.T, a.qr);
    else
      qr_rows_kernel<N, false><<<grid, threads, 0, st>>>(a.X.ptr, a.X.mode, a.r.ptr, a.r.mode, a.mode_qr, a.cnt_qr,
                                                          a.K, a.T, a.qr);
  } else {
    qr_identity_kernel<N><<<(unsigned)((a.cnt_qr + threads - 1) / threads), threads, 0, st>>>(
        a.X.ptr, a.X.mode, a.r.ptr, a.r.mode, a.mode_qr, a.cnt_qr, a.K, a.T, a.qr);
  }
  count_launch();
}

// The derived coefficients of problem p into the given arrays (Lt, Q, qr, Ku
// laid out as the Layout's modes say); cf describes p's coefficients with
// those arrays.  Q is written only when H is given.
cudaError_t launch_prepare_into(const lqt_problem& p, const Layout& lay, double* Lt, double* Q, double* qr,
                                double* Ku, Coefs& cf, cudaStream_t st) {
  PrepArgs a;
  a.n = p.n; a.m = p.m; a.nr = p.nr; a.K = p.K; a.M = lay.M; a.T = p.T;
  a.L = {p.L.ptr, p.L.mode};
  a.U = {p.U.ptr, p.U.mode};
  a.H = {p.H.ptr, p.H.mode};
  a.X = {p.X.ptr, p.X.mode};
  a.r = {p.r.ptr, p.r.mode};
  a.mode_Lt = lay.mode_Lt; a.mode_Q = lay.mode_Q; a.mode_qr = lay.mode_qr;
  a.cnt_Lt = sample_count(lay.mode_Lt, p.T, p.K);
  a.cnt_Q = sample_count(lay.mode_Q, p.T, p.K);
  a.cnt_qr = sample_count(lay.mode_qr, p.T, p.K);
  const bool ku_const = p.L.mode == LQT_CONST && p.U.mode == LQT_CONST;
  a.cnt_Ku = ku_const ? 1 : p.T + 1;
  a.Lt = Lt;
  a.Q = Q;
  a.qr = qr;
  a.Ku = Ku;
  // Lt and Ku always; H^T X H only when H is given; H^T X r by the dedicated
  // kernel when H is the identity.
  const bool h_identity = p.H.ptr == nullptr;
  int64_t most = a.cnt_Lt > a.cnt_Ku ? a.cnt_Lt : a.cnt_Ku;
  if (!h_identity) {
    if (a.cnt_Q > most) most = a.cnt_Q;
    if (a.cnt_qr > most) most = a.cnt_qr;
  }
  const int threads = 128;
  const int64_t blocks = (most + threads - 1) / threads;
  if (h_identity) {
    // which = 0 (Lt) and 3 (Ku): map blockIdx.y 0 -> 0, 1 -> 3
    prepare_kernel<<<dim3((unsigned)blocks, 2), threads, 0, st>>>(a);
    count_launch();
    switch (p.n) {
      case 1: launch_qr_identity<1>(a, st); break;
      case 2: launch_qr_identity<2>(a, st); break;
      case 3: launch_qr_identity<3>(a, st); break;
      case 4: launch_qr_identity<4>(a, st); break;
      case 8: launch_qr_identity<8>(a, st); break;
      case 16: launch_qr_identity<16>(a, st); break;
      case 64: launch_qr_identity<64>(a, st); break;
      default: return cudaErrorInvalidValue;
    }
  } else {
    prepare_kernel<<<dim3((unsigned)blocks, 4), threads, 0, st>>>(a);
    count_launch();
  }
  cf = coefs_view(p, lay, Lt, Q, qr, Ku);
  return cudaGetLastError();
}

Coefs coefs_view(const lqt_problem& p, const Layout& lay, double* Lt, double* Q, double* qr, double* Ku) {
  const bool h_identity = p.H.ptr == nullptr;
  const bool ku_const = p.L.mode == LQT_CONST && p.U.mode == LQT_CONST;
  Coefs cf;
  cf.F = {p.F.ptr, p.F.mode};
  cf.c = {p.c.ptr, p.c.ptr ? p.c.mode : kConst};
  cf.Lt = {Lt, lay.mode_Lt};
  cf.Q = h_identity ? Coef{p.X.ptr, p.X.mode} : Coef{Q, lay.mode_Q};
  cf.qr = {qr, lay.mode_qr};
  cf.Ku = Ku;
  cf.Ku_per_boundary = ku_const ? 0 : 1;
  cf.M = lay.M;
  return cf;
}

cudaError_t launch_prepare_coefs(const lqt_problem& p, const Layout& lay, char* ws, Coefs& cf, cudaStream_t st) {
  return launch_prepare_into(p, lay, (double*)(ws + lay.off_Lt), (double*)(ws + lay.off_Q),
                             (double*)(ws + lay.off_qr), (double*)(ws + lay.off_Ku), cf, st);
}

// ---------------------------------------------------------------------------
// element build
// ---------------------------------------------------------------------------

// Right-hand side of the backward conditional HJB ODEs in s:
//   dA/ds    =  A B J - A F                = AL P^T - A F
//   db/ds    = -A B eta - A c               = -AL w - A c
//   dC/ds    = -A B A^T                     = -AL AL^T
//   deta/ds  = -q - F^T eta + J c + J B eta = -q - F^T eta + J c + P w
//   dJ/ds    = -Q - J F - F^T J + J B J     = -Q - JF - (JF)^T + P P^T
//   dzeta/ds = -rho/2 + eta^T B eta / 2 + eta^T c = -rho/2 + |w|^2/2 + eta^T c
// with AL = A Lt, P = J Lt, w = Lt^T eta, q = H^T X r, rho = r^T X r.
template <int N, int M>
__device__ __forceinline__ void element_rhs(const Elem<N>& y, const double* __restrict__ F,
                                            const double* __restrict__ c, const double* __restrict__ Lt,
                                            const double* __restrict__ Q, const double* __restrict__ qr,
                                            Elem<N>& k) {
  double AL[N * M], P[N * M], w[M];
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int a = 0; a < M; ++a) {
      double s1 = 0.0, s2 = 0.0;
#pragma unroll
      for (int l = 0; l < N; ++l) {
        const double lt = Lt[l * M + a];
        s1 = fma(y.A[i * N + l], lt, s1);
        s2 = fma(y.J[sidx<N>(i, l)], lt, s2);
      }
      AL[i * M + a] = s1;
      P[i * M + a] = s2;
    }
#pragma unroll
  for (int a = 0; a < M; ++a) {
    double s = 0.0;
#pragma unroll
    for (int l = 0; l < N; ++l) s = fma(Lt[l * M + a], y.eta[l], s);
    w[a] = s;
  }
  // dA = AL P^T - A F
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = 0; j < N; ++j) {
      double s = 0.0;
#pragma unroll
      for (int a = 0; a < M; ++a) s = fma(AL[i * M + a], P[j * M + a], s);
#pragma unroll
      for (int l = 0; l < N; ++l) s = fma(-y.A[i * N + l], F[l * N + j], s);
      k.A[i * N + j] = s;
    }
  // db = -AL w - A c
#pragma unroll
  for (int i = 0; i < N; ++i) {
    double s = 0.0;
#pragma unroll
    for (int a = 0; a < M; ++a) s = fma(-AL[i * M + a], w[a], s);
    if (c) {
#pragma unroll
      for (int l = 0; l < N; ++l) s = fma(-y.A[i * N + l], c[l], s);
    }
    k.b[i] = s;
  }
  // dC = -AL AL^T
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = i; j < N; ++j) {
      double s = 0.0;
#pragma unroll
      for (int a = 0; a < M; ++a) s = fma(-AL[i * M + a], AL[j * M + a], s);
      k.C[sidx<N>(i, j)] = s;
    }
  // deta = -q - F^T eta + J c + P w
#pragma unroll
  for (int i = 0; i < N; ++i) {
    double s = -qr[i];
#pragma unroll
    for (int l = 0; l < N; ++l) s = fma(-F[l * N + i], y.eta[l], s);
    if (c) {
#pragma unroll
      for (int l = 0; l < N; ++l) s = fma(y.J[sidx<N>(i, l)], c[l], s);
    }
#pragma unroll
    for (int a = 0; a < M; ++a) s = fma(P[i * M + a], w[a], s);
    k.eta[i] = s;
  }
  // dJ = -Q - JF - (JF)^T + P P^T
  double JF[N * N];
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = 0; j < N; ++j) {
      double s = 0.0;
#pragma unroll
      for (int l = 0; l < N; ++l) s = fma(y.J[sidx<N>(i, l)], F[l * N + j], s);
      JF[i * N + j] = s;
    }
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = i; j < N; ++j) {
      double s = -Q[i * N + j] - JF[i * N + j] - JF[j * N + i];
#pragma unroll
      for (int a = 0; a < M; ++a) s = fma(P[i * M + a], P[j * M + a], s);
      k.J[sidx<N>(i, j)] = s;
    }
  // dzeta
  double z = -0.5 * qr[N];
#pragma unroll
  for (int a = 0; a < M; ++a) z = fma(0.5 * w[a], w[a], z);
  if (c) {
#pragma unroll
    for (int l = 0; l < N; ++l) z = fma(y.eta[l], c[l], z);
  }
  k.zeta = z;
}

// y <- base + s * k over every field.
template <int N>
__device__ __forceinline__ void axpy_to(Elem<N>& y, const Elem<N>& base, double s, const Elem<N>& k) {
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

struct BuildArgs {
  int64_t T;
  int32_t K;
  const double* t;
  Coefs cf;
  ElemPtrs out;
};

template <int N>
__device__ __forceinline__ const double* coef_at(const Coef& c, int64_t j, int32_t p, int32_t K, int stride) {
  return c.ptr + sample_index(c.mode, j, p, K) * stride;
}

// Element y in the full layout (A, b, C, eta, J with C and J written in full,
// zeta): 3 N^2 + 2 N + 1 doubles at dst.
template <int N>
__device__ __forceinline__ void store_full(const Elem<N>& y, double* dst) {
  double* o = dst;
#pragma unroll
  for (int i = 0; i < N * N; ++i) *o++ = y.A[i];
#pragma unroll
  for (int i = 0; i < N; ++i) *o++ = y.b[i];
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int c = 0; c < N; ++c) *o++ = y.C[sidx<N>(i, c)];
#pragma unroll
  for (int i = 0; i < N; ++i) *o++ = y.eta[i];
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int c = 0; c < N; ++c) *o++ = y.J[sidx<N>(i, c)];
  *o = y.zeta;
}

// K classical RK4 steps of the backward conditional HJB ODEs for sub-interval
// j, from the boundary A = I, b = C = eta = J = 0, zeta = 0 at s = t_{j+1}
// down to s = t_j (Sec. IV-B, eq. abcej_boundary).  With kStages the four
// stage inputs of every step go to stages[i][0..3] (full layout), for the
// discrete adjoint's reverse sweep.
template <int N, int M, bool kStages = false>
__device__ __forceinline__ void build_one(const Coefs& cf, const double* t, int64_t j, int32_t K, Elem<N>& y,
                                          double* stages = nullptr) {
  constexpr int FS = 3 * N * N + 2 * N + 1;
  const double h = (t[j + 1] - t[j]) / K;
  Elem<N> yn, yt, k;
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
  for (int32_t i = K - 1; i >= 0; --i) {
    // stage times (in half steps from t_j): 2i+2, 2i+1, 2i+1, 2i
    const int32_t ps[3] = {2 * i + 2, 2 * i + 1, 2 * i};
    const double* F[3];
    const double* c[3];
    const double* Lt[3];
    const double* Q[3];
    const double* qr[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      F[q] = coef_at<N>(cf.F, j, ps[q], K, N * N);
      c[q] = cf.c.ptr ? coef_at<N>(cf.c, j, ps[q], K, N) : nullptr;
      Lt[q] = coef_at<N>(cf.Lt, j, ps[q], K, N * M);
      Q[q] = coef_at<N>(cf.Q, j, ps[q], K, N * N);
      qr[q] = coef_at<N>(cf.qr, j, ps[q], K, N + 1);
    }
    double* st = kStages ? stages + (int64_t)i * 4 * FS : nullptr;
    if constexpr (kStages) store_full<N>(y, st);
    element_rhs<N, M>(y, F[0], c[0], Lt[0], Q[0], qr[0], k);
    axpy_to(yn, y, -h / 6.0, k);
    axpy_to(yt, y, -0.5 * h, k);
    if constexpr (kStages) store_full<N>(yt, st + FS);
    element_rhs<N, M>(yt, F[1], c[1], Lt[1], Q[1], qr[1], k);
    axpy_to(yn, yn, -h / 3.0, k);
    axpy_to(yt, y, -0.5 * h, k);
    if constexpr (kStages) store_full<N>(yt, st + 2 * FS);
    element_rhs<N, M>(yt, F[1], c[1], Lt[1], Q[1], qr[1], k);
    axpy_to(yn, yn, -h / 3.0, k);
    axpy_to(yt, y, -h, k);
    if constexpr (kStages) store_full<N>(yt, st + 3 * FS);
    element_rhs<N, M>(yt, F[2], c[2], Lt[2], Q[2], qr[2], k);
    axpy_to(y, yn, -h / 6.0, k);
  }
}

template <int N, int M>
__global__ void __launch_bounds__(128) build_kernel(BuildArgs a) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= a.T) return;
  Elem<N> y;
  build_one<N, M>(a.cf, a.t, j, a.K, y);
  store_public<N>(a.out, j, y);
}

// The same for sub-intervals j0 .. j0 + T - 1 (a.T counts the range), writing
// every RK4 stage input of sub-interval j0 + i to stages + i K 4 (3N^2 + 2N + 1)
// (full layout, step i = K-1 .. 0 at slot i); the element itself is stored
// only when a.out.A is not null.
template <int N, int M>
__global__ void __launch_bounds__(128) build_stages_kernel(BuildArgs a, int64_t j0, double* stages) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.T) return;
  constexpr int FS = 3 * N * N + 2 * N + 1;
  Elem<N> y;
  build_one<N, M, true>(a.cf, a.t, j0 + i, a.K, y, stages + i * (int64_t)a.K * 4 * FS);
  if (a.out.A) store_public<N>(a.out, j0 + i, y);
}

// Terminal element a_T: A = b = C = 0, J = Hf^T Xf Hf, eta = Hf^T Xf rf,
// zeta = 1/2 rf^T Xf rf.  One thread per (i, j) entry of the n x n blocks.
__device__ __forceinline__ double hf_at(const double* Hf, int k, int i, int n) {
  return Hf ? Hf[k * n + i] : (k == i ? 1.0 : 0.0);
}

struct TermArgs {
  int32_t n, nr;
  const double *Hf, *Xf, *rf;
  double *A, *b, *C, *eta, *J, *zeta;  // the terminal record (any of A, b, C, zeta may be null)
};

__global__ void terminal_kernel(TermArgs a) {
  const int n = a.n, nr = a.nr;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * n) return;
  const int i = e / n, j = e % n;
  double vij = 0.0, vji = 0.0;
  for (int k = 0; k < nr; ++k) {
    double xhj = 0.0, xhi = 0.0;
    for (int l = 0; l < nr; ++l) {
      xhj = fma(a.Xf[k * nr + l], hf_at(a.Hf, l, j, n), xhj);
      xhi = fma(a.Xf[k * nr + l], hf_at(a.Hf, l, i, n), xhi);
    }
    vij = fma(hf_at(a.Hf, k, i, n), xhj, vij);
    vji = fma(hf_at(a.Hf, k, j, n), xhi, vji);
  }
  a.J[e] = 0.5 * (vij + vji);
  if (a.A) a.A[e] = 0.0;
  if (a.C) a.C[e] = 0.0;
  if (j == 0) {
    if (a.b) a.b[i] = 0.0;
    double et = 0.0;
    if (a.rf)
      for (int k = 0; k < nr; ++k) {
        double xr = 0.0;
        for (int l = 0; l < nr; ++l) xr = fma(a.Xf[k * nr + l], a.rf[l], xr);
        et = fma(hf_at(a.Hf, k, i, n), xr, et);
      }
    a.eta[i] = et;
  }
  if (e == 0 && a.zeta) {
    double rho = 0.0;
    if (a.rf)
      for (int k = 0; k < nr; ++k) {
        double xr = 0.0;
        for (int l = 0; l < nr; ++l) xr = fma(a.Xf[k * nr + l], a.rf[l], xr);
        rho = fma(a.rf[k], xr, rho);
      }
    *a.zeta = 0.5 * rho;
  }
}

cudaError_t launch_terminal_values(const lqt_problem& p, double* J, double* eta, double* zeta, cudaStream_t st) {
  TermArgs t{p.n, p.nr, p.Hf, p.Xf, p.rf, nullptr, nullptr, nullptr, eta, J, zeta};
  terminal_kernel<<<(p.n * p.n + 255) / 256, 256, 0, st>>>(t);
  count_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// batches: coefficient preparation and element build over the concatenation
// ---------------------------------------------------------------------------

// which = 0: Lt and Ku of every problem (constant L, U); which = 1: q = X r,
// rho = r'Xr of every qr sample (X constant, H = identity).
__global__ void batch_prepare_kernel(BatchDev bd, int which) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int n = bd.n, m = bd.m;
  if (which == 0) {
    if (g >= bd.B) return;
    const BatchProb& P = bd.probs[g];
    double R[kMaxM * kMaxM];
    for (int i = 0; i < m * m; ++i) R[i] = P.U[i];
    cholesky_lower(R, m);
    double* Lt = const_cast<double*>(P.cf.Lt.ptr);
    for (int i = 0; i < n; ++i) {
      double row[kMaxM];
      for (int c = 0; c < m; ++c) {
        double v = P.L[i * m + c];
        for (int k = 0; k < c; ++k) v -= row[k] * R[c * m + k];
        row[c] = v / R[c * m + c];
      }
      for (int c = 0; c < bd.M; ++c) Lt[i * bd.M + c] = c < m ? row[c] : 0.0;
    }
    double* Ku = const_cast<double*>(P.cf.Ku);
    for (int col = 0; col < n; ++col) {
      double y[kMaxM];
      for (int i = 0; i < m; ++i) {
        double v = P.L[col * m + i];
        for (int k = 0; k < i; ++k) v -= R[i * m + k] * y[k];
        y[i] = v / R[i * m + i];
      }
      for (int i = m - 1; i >= 0; --i) {
        double v = y[i];
        for (int k = i + 1; k < m; ++k) v -= R[k * m + i] * y[k];
        y[i] = v / R[i * m + i];
      }
      for (int i = 0; i < m; ++i) Ku[i * n + col] = y[i];
    }
  } else {
    if (g >= bd.total_qr) return;
    const int32_t b = batch_find(bd.off_qr, bd.B, g);
    const BatchProb& P = bd.probs[b];
    const int64_t s = g - bd.off_qr[b];
    const double* r = P.r ? P.r + (P.r_mode == kConst ? 0 : s) * n : nullptr;
    double* out = const_cast<double*>(P.cf.qr.ptr) + s * (n + 1);
    double rho = 0.0;
    for (int i = 0; i < n; ++i) {
      double v = 0.0;
      if (r)
        for (int l = 0; l < n; ++l) v = fma(P.X[i * n + l], r[l], v);
      out[i] = v;
      if (r) rho = fma(r[i], v, rho);
    }
    out[n] = rho;
  }
}

cudaError_t batch_prepare(const BatchDev& bd, cudaStream_t st) {
  batch_prepare_kernel<<<(unsigned)((bd.B + 127) / 128), 128, 0, st>>>(bd, 0);
  count_launch();
  batch_prepare_kernel<<<(unsigned)((bd.total_qr + 127) / 128), 128, 0, st>>>(bd, 1);
  count_launch();
  return cudaGetLastError();
}

// One thread per boundary of the concatenation: element j of problem b, or its
// terminal element (j = T_b; Hf = identity: J = Xf, eta = Xf rf,
// zeta = rf'Xf rf / 2).
template <int N, int M>
__global__ void __launch_bounds__(128) batch_build_kernel(BatchDev bd, ElemPtrs out) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= bd.total) return;
  const int32_t b = batch_find(bd.off, bd.B, g);
  const BatchProb& P = bd.probs[b];
  const int64_t j = g - P.off;
  Elem<N> y;
  if (j < P.T) {
    build_one<N, M>(P.cf, P.t, j, bd.K, y);
  } else {
#pragma unroll
    for (int i = 0; i < N * N; ++i) y.A[i] = 0.0;
#pragma unroll
    for (int i = 0; i < N; ++i) {
      y.b[i] = 0.0;
      double e = 0.0;
      if (P.rf)
        for (int l = 0; l < N; ++l) e = fma(P.Xf[i * N + l], P.rf[l], e);
      y.eta[i] = e;
    }
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
      for (int c = i; c < N; ++c) {
        y.C[sidx<N>(i, c)] = 0.0;
        y.J[sidx<N>(i, c)] = 0.5 * (P.Xf[i * N + c] + P.Xf[c * N + i]);
      }
    double z = 0.0;
    if (P.rf)
      for (int i = 0; i < N; ++i) z = fma(P.rf[i], y.eta[i], z);
    y.zeta = 0.5 * z;
  }
  store_public<N>(out, g, y);
}

template <int N, int M>
static void launch_batch_build_nm(const BatchDev& bd, const ElemPtrs& el, cudaStream_t st) {
  batch_build_kernel<N, M><<<(unsigned)((bd.total + 127) / 128), 128, 0, st>>>(bd, el);
  count_launch();
}

cudaError_t batch_build(const BatchDev& bd, const ElemPtrs& el, char* team_scratch, cudaStream_t st) {
  switch (bd.n) {
    case 1: launch_batch_build_nm<1, 1>(bd, el, st); break;
    case 2:
      if (bd.M == 1) launch_batch_build_nm<2, 1>(bd, el, st);
      else launch_batch_build_nm<2, 2>(bd, el, st);
      break;
    case 3:
      if (bd.M == 1) launch_batch_build_nm<3, 1>(bd, el, st);
      else if (bd.M == 2) launch_batch_build_nm<3, 2>(bd, el, st);
      else launch_batch_build_nm<3, 4>(bd, el, st);
      break;
    case 4:
      if (bd.M == 1) launch_batch_build_nm<4, 1>(bd, el, st);
      else if (bd.M == 2) launch_batch_build_nm<4, 2>(bd, el, st);
      else launch_batch_build_nm<4, 4>(bd, el, st);
      break;
    case 8:
      if (bd.M == 1) launch_batch_build_nm<8, 1>(bd, el, st);
      else if (bd.M == 2) launch_batch_build_nm<8, 2>(bd, el, st);
      else if (bd.M == 4) launch_batch_build_nm<8, 4>(bd, el, st);
      else launch_batch_build_nm<8, 8>(bd, el, st);
      break;
    case 16:
    case 64: return batch_build_team(bd, el, (double*)team_scratch, st);
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <int N, int M>
static void launch_build_nm(const BuildArgs& a, cudaStream_t st, double* stages, int64_t j0) {
  const int threads = 128;
  const int64_t blocks = (a.T + threads - 1) / threads;
  if (stages)
    build_stages_kernel<N, M><<<(unsigned)blocks, threads, 0, st>>>(a, j0, stages);
  else
    build_kernel<N, M><<<(unsigned)blocks, threads, 0, st>>>(a);
  count_launch();
}

template <int N>
static cudaError_t launch_build_n(const BuildArgs& a, int M, cudaStream_t st, double* stages = nullptr,
                                  int64_t j0 = 0) {
  switch (M) {
    case 1: launch_build_nm<N, 1>(a, st, stages, j0); break;
    case 2: if constexpr (N >= 2) { launch_build_nm<N, 2>(a, st, stages, j0); break; } else return cudaErrorInvalidValue;
    case 4: if constexpr (N >= 3) { launch_build_nm<N, 4>(a, st, stages, j0); break; } else return cudaErrorInvalidValue;
    case 8: if constexpr (N >= 8) { launch_build_nm<N, 8>(a, st, stages, j0); break; } else return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
  }
  return cudaSuccess;
}

// The RK4 stage inputs of sub-intervals j0 .. j0 + cnt - 1 of p (n <= 8), the
// stages of sub-interval j0 + i at stages + i K 4 (3n^2 + 2n + 1) (full
// layout); the elements themselves go to `out` when out.A is not null.
cudaError_t launch_build_stages_range(const lqt_problem& p, const Layout& lay, const Coefs& cf, int64_t j0,
                                      int64_t cnt, double* stages, cudaStream_t st, const ElemPtrs& out) {
  BuildArgs a{};
  a.T = cnt; a.K = p.K; a.t = p.t; a.cf = cf; a.out = out;
  if (team_build_preferred(p.n, cnt)) return team_launch_build_small(p, lay, cf, j0, cnt, stages, out, st);
  switch (p.n) {
    case 1: return launch_build_n<1>(a, lay.M, st, stages, j0);
    case 2: return launch_build_n<2>(a, lay.M, st, stages, j0);
    case 3: return launch_build_n<3>(a, lay.M, st, stages, j0);
    case 4: return launch_build_n<4>(a, lay.M, st, stages, j0);
    case 8: return launch_build_n<8>(a, lay.M, st, stages, j0);
    default: return cudaErrorInvalidValue;
  }
}

// Elements 0..T-1 of p alone (no terminal element), n <= 8.
cudaError_t launch_build_range(const lqt_problem& p, const Layout& lay, const Coefs& cf, const ElemPtrs& out,
                               cudaStream_t st) {
  BuildArgs a;
  a.T = p.T; a.K = p.K; a.t = p.t; a.cf = cf; a.out = out;
  switch (p.n) {
    case 1: return launch_build_n<1>(a, lay.M, st);
    case 2: return launch_build_n<2>(a, lay.M, st);
    case 3: return launch_build_n<3>(a, lay.M, st);
    case 4: return launch_build_n<4>(a, lay.M, st);
    case 8: return launch_build_n<8>(a, lay.M, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_build(const lqt_problem& p, const Layout& lay, const Coefs& cf, const ElemPtrs& out,
                         cudaStream_t st, double* team_scratch) {
  BuildArgs a;
  a.T = p.T; a.K = p.K; a.t = p.t; a.cf = cf; a.out = out;
  cudaError_t e;
  if (team_build_preferred(p.n, p.T)) {
    e = team_launch_build_small(p, lay, cf, 0, p.T, nullptr, out, st);
    if (e != cudaSuccess) return e;
    return launch_terminal_element(p, out, st);
  }
  switch (p.n) {
    case 1: e = launch_build_n<1>(a, lay.M, st); break;
    case 2: e = launch_build_n<2>(a, lay.M, st); break;
    case 3: e = launch_build_n<3>(a, lay.M, st); break;
    case 4: e = launch_build_n<4>(a, lay.M, st); break;
    case 8: e = launch_build_n<8>(a, lay.M, st); break;
    case 16:
    case 64: e = team_launch_build(p, lay, cf, out, team_scratch, st); break;
    default: return cudaErrorInvalidValue;
  }
  if (e != cudaSuccess) return e;
  return launch_terminal_element(p, out, st);
}

// Terminal element a_T into index T of the public arrays.
cudaError_t launch_terminal_element(const lqt_problem& p, const ElemPtrs& out, cudaStream_t st) {
  const int64_t T = p.T;
  const int n = p.n;
  TermArgs t{p.n, p.nr, p.Hf, p.Xf, p.rf, out.A + T * n * n, out.b + T * n, out.C + T * n * n,
             out.eta + T * n, out.J + T * n * n, out.zeta ? out.zeta + T : nullptr};
  terminal_kernel<<<(n * n + 255) / 256, 256, 0, st>>>(t);
  count_launch();
  return cudaGetLastError();
}

}  // namespace lqt
