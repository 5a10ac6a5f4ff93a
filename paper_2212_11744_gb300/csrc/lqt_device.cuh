// Device-side building blocks of the LQT solver: register-resident small
// matrices (one CUDA thread owns one n x n problem), the LQT combination rule
// of Sec. IV-A (eq. lqt_comb) in full and in value form, and LU with partial
// pivoting written without dynamic register indexing.
//
// Storage inside a thread: general n x n matrices row-major in double[N*N];
// symmetric ones (C, J, S) as the upper triangle, row by row, in
// double[N*(N+1)/2] (index sidx<N>(i, j)).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "lqt_internal.h"

namespace lqt {

template <int N>
struct Dim {
  static constexpr int NN = N * N;
  static constexpr int NS = N * (N + 1) / 2;
};

// Position of (i, j) in the packed upper triangle.
template <int N>
__host__ __device__ constexpr int sidx(int i, int j) {
  return i <= j ? i * N - (i * (i - 1)) / 2 + (j - i) : j * N - (j * (j - 1)) / 2 + (i - j);
}

// Conditional value function element (Sec. IV-A, eq. LQT_V_form2).
template <int N>
struct Elem {
  double A[N * N];
  double b[N];
  double C[Dim<N>::NS];
  double eta[N];
  double J[Dim<N>::NS];
  double zeta;
};

// Value function (eq. V_quadratic_LQT): V(x) = zeta + 1/2 x'Sx - v'x.
template <int N>
struct Val {
  double S[Dim<N>::NS];
  double v[N];
  double zeta;
};

// Packed element size in doubles (A, b, C packed, eta, J packed, zeta).
template <int N>
__host__ __device__ constexpr int packed_elem_doubles() {
  return N * N + N + Dim<N>::NS + N + Dim<N>::NS + 1;
}
template <int N>
__host__ __device__ constexpr int packed_val_doubles() {
  return Dim<N>::NS + N + 1;
}

// ---------------------------------------------------------------------------
// status word
// ---------------------------------------------------------------------------

__device__ __forceinline__ void flag(unsigned bits) { atomicOr(&g_status_word, bits); }

__device__ __forceinline__ bool finite(double x) { return isfinite(x); }

// ---------------------------------------------------------------------------
// packed element / value I/O (each thread moves its own contiguous record)
// ---------------------------------------------------------------------------

template <int N>
__device__ __forceinline__ void load_packed(const double* __restrict__ p, Elem<N>& e) {
  int o = 0;
#pragma unroll
  for (int i = 0; i < N * N; ++i) e.A[i] = p[o++];
#pragma unroll
  for (int i = 0; i < N; ++i) e.b[i] = p[o++];
#pragma unroll
  for (int i = 0; i < Dim<N>::NS; ++i) e.C[i] = p[o++];
#pragma unroll
  for (int i = 0; i < N; ++i) e.eta[i] = p[o++];
#pragma unroll
  for (int i = 0; i < Dim<N>::NS; ++i) e.J[i] = p[o++];
  e.zeta = p[o];
}

template <int N>
__device__ __forceinline__ void store_packed(double* __restrict__ p, const Elem<N>& e) {
  int o = 0;
#pragma unroll
  for (int i = 0; i < N * N; ++i) p[o++] = e.A[i];
#pragma unroll
  for (int i = 0; i < N; ++i) p[o++] = e.b[i];
#pragma unroll
  for (int i = 0; i < Dim<N>::NS; ++i) p[o++] = e.C[i];
#pragma unroll
  for (int i = 0; i < N; ++i) p[o++] = e.eta[i];
#pragma unroll
  for (int i = 0; i < Dim<N>::NS; ++i) p[o++] = e.J[i];
  p[o] = e.zeta;
}

// Element k from the public SoA layout (full symmetric matrices).
template <int N>
__device__ __forceinline__ void load_public(const ElemPtrs& el, int64_t k, Elem<N>& e) {
  const double* A = el.A + k * N * N;
  const double* b = el.b + k * N;
  const double* C = el.C + k * N * N;
  const double* eta = el.eta + k * N;
  const double* J = el.J + k * N * N;
#pragma unroll
  for (int i = 0; i < N * N; ++i) e.A[i] = A[i];
#pragma unroll
  for (int i = 0; i < N; ++i) {
    e.b[i] = b[i];
    e.eta[i] = eta[i];
  }
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = i; j < N; ++j) {
      e.C[sidx<N>(i, j)] = C[i * N + j];
      e.J[sidx<N>(i, j)] = J[i * N + j];
    }
  e.zeta = el.zeta ? el.zeta[k] : 0.0;
}

template <int N>
__device__ __forceinline__ void store_public(const ElemPtrs& el, int64_t k, const Elem<N>& e) {
  double* A = el.A + k * N * N;
  double* b = el.b + k * N;
  double* C = el.C + k * N * N;
  double* eta = el.eta + k * N;
  double* J = el.J + k * N * N;
#pragma unroll
  for (int i = 0; i < N * N; ++i) A[i] = e.A[i];
#pragma unroll
  for (int i = 0; i < N; ++i) {
    b[i] = e.b[i];
    eta[i] = e.eta[i];
  }
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = 0; j < N; ++j) {
      C[i * N + j] = e.C[sidx<N>(i, j)];
      J[i * N + j] = e.J[sidx<N>(i, j)];
    }
  if (el.zeta) el.zeta[k] = e.zeta;
}

// Full-matrix record layouts shared with the team kernels (lqt_team.cuh):
// element = A (N*N), b (N), C (N*N), eta (N), J (N*N), zeta; value = S (N*N),
// v (N), zeta.
template <int N>
__host__ __device__ constexpr int full_elem_doubles() {
  return 3 * N * N + 2 * N + 1;
}
template <int N>
__host__ __device__ constexpr int full_val_doubles() {
  return N * N + N + 1;
}

template <int N>
__device__ __forceinline__ void store_full(double* __restrict__ p, const Elem<N>& e) {
  double* A = p;
  double* b = A + N * N;
  double* C = b + N;
  double* eta = C + N * N;
  double* J = eta + N;
#pragma unroll
  for (int i = 0; i < N * N; ++i) A[i] = e.A[i];
#pragma unroll
  for (int i = 0; i < N; ++i) {
    b[i] = e.b[i];
    eta[i] = e.eta[i];
  }
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = 0; j < N; ++j) {
      C[i * N + j] = e.C[sidx<N>(i, j)];
      J[i * N + j] = e.J[sidx<N>(i, j)];
    }
  J[N * N] = e.zeta;
}

template <int N>
__device__ __forceinline__ void load_full(const double* __restrict__ p, Elem<N>& e) {
  const double* A = p;
  const double* b = A + N * N;
  const double* C = b + N;
  const double* eta = C + N * N;
  const double* J = eta + N;
#pragma unroll
  for (int i = 0; i < N * N; ++i) e.A[i] = A[i];
#pragma unroll
  for (int i = 0; i < N; ++i) {
    e.b[i] = b[i];
    e.eta[i] = eta[i];
  }
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = i; j < N; ++j) {
      e.C[sidx<N>(i, j)] = C[i * N + j];
      e.J[sidx<N>(i, j)] = J[i * N + j];
    }
  e.zeta = J[N * N];
}

template <int N>
__device__ __forceinline__ void store_val_full(double* __restrict__ p, const Val<N>& v) {
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = 0; j < N; ++j) p[i * N + j] = v.S[sidx<N>(i, j)];
#pragma unroll
  for (int i = 0; i < N; ++i) p[N * N + i] = v.v[i];
  p[N * N + N] = v.zeta;
}

template <int N>
__device__ __forceinline__ void load_val_full(const double* __restrict__ p, Val<N>& v) {
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = i; j < N; ++j) v.S[sidx<N>(i, j)] = p[i * N + j];
#pragma unroll
  for (int i = 0; i < N; ++i) v.v[i] = p[N * N + i];
  v.zeta = p[N * N + N];
}

template <int N>
__device__ __forceinline__ void zero_val(Val<N>& v) {
#pragma unroll
  for (int i = 0; i < Dim<N>::NS; ++i) v.S[i] = 0.0;
#pragma unroll
  for (int i = 0; i < N; ++i) v.v[i] = 0.0;
  v.zeta = 0.0;
}

template <int N>
__device__ __forceinline__ void load_val(const double* __restrict__ p, Val<N>& v) {
#pragma unroll
  for (int i = 0; i < Dim<N>::NS; ++i) v.S[i] = p[i];
#pragma unroll
  for (int i = 0; i < N; ++i) v.v[i] = p[Dim<N>::NS + i];
  v.zeta = p[Dim<N>::NS + N];
}

template <int N>
__device__ __forceinline__ void store_val(double* __restrict__ p, const Val<N>& v) {
#pragma unroll
  for (int i = 0; i < Dim<N>::NS; ++i) p[i] = v.S[i];
#pragma unroll
  for (int i = 0; i < N; ++i) p[Dim<N>::NS + i] = v.v[i];
  p[Dim<N>::NS + N] = v.zeta;
}

// ---------------------------------------------------------------------------
// LU with partial pivoting, applied to an augmented right-hand side block
// ---------------------------------------------------------------------------

// Magnitude key of a double: its bit pattern without the sign.  For finite
// values (and +inf) comparing keys as unsigned integers orders them like |x|,
// on the integer pipes (FP64 compares share the slow FP64 pipe).
__device__ __forceinline__ unsigned long long mag_key(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
}
__device__ __forceinline__ unsigned long long umax64(unsigned long long a, unsigned long long b) {
  return a > b ? a : b;
}
// Relative pivot tolerance 2^-40 (about 9.1e-13): a pivot this small next to
// its row's original scale means a condition number beyond ~1e12, where an
// FP64 solve no longer carries the digits a 1e-9 result needs.  Applied to the
// key: subtracting 40 from the exponent field multiplies a normal double by
// 2^-40 (row scales below 2^-982 get the threshold 0).
constexpr unsigned long long kPivotTolExpShift = 40ull << 52;
__device__ __forceinline__ bool pivot_too_small(double piv, unsigned long long row_key) {
  const unsigned long long thr = row_key > kPivotTolExpShift ? row_key - kPivotTolExpShift : 0ull;
  return mag_key(piv) <= thr;
}

// Solves W X = R in place (W: N x N, R: N x Q, both row-major in registers).
// Row exchanges are done with predicated selects so every register index stays
// a compile-time constant.  W = I + P (P = C J or C S in every use): a pivot no
// larger than 2^-40 times its row's original scale, max(1, max_j |W_ij|) (the
// identity's 1 included, so that cancellation between I and P counts), sets
// the SINGULAR status bit: the system is then singular to working precision
// and the solution meaningless (but finite work).
template <int N, int Q>
__device__ __forceinline__ void lu_solve(double (&W)[N * N], double (&R)[N * Q]) {
  unsigned long long rk[N];  // original row scales, as magnitude keys
#pragma unroll
  for (int i = 0; i < N; ++i) {
    rk[i] = mag_key(1.0);
#pragma unroll
    for (int j = 0; j < N; ++j) rk[i] = umax64(rk[i], mag_key(W[i * N + j]));
  }
#pragma unroll
  for (int k = 0; k < N; ++k) {
    // bring the largest |W[i][k]|, i >= k, to row k
#pragma unroll
    for (int i = k + 1; i < N; ++i) {
      const bool sw = fabs(W[i * N + k]) > fabs(W[k * N + k]);
#pragma unroll
      for (int j = k; j < N; ++j) {
        const double a = W[k * N + j], c = W[i * N + j];
        W[k * N + j] = sw ? c : a;
        W[i * N + j] = sw ? a : c;
      }
#pragma unroll
      for (int j = 0; j < Q; ++j) {
        const double a = R[k * Q + j], c = R[i * Q + j];
        R[k * Q + j] = sw ? c : a;
        R[i * Q + j] = sw ? a : c;
      }
      const unsigned long long a = rk[k], c = rk[i];
      rk[k] = sw ? c : a;
      rk[i] = sw ? a : c;
    }
    const double piv = W[k * N + k];
    if (pivot_too_small(piv, rk[k])) flag(kStatusSingular);
    const double inv = 1.0 / piv;
#pragma unroll
    for (int i = k + 1; i < N; ++i) {
      const double f = W[i * N + k] * inv;
#pragma unroll
      for (int j = k + 1; j < N; ++j) W[i * N + j] = fma(-f, W[k * N + j], W[i * N + j]);
#pragma unroll
      for (int j = 0; j < Q; ++j) R[i * Q + j] = fma(-f, R[k * Q + j], R[i * Q + j]);
    }
    // scale row k once so back substitution needs no divisions
#pragma unroll
    for (int j = k + 1; j < N; ++j) W[k * N + j] *= inv;
#pragma unroll
    for (int j = 0; j < Q; ++j) R[k * Q + j] *= inv;
  }
#pragma unroll
  for (int k = N - 1; k >= 0; --k)
#pragma unroll
    for (int i = 0; i < k; ++i) {
      const double f = W[i * N + k];
#pragma unroll
      for (int j = 0; j < Q; ++j) R[i * Q + j] = fma(-f, R[k * Q + j], R[i * Q + j]);
    }
}

// ---------------------------------------------------------------------------
// combination rule (Sec. IV-A, eq. lqt_comb)
// ---------------------------------------------------------------------------

// G is the type the matrix products are accumulated in: double for the FP64
// path; float for the mixed-precision path, where every product runs in FP32
// while W = I + C J is promoted to FP64 for the LU solve, which stays FP64.
template <typename G>
__device__ __forceinline__ G gf(double x) {
  return (G)x;
}

// out = e1 (x) e2 for general elements.  With W = I + C1 J2 and
// M = W^-1, (I + J2 C1)^-1 = M^T:
//   K1 = M A1, MC1 = M C1, z0 = M (b1 + C1 eta2)          (one LU, 2N+1 rhs)
//   A   = A2 K1,        b = A2 z0 + b2,    C = A2 MC1 A2^T + C2
//   eta = K1^T (eta2 - J2 b1) + eta1,      J = K1^T (J2 A1) + J1
//   zeta = zeta1 + zeta2 + 1/2 l0'C1 l0 + 1/2 z0'J2 z0 - z0'eta2,
//          l0 = J2 z0 - eta2                                 (minimiser at x=0)
// `out` may alias e2 (it is written after e2's last read of each field).
template <int N, typename G = double>
__device__ __forceinline__ void combine(const Elem<N>& e1, const Elem<N>& e2, Elem<N>& out) {
  constexpr int Q = 2 * N + 1;
  double W[N * N];
  double R[N * Q];
  // W = I + C1 J2 ; R = [A1 | C1 | b1 + C1 eta2]
#pragma unroll
  for (int i = 0; i < N; ++i) {
#pragma unroll
    for (int j = 0; j < N; ++j) {
      G s = (i == j) ? G(1) : G(0);
#pragma unroll
      for (int l = 0; l < N; ++l) s = fma(gf<G>(e1.C[sidx<N>(i, l)]), gf<G>(e2.J[sidx<N>(l, j)]), s);
      W[i * N + j] = (double)s;
      R[i * Q + j] = e1.A[i * N + j];
      R[i * Q + N + j] = e1.C[sidx<N>(i, j)];
    }
    G s = gf<G>(e1.b[i]);
#pragma unroll
    for (int l = 0; l < N; ++l) s = fma(gf<G>(e1.C[sidx<N>(i, l)]), gf<G>(e2.eta[l]), s);
    R[i * Q + 2 * N] = (double)s;
  }
  lu_solve<N, Q>(W, R);
  // R = [K1 | MC1 | z0]
  G z0[N], l0[N], J2z0[N];
#pragma unroll
  for (int i = 0; i < N; ++i) z0[i] = gf<G>(R[i * Q + 2 * N]);
  // zeta
  G zeta = gf<G>(e1.zeta) + gf<G>(e2.zeta);
#pragma unroll
  for (int i = 0; i < N; ++i) {
    G s = 0;
#pragma unroll
    for (int l = 0; l < N; ++l) s = fma(gf<G>(e2.J[sidx<N>(i, l)]), z0[l], s);
    J2z0[i] = s;
    l0[i] = s - gf<G>(e2.eta[i]);
  }
#pragma unroll
  for (int i = 0; i < N; ++i) {
    G s = 0;
#pragma unroll
    for (int l = 0; l < N; ++l) s = fma(gf<G>(e1.C[sidx<N>(i, l)]), l0[l], s);
    zeta = fma(G(0.5) * l0[i], s, zeta);
    zeta = fma(z0[i], fma(G(0.5), J2z0[i], -gf<G>(e2.eta[i])), zeta);
  }
  // eta = K1^T (eta2 - J2 b1) + eta1
  G w[N];
#pragma unroll
  for (int i = 0; i < N; ++i) {
    G s = gf<G>(e2.eta[i]);
#pragma unroll
    for (int l = 0; l < N; ++l) s = fma(-gf<G>(e2.J[sidx<N>(i, l)]), gf<G>(e1.b[l]), s);
    w[i] = s;
  }
  double eta_new[N];
#pragma unroll
  for (int i = 0; i < N; ++i) {
    G s = gf<G>(e1.eta[i]);
#pragma unroll
    for (int l = 0; l < N; ++l) s = fma(gf<G>(R[l * Q + i]), w[l], s);
    eta_new[i] = (double)s;
  }
  // J = K1^T (J2 A1) + J1   (upper triangle)
  G T1[N * N];
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = 0; j < N; ++j) {
      G s = 0;
#pragma unroll
      for (int l = 0; l < N; ++l) s = fma(gf<G>(e2.J[sidx<N>(i, l)]), gf<G>(e1.A[l * N + j]), s);
      T1[i * N + j] = s;
    }
  double J_new[Dim<N>::NS];
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = i; j < N; ++j) {
      G s = gf<G>(e1.J[sidx<N>(i, j)]);
#pragma unroll
      for (int l = 0; l < N; ++l) s = fma(gf<G>(R[l * Q + i]), T1[l * N + j], s);
      J_new[sidx<N>(i, j)] = (double)s;
    }
  // b = A2 z0 + b2
  double b_new[N];
#pragma unroll
  for (int i = 0; i < N; ++i) {
    G s = gf<G>(e2.b[i]);
#pragma unroll
    for (int l = 0; l < N; ++l) s = fma(gf<G>(e2.A[i * N + l]), z0[l], s);
    b_new[i] = (double)s;
  }
  // T1 = A2 MC1 ; C = T1 A2^T + C2 (upper triangle)
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = 0; j < N; ++j) {
      G s = 0;
#pragma unroll
      for (int l = 0; l < N; ++l) s = fma(gf<G>(e2.A[i * N + l]), gf<G>(R[l * Q + N + j]), s);
      T1[i * N + j] = s;
    }
  double C_new[Dim<N>::NS];
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = i; j < N; ++j) {
      G s = gf<G>(e2.C[sidx<N>(i, j)]);
#pragma unroll
      for (int l = 0; l < N; ++l) s = fma(T1[i * N + l], gf<G>(e2.A[j * N + l]), s);
      C_new[sidx<N>(i, j)] = (double)s;
    }
  // A = A2 K1
  double A_new[N * N];
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = 0; j < N; ++j) {
      G s = 0;
#pragma unroll
      for (int l = 0; l < N; ++l) s = fma(gf<G>(e2.A[i * N + l]), gf<G>(R[l * Q + j]), s);
      A_new[i * N + j] = (double)s;
    }
#pragma unroll
  for (int i = 0; i < N * N; ++i) out.A[i] = A_new[i];
#pragma unroll
  for (int i = 0; i < N; ++i) {
    out.b[i] = b_new[i];
    out.eta[i] = eta_new[i];
  }
#pragma unroll
  for (int i = 0; i < Dim<N>::NS; ++i) {
    out.C[i] = C_new[i];
    out.J[i] = J_new[i];
  }
  out.zeta = (double)zeta;
}

// Value-form combination: e (x) V where V = (S2, v2, zeta2) is a value
// function (an element with A = b = C = 0).  Returns the new value and the
// one-sub-interval optimal-state map x' = Psi x + alpha with
// Psi = (I + C S2)^-1 A and alpha = (I + C S2)^-1 (b + C v2)
// (Method 2 of Sec. IV-E over one sub-interval).
//   S    = Psi^T (S2 A) + J,   v = Psi^T (v2 - S2 b) + eta
//   zeta = zeta_e + zeta2 + 1/2 l0'C l0 + 1/2 z0'S2 z0 - z0'v2,
//          z0 = alpha, l0 = S2 z0 - v2
template <int N, typename G = double>
__device__ __forceinline__ void combine_value(const Elem<N>& e, const Val<N>& V, Val<N>& out, double (&Psi)[N * N],
                                              double (&alpha)[N], double* zeta_inc = nullptr) {
  constexpr int Q = N + 1;
  double W[N * N];
  double R[N * Q];
  // W = I + C S2 and b + C v2 in FP64 whatever G is: they define the
  // one-sub-interval map (Psi, alpha) that the state scan composes T times,
  // where FP32 rounding would accumulate
#pragma unroll
  for (int i = 0; i < N; ++i) {
#pragma unroll
    for (int j = 0; j < N; ++j) {
      double s = (i == j) ? 1.0 : 0.0;
#pragma unroll
      for (int l = 0; l < N; ++l) s = fma(e.C[sidx<N>(i, l)], V.S[sidx<N>(l, j)], s);
      W[i * N + j] = s;
      R[i * Q + j] = e.A[i * N + j];
    }
    double s = e.b[i];
#pragma unroll
    for (int l = 0; l < N; ++l) s = fma(e.C[sidx<N>(i, l)], V.v[l], s);
    R[i * Q + N] = s;
  }
  lu_solve<N, Q>(W, R);
#pragma unroll
  for (int i = 0; i < N; ++i) {
#pragma unroll
    for (int j = 0; j < N; ++j) Psi[i * N + j] = R[i * Q + j];
    alpha[i] = R[i * Q + N];
  }
  G Sz[N], l0[N];
  // the element's own share of zeta (its zeta and the saddle-point terms);
  // the carry's zeta is added to it in FP64
  G zeta = gf<G>(e.zeta);
#pragma unroll
  for (int i = 0; i < N; ++i) {
    G s = 0;
#pragma unroll
    for (int l = 0; l < N; ++l) s = fma(gf<G>(V.S[sidx<N>(i, l)]), gf<G>(alpha[l]), s);
    Sz[i] = s;
    l0[i] = s - gf<G>(V.v[i]);
  }
#pragma unroll
  for (int i = 0; i < N; ++i) {
    G s = 0;
#pragma unroll
    for (int l = 0; l < N; ++l) s = fma(gf<G>(e.C[sidx<N>(i, l)]), l0[l], s);
    zeta = fma(G(0.5) * l0[i], s, zeta);
    zeta = fma(gf<G>(alpha[i]), fma(G(0.5), Sz[i], -gf<G>(V.v[i])), zeta);
  }
  // w = v2 - S2 b
  G w[N];
#pragma unroll
  for (int i = 0; i < N; ++i) {
    G s = gf<G>(V.v[i]);
#pragma unroll
    for (int l = 0; l < N; ++l) s = fma(-gf<G>(V.S[sidx<N>(i, l)]), gf<G>(e.b[l]), s);
    w[i] = s;
  }
  // T1 = S2 A
  G T1[N * N];
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = 0; j < N; ++j) {
      G s = 0;
#pragma unroll
      for (int l = 0; l < N; ++l) s = fma(gf<G>(V.S[sidx<N>(i, l)]), gf<G>(e.A[l * N + j]), s);
      T1[i * N + j] = s;
    }
#pragma unroll
  for (int i = 0; i < N; ++i) {
    G s = gf<G>(e.eta[i]);
#pragma unroll
    for (int l = 0; l < N; ++l) s = fma(gf<G>(Psi[l * N + i]), w[l], s);
    out.v[i] = (double)s;
  }
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = i; j < N; ++j) {
      G s = gf<G>(e.J[sidx<N>(i, j)]);
#pragma unroll
      for (int l = 0; l < N; ++l) s = fma(gf<G>(Psi[l * N + i]), T1[l * N + j], s);
      out.S[sidx<N>(i, j)] = (double)s;
    }
  out.zeta = (double)zeta + V.zeta;
  if (zeta_inc) *zeta_inc = (double)zeta;
}

// ---------------------------------------------------------------------------
// prefix form of the combination (Method 2, Sec. IV-E)
// ---------------------------------------------------------------------------

// The (A, b, C) part of a prefix V(., t_0; ., t_k): only these enter the
// Method 2 states, and only these of a left operand enter the (A, b, C) of a
// combination.
template <int N>
struct Prefix {
  double A[N * N];
  double b[N];
  double C[Dim<N>::NS];
};

template <int N>
__device__ __forceinline__ void identity_prefix(Prefix<N>& P) {
#pragma unroll
  for (int i = 0; i < N * N; ++i) P.A[i] = (i % (N + 1) == 0) ? 1.0 : 0.0;
#pragma unroll
  for (int i = 0; i < N; ++i) P.b[i] = 0.0;
#pragma unroll
  for (int i = 0; i < Dim<N>::NS; ++i) P.C[i] = 0.0;
}

// The (A, b, C) part of a full-matrix record (full_elem_doubles layout).
template <int N>
__device__ __forceinline__ void load_prefix_full(const double* __restrict__ p, Prefix<N>& P) {
  const double* A = p;
  const double* b = A + N * N;
  const double* C = b + N;
#pragma unroll
  for (int i = 0; i < N * N; ++i) P.A[i] = A[i];
#pragma unroll
  for (int i = 0; i < N; ++i) P.b[i] = b[i];
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = i; j < N; ++j) P.C[sidx<N>(i, j)] = C[i * N + j];
}

// P <- P (x) e, (A, b, C) part only (Lemma LQT_combination with the prefix as
// the left operand): W = I + C_P J_e, [K | MC | z0] = W^-1 [A_P | C_P |
// b_P + C_P eta_e]; A = A_e K, b = A_e z0 + b_e, C = A_e MC A_e^T + C_e.
template <int N>
__device__ __forceinline__ void combine_prefix(Prefix<N>& P, const Elem<N>& e) {
  constexpr int Q = 2 * N + 1;
  double W[N * N];
  double R[N * Q];
#pragma unroll
  for (int i = 0; i < N; ++i) {
#pragma unroll
    for (int j = 0; j < N; ++j) {
      double s = (i == j) ? 1.0 : 0.0;
#pragma unroll
      for (int l = 0; l < N; ++l) s = fma(P.C[sidx<N>(i, l)], e.J[sidx<N>(l, j)], s);
      W[i * N + j] = s;
      R[i * Q + j] = P.A[i * N + j];
      R[i * Q + N + j] = P.C[sidx<N>(i, j)];
    }
    double s = P.b[i];
#pragma unroll
    for (int l = 0; l < N; ++l) s = fma(P.C[sidx<N>(i, l)], e.eta[l], s);
    R[i * Q + 2 * N] = s;
  }
  lu_solve<N, Q>(W, R);
  double T1[N * N];
#pragma unroll
  for (int i = 0; i < N; ++i) {
    double s = e.b[i];
#pragma unroll
    for (int l = 0; l < N; ++l) s = fma(e.A[i * N + l], R[l * Q + 2 * N], s);
    P.b[i] = s;
#pragma unroll
    for (int j = 0; j < N; ++j) {
      double t = 0.0;
#pragma unroll
      for (int l = 0; l < N; ++l) t = fma(e.A[i * N + l], R[l * Q + N + j], t);
      T1[i * N + j] = t;
    }
  }
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = i; j < N; ++j) {
      double s = e.C[sidx<N>(i, j)];
#pragma unroll
      for (int l = 0; l < N; ++l) s = fma(T1[i * N + l], e.A[j * N + l], s);
      P.C[sidx<N>(i, j)] = s;
    }
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = 0; j < N; ++j) {
      double s = 0.0;
#pragma unroll
      for (int l = 0; l < N; ++l) s = fma(e.A[i * N + l], R[l * Q + j], s);
      P.A[i * N + j] = s;
    }
}

}  // namespace lqt
