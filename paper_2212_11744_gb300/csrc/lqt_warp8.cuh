// One warp per combination for n <= 8 at the upper scan levels: the
// combination rule of Sec. IV-A (eq. lqt_comb, full and value form) with the
// linear solve of I + C1 J2 (App. B) as a register-resident Gauss-Jordan
// elimination across the warp's lanes.
//
// Why: an upper level with few pairs is latency-bound: its time is one
// combination's chain of dependent steps.  Spread over a warp with the
// operands in shared memory and a barrier per elimination step, that chain was
// ~30-55 us at n = 8 (about 27 such levels at T = 2^14).  Here lane c owns
// column c of [W | X1 | X2 | x] in registers (lanes 0..N-1: W, N..2N-1: X1,
// 2N..3N-1: X2, lane 3N: x), so one elimination step is a pivot search inside
// one lane, N shuffles for the pivot column and N independent FMAs per lane,
// with no shared-memory traffic and no barrier.
//
// Records are the full-matrix layout of the upper levels (A, b, C, eta, J,
// zeta; full_elem_doubles) and the value layout (S, v, zeta;
// full_val_doubles), staged in shared memory by plain coalesced loads.
#pragma once

#include <cuda_runtime.h>

#include "lqt_device.cuh"
#include "lqt_internal.h"

namespace lqt {
namespace w8 {

constexpr unsigned kFull = 0xffffffffu;

template <int N>
struct Lay {
  static constexpr int A = 0, B = N * N, C = N * N + N, ETA = 2 * N * N + N, J = 2 * N * N + 2 * N,
                       ZETA = 3 * N * N + 2 * N, REC = 3 * N * N + 2 * N + 1;
  static constexpr int VAL = N * N + N + 1;  // S, v, zeta
  static constexpr int LD = N + 1;           // row stride of the scratch matrices
  static constexpr int RLD = 3 * N + 1;      // row stride of the solved block [X1 | X2 | x]
  // scratch: W, T1, R (N x RLD), vectors
  static constexpr int W = 0, T1 = N * LD, R = 2 * N * LD, V = 2 * N * LD + N * RLD;
  static constexpr int SCRATCH = V + 6 * N;
};

// out(i, j) <- sum_l a(i, l) b(l, j) over the N x N outputs, lane o owning
// outputs o, o + 32, ...
template <int N, typename G, class FA, class FB, class FO>
__device__ __forceinline__ void gemm(int lane, FA a, FB b, FO out) {
  for (int o = lane; o < N * N; o += 32) {
    const int i = o / N, j = o % N;
    G s = (G)0;
#pragma unroll
    for (int l = 0; l < N; ++l) s = fma((G)a(i, l), (G)b(l, j), s);
    out(i, j, s);
  }
}

// y(i) = base(i) + sum_l m(i, l) x(l): lane (i = lane % N, q = lane / N) sums
// the terms l = q, q + Q, ... (Q = 32 / N groups), the groups added by
// shuffles; every lane returns y(lane % N).
template <int N, typename G, class FM, class FX>
__device__ __forceinline__ G matvec(int lane, FM m, FX x, G base) {
  constexpr int Q = 32 / N;
  const int i = lane % N, q = lane / N;
  G s = q == 0 ? base : (G)0;
#pragma unroll
  for (int l = q; l < N; l += Q) s = fma((G)m(i, l), (G)x(l), s);
#pragma unroll
  for (int o = N; o < 32; o <<= 1) s += __shfl_xor_sync(kFull, s, o);
  return s;
}

__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
  return x;
}

// Gauss-Jordan elimination with partial pivoting.  On entry lane c < N holds
// column c of W in col[], lanes N .. 3N the right-hand-side columns (others
// zero); rk[i] is the magnitude key of row i's scale max(1, max_j |W_ij|), in
// every lane.  On return the right-hand-side lanes hold W^-1 times their
// column.  A pivot no larger than 2^-40 of its row's scale sets the SINGULAR
// status bit (pivot_too_small).
template <int N>
__device__ __forceinline__ void gauss_jordan(int lane, double (&col)[N], unsigned long long (&rk)[N]) {
#pragma unroll
  for (int k = 0; k < N; ++k) {
    // pivot: the largest |W(i, k)|, i >= k, lowest i on ties (lane k's column)
    unsigned long long best = mag_key(col[k]);
    int p = k;
#pragma unroll
    for (int i = k + 1; i < N; ++i) {
      const unsigned long long key = mag_key(col[i]);
      if (key > best) {
        best = key;
        p = i;
      }
    }
    p = __shfl_sync(kFull, p, k);
    best = __shfl_sync(kFull, best, k);
    // exchange rows k and p: every lane's column and the row scales
    {
      double ck = col[k];
      unsigned long long rkk = rk[k];
#pragma unroll
      for (int i = k + 1; i < N; ++i) {
        const bool s = (p == i);
        const double ci = col[i];
        const unsigned long long ri = rk[i];
        col[i] = s ? col[k] : ci;
        rk[i] = s ? rk[k] : ri;
        ck = s ? ci : ck;
        rkk = s ? ri : rkk;
      }
      col[k] = ck;
      rk[k] = rkk;
    }
    if (lane == 0 && pivot_too_small(__longlong_as_double((long long)best), rk[k])) flag(kStatusSingular);
    const double d = __shfl_sync(kFull, col[k], k);
    const double inv = 1.0 / d;
    // new row k = row k / d; row i -= W(i, k) (new row k) for i != k
    const double pr = col[k] * inv;
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const double f = __shfl_sync(kFull, col[i], k);
      if (i != k) col[i] = fma(-f, pr, col[i]);
    }
    col[k] = pr;
  }
}

// Row scale keys of W (row stride LD) in every lane.
template <int N>
__device__ __forceinline__ void row_scales(const double* W, unsigned long long (&rk)[N]) {
#pragma unroll
  for (int i = 0; i < N; ++i) {
    unsigned long long r = mag_key(1.0);
#pragma unroll
    for (int j = 0; j < N; ++j) r = umax64(r, mag_key(W[i * Lay<N>::LD + j]));
    rk[i] = r;
  }
}

// out = e1 (x) e2 (full records in shared memory; out may alias neither).
// G: the type of the products (double, or float for the mixed path); the
// solve is FP64 in both.
template <int N, typename G>
__device__ void combine(int lane, const double* e1, const double* e2, double* out, double* scr) {
  using L = Lay<N>;
  double* W = scr + L::W;
  double* T1 = scr + L::T1;
  double* R = scr + L::R;
  double* z0 = scr + L::V;
  double* J2z = z0 + N;
  double* l0 = J2z + N;
  double* wv = l0 + N;
  const double* A1 = e1 + L::A;
  const double* C1 = e1 + L::C;
  const double* b1 = e1 + L::B;
  const double* A2 = e2 + L::A;
  const double* C2 = e2 + L::C;
  const double* J2 = e2 + L::J;
  const double* b2 = e2 + L::B;
  const double* eta2 = e2 + L::ETA;
  const int i = lane % N;
  // W = I + C1 J2 ; T1 = J2 A1 ; r = b1 + C1 eta2 ; wv = eta2 - J2 b1
  gemm<N, G>(lane, [&](int r, int l) { return C1[r * N + l]; }, [&](int l, int c) { return J2[l * N + c]; },
             [&](int r, int c, G v) { W[r * L::LD + c] = (double)v + (r == c ? 1.0 : 0.0); });
  gemm<N, G>(lane, [&](int r, int l) { return J2[r * N + l]; }, [&](int l, int c) { return A1[l * N + c]; },
             [&](int r, int c, G v) { T1[r * L::LD + c] = (double)v; });
  const double rv = (double)matvec<N, G>(lane, [&](int r, int l) { return C1[r * N + l]; },
                                         [&](int l) { return eta2[l]; }, (G)b1[i]);
  const double w = (double)matvec<N, G>(lane, [&](int r, int l) { return -J2[r * N + l]; },
                                        [&](int l) { return b1[l]; }, (G)eta2[i]);
  if (lane < N) wv[lane] = w;
  __syncwarp();
  // [K1 | MC1 | z0] = W^-1 [A1 | C1 | r] (FP64)
  {
    double col[N];
    unsigned long long rk[N];
    row_scales<N>(W, rk);
#pragma unroll
    for (int r = 0; r < N; ++r) {
      double v = 0.0;
      if (lane < N) v = W[r * L::LD + lane];
      else if (lane < 2 * N) v = A1[r * N + lane - N];
      else if (lane < 3 * N) v = C1[r * N + lane - 2 * N];
      col[r] = v;
    }
    // column 3N: r, lane i's value moved to lane 3N's register r
#pragma unroll
    for (int r = 0; r < N; ++r) {
      const double rr = __shfl_sync(kFull, rv, r);
      if (lane == 3 * N) col[r] = rr;
    }
    gauss_jordan<N>(lane, col, rk);
    if (lane >= N && lane <= 3 * N) {
#pragma unroll
      for (int r = 0; r < N; ++r) R[r * L::RLD + (lane - N)] = col[r];
    }
    if (lane == 3 * N) {
#pragma unroll
      for (int r = 0; r < N; ++r) z0[r] = col[r];
    }
  }
  __syncwarp();
  // J2 z0, l0 = J2 z0 - eta2 ; zeta ; eta = K1^T wv + eta1 ; b = A2 z0 + b2
  {
    const G jz = matvec<N, G>(lane, [&](int r, int l) { return J2[r * N + l]; }, [&](int l) { return z0[l]; },
                              (G)0);
    if (lane < N) {
      J2z[lane] = (double)jz;
      l0[lane] = (double)jz - eta2[lane];
    }
    const G et = matvec<N, G>(lane, [&](int r, int l) { return R[l * L::RLD + r]; }, [&](int l) { return wv[l]; },
                              (G)e1[L::ETA + i]);
    const G bo = matvec<N, G>(lane, [&](int r, int l) { return A2[r * N + l]; }, [&](int l) { return z0[l]; },
                              (G)b2[i]);
    __syncwarp();
    const G cl = matvec<N, G>(lane, [&](int r, int l) { return C1[r * N + l]; }, [&](int l) { return l0[l]; },
                              (G)0);
    const double zt = (lane < N) ? fma(0.5 * l0[lane], (double)cl, z0[lane] * fma(0.5, J2z[lane], -eta2[lane]))
                                 : 0.0;
    const double z = warp_sum(zt);
    if (lane < N) {
      out[L::ETA + lane] = (double)et;
      out[L::B + lane] = (double)bo;
    }
    if (lane == 0) out[L::ZETA] = e1[L::ZETA] + e2[L::ZETA] + z;
  }
  // W <- K1^T T1 ; A = A2 K1
  gemm<N, G>(lane, [&](int r, int l) { return R[l * L::RLD + r]; }, [&](int l, int c) { return T1[l * L::LD + c]; },
             [&](int r, int c, G v) { W[r * L::LD + c] = (double)v; });
  gemm<N, G>(lane, [&](int r, int l) { return A2[r * N + l]; }, [&](int l, int c) { return R[l * L::RLD + c]; },
             [&](int r, int c, G v) { out[L::A + r * N + c] = (double)v; });
  __syncwarp();
  // J = J1 + sym(K1^T T1) ; T1 <- A2 MC1
  for (int e = lane; e < N * N; e += 32) {
    const int r = e / N, c = e % N;
    out[L::J + e] = e1[L::J + e] + 0.5 * (W[r * L::LD + c] + W[c * L::LD + r]);
  }
  gemm<N, G>(lane, [&](int r, int l) { return A2[r * N + l]; }, [&](int l, int c) { return R[l * L::RLD + N + c]; },
             [&](int r, int c, G v) { T1[r * L::LD + c] = (double)v; });
  __syncwarp();
  // C = C2 + sym(T1 A2^T)
  gemm<N, G>(lane, [&](int r, int l) { return T1[r * L::LD + l]; }, [&](int l, int c) { return A2[c * N + l]; },
             [&](int r, int c, G v) { W[r * L::LD + c] = (double)v; });
  __syncwarp();
  for (int e = lane; e < N * N; e += 32) {
    const int r = e / N, c = e % N;
    out[L::C + e] = C2[e] + 0.5 * (W[r * L::LD + c] + W[c * L::LD + r]);
  }
  __syncwarp();
}

// out = e (x) V in value form (V = S, v, zeta; out may not alias V or e).
// W = I + C S2 and b + C v2 in FP64 whatever G is.
template <int N, typename G>
__device__ void combine_value(int lane, const double* e, const double* V, double* out, double* scr) {
  using L = Lay<N>;
  double* W = scr + L::W;
  double* T1 = scr + L::T1;
  double* R = scr + L::R;  // [Psi | alpha]
  double* alpha = scr + L::V;
  double* Sz = alpha + N;
  double* l0 = Sz + N;
  double* wv = l0 + N;
  const double* A = e + L::A;
  const double* C = e + L::C;
  const double* b = e + L::B;
  const double* S2 = V;
  const double* v2 = V + N * N;
  const int i = lane % N;
  gemm<N, double>(lane, [&](int r, int l) { return C[r * N + l]; }, [&](int l, int c) { return S2[l * N + c]; },
                  [&](int r, int c, double v) { W[r * L::LD + c] = v + (r == c ? 1.0 : 0.0); });
  gemm<N, G>(lane, [&](int r, int l) { return S2[r * N + l]; }, [&](int l, int c) { return A[l * N + c]; },
             [&](int r, int c, G v) { T1[r * L::LD + c] = (double)v; });
  const double rv = matvec<N, double>(lane, [&](int r, int l) { return C[r * N + l]; },
                                      [&](int l) { return v2[l]; }, b[i]);
  const double w = (double)matvec<N, G>(lane, [&](int r, int l) { return -S2[r * N + l]; },
                                        [&](int l) { return b[l]; }, (G)v2[i]);
  if (lane < N) wv[lane] = w;
  __syncwarp();
  {
    double col[N];
    unsigned long long rk[N];
    row_scales<N>(W, rk);
#pragma unroll
    for (int r = 0; r < N; ++r) {
      double v = 0.0;
      if (lane < N) v = W[r * L::LD + lane];
      else if (lane < 2 * N) v = A[r * N + lane - N];
      col[r] = v;
    }
#pragma unroll
    for (int r = 0; r < N; ++r) {
      const double rr = __shfl_sync(kFull, rv, r);
      if (lane == 2 * N) col[r] = rr;
    }
    gauss_jordan<N>(lane, col, rk);
    if (lane >= N && lane < 2 * N) {
#pragma unroll
      for (int r = 0; r < N; ++r) R[r * L::RLD + (lane - N)] = col[r];
    }
    if (lane == 2 * N) {
#pragma unroll
      for (int r = 0; r < N; ++r) alpha[r] = col[r];
    }
  }
  __syncwarp();
  {
    const G sz = matvec<N, G>(lane, [&](int r, int l) { return S2[r * N + l]; }, [&](int l) { return alpha[l]; },
                              (G)0);
    if (lane < N) {
      Sz[lane] = (double)sz;
      l0[lane] = (double)sz - v2[lane];
    }
    const G vo = matvec<N, G>(lane, [&](int r, int l) { return R[l * L::RLD + r]; }, [&](int l) { return wv[l]; },
                              (G)e[L::ETA + i]);
    gemm<N, G>(lane, [&](int r, int l) { return R[l * L::RLD + r]; },
               [&](int l, int c) { return T1[l * L::LD + c]; }, [&](int r, int c, G v) { W[r * L::LD + c] = (double)v; });
    __syncwarp();
    const G cl = matvec<N, G>(lane, [&](int r, int l) { return C[r * N + l]; }, [&](int l) { return l0[l]; },
                              (G)0);
    const double zt = (lane < N) ? fma(0.5 * l0[lane], (double)cl, alpha[lane] * fma(0.5, Sz[lane], -v2[lane]))
                                 : 0.0;
    const double z = warp_sum(zt);
    if (lane < N) out[N * N + lane] = (double)vo;
    if (lane == 0) out[N * N + N] = e[L::ZETA] + z + V[N * N + N];
  }
  for (int q = lane; q < N * N; q += 32) {
    const int r = q / N, c = q % N;
    out[q] = e[L::J + q] + 0.5 * (W[r * L::LD + c] + W[c * L::LD + r]);
  }
  __syncwarp();
}

}  // namespace w8
}  // namespace lqt
