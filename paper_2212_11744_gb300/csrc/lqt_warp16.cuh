// One warp per combination for n = 16: the combination rule of Sec. IV-A (eq.
// lqt_comb, full and value form) with the warp's 32 lanes used on every FP64
// instruction, and the linear solve of I + C1 J2 (App. B) as a register
// resident Gauss-Jordan elimination.
//
// Why: on this GPU a warp's FP64 instruction occupies its sub-partition for
// 64 cycles whatever the number of active lanes, and the solve is a chain of
// 16 dependent pivot steps.  Written as an LU in shared memory with a barrier
// after every step (and a second pass for the back substitution), the chain
// left the FP64 pipe idle most of the time.  Here each lane owns one column of
// [W | X1] in registers (lanes 0..15: W, lanes 16..31: X1) and one row slice
// of X2 and of the vector x, so one pass of 16 steps solves
// W [X1 | X2 | x] = [X1 | X2 | x]_in with 16-26 independent FMAs per lane per
// step, no shared-memory traffic and no barriers inside the elimination.
//
// The element operand of every combination is staged in shared memory by the
// TMA unit (cp.async.bulk, completion on an mbarrier with a bounded wait),
// from the public element arrays when they are 16-byte aligned; otherwise by
// coalesced plain loads.
#pragma once

#include <cuda_runtime.h>

#include "lqt_device.cuh"
#include "lqt_internal.h"

namespace lqt {
namespace w16 {

constexpr int N = 16;
constexpr unsigned kFull = 0xffffffffu;
// element record in shared memory: A (256), b (16), C (256), eta (16), J
// (256), zeta (1): the packed record order; every matrix and vector starts on
// a 16-byte boundary
constexpr int kOffA = 0, kOffB = 256, kOffC = 272, kOffEta = 528, kOffJ = 544, kOffZeta = 800;
constexpr int kRec = 801;
constexpr int kRecPad = 802;  // keeps the next buffer 16-byte aligned
constexpr int kWld = 17;      // row stride of W (odd: row and column accesses are both conflict-free)
constexpr int kRld = 33;      // row stride of the solved block [K1 | MC1 | z0]
// bounded waits: iterations of mbarrier try_wait before the wait gives up
constexpr unsigned kWaitLimit = 1u << 24;

// ---------------------------------------------------------------------------
// TMA bulk copies into shared memory, completion on an mbarrier
// ---------------------------------------------------------------------------

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// global -> shared bulk copy of `bytes` (a multiple of 16; both addresses
// 16-byte aligned), counted on `bar`
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// orders this thread's earlier generic-proxy shared-memory accesses before
// later async-proxy (TMA) accesses
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Waits for phase `parity` of `bar`, at most kWaitLimit polls.  On time-out
// the status word gets kStatusTimeout, and the wait is retried once more
// (bounded again) so that no copy is left landing in shared memory after the
// caller moves on.
__device__ __forceinline__ void mbar_wait_bounded(unsigned long long* bar, unsigned parity) {
  unsigned it = 0;
  while (!mbar_try_wait(bar, parity)) {
    if (++it >= kWaitLimit) {
      flag(kStatusTimeout);
      for (unsigned j = 0; j < kWaitLimit && !mbar_try_wait(bar, parity); ++j) {
      }
      return;
    }
  }
}

// Where element k of a scan level lives: the public arrays (level 0) or a
// packed record (levels above).
struct ElemSrc {
  ElemPtrs el;         // public layout (level 0)
  const double* rec;   // packed records (levels >= 1), or null
  bool bulk;           // public arrays 16-byte aligned: stage by TMA
};

// Stages element k into the shared record `dst` (kRec doubles).  The whole warp
// calls it; on return (after a __syncwarp) the record is complete.  `bar` is
// this warp's mbarrier and `phase` its parity, flipped per use.
__device__ __forceinline__ void stage(int lane, const ElemSrc& s, int64_t k, double* dst, unsigned long long* bar,
                                      unsigned& phase, const double* zero_zeta) {
  if (s.rec == nullptr && s.bulk) {
    fence_proxy_async();  // this lane's earlier reads of dst before the copy's writes
    __syncwarp();
    if (lane == 0) {
      mbar_expect_tx(bar, (3 * 256 + 2 * 16) * 8);
      bulk_g2s(dst + kOffA, s.el.A + k * 256, 256 * 8, bar);
      bulk_g2s(dst + kOffB, s.el.b + k * 16, 16 * 8, bar);
      bulk_g2s(dst + kOffC, s.el.C + k * 256, 256 * 8, bar);
      bulk_g2s(dst + kOffEta, s.el.eta + k * 16, 16 * 8, bar);
      bulk_g2s(dst + kOffJ, s.el.J + k * 256, 256 * 8, bar);
      dst[kOffZeta] = s.el.zeta ? s.el.zeta[k] : *zero_zeta;
    }
    mbar_wait_bounded(bar, phase);
    phase ^= 1u;
  } else if (s.rec == nullptr) {
    for (int e = lane; e < 256; e += 32) {
      dst[kOffA + e] = s.el.A[k * 256 + e];
      dst[kOffC + e] = s.el.C[k * 256 + e];
      dst[kOffJ + e] = s.el.J[k * 256 + e];
    }
    if (lane < 16) {
      dst[kOffB + lane] = s.el.b[k * 16 + lane];
      dst[kOffEta + lane] = s.el.eta[k * 16 + lane];
    }
    if (lane == 0) dst[kOffZeta] = s.el.zeta ? s.el.zeta[k] : *zero_zeta;
  } else {
    const double* r = s.rec + k * kRec;
    for (int e = lane; e < kRec; e += 32) dst[e] = r[e];
  }
  __syncwarp();
}

// ---------------------------------------------------------------------------
// products and vectors
// ---------------------------------------------------------------------------

// out(i, j) <- sum_l a(i, l) b(l, j), 16 x 16 x 16: lane (j = lane & 15,
// h = lane >> 4) owns rows 8h..8h+7 of column j (8 independent accumulators);
// a(i, l) is read by the 16 lanes of a half at one address, b(l, j) by
// consecutive lanes at consecutive addresses.
template <typename G, class FA, class FB, class FO>
__device__ __forceinline__ void gemm(int lane, FA a, FB b, FO out) {
  const int j = lane & 15, i0 = (lane >> 4) * 8;
  G acc[8];
#pragma unroll
  for (int r = 0; r < 8; ++r) acc[r] = (G)0;
#pragma unroll 4
  for (int l = 0; l < 16; ++l) {
    const G bv = (G)b(l, j);
#pragma unroll
    for (int r = 0; r < 8; ++r) acc[r] = fma((G)a(i0 + r, l), bv, acc[r]);
  }
#pragma unroll
  for (int r = 0; r < 8; ++r) out(i0 + r, j, acc[r]);
}

// y(i) = base(i) + sum_l m(i, l) x(l): lane (i = lane & 15, h) sums l in
// 8h..8h+7, the halves are added with one shuffle; every lane returns y(its i).
template <typename G, class FM, class FX>
__device__ __forceinline__ G matvec(int lane, FM m, FX x, G base) {
  const int i = lane & 15, l0 = (lane >> 4) * 8;
  G s = (lane >> 4) ? (G)0 : base;
#pragma unroll
  for (int l = 0; l < 8; ++l) s = fma((G)m(i, l0 + l), (G)x(l0 + l), s);
  return s + __shfl_xor_sync(kFull, s, 16);
}

__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
  return x;
}

// ---------------------------------------------------------------------------
// Gauss-Jordan elimination with partial pivoting on [W | X1 | X2 | x]
// ---------------------------------------------------------------------------

// On entry lane c < 16 holds column c of W in col[], lane 16 + c column c of
// X1; lane l holds x(l & 15) in xv and, when HAS_X2, row (l & 15) of X2,
// columns 8 (l >> 4) .. +7, in row[]; rk is the magnitude key of row (l & 15)'s
// scale max(1, max_j |W_lj|).  On return X1, X2, x are replaced by
// W^-1 X1, W^-1 X2, W^-1 x in the same places.  A pivot no larger than 2^-40
// of its row's scale sets the SINGULAR status bit (pivot_too_small).
template <bool HAS_X2>
__device__ __forceinline__ void gauss_jordan(int lane, double (&col)[16], double (&row)[8], double& xv,
                                             unsigned long long rk) {
  const int myrow = lane & 15, half = lane >> 4;
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    // pivot: the largest |W(i, k)|, i >= k, lowest i on ties (lane k's column)
    unsigned long long best = mag_key(col[k]);
    int p = k;
#pragma unroll
    for (int i = k + 1; i < 16; ++i) {
      const unsigned long long key = mag_key(col[i]);
      if (key > best) {
        best = key;
        p = i;
      }
    }
    p = __shfl_sync(kFull, p, k);
    best = __shfl_sync(kFull, best, k);
    const unsigned long long rk_k = __shfl_sync(kFull, rk, k), rk_p = __shfl_sync(kFull, rk, p);
    if (myrow == k) rk = rk_p;
    else if (myrow == p) rk = rk_k;
    if (lane == 0 && pivot_too_small(__longlong_as_double((long long)best), rk_p)) flag(kStatusSingular);
    // exchange rows k and p: the column registers by predicated selects, the
    // row-distributed values between the lanes that hold rows k and p
    {
      double nk = col[k];
#pragma unroll
      for (int i = k + 1; i < 16; ++i) {
        const bool s = (p == i);
        const double ci = col[i];
        col[i] = s ? col[k] : ci;
        nk = s ? ci : nk;
      }
      col[k] = nk;
      const int src = myrow == k ? p + 16 * half : (myrow == p ? k + 16 * half : lane);
      if constexpr (HAS_X2) {
#pragma unroll
        for (int j = 0; j < 8; ++j) row[j] = __shfl_sync(kFull, row[j], src);
      }
      xv = __shfl_sync(kFull, xv, src);
    }
    const double d = __shfl_sync(kFull, col[k], k);
    const double inv = 1.0 / d;
    double rkrow[8];
    if constexpr (HAS_X2) {
#pragma unroll
      for (int j = 0; j < 8; ++j) rkrow[j] = __shfl_sync(kFull, row[j], k + 16 * half);
    }
    const double xk = __shfl_sync(kFull, xv, k);
    // new row k = row k / d; row i -= W(i, k) (new row k) for i != k
    const double pr = col[k] * inv;
    double myf = 0.0;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const double f = __shfl_sync(kFull, col[i], k);
      myf = (i == myrow) ? f : myf;
      if (i != k) col[i] = fma(-f, pr, col[i]);
    }
    col[k] = pr;
    // the row-distributed values: one fma each, a = inv - 1 on row k itself
    const double a = (myrow == k) ? inv - 1.0 : -myf * inv;
    if constexpr (HAS_X2) {
#pragma unroll
      for (int j = 0; j < 8; ++j) row[j] = fma(a, rkrow[j], row[j]);
    }
    xv = fma(a, xk, xv);
  }
}

// Row scale key of row (lane & 15) of W (row stride kWld): max(1, max_j |W_ij|).
__device__ __forceinline__ unsigned long long row_scale(int lane, const double* W) {
  const int i = lane & 15, j0 = (lane >> 4) * 8;
  unsigned long long rk = mag_key(1.0);
#pragma unroll
  for (int j = 0; j < 8; ++j) rk = umax64(rk, mag_key(W[i * kWld + j0 + j]));
  return umax64(rk, __shfl_xor_sync(kFull, rk, 16));
}

// ---------------------------------------------------------------------------
// the combinations
// ---------------------------------------------------------------------------

// Scratch of combine(): W (16 x 17), R (16 x 33), T1 (16 x 17), vectors.
constexpr int kScrW = 0, kScrR = 16 * kWld, kScrT = kScrR + 16 * kRld, kScrV = kScrT + 16 * kWld;
constexpr int kScratch = kScrV + 6 * 16;

// e1 <- e1 (x) e2 in place (both full records in shared memory, kRec layout).
// G: the type the products are formed in (double, or float for the mixed
// path); the solve is FP64 in both.
template <typename G>
__device__ void combine(int lane, double* e1, const double* e2, double* scr) {
  double* W = scr + kScrW;
  double* R = scr + kScrR;
  double* T1 = scr + kScrT;
  double* z0 = scr + kScrV;
  double* J2z = z0 + 16;
  double* l0 = J2z + 16;
  double* wv = l0 + 16;
  const double* A1 = e1 + kOffA;
  const double* C1 = e1 + kOffC;
  const double* b1 = e1 + kOffB;
  const double* A2 = e2 + kOffA;
  const double* C2 = e2 + kOffC;
  const double* J2 = e2 + kOffJ;
  const double* b2 = e2 + kOffB;
  const double* eta2 = e2 + kOffEta;
  const int i = lane & 15, h = lane >> 4;
  // W = I + C1 J2 ; T1 = J2 A1 ; r = b1 + C1 eta2 ; wv = eta2 - J2 b1 (C1, J2
  // symmetric: their rows are read as columns)
  gemm<G>(lane, [&](int r, int l) { return C1[r * 16 + l]; }, [&](int l, int c) { return J2[l * 16 + c]; },
          [&](int r, int c, G v) { W[r * kWld + c] = (double)v + (r == c ? 1.0 : 0.0); });
  gemm<G>(lane, [&](int r, int l) { return J2[r * 16 + l]; }, [&](int l, int c) { return A1[l * 16 + c]; },
          [&](int r, int c, G v) { T1[r * kWld + c] = (double)v; });
  const double rv = (double)matvec<G>(lane, [&](int r, int l) { return C1[l * 16 + r]; },
                                      [&](int l) { return eta2[l]; }, (G)b1[i]);
  const double w = (double)matvec<G>(lane, [&](int r, int l) { return -J2[l * 16 + r]; },
                                     [&](int l) { return b1[l]; }, (G)eta2[i]);
  if (h == 0) wv[i] = w;
  __syncwarp();
  // [K1 | MC1 | z0] = W^-1 [A1 | C1 | r] (FP64)
  {
    double col[16], row[8];
    const double* src = lane < 16 ? W + lane : A1 + (lane - 16);
    const int ld = lane < 16 ? kWld : 16;
#pragma unroll
    for (int r = 0; r < 16; ++r) col[r] = src[r * ld];
#pragma unroll
    for (int j = 0; j < 8; ++j) row[j] = C1[(8 * h + j) * 16 + i];
    double xv = rv;
    const unsigned long long rk = row_scale(lane, W);
    gauss_jordan<true>(lane, col, row, xv, rk);
    if (lane >= 16) {
#pragma unroll
      for (int r = 0; r < 16; ++r) R[r * kRld + (lane - 16)] = col[r];
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) R[i * kRld + 16 + 8 * h + j] = row[j];
    if (h == 0) {
      R[i * kRld + 32] = xv;
      z0[i] = xv;
    }
  }
  __syncwarp();
  // J2 z0, l0 = J2 z0 - eta2 ; zeta ; eta = K1^T wv + eta1 ; b = A2 z0 + b2
  {
    const G jz = matvec<G>(lane, [&](int r, int l) { return J2[l * 16 + r]; }, [&](int l) { return z0[l]; }, (G)0);
    if (h == 0) {
      J2z[i] = (double)jz;
      l0[i] = (double)jz - eta2[i];
    }
    const G et = matvec<G>(lane, [&](int r, int l) { return R[l * kRld + r]; }, [&](int l) { return wv[l]; },
                           (G)e1[kOffEta + i]);
    const G bo = matvec<G>(lane, [&](int r, int l) { return A2[r * 16 + l]; }, [&](int l) { return z0[l]; },
                           (G)b2[i]);
    __syncwarp();
    const G cl = matvec<G>(lane, [&](int r, int l) { return C1[l * 16 + r]; }, [&](int l) { return l0[l]; }, (G)0);
    double zt = (h == 0) ? fma(0.5 * l0[i], (double)cl, z0[i] * fma(0.5, J2z[i], -eta2[i])) : 0.0;
    const double z = warp_sum(zt);
    __syncwarp();
    if (h == 0) {
      e1[kOffEta + i] = (double)et;
      e1[kOffB + i] = (double)bo;
    }
    if (lane == 0) e1[kOffZeta] = e1[kOffZeta] + e2[kOffZeta] + z;
  }
  // W <- K1^T T1 ; A1 <- A2 K1 (A1 was consumed by the solve and T1)
  gemm<G>(lane, [&](int r, int l) { return R[l * kRld + r]; }, [&](int l, int c) { return T1[l * kWld + c]; },
          [&](int r, int c, G v) { W[r * kWld + c] = (double)v; });
  gemm<G>(lane, [&](int r, int l) { return A2[r * 16 + l]; }, [&](int l, int c) { return R[l * kRld + c]; },
          [&](int r, int c, G v) { e1[kOffA + r * 16 + c] = (double)v; });
  __syncwarp();
  // J = J1 + sym(K1^T T1) ; T1 <- (A2 MC1)^T
  for (int e = lane; e < 256; e += 32) {
    const int r = e >> 4, c = e & 15;
    e1[kOffJ + e] += 0.5 * (W[r * kWld + c] + W[c * kWld + r]);
  }
  gemm<G>(lane, [&](int r, int l) { return A2[r * 16 + l]; }, [&](int l, int c) { return R[l * kRld + 16 + c]; },
          [&](int r, int c, G v) { T1[c * kWld + r] = (double)v; });
  __syncwarp();
  // C = C2 + sym(A2 (A2 MC1)^T)
  gemm<G>(lane, [&](int r, int l) { return A2[r * 16 + l]; }, [&](int l, int c) { return T1[l * kWld + c]; },
          [&](int r, int c, G v) { W[r * kWld + c] = (double)v; });
  __syncwarp();
  for (int e = lane; e < 256; e += 32) {
    const int r = e >> 4, c = e & 15;
    e1[kOffC + e] = C2[e] + 0.5 * (W[r * kWld + c] + W[c * kWld + r]);
  }
  __syncwarp();
}

// Value record: S (256), v (16), zeta.
constexpr int kVal = 273;
// Scratch of combine_value(): W (16 x 17), T1 (16 x 17), vectors.
constexpr int kVScrW = 0, kVScrT = 16 * kWld, kVScrV = kVScrT + 16 * kWld;
constexpr int kVScratch = kVScrV + 4 * 16;

// out = e (x) V (value form, out may not alias V), and the one-sub-interval
// map Psi (16 x 16 row-major), alpha (16).  e: full record in shared memory.
// W = I + C S2 and b + C v2 are formed in FP64 whatever G is: they define the
// map the state scan composes T times.
template <typename G>
__device__ void combine_value(int lane, const double* e, const double* V, double* out, double* Psi, double* alpha,
                              double* scr, double* zeta_inc = nullptr) {
  double* W = scr + kVScrW;
  double* T1 = scr + kVScrT;
  double* wv = scr + kVScrV;
  double* Sz = wv + 16;
  double* l0 = Sz + 16;
  const double* A = e + kOffA;
  const double* C = e + kOffC;
  const double* b = e + kOffB;
  const double* S2 = V;
  const double* v2 = V + 256;
  const int i = lane & 15, h = lane >> 4;
  gemm<double>(lane, [&](int r, int l) { return C[r * 16 + l]; }, [&](int l, int c) { return S2[l * 16 + c]; },
               [&](int r, int c, double v) { W[r * kWld + c] = v + (r == c ? 1.0 : 0.0); });
  gemm<G>(lane, [&](int r, int l) { return S2[r * 16 + l]; }, [&](int l, int c) { return A[l * 16 + c]; },
          [&](int r, int c, G v) { T1[r * kWld + c] = (double)v; });
  const double rv = matvec<double>(lane, [&](int r, int l) { return C[l * 16 + r]; }, [&](int l) { return v2[l]; },
                                   b[i]);
  const double w = (double)matvec<G>(lane, [&](int r, int l) { return -S2[l * 16 + r]; },
                                     [&](int l) { return b[l]; }, (G)v2[i]);
  if (h == 0) wv[i] = w;
  __syncwarp();
  {
    double col[16], row[8];
    const double* src = lane < 16 ? W + lane : A + (lane - 16);
    const int ld = lane < 16 ? kWld : 16;
#pragma unroll
    for (int r = 0; r < 16; ++r) col[r] = src[r * ld];
    double xv = rv;
    const unsigned long long rk = row_scale(lane, W);
    gauss_jordan<false>(lane, col, row, xv, rk);
    if (lane >= 16) {
#pragma unroll
      for (int r = 0; r < 16; ++r) Psi[r * 16 + (lane - 16)] = col[r];
    }
    if (h == 0) alpha[i] = xv;
  }
  __syncwarp();
  // Sz = S2 alpha, l0 = Sz - v2 ; v = eta + Psi^T wv ; W <- Psi^T T1 ; zeta
  {
    const G sz = matvec<G>(lane, [&](int r, int l) { return S2[l * 16 + r]; }, [&](int l) { return alpha[l]; },
                           (G)0);
    if (h == 0) {
      Sz[i] = (double)sz;
      l0[i] = (double)sz - v2[i];
    }
    const G vo = matvec<G>(lane, [&](int r, int l) { return Psi[l * 16 + r]; }, [&](int l) { return wv[l]; },
                           (G)e[kOffEta + i]);
    gemm<G>(lane, [&](int r, int l) { return Psi[l * 16 + r]; }, [&](int l, int c) { return T1[l * kWld + c]; },
            [&](int r, int c, G v) { W[r * kWld + c] = (double)v; });
    __syncwarp();
    const G cl = matvec<G>(lane, [&](int r, int l) { return C[l * 16 + r]; }, [&](int l) { return l0[l]; }, (G)0);
    const double zt = (h == 0) ? fma(0.5 * l0[i], (double)cl, alpha[i] * fma(0.5, Sz[i], -v2[i])) : 0.0;
    const double z = warp_sum(zt);
    if (h == 0) out[256 + i] = (double)vo;
    if (lane == 0) {
      const double inc = e[kOffZeta] + z;  // the element's own share; the carry's zeta added after
      out[272] = inc + V[272];
      if (zeta_inc) *zeta_inc = inc;
    }
  }
  for (int q = lane; q < 256; q += 32) {
    const int r = q >> 4, c = q & 15;
    out[q] = e[kOffJ + q] + 0.5 * (W[r * kWld + c] + W[c * kWld + r]);
  }
  __syncwarp();
}

// (P, p) <- (P Psi, P alpha + p); Tm: 16 x 17 scratch.
__device__ __forceinline__ void compose_right(int lane, double* P, double* p, const double* Psi, const double* alpha,
                                              double* Tm) {
  gemm<double>(lane, [&](int r, int l) { return P[r * 16 + l]; }, [&](int l, int c) { return Psi[l * 16 + c]; },
               [&](int r, int c, double v) { Tm[r * kWld + c] = v; });
  const double pa = matvec<double>(lane, [&](int r, int l) { return P[r * 16 + l]; },
                                   [&](int l) { return alpha[l]; }, p[lane & 15]);
  __syncwarp();
  for (int q = lane; q < 256; q += 32) P[q] = Tm[(q >> 4) * kWld + (q & 15)];
  if (lane < 16) p[lane] = pa;
  __syncwarp();
}

}  // namespace w16
}  // namespace lqt
