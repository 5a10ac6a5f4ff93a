// Cooperative ("team") versions of the element build and the combination rule
// for larger state dimensions (n = 16, 64), where one thread cannot hold an
// element.  A team of TEAM threads (one warp for n = 16, one CTA of 256
// threads for n = 64) owns one element; matrices are full n x n row-major in
// buffers the caller places in shared or global memory; the team spreads the
// entries of every product over its lanes.  On this GPU the FP64 pipe is the
// limit (one FP64 warp instruction per 64 cycles per sub-partition), so
// operands are read straight from the buffers without register blocking.
//
// Math: Sec. IV-B Theorem Backward_HJB_LQT (right-hand side, with the factor
// B = Lt Lt^T), Sec. IV-A eq. lqt_comb (full and value-form combination),
// Sec. IV-E (one-sub-interval optimal-state map).
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

#include "lqt_device.cuh"
#include "lqt_internal.h"
#include "lqt_tc64.cuh"

namespace lqt {
namespace team {

template <int TEAM>
__device__ __forceinline__ void sync() {
  if constexpr (TEAM <= 32)
    __syncwarp();
  else
    __syncthreads();
}

// (i, j) of the t-th entry of the upper triangle (row by row).
__device__ __forceinline__ void upper_ij(int N, int t, int& i, int& j) {
  int r = 0;
  while (t >= N - r) {
    t -= N - r;
    ++r;
  }
  i = r;
  j = r + t;
}

// Register-blocked product over a team: out(i, j, s) receives
// s = sum_{l < INNER} a(i, l) b(l, j) for i < ROWS, j < COLS.  Each thread owns
// an RB x CB set of outputs, RB consecutive rows by CB columns a block-count
// apart (RB * CB accumulators, RB + CB operand loads per
// step of l), with the block shape chosen so that the blocks just cover the
// team; the mapping depends only on (ROWS, COLS, TEAM), so two products of one
// shape give every thread the same outputs (a thread may then accumulate
// into its outputs without a barrier).  G is the product type.
//
// Shapes: a warp-sized team (n = 16, buffers in shared memory) gives each lane
// one column and RB consecutive rows, so that consecutive lanes read
// consecutive words of b and share rows of a (an operand read from several
// rows of one column would hit one shared-memory bank: the row stride is a
// multiple of 32 words); a larger team (n = 64) takes 4 x 4 sets, which need
// the fewest loads per FMA.
template <int ROWS, int COLS, int TEAM>
struct GemmShape {
  static constexpr int cb() {
    if (TEAM <= 32) return 1;
    int c = 1;
    while (c < 4 && COLS % (2 * c) == 0 && ROWS * COLS / (2 * c) >= TEAM) c *= 2;
    return c;
  }
  static constexpr int CB = cb();
  static constexpr int rb() {
    int r = 1;
    const int lim = TEAM <= 32 ? 8 : 4;
    while (r < lim && ROWS % (2 * r) == 0 && ROWS * COLS / (CB * 2 * r) >= TEAM) r *= 2;
    return r;
  }
  static constexpr int RB = rb();
};

template <int ROWS, int COLS, int INNER, int TEAM, typename G, class FA, class FB, class FO>
__device__ __forceinline__ void gemm(int lane, FA a, FB b, FO out) {
  constexpr int RB = GemmShape<ROWS, COLS, TEAM>::RB, CB = GemmShape<ROWS, COLS, TEAM>::CB;
  constexpr int NBC = COLS / CB, NB = (ROWS / RB) * NBC;
  // a thread's CB columns are jb, jb + NBC, ...: consecutive threads then read
  // consecutive words of a row of b (one shared-memory wavefront for 16
  // doubles) rather than words 32 bytes apart
  for (int blk = lane; blk < NB; blk += TEAM) {
    const int i0 = (blk / NBC) * RB, jb = blk % NBC;
    G acc[RB][CB];
#pragma unroll
    for (int r = 0; r < RB; ++r)
#pragma unroll
      for (int c = 0; c < CB; ++c) acc[r][c] = (G)0;
#pragma unroll 4
    for (int l = 0; l < INNER; ++l) {
      G av[RB], bv[CB];
#pragma unroll
      for (int r = 0; r < RB; ++r) av[r] = (G)a(i0 + r, l);
#pragma unroll
      for (int c = 0; c < CB; ++c) bv[c] = (G)b(l, jb + c * NBC);
#pragma unroll
      for (int r = 0; r < RB; ++r)
#pragma unroll
        for (int c = 0; c < CB; ++c) acc[r][c] = fma(av[r], bv[c], acc[r][c]);
    }
#pragma unroll
    for (int r = 0; r < RB; ++r)
#pragma unroll
      for (int c = 0; c < CB; ++c) out(i0 + r, jb + c * NBC, acc[r][c]);
  }
}

// A product of the combination rule in the type G: on the tensor core
// (lqt_tc64.cuh) for the FP32 products of n = 64 when the kernel set up a
// tensor-core context, else the team product above.
template <int N, int TEAM, typename G, class FA, class FB, class FO>
__device__ __forceinline__ void pgemm(int lane, tc::Ctx* tcx, FA a, FB b, FO out) {
  if constexpr (N == 64 && TEAM == tc::kTeam && std::is_same<G, float>::value) {
    if (tcx) {
      tc::gemm64(*tcx, a, b, out);
      return;
    }
  }
  gemm<N, N, N, TEAM, G>(lane, a, b, out);
}

// An element as six field pointers (full n x n matrices), so that a record can
// live in a packed buffer (A, b, C, eta, J, zeta back to back) or in the public
// SoA arrays.
template <int N>
struct Rec {
  static constexpr int SIZE = 3 * N * N + 2 * N + 1;
  double *a_, *b_, *c_, *e_, *j_, *z_;
  __device__ __forceinline__ double* A() const { return a_; }
  __device__ __forceinline__ double* b() const { return b_; }
  __device__ __forceinline__ double* C() const { return c_; }
  __device__ __forceinline__ double* eta() const { return e_; }
  __device__ __forceinline__ double* J() const { return j_; }
  __device__ __forceinline__ double* zeta() const { return z_; }
  // packed record at p
  __device__ __forceinline__ static Rec packed(double* p) {
    return Rec{p, p + N * N, p + N * N + N, p + 2 * N * N + N, p + 2 * N * N + 2 * N, p + 3 * N * N + 2 * N};
  }
  // the fields that drive the element flow (A, eta, J) alone, FLOW doubles at
  // p: the RK4 stage buffers of the build (b, C, zeta are quadratures)
  static constexpr int FLOW = 2 * N * N + N;
  __device__ __forceinline__ static Rec flow(double* p) {
    return Rec{p, nullptr, nullptr, p + N * N, p + N * N + N, nullptr};
  }
  // element k of the public arrays
  __device__ __forceinline__ static Rec pub(const ElemPtrs& el, int64_t k, double* zeta_fallback) {
    return Rec{el.A + k * N * N, el.b + k * N, el.C + k * N * N, el.eta + k * N, el.J + k * N * N,
               el.zeta ? el.zeta + k : zeta_fallback};
  }
};
// ---------------------------------------------------------------------------
// element build right-hand side (factor form, see build_kernel)
// ---------------------------------------------------------------------------

// Sum of x over the S consecutive lanes of an aligned group (S a power of two
// <= 32); every lane of the warp calls it.
template <int S>
__device__ __forceinline__ double group_sum(double x) {
#pragma unroll
  for (int o = S / 2; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// Lanes per output when `outputs` sums are spread over a team: the largest
// power of two <= team / outputs, at most a warp.
__host__ __device__ constexpr int split_lanes(int outputs, int team) {
  int s = 1;
  while (2 * s * outputs <= team && 2 * s <= 32) s *= 2;
  return s;
}

// k = f(y) for the flow fields (A, eta, J); the quadrature fields' rates
// (db, dC, dzeta: nothing reads b, C or zeta) are added, times the RK4 weight
// sq, straight into qacc's b, C, zeta, in the order the four-stage sum takes
// them.  y and k may be flow records.  Scratch: AL, P (N x M), w (M).
// Outputs that fill the team (AL, P, dA and whole passes of the C, J upper
// triangles) take one thread each; outputs fewer than the team (w, db, deta,
// the last partial pass of C and J, dzeta) have each sum spread over a group
// of lanes, strided terms, and the group's partial sums added by shuffles,
// so that every lane issues FP64 work: on this GPU a warp's FP64 instruction
// costs its sub-partition the same 64 cycles whatever the active lanes.  The
// symmetric C, J are formed on their upper triangles.
//
// A CTA (n = 64, buffers in global memory): one output per thread at a time
// needs two operand loads per FMA, and the loads, not the FP64 pipe, then set
// the pace (the LSU queue full, 71% FP64 busy).  So there AL, P and dA are
// register-blocked team products (gemm: 4 x 4 blocks, half a load per FMA),
// and dJ's J F + (J F)^T is one blocked product J F into shared memory, read
// twice.
template <int N, int M, int TEAM>
__device__ void rhs(int lane, Rec<N> y, Rec<N> k, const double* __restrict__ F, const double* __restrict__ c,
                    const double* __restrict__ Lt, const double* __restrict__ Q, const double* __restrict__ qr,
                    double* AL, double* P, double* w, double sq, Rec<N> qacc) {
  const double* A = y.A();
  const double* J = y.J();
  const double* eta = y.eta();
  double* JF = nullptr;
  if constexpr (TEAM > 32) {
    __shared__ double jf_smem[N * N];
    JF = jf_smem;
    gemm<N, M, N, TEAM, double>(
        lane, [&](int i, int l) { return A[i * N + l]; }, [&](int l, int a) { return Lt[l * M + a]; },
        [&](int i, int a, double s) { AL[i * M + a] = s; });
    gemm<N, M, N, TEAM, double>(
        lane, [&](int i, int l) { return J[i * N + l]; }, [&](int l, int a) { return Lt[l * M + a]; },
        [&](int i, int a, double s) { P[i * M + a] = s; });
    gemm<N, N, N, TEAM, double>(
        lane, [&](int i, int l) { return J[i * N + l]; }, [&](int l, int j) { return F[l * N + j]; },
        [&](int i, int j, double s) { JF[i * N + j] = s; });
  } else {
  for (int e = lane; e < N * M; e += TEAM) {
    const int i = e / M, a = e % M;
    double s1 = 0.0, s2 = 0.0;
    for (int l = 0; l < N; ++l) {
      s1 = fma(A[i * N + l], Lt[l * M + a], s1);
      s2 = fma(J[i * N + l], Lt[l * M + a], s2);
    }
    AL[e] = s1;
    P[e] = s2;
  }
  }
  {  // w = Lt^T eta
    constexpr int S = split_lanes(M, TEAM);
    const int o = lane / S, sub = lane % S;
    double s = 0.0;
    if (o < M)
      for (int l = sub; l < N; l += S) s = fma(Lt[l * M + o], eta[l], s);
    s = group_sum<S>(s);
    if (sub == 0 && o < M) w[o] = s;
  }
  sync<TEAM>();
  constexpr int NS = N * (N + 1) / 2;
  // dA = AL P^T - A F
  if constexpr (TEAM > 32) {
    double* kA = k.A();
    gemm<N, N, M, TEAM, double>(
        lane, [&](int i, int a) { return AL[i * M + a]; }, [&](int a, int j) { return P[j * M + a]; },
        [&](int i, int j, double s) { kA[i * N + j] = s; });
    gemm<N, N, N, TEAM, double>(
        lane, [&](int i, int l) { return A[i * N + l]; }, [&](int l, int j) { return F[l * N + j]; },
        [&](int i, int j, double s) { kA[i * N + j] -= s; });
  } else {
    for (int t = lane; t < N * N; t += TEAM) {
      const int i = t / N, j = t % N;
      double s = 0.0;
      for (int a = 0; a < M; ++a) s = fma(AL[i * M + a], P[j * M + a], s);
      for (int l = 0; l < N; ++l) s = fma(-A[i * N + l], F[l * N + j], s);
      k.A()[t] = s;
    }
  }
  {  // db = -AL w - A c ; deta = -q - F^T eta + J c + P w
    constexpr int S = split_lanes(N, TEAM);
    const int o = lane / S, sub = lane % S;
    double s = 0.0, se = 0.0;
    if (o < N) {
      if (sub == 0) se = -qr[o];
      for (int a = sub; a < M; a += S) {
        s = fma(-AL[o * M + a], w[a], s);
        se = fma(P[o * M + a], w[a], se);
      }
      for (int l = sub; l < N; l += S) se = fma(-F[l * N + o], eta[l], se);
      if (c)
        for (int l = sub; l < N; l += S) {
          s = fma(-A[o * N + l], c[l], s);
          se = fma(J[o * N + l], c[l], se);
        }
    }
    s = group_sum<S>(s);
    se = group_sum<S>(se);
    if (sub == 0 && o < N) {
      qacc.b()[o] = fma(sq, s, qacc.b()[o]);
      k.eta()[o] = se;
    }
  }
  // dC = -AL AL^T ; dJ = -Q - JF - (JF)^T + P P^T  (upper triangles, mirrored):
  // whole passes one entry per thread, the remainder spread over lane groups
  if constexpr (TEAM > 32) {
    for (int t = lane; t < NS; t += TEAM) {
      int i, j;
      upper_ij(N, t, i, j);
      double sc = 0.0, sj = -Q[i * N + j] - JF[i * N + j] - JF[j * N + i];
      for (int a = 0; a < M; ++a) {
        sc = fma(-AL[i * M + a], AL[j * M + a], sc);
        sj = fma(P[i * M + a], P[j * M + a], sj);
      }
      const double cn = fma(sq, sc, qacc.C()[i * N + j]);
      qacc.C()[i * N + j] = cn;
      qacc.C()[j * N + i] = cn;
      k.J()[i * N + j] = sj;
      k.J()[j * N + i] = sj;
    }
  } else {
  constexpr int NSF = NS - NS % TEAM;
  for (int t = lane; t < NSF; t += TEAM) {
    int i, j;
    upper_ij(N, t, i, j);
    double sc = 0.0, sj = -Q[i * N + j];
    for (int a = 0; a < M; ++a) {
      sc = fma(-AL[i * M + a], AL[j * M + a], sc);
      sj = fma(P[i * M + a], P[j * M + a], sj);
    }
    for (int l = 0; l < N; ++l) {
      sj = fma(-J[i * N + l], F[l * N + j], sj);
      sj = fma(-J[j * N + l], F[l * N + i], sj);
    }
    const double cn = fma(sq, sc, qacc.C()[i * N + j]);
    qacc.C()[i * N + j] = cn;
    qacc.C()[j * N + i] = cn;
    k.J()[i * N + j] = sj;
    k.J()[j * N + i] = sj;
  }
  if constexpr (NS % TEAM != 0) {
    constexpr int R = NS % TEAM;
    constexpr int S = split_lanes(R, TEAM);
    const int o = lane / S, sub = lane % S;
    int i = 0, j = 0;
    double sc = 0.0, sj = 0.0;
    if (o < R) {
      upper_ij(N, NSF + o, i, j);
      if (sub == 0) sj = -Q[i * N + j];
      for (int a = sub; a < M; a += S) {
        sc = fma(-AL[i * M + a], AL[j * M + a], sc);
        sj = fma(P[i * M + a], P[j * M + a], sj);
      }
      for (int l = sub; l < N; l += S) {
        sj = fma(-J[i * N + l], F[l * N + j], sj);
        sj = fma(-J[j * N + l], F[l * N + i], sj);
      }
    }
    sc = group_sum<S>(sc);
    sj = group_sum<S>(sj);
    if (sub == 0 && o < R) {
      const double cn = fma(sq, sc, qacc.C()[i * N + j]);
      qacc.C()[i * N + j] = cn;
      qacc.C()[j * N + i] = cn;
      k.J()[i * N + j] = sj;
      k.J()[j * N + i] = sj;
    }
  }
  }
  if (lane < 32) {  // dzeta = -rho/2 + |w|^2/2 + eta^T c, over the first warp
    double z = 0.0;
    for (int a = lane; a < M; a += 32) z = fma(0.5 * w[a], w[a], z);
    if (c)
      for (int l = lane; l < N; l += 32) z = fma(eta[l], c[l], z);
    z = group_sum<32>(z);
    if (lane == 0) *qacc.zeta() = fma(sq, z - 0.5 * qr[N], *qacc.zeta());
  }
  sync<TEAM>();
}

// out = base + s * k over the flow fields A, eta, J (out may alias base).
template <int N, int TEAM>
__device__ __forceinline__ void axpy_flow(int lane, Rec<N> out, Rec<N> base, double s, Rec<N> k) {
  for (int e = lane; e < N * N; e += TEAM) {
    out.A()[e] = fma(s, k.A()[e], base.A()[e]);
    out.J()[e] = fma(s, k.J()[e], base.J()[e]);
  }
  for (int e = lane; e < N; e += TEAM) out.eta()[e] = fma(s, k.eta()[e], base.eta()[e]);
  sync<TEAM>();
}


// ---------------------------------------------------------------------------
// forward conditional ODEs (Sec. IV-C, Theorem Forward_HJB_LQT), full records
// ---------------------------------------------------------------------------

// k = f(y) for the forward element flow in tau, with B = Lt Lt^T,
// Q = H^T X H, q = H^T X r, rho = r^T X r (qr = [q | rho]):
//   dA = F A - C Q A             db = c + F b + C w      (w = q - Q b)
//   dC = B + F C + (F C)^T - C Q C
//   deta = A^T w                 dJ = A^T Q A
//   dzeta = rho/2 - b^T (w + q)/2
// y, k: packed records (k must not alias y).  Scratch QA, CQ (N x N), w (N).
// Products that share a shape give every thread the same outputs (gemm), so
// the terms of dA and dC are accumulated without barriers between them.
template <int N, int M, int TEAM>
__device__ void forward_rhs(int lane, Rec<N> y, Rec<N> k, const double* __restrict__ F, const double* __restrict__ c,
                            const double* __restrict__ Lt, const double* __restrict__ Q,
                            const double* __restrict__ qr, double* QA, double* CQ, double* w) {
  const double* A = y.A();
  const double* C = y.C();
  const double* b = y.b();
  gemm<N, N, N, TEAM, double>(
      lane, [&](int i, int l) { return Q[i * N + l]; }, [&](int l, int j) { return A[l * N + j]; },
      [&](int i, int j, double s) { QA[i * N + j] = s; });
  gemm<N, N, N, TEAM, double>(
      lane, [&](int i, int l) { return C[i * N + l]; }, [&](int l, int j) { return Q[l * N + j]; },
      [&](int i, int j, double s) { CQ[i * N + j] = s; });
  for (int i = lane; i < N; i += TEAM) {
    double s = qr[i];
    for (int l = 0; l < N; ++l) s = fma(-Q[i * N + l], b[l], s);
    w[i] = s;
  }
  sync<TEAM>();
  double* kA = k.A();
  double* kC = k.C();
  double* kJ = k.J();
  // dA = F A - C (Q A)
  gemm<N, N, N, TEAM, double>(
      lane, [&](int i, int l) { return F[i * N + l]; }, [&](int l, int j) { return A[l * N + j]; },
      [&](int i, int j, double s) { kA[i * N + j] = s; });
  gemm<N, N, N, TEAM, double>(
      lane, [&](int i, int l) { return C[i * N + l]; }, [&](int l, int j) { return QA[l * N + j]; },
      [&](int i, int j, double s) { kA[i * N + j] -= s; });
  // dC = F C + C F^T - (C Q) C + Lt Lt^T  (C F^T = (F C)^T, C symmetric)
  gemm<N, N, N, TEAM, double>(
      lane, [&](int i, int l) { return F[i * N + l]; }, [&](int l, int j) { return C[l * N + j]; },
      [&](int i, int j, double s) { kC[i * N + j] = s; });
  gemm<N, N, N, TEAM, double>(
      lane, [&](int i, int l) { return C[i * N + l]; }, [&](int l, int j) { return F[j * N + l]; },
      [&](int i, int j, double s) { kC[i * N + j] += s; });
  gemm<N, N, N, TEAM, double>(
      lane, [&](int i, int l) { return CQ[i * N + l]; }, [&](int l, int j) { return C[l * N + j]; },
      [&](int i, int j, double s) {
        double bij = kC[i * N + j] - s;
        for (int a = 0; a < M; ++a) bij = fma(Lt[i * M + a], Lt[j * M + a], bij);
        kC[i * N + j] = bij;
      });
  // dJ = A^T (Q A)
  gemm<N, N, N, TEAM, double>(
      lane, [&](int i, int l) { return A[l * N + i]; }, [&](int l, int j) { return QA[l * N + j]; },
      [&](int i, int j, double s) { kJ[i * N + j] = s; });
  // db = c + F b + C w ; deta = A^T w
  for (int i = lane; i < N; i += TEAM) {
    double s = c ? c[i] : 0.0, se = 0.0;
    for (int l = 0; l < N; ++l) {
      s = fma(F[i * N + l], b[l], s);
      s = fma(C[i * N + l], w[l], s);
      se = fma(A[l * N + i], w[l], se);
    }
    k.b()[i] = s;
    k.eta()[i] = se;
  }
  if (lane == 0) {
    double z = 0.5 * qr[N];
    for (int i = 0; i < N; ++i) z = fma(-0.5 * b[i], w[i] + qr[i], z);
    *k.zeta() = z;
  }
  sync<TEAM>();
}

// out1 = base1 + s1 k and out2 = base2 + s2 k over whole packed records (out1
// may alias base1; out2 may not alias base1).
template <int N, int TEAM>
__device__ __forceinline__ void axpy2_rec(int lane, double* out1, const double* base1, double s1, double* out2,
                                         const double* base2, double s2, const double* k) {
  for (int e = lane; e < Rec<N>::SIZE; e += TEAM) {
    const double ke = k[e];
    out1[e] = fma(s1, ke, base1[e]);
    if (out2) out2[e] = fma(s2, ke, base2[e]);
  }
  sync<TEAM>();
}

// copy a record (any layout) to another
template <int N, int TEAM>
__device__ __forceinline__ void copy_rec(int lane, Rec<N> dst, Rec<N> src) {
  for (int e = lane; e < Rec<N>::SIZE; e += TEAM) {
    if (e < N * N) dst.A()[e] = src.A()[e];
    else if (e < N * N + N) dst.b()[e - N * N] = src.b()[e - N * N];
    else if (e < 2 * N * N + N) dst.C()[e - N * N - N] = src.C()[e - N * N - N];
    else if (e < 2 * N * N + 2 * N) dst.eta()[e - 2 * N * N - N] = src.eta()[e - 2 * N * N - N];
    else if (e < 3 * N * N + 2 * N) dst.J()[e - 2 * N * N - 2 * N] = src.J()[e - 2 * N * N - 2 * N];
    else *dst.zeta() = *src.zeta();
  }
  sync<TEAM>();
}

// ---------------------------------------------------------------------------
// LU with partial pivoting on W (N x N), applied to R (N x Q); both in the
// caller's buffers.  Scratch: fscratch 2 * TEAM doubles (the pivot
// reciprocals at TEAM.. for a warp; a CTA keeps its row scales at TEAM.. and
// its pivot reciprocals at TEAM + 64..), iscratch TEAM ints.
// The pivot search compares magnitude keys (mag_key) on the integer pipes.
// W = I + P in every use (P = C J or C S): a pivot no larger than 2^-40 times
// its row's original scale max(1, max_j |W_ij|) sets the SINGULAR status bit
// (pivot_too_small).
// ---------------------------------------------------------------------------

template <int N, int TEAM, int Q>
__device__ void lu_solve(int lane, double* W, double* R, double* fscratch, int* iscratch) {
  static_assert(N <= TEAM, "one row scale per thread");
  // original row scales: in a register of lane i (a warp), or in shared
  // scratch (a larger team)
  unsigned long long* rks = reinterpret_cast<unsigned long long*>(fscratch + TEAM);
  unsigned long long rk = mag_key(1.0);
  if (lane < N)
    for (int j = 0; j < N; ++j) rk = umax64(rk, mag_key(W[lane * N + j]));
  if constexpr (TEAM > 32) {
    if (lane < N) rks[lane] = rk;
    __syncthreads();
  }
  for (int k = 0; k < N; ++k) {
    // arg max |W[i][k]|, i >= k (lowest index on ties)
    unsigned long long best = 0;
    int bi = N;
    if constexpr (TEAM <= 32) {
      for (int i = k + lane; i < N; i += TEAM) {
        const unsigned long long a = mag_key(W[i * N + k]);
        if (bi == N || a > best) { best = a; bi = i; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (oi < N && (bi == N || ob > best || (ob == best && oi < bi))) { best = ob; bi = oi; }
      }
      // exchange the row scales of rows k and bi with the rows
      const unsigned long long rk_k = __shfl_sync(0xffffffffu, rk, k);
      const unsigned long long rk_b = __shfl_sync(0xffffffffu, rk, bi);
      if (lane == k) rk = rk_b;
      else if (lane == bi) rk = rk_k;
      if (lane == 0 && pivot_too_small(__longlong_as_double((long long)best), rk_b)) flag(kStatusSingular);
    } else {
      // the first warp searches the (at most 64) candidate rows with shuffles
      // and publishes the pivot row: one barrier per step
      static_assert(N <= 64, "two candidate rows per lane of the first warp");
      unsigned long long* kb = reinterpret_cast<unsigned long long*>(fscratch);
      if (lane < 32) {
        unsigned long long wb = 0;
        int wi = N;
        for (int i = k + lane; i < N; i += 32) {
          const unsigned long long a = mag_key(W[i * N + k]);
          if (wi == N || a > wb) { wb = a; wi = i; }
        }
        for (int o = 16; o > 0; o >>= 1) {
          const unsigned long long ob = __shfl_xor_sync(0xffffffffu, wb, o);
          const int oi = __shfl_xor_sync(0xffffffffu, wi, o);
          if (oi < N && (wi == N || ob > wb || (ob == wb && oi < wi))) { wb = ob; wi = oi; }
        }
        if (lane == 0) {
          kb[0] = wb;
          iscratch[0] = wi;
          const unsigned long long rk_b = rks[wi];
          if (pivot_too_small(__longlong_as_double((long long)wb), rk_b)) flag(kStatusSingular);
          rks[wi] = rks[k];
          rks[k] = rk_b;
          // 1 / pivot, once for the team (the elimination and the back
          // substitution read it)
          fscratch[TEAM + 64 + k] = 1.0 / W[wi * N + k];
        }
      }
      __syncthreads();
      bi = iscratch[0];
      best = kb[0];
    }
    if (bi != k) {
      for (int j = lane; j < N + Q; j += TEAM) {
        double* a = j < N ? &W[k * N + j] : &R[k * Q + (j - N)];
        double* b = j < N ? &W[bi * N + j] : &R[bi * Q + (j - N)];
        const double t = *a;
        *a = *b;
        *b = t;
      }
    }
    sync<TEAM>();
    const int wc = N - k - 1, cols = wc + Q;
    if constexpr (TEAM > 32) {
      // a CTA: warp w updates rows k+1+w, k+1+w+8, ..., forming each row's
      // multiplier itself (one instruction per row), the lanes over the
      // row's columns
      const double inv = fscratch[TEAM + 64 + k];
      const int warp = lane >> 5, wl = lane & 31;
      for (int i = k + 1 + warp; i < N; i += TEAM / 32) {
        const double f = W[i * N + k] * inv;
        for (int c = wl; c < cols; c += 32) {
          if (c < wc) {
            const int j = k + 1 + c;
            W[i * N + j] = fma(-f, W[k * N + j], W[i * N + j]);
          } else {
            const int j = c - wc;
            R[i * Q + j] = fma(-f, R[k * Q + j], R[i * Q + j]);
          }
        }
      }
      sync<TEAM>();
      continue;
    }
    // multipliers into column k (below the diagonal); 1 / pivot kept for the
    // back substitution
    const double inv = 1.0 / W[k * N + k];
    if (lane == 0) fscratch[TEAM + k] = inv;
    for (int i = k + 1 + lane; i < N; i += TEAM) W[i * N + k] *= inv;
    sync<TEAM>();
    // rank-1 update of the trailing rows
    if constexpr (TEAM <= 32) {
      // a warp: one row at a time, the lanes over its columns (no division by
      // the step-dependent row length in the warp's instruction stream)
      for (int i = k + 1; i < N; ++i) {
        const double f = W[i * N + k];
        for (int c = lane; c < cols; c += TEAM) {
          if (c < wc) {
            const int j = k + 1 + c;
            W[i * N + j] = fma(-f, W[k * N + j], W[i * N + j]);
          } else {
            const int j = c - wc;
            R[i * Q + j] = fma(-f, R[k * Q + j], R[i * Q + j]);
          }
        }
      }
    } else {
      // a CTA: the threads over all (row, column) entries of the update
      for (int e = lane; e < wc * cols; e += TEAM) {
        const int i = k + 1 + e / cols, c = e % cols;
        const double f = W[i * N + k];
        if (c < wc) {
          const int j = k + 1 + c;
          W[i * N + j] = fma(-f, W[k * N + j], W[i * N + j]);
        } else {
          const int j = c - wc;
          R[i * Q + j] = fma(-f, R[k * Q + j], R[i * Q + j]);
        }
      }
    }
    sync<TEAM>();
  }
  // back substitution, one pivot row at a time
  for (int k = N - 1; k >= 0; --k) {
    double inv;
    if constexpr (TEAM > 32) inv = fscratch[TEAM + 64 + k];
    else inv = fscratch[TEAM + k];
    for (int j = lane; j < Q; j += TEAM) R[k * Q + j] *= inv;
    sync<TEAM>();
    for (int e = lane; e < k * Q; e += TEAM) {
      const int i = e / Q, j = e % Q;
      R[i * Q + j] = fma(-W[i * N + k], R[k * Q + j], R[i * Q + j]);
    }
    sync<TEAM>();
  }
}

// Sum of one value per thread over the team (every thread gets the sum).
// scratch: TEAM doubles (teams larger than a warp).
template <int TEAM>
__device__ __forceinline__ double team_sum(int lane, double x, double* scratch) {
  if constexpr (TEAM <= 32) {
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
  } else {
    scratch[lane] = x;
    __syncthreads();
    for (int w = TEAM / 2; w > 0; w >>= 1) {
      if (lane < w) scratch[lane] += scratch[lane + w];
      __syncthreads();
    }
    const double r = scratch[0];
    __syncthreads();
    return r;
  }
}

// ---------------------------------------------------------------------------
// combination rule
// ---------------------------------------------------------------------------

// Scratch needs for combine(): W (N^2), R (N (2N+1)), T1 (N^2), vectors 4N,
// plus lu scratch (2 TEAM doubles, TEAM ints).
template <int N>
__host__ __device__ constexpr int combine_scratch_doubles() {
  return N * N + N * (2 * N + 1) + N * N + 4 * N;
}

// out = e1 (x) e2 (full elements; out must not alias e1 or e2).  The O(N^3)
// products are register-blocked team products (gemm above); the symmetric
// results J, C are formed in full and stored as (X + X^T)/2.  Scratch: W, R,
// T1, vectors back to back at scr, or T1 at t1 (when given) and the rest at
// scr.
template <int N, int TEAM, typename G = double>
__device__ void combine(int lane, Rec<N> e1, Rec<N> e2, Rec<N> out, double* scr, double* fs, int* is,
                        tc::Ctx* tcx = nullptr, double* t1 = nullptr) {
  constexpr int Q = 2 * N + 1;
  double* W = scr;
  double* R = W + N * N;
  double* T1 = t1 ? t1 : R + N * Q;
  double* z0 = t1 ? R + N * Q : T1 + N * N;
  double* l0 = z0 + N;
  double* J2z = l0 + N;
  double* wv = J2z + N;
  const double* A1 = e1.A();
  const double* C1 = e1.C();
  const double* A2 = e2.A();
  const double* J2 = e2.J();
  // W = I + C1 J2 ; R = [A1 | C1 | b1 + C1 eta2]
  pgemm<N, TEAM, G>(lane, tcx, [&](int i, int l) { return C1[i * N + l]; }, [&](int l, int j) { return J2[l * N + j]; },
                         [&](int i, int j, G v) { W[i * N + j] = (double)v + (i == j ? 1.0 : 0.0); });
  for (int e = lane; e < 2 * N * N; e += TEAM) {
    const int i = e / (2 * N), j = e % (2 * N);
    R[i * Q + j] = j < N ? A1[i * N + j] : C1[i * N + (j - N)];
  }
  for (int i = lane; i < N; i += TEAM) {
    G g = (G)(e1.b()[i]);
    for (int l = 0; l < N; ++l) g = fma((G)(C1[i * N + l]), (G)(e2.eta()[l]), g);
    R[i * Q + 2 * N] = (double)g;
  }
  sync<TEAM>();
  lu_solve<N, TEAM, Q>(lane, W, R, fs, is);
  // R = [K1 | MC1 | z0]
  for (int i = lane; i < N; i += TEAM) z0[i] = R[i * Q + 2 * N];
  sync<TEAM>();
  // J2 z0, l0 = J2 z0 - eta2, w = eta2 - J2 b1 ; T1 = J2 A1
  for (int e = lane; e < N; e += TEAM) {
    G s = (G)(0.0);
    for (int l = 0; l < N; ++l) s = fma((G)(J2[e * N + l]), (G)(z0[l]), s);
    J2z[e] = s;
    l0[e] = s - e2.eta()[e];
    G w = (G)(e2.eta()[e]);
    for (int l = 0; l < N; ++l) w = fma((G)(-J2[e * N + l]), (G)(e1.b()[l]), w);
    wv[e] = w;
  }
  pgemm<N, TEAM, G>(lane, tcx, [&](int i, int l) { return J2[i * N + l]; }, [&](int l, int j) { return A1[l * N + j]; },
                         [&](int i, int j, G v) { T1[i * N + j] = v; });
  sync<TEAM>();
  // eta = K1^T w + eta1 ; b = A2 z0 + b2 ; W <- K1^T T1 ; A = A2 K1 ; zeta
  for (int t = lane; t < N; t += TEAM) {
    G s = (G)(e1.eta()[t]);
    for (int l = 0; l < N; ++l) s = fma((G)(R[l * Q + t]), (G)(wv[l]), s);
    out.eta()[t] = s;
    G sb = (G)(e2.b()[t]);
    for (int l = 0; l < N; ++l) sb = fma((G)(A2[t * N + l]), (G)(z0[l]), sb);
    out.b()[t] = sb;
  }
  pgemm<N, TEAM, G>(lane, tcx, [&](int i, int l) { return R[l * Q + i]; }, [&](int l, int j) { return T1[l * N + j]; },
                         [&](int i, int j, G v) { W[i * N + j] = v; });
  double* oA = out.A();
  pgemm<N, TEAM, G>(lane, tcx, [&](int i, int l) { return A2[i * N + l]; }, [&](int l, int j) { return R[l * Q + j]; },
                         [&](int i, int j, G v) { oA[i * N + j] = v; });
  {
    double zt = 0.0;
    for (int i = lane; i < N; i += TEAM) {
      G s = (G)(0.0);
      for (int l = 0; l < N; ++l) s = fma((G)(C1[i * N + l]), (G)(l0[l]), s);
      zt = fma(0.5 * l0[i], s, zt);
      zt = fma(z0[i], fma(0.5, J2z[i], -e2.eta()[i]), zt);
    }
    const double z = team_sum<TEAM>(lane, zt, fs);
    if (lane == 0) *out.zeta() = *e1.zeta() + *e2.zeta() + z;
  }
  sync<TEAM>();
  // J = J1 + sym(K1^T T1) ; T1 <- A2 MC1
  double* oJ = out.J();
  for (int e = lane; e < N * N; e += TEAM) {
    const int i = e / N, j = e % N;
    oJ[e] = e1.J()[e] + 0.5 * (W[i * N + j] + W[j * N + i]);
  }
  pgemm<N, TEAM, G>(lane, tcx, [&](int i, int l) { return A2[i * N + l]; },
                         [&](int l, int j) { return R[l * Q + N + j]; }, [&](int i, int j, G v) { T1[i * N + j] = v; });
  sync<TEAM>();
  // C = C2 + sym(T1 A2^T)
  pgemm<N, TEAM, G>(lane, tcx, [&](int i, int l) { return T1[i * N + l]; }, [&](int l, int j) { return A2[j * N + l]; },
                         [&](int i, int j, G v) { W[i * N + j] = v; });
  sync<TEAM>();
  double* oC = out.C();
  for (int e = lane; e < N * N; e += TEAM) {
    const int i = e / N, j = e % N;
    oC[e] = e2.C()[e] + 0.5 * (W[i * N + j] + W[j * N + i]);
  }
  sync<TEAM>();
}

// Value form: out = e (x) V, V = (S2 full N^2, v2 N, zeta2); also Psi (N^2) and
// alpha (N) of the one-sub-interval map.  Value record layout: S (N^2), v (N),
// zeta.  Scratch: W (N^2), R (N (N+1)), T1 (N^2), 3 vectors (T1 at t1 when
// given, as in combine()).
template <int N>
__host__ __device__ constexpr int value_scratch_doubles() {
  return N * N + N * (N + 1) + N * N + 3 * N;
}
template <int N>
__host__ __device__ constexpr int val_doubles() {
  return N * N + N + 1;
}

template <int N, int TEAM, typename G = double>
__device__ void combine_value(int lane, Rec<N> e, const double* V, double* out, double* Psi, double* alpha,
                              double* scr, double* fs, int* is, double* zeta_inc = nullptr,
                              tc::Ctx* tcx = nullptr, double* t1 = nullptr) {
  constexpr int Q = N + 1;
  const double* S2 = V;
  const double* v2 = V + N * N;
  const double zeta2 = V[N * N + N];
  double* W = scr;
  double* R = W + N * N;
  double* T1 = t1 ? t1 : R + N * Q;
  double* Sz = t1 ? R + N * Q : T1 + N * N;
  double* l0 = Sz + N;
  double* wv = l0 + N;
  const double* A = e.A();
  const double* C = e.C();
  // W = I + C S2 ; R = [A | b + C v2], in FP64 whatever G is: they define
  // the one-sub-interval map (Psi, alpha) that the state scan composes T
  // times, where FP32 rounding would accumulate
  gemm<N, N, N, TEAM, double>(lane, [&](int i, int l) { return C[i * N + l]; },
                              [&](int l, int j) { return S2[l * N + j]; },
                              [&](int i, int j, double v) { W[i * N + j] = v + (i == j ? 1.0 : 0.0); });
  for (int t = lane; t < N * N; t += TEAM) R[(t / N) * Q + (t % N)] = A[t];
  for (int i = lane; i < N; i += TEAM) {
    double g = e.b()[i];
    for (int l = 0; l < N; ++l) g = fma(C[i * N + l], v2[l], g);
    R[i * Q + N] = g;
  }
  sync<TEAM>();
  lu_solve<N, TEAM, Q>(lane, W, R, fs, is);
  for (int t = lane; t < N * N + N; t += TEAM) {
    if (t < N * N) Psi[t] = R[(t / N) * Q + (t % N)];
    else alpha[t - N * N] = R[(t - N * N) * Q + N];
  }
  sync<TEAM>();
  // Sz = S2 alpha, l0 = Sz - v2, w = v2 - S2 b ; T1 = S2 A
  for (int t = lane; t < N; t += TEAM) {
    G s = (G)(0.0);
    for (int l = 0; l < N; ++l) s = fma((G)(S2[t * N + l]), (G)(alpha[l]), s);
    Sz[t] = s;
    l0[t] = s - v2[t];
    G w = (G)(v2[t]);
    for (int l = 0; l < N; ++l) w = fma((G)(-S2[t * N + l]), (G)(e.b()[l]), w);
    wv[t] = w;
  }
  pgemm<N, TEAM, G>(lane, tcx, [&](int i, int l) { return S2[i * N + l]; }, [&](int l, int j) { return A[l * N + j]; },
                         [&](int i, int j, G v) { T1[i * N + j] = v; });
  sync<TEAM>();
  double* So = out;
  double* vo = out + N * N;
  for (int t = lane; t < N; t += TEAM) {
    G s = (G)(e.eta()[t]);
    for (int l = 0; l < N; ++l) s = fma((G)(Psi[l * N + t]), (G)(wv[l]), s);
    vo[t] = s;
  }
  // W <- Psi^T T1 ; S = J + sym(W)
  pgemm<N, TEAM, G>(lane, tcx, [&](int i, int l) { return Psi[l * N + i]; },
                         [&](int l, int j) { return T1[l * N + j]; }, [&](int i, int j, G v) { W[i * N + j] = v; });
  {
    double zt = 0.0;
    for (int i = lane; i < N; i += TEAM) {
      G s = (G)(0.0);
      for (int l = 0; l < N; ++l) s = fma((G)(C[i * N + l]), (G)(l0[l]), s);
      zt = fma(0.5 * l0[i], s, zt);
      zt = fma(alpha[i], fma(0.5, Sz[i], -v2[i]), zt);
    }
    const double z = team_sum<TEAM>(lane, zt, fs);
    if (lane == 0) {
      const double inc = *e.zeta() + z;  // the element's own share; the carry's zeta added after
      out[N * N + N] = inc + zeta2;
      if (zeta_inc) *zeta_inc = inc;
    }
  }
  sync<TEAM>();
  for (int t = lane; t < N * N; t += TEAM) {
    const int i = t / N, j = t % N;
    So[t] = e.J()[t] + 0.5 * (W[i * N + j] + W[j * N + i]);
  }
  sync<TEAM>();
}

// (P, p) <- (P Psi, P alpha + p) ; T scratch N^2 + N.
template <int N, int TEAM>
__device__ void compose_right(int lane, double* P, double* p, const double* Psi, const double* alpha, double* Tm) {
  for (int t = lane; t < N * N + N; t += TEAM) {
    if (t < N * N) {
      const int i = t / N, j = t % N;
      double s = 0.0;
      for (int l = 0; l < N; ++l) s = fma(P[i * N + l], Psi[l * N + j], s);
      Tm[t] = s;
    } else {
      const int i = t - N * N;
      double s = p[i];
      for (int l = 0; l < N; ++l) s = fma(P[i * N + l], alpha[l], s);
      Tm[t] = s;
    }
  }
  sync<TEAM>();
  for (int t = lane; t < N * N + N; t += TEAM) {
    if (t < N * N) P[t] = Tm[t];
    else p[t - N * N] = Tm[t];
  }
  sync<TEAM>();
}

}  // namespace team
}  // namespace lqt

namespace lqt {
namespace team {

// (P, p) <- (Psi P, Psi p + alpha): apply the group's earlier maps first.
template <int N, int TEAM>
__device__ void compose_left(int lane, double* P, double* p, const double* Psi, const double* alpha, double* Tm) {
  for (int t = lane; t < N * N + N; t += TEAM) {
    if (t < N * N) {
      const int i = t / N, j = t % N;
      double s = 0.0;
      for (int l = 0; l < N; ++l) s = fma(Psi[i * N + l], P[l * N + j], s);
      Tm[t] = s;
    } else {
      const int i = t - N * N;
      double s = alpha[i];
      for (int l = 0; l < N; ++l) s = fma(Psi[i * N + l], p[l], s);
      Tm[t] = s;
    }
  }
  sync<TEAM>();
  for (int t = lane; t < N * N + N; t += TEAM) {
    if (t < N * N) P[t] = Tm[t];
    else p[t - N * N] = Tm[t];
  }
  sync<TEAM>();
}

// y = Psi x + alpha
template <int N, int TEAM>
__device__ void apply_map(int lane, const double* Psi, const double* alpha, const double* x, double* y) {
  for (int i = lane; i < N; i += TEAM) {
    double s = alpha[i];
    for (int l = 0; l < N; ++l) s = fma(Psi[i * N + l], x[l], s);
    y[i] = s;
  }
  sync<TEAM>();
}

}  // namespace team
}  // namespace lqt
