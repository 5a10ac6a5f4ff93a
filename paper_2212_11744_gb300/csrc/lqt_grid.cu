// The general method on a state grid: the nonlinear scalar example of
// Sec. VI-B (dx/dt = d0 + d1 x + d2 x^2 + u, running cost q x^2/2 + rho u^2/2,
// terminal cost qf x^2/2), each conditional value function held as the G x G
// array V(x_i, s; x_j, s') on the grid x_i = x_min + i dx, combined by the
// minimisation of Theorem HJB-comb over the grid and refined by the
// quadratic interpolation of App. E.
//
//   block    the one-step function (an explicit Euler step with any control)
//            combined with itself `substeps` times, left to right;
//   combine  out(i, j) = min_k A(i, k) + B(k, j), refined;
//   values   V(., t_k) for k = 0..T.  The model is time-invariant, so every
//            block has the same conditional value function (Sec. VI-B) and
//            the scan's partial products are its powers.  The powers
//            P_{l+1} = P_l (x) P_l are formed once (log2 T products); then for
//            each bit l, lowest first, every k whose T - k has bit l set
//            updates w_k <- P_l (x) w_k, all such k and all grid points in one
//            launch.  After the last bit w_k = V(., t_k).
//
// Both products are one kernel: a 16 x 16 tile of outputs per CTA, one output
// per thread, the reduction index in steps of 64 staged in shared memory.  The
// minimum is defined on FP64 sums, ascending k, strict improvement only (the
// lowest index wins a tie).  GB300 retires FP64 adds at 1/64 of its FP32
// rate, so every candidate is first screened in FP32 (a bracket around its
// sum) and only the few whose bracket reaches the smallest upper bound are
// summed in FP64; the screen provably keeps every k that could be the FP64
// minimum, so the result is the one of the plain FP64 scan (which remains the
// path for operands outside the screen's float range).  FP64 comparisons run
// on integer keys that order doubles like the FP64 comparison does (the two
// zeros equal).  This is tropical (min, +) algebra: no multiply-accumulate, so
// no tensor-core form applies.
//
// Every floating-point expression uses explicit round-to-nearest intrinsics,
// in the order the definitions state them, so no multiply-add contraction
// changes a rounding: on the same inputs the grid minimisers are the same as
// those of any evaluation that follows the same formulas in IEEE double.
#include <climits>

#include <cuda_runtime.h>

#include "lqt_device.cuh"
#include "lqt_internal.h"

namespace lqt {

namespace {

struct GridArgs {
  int32_t G;
  double x_min, dx, d0, d1, d2, q, rho, qf, tau;
  int32_t substeps;
  int64_t T;
  int32_t interp;
};

GridArgs grid_args(const lqt_grid_problem& p) {
  return GridArgs{p.G, p.x_min, p.dx, p.d0, p.d1, p.d2, p.q, p.rho, p.qf, p.tau, p.substeps, p.T, p.interp};
}

constexpr int kGT = 16;  // output tile edge
constexpr int kGK = 64;  // reduction step staged in shared memory (a grid of <= 64 points: one tile)

__device__ __forceinline__ double grid_x(const GridArgs& a, int i) { return __dadd_rn(a.x_min, __dmul_rn((double)i, a.dx)); }

// Integer key with key(u) < key(v) exactly when u < v for non-NaN doubles
// (and key(-0) == key(+0)): the bit pattern for u >= +0, its negated
// magnitude for u <= -0.
__device__ __forceinline__ long long order_key(double v) {
  const long long b = __double_as_longlong(v);
  return b < 0 ? LLONG_MIN - b : b;
}

// App. E: the curvature a = (p + m - 2 c) / (2 dx^2) and slope
// b = (p - m) / (2 dx) of the quadratic through (m, c, p) at (k-1, k, k+1).
__device__ __forceinline__ double2 curvature(const GridArgs& a, double m, double c, double p) {
  const double den2 = __dmul_rn(2.0, __dmul_rn(a.dx, a.dx));
  const double den1 = __dmul_rn(2.0, a.dx);
  return make_double2(__ddiv_rn(__dsub_rn(__dadd_rn(p, m), __dmul_rn(2.0, c)), den2), __ddiv_rn(__dsub_rn(p, m), den1));
}

// App. E: the grid minimum `best` = g_k + f_k lowered by b^2 / (4a), with
// a = a_g + a_f and b = b_g + b_f; unchanged when a <= 0.
__device__ __forceinline__ double refine_with(double best, double2 g, double2 f) {
  const double cv = __dadd_rn(g.x, f.x), sl = __dadd_rn(g.y, f.y);
  if (!(cv > 0.0)) return best;
  return __dsub_rn(best, __ddiv_rn(__dmul_rn(sl, sl), __dmul_rn(4.0, cv)));
}

// Curvature and slope of every power's rows at every interior k, as pairs
// tab[l][i][k] (zero at k = 0 and G-1): they depend on (l, i, k) alone, so the
// values levels read them instead of dividing again for every row of w.
__global__ void grid_curv_kernel(GridArgs a, const double* __restrict__ pw, int L, double2* __restrict__ tab) {
  const int64_t GG = (int64_t)a.G * a.G;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= L * GG) return;
  const int k = (int)(e % a.G);
  tab[e] = (k > 0 && k < a.G - 1) ? curvature(a, pw[e - 1], pw[e], pw[e + 1]) : make_double2(0.0, 0.0);
}

// C(i, j): from x_i to x_j in one step dt = tau / substeps of
// x' = x + dt (drift(x) + u), so u = (x_j - x_i)/dt - drift(x_i) and the cost
// is dt (q x_i^2 + rho u^2) / 2.
__global__ void grid_one_step_kernel(GridArgs a, double* __restrict__ C) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)a.G * a.G) return;
  const int i = (int)(e / a.G), j = (int)(e % a.G);
  const double dt = __ddiv_rn(a.tau, (double)a.substeps);
  const double xi = grid_x(a, i), xj = grid_x(a, j);
  const double drift = __dadd_rn(__dadd_rn(a.d0, __dmul_rn(a.d1, xi)), __dmul_rn(__dmul_rn(a.d2, xi), xi));
  const double u = __dsub_rn(__ddiv_rn(__dsub_rn(xj, xi), dt), drift);
  C[e] = __dmul_rn(__dmul_rn(dt, 0.5), __dadd_rn(__dmul_rn(__dmul_rn(a.q, xi), xi), __dmul_rn(__dmul_rn(a.rho, u), u)));
}

// Values mode: column c of the product is the c-th k (ascending e = T - k)
// whose e has bit l set.  Such e run in blocks of 2^l: e = (2m+1) 2^l + r.
// Row k starts in buffer popc(e) & 1 and moves to the other buffer at every
// set bit of e, so before level l it is in buffer popc(e >> l) & 1 and after
// its last set bit in buffer 0.
struct ValCol {
  const double* in;
  double* out;
};

__device__ __forceinline__ ValCol value_column(const GridArgs& a, int l, int64_t c, double* X0, double* X1) {
  const int64_t low = ((int64_t)1 << l) - 1;
  const int64_t e = ((2 * (c >> l) + 1) << l) + (c & low);
  const int64_t k = a.T - e;
  const bool odd = __popcll((unsigned long long)(e >> l)) & 1;
  const int64_t off = k * a.G;
  return odd ? ValCol{X1 + off, X0 + off} : ValCol{X0 + off, X1 + off};
}

// Operands of one product.  kValues = false: A(i, k), B(k, j), out(i, j), all
// G x G row-major.  kValues = true: A = P_l, column c of B is w_in of the c-th
// updated row (see value_column), out column c is its w_out.
template <bool kValues>
struct Operands {
  const GridArgs& a;
  const double* __restrict__ A;
  const double* Bm;
  double* Om;
  double* X0;
  double* X1;
  int l;
  __device__ __forceinline__ double av(int i, int k) const { return A[(int64_t)i * a.G + k]; }
  // Column c of B: combine mode strides by G, values mode is contiguous.
  __device__ __forceinline__ const double* bcol(int64_t c) const {
    return kValues ? value_column(a, l, c, X0, X1).in : Bm + c;
  }
  __device__ __forceinline__ double bv(const double* col, int k) const {
    return kValues ? col[k] : col[(int64_t)k * a.G];
  }
};

// FP32 screen of a grid minimum (exactness argument below).  The operands are
// truncated to float by bit operations (relative error < 2^-23; magnitudes
// below 2^-126 become 0), summed in float, and bracketed:
//   lo_k = s_k - c t_k - d  <=  g_k + f_k  <=  hi_k = s_k + c t_k,
// t_k = |a_k| + |b_k|, c = 2^-20, d = 2^-100, with margins of more than four
// times the truncation and rounding errors and of the gap between two doubles
// that round to the same FP64 sum.  With U = min_k hi_k (+ d), every k whose
// FP64 sum g_k + f_k equals the FP64 minimum has lo_k <= U; every k with
// lo_k > U has a larger FP64 sum.  So the exact minimum, with the lowest-index
// rule, is taken over the survivors lo_k <= U alone, in ascending k, in FP64.
// Operands of magnitude >= 2^100 (or not finite) fall outside the screen's
// float range: a CTA that meets one takes the FP64 path for all its outputs.
constexpr float kScreenC = 9.5367431640625e-07f;  // 2^-20
constexpr float kScreenD = 7.888609052210118e-31f;  // 2^-100
constexpr float kScreenPad = 1.329227995784916e+36f;  // 2^120: k beyond the grid
constexpr int kMaxSurvivors = 4;

__device__ __forceinline__ bool screen_range(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  return ((b >> 52) & 0x7ff) < 1023 + 100;
}

// Truncation toward zero of a double in the screen's range to float.
__device__ __forceinline__ float screen_float(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int eb = (int)((b >> 52) & 0x7ff);
  if (eb < 1023 - 126) return 0.0f;
  const unsigned fb = ((unsigned)(b >> 63) << 31) | ((unsigned)(eb - 1023 + 127) << 23) |
                      (unsigned)((b >> 29) & 0x7fffff);
  return __uint_as_float(fb);
}

union GridSmem {
  struct {
    double A[kGT][kGK + 1];
    double B[kGK][kGT + 1];
  } d;  // FP64 path
  struct {
    float A[kGT][kGK + 2];
    float Bt[kGT][kGK + 2];  // B transposed: one row of k per output column
  } f;  // screen; rows of 66 floats keep float2 reads aligned and conflict-free
};

__device__ __forceinline__ float screen_hi(float a, float b) {
  return __fmaf_rn(kScreenC, __fadd_rn(fabsf(a), fabsf(b)), __fadd_rn(a, b));
}
__device__ __forceinline__ float screen_lo(float a, float b) {
  return __fmaf_rn(-kScreenC, __fadd_rn(fabsf(a), fabsf(b)), __fadd_rn(a, b));
}

// Float tiles of A (rows i0.., reduction k0..) and B (reduction k0..,
// columns c0..); k beyond the grid holds kScreenPad.  Returns whether an
// operand lies outside the screen's range.
template <bool kValues>
__device__ __forceinline__ bool stage_float(const Operands<kValues>& op, GridSmem& sm, int t, int i0, int64_t c0,
                                            int64_t ncols, int k0) {
  const int G = op.a.G;
  bool bad = false;
  for (int e = t; e < kGT * kGK; e += kGT * kGT) {
    const int r = e / kGK, kk = e % kGK;
    const int gi = i0 + r, gk = k0 + kk;
    float v = kScreenPad;
    if (gk < G) {
      v = 0.0f;
      if (gi < G) {
        const double x = op.av(gi, gk);
        bad |= !screen_range(x);
        v = screen_float(x);
      }
    }
    sm.f.A[r][kk] = v;
  }
  for (int e = t; e < kGT * kGK; e += kGT * kGT) {
    int kk, cc;
    if (kValues) {
      cc = e / kGK; kk = e % kGK;
    } else {
      kk = e / kGT; cc = e % kGT;
    }
    const int gk = k0 + kk;
    const int64_t gc = c0 + cc;
    float v = kScreenPad;
    if (gk < G) {
      v = 0.0f;
      if (gc < ncols) {
        const double x = op.bv(op.bcol(gc), gk);
        bad |= !screen_range(x);
        v = screen_float(x);
      }
    }
    sm.f.Bt[cc][kk] = v;
  }
  return bad;
}

// The FP64 evaluation of every candidate (CTAs whose operands leave the
// screen's range): double tiles, ascending k, strict improvement.
template <bool kValues>
__device__ __forceinline__ void fp64_scan(const Operands<kValues>& op, GridSmem& sm, int t, int i0, int64_t c0,
                                          int64_t ncols, int r_loc, int c_loc, double& best, int& bk) {
  const int G = op.a.G;
  long long bestk = LLONG_MAX;
  for (int k0 = 0; k0 < G; k0 += kGK) {
    for (int e = t; e < kGT * kGK; e += kGT * kGT) {
      const int r = e / kGK, kk = e % kGK;
      const int gi = i0 + r, gk = k0 + kk;
      sm.d.A[r][kk] = (gi < G && gk < G) ? op.av(gi, gk) : 0.0;
    }
    for (int e = t; e < kGT * kGK; e += kGT * kGT) {
      int kk, cc;
      if (kValues) {
        cc = e / kGK; kk = e % kGK;
      } else {
        kk = e / kGT; cc = e % kGT;
      }
      const int gk = k0 + kk;
      const int64_t gc = c0 + cc;
      sm.d.B[kk][cc] = (gk < G && gc < ncols) ? op.bv(op.bcol(gc), gk) : 0.0;
    }
    __syncthreads();
    const int kend = G - k0 < kGK ? G - k0 : kGK;
    for (int kk = 0; kk < kend; ++kk) {
      const double v = __dadd_rn(sm.d.A[r_loc][kk], sm.d.B[kk][c_loc]);
      const long long key = order_key(v);
      if (key < bestk) {
        bestk = key;
        best = v;
        bk = k0 + kk;
      }
    }
    __syncthreads();
  }
}

// One output (i, c) per thread, a 16 x 16 tile per CTA: the FP32 screen over
// all k (two passes: the bound U, then the survivors), the FP64 minimum over
// the survivors, App. E's refinement, the store.  Rows run over i (grid y),
// columns over j or c (grid x); in the values mode consecutive threads walk i
// so that the w_out stores are coalesced.
template <bool kValues>
__global__ void __launch_bounds__(kGT* kGT, 4)
    grid_minplus_kernel(GridArgs a, const double* __restrict__ A, const double* Bm, double* Om, double* X0,
                        double* X1, int l, int64_t ncols, const double2* __restrict__ tab) {
  __shared__ GridSmem sm;
  const Operands<kValues> op{a, A, Bm, Om, X0, X1, l};
  const int G = a.G;
  const int t = threadIdx.x;
  const int r_loc = kValues ? t % kGT : t / kGT;  // output row inside the tile
  const int c_loc = kValues ? t / kGT : t % kGT;  // output column inside the tile
  const int i0 = blockIdx.y * kGT;
  const int64_t c0 = (int64_t)blockIdx.x * kGT;
  const int i = i0 + r_loc;
  const int64_t c = c0 + c_loc;
  const bool valid = i < G && c < ncols;

  double best = 0.0;
  int bk = 0;
  // pass 1: U = min_k hi_k
  bool bad = false;
  float U = __int_as_float(0x7f800000);  // +inf
  for (int k0 = 0; k0 < G; k0 += kGK) {
    bad |= stage_float(op, sm, t, i0, c0, ncols, k0);
    __syncthreads();
    const int kend = G - k0 < kGK ? G - k0 : kGK;
    float U1 = U;  // two chains
    for (int kk = 0; kk < kend; kk += 2) {  // an odd kend reads one padded k
      const float2 a2 = *reinterpret_cast<const float2*>(&sm.f.A[r_loc][kk]);
      const float2 b2 = *reinterpret_cast<const float2*>(&sm.f.Bt[c_loc][kk]);
      U = fminf(U, screen_hi(a2.x, b2.x));
      U1 = fminf(U1, screen_hi(a2.y, b2.y));
    }
    U = fminf(U, U1);
    __syncthreads();
  }
  if (__syncthreads_or(bad)) {
    fp64_scan(op, sm, t, i0, c0, ncols, r_loc, c_loc, best, bk);
  } else {
    // pass 2: survivors lo_k <= U + d, ascending, up to kMaxSurvivors packed
    // as 16-bit indices (G <= 16384)
    const float Ub = __fadd_ru(U, kScreenD);
    unsigned long long pk = 0;
    int ns = 0;
    for (int k0 = 0; k0 < G; k0 += kGK) {
      if (G > kGK) {  // one tile: pass 1's staging is still in place
        stage_float(op, sm, t, i0, c0, ncols, k0);
        __syncthreads();
      }
      const int kend = G - k0 < kGK ? G - k0 : kGK;
      for (int kk = 0; kk < kend; kk += 2) {
        const float2 a2 = *reinterpret_cast<const float2*>(&sm.f.A[r_loc][kk]);
        const float2 b2 = *reinterpret_cast<const float2*>(&sm.f.Bt[c_loc][kk]);
        if (screen_lo(a2.x, b2.x) <= Ub) {
          if (ns < kMaxSurvivors) pk |= (unsigned long long)(k0 + kk) << (16 * ns);
          ++ns;
        }
        if (screen_lo(a2.y, b2.y) <= Ub) {  // a padded k never passes
          if (ns < kMaxSurvivors) pk |= (unsigned long long)(k0 + kk + 1) << (16 * ns);
          ++ns;
        }
      }
      __syncthreads();
    }
    if (!valid) return;
    const double* col = op.bcol(c);
    long long bestk = LLONG_MAX;
    const int cnt = ns <= kMaxSurvivors ? ns : G;  // too many survivors: every k
    for (int r = 0; r < cnt; ++r) {
      const int k = ns <= kMaxSurvivors ? (int)((pk >> (16 * r)) & 0xffff) : r;
      const double v = __dadd_rn(op.av(i, k), op.bv(col, k));
      const long long key = order_key(v);
      if (key < bestk) {
        bestk = key;
        best = v;
        bk = k;
      }
    }
  }
  if (!valid) return;
  const double* col = op.bcol(c);
  double res = best;
  if (a.interp && bk > 0 && bk < G - 1) {
    const double2 gc = tab ? tab[(int64_t)i * G + bk] : curvature(a, op.av(i, bk - 1), op.av(i, bk), op.av(i, bk + 1));
    res = refine_with(best, gc, curvature(a, op.bv(col, bk - 1), op.bv(col, bk), op.bv(col, bk + 1)));
  }
  if (kValues) value_column(a, l, c, X0, X1).out[i] = res;
  else Om[(int64_t)i * G + c] = res;
  if (!isfinite(res)) flag(kStatusNonFinite);
}

// Row k of the values starts as phi(x_i) = qf x_i^2 / 2 in the buffer it
// occupies before level 0: X0 when popc(T - k) is even, so that after its
// last update it lands in X0.
__global__ void grid_terminal_kernel(GridArgs a, double* __restrict__ X0, double* __restrict__ X1) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (a.T + 1) * a.G) return;
  const int64_t k = e / a.G;
  const double x = grid_x(a, (int)(e % a.G));
  const double phi = __dmul_rn(__dmul_rn(__dmul_rn(0.5, a.qf), x), x);
  const bool odd = __popcll((unsigned long long)(a.T - k)) & 1;
  (odd ? X1 : X0)[e] = phi;
}

unsigned cdiv_u(int64_t x, int64_t y) { return (unsigned)((x + y - 1) / y); }

int grid_levels(int64_t T) {
  int L = 0;
  while (((int64_t)1 << L) <= T) ++L;
  return L;
}

// Number of e in [1, T] with bit l set.
int64_t set_count(int64_t T, int l) {
  const int64_t blk = (int64_t)1 << (l + 1), half = (int64_t)1 << l;
  const int64_t full = (T + 1) / blk, rem = (T + 1) % blk;
  return full * half + (rem > half ? rem - half : 0);
}

cudaError_t launch_combine(const GridArgs& a, const double* A, const double* B, double* out, cudaStream_t st) {
  const dim3 grid(cdiv_u(a.G, kGT), cdiv_u(a.G, kGT));
  grid_minplus_kernel<false><<<grid, kGT * kGT, 0, st>>>(a, A, B, out, nullptr, nullptr, 0, a.G, nullptr);
  count_launch();
  return cudaGetLastError();
}

}  // namespace

size_t grid_workspace_bytes(const lqt_grid_problem& p, int which) {
  const size_t GG = (size_t)p.G * p.G;
  if (which == 0) return 2 * GG * sizeof(double);
  // powers, one double of alignment slack, their (curvature, slope) pairs, the
  // second buffer of the values
  return ((size_t)grid_levels(p.T) * GG * 3 + 1 + ((size_t)p.T + 1) * p.G) * sizeof(double);
}

cudaError_t run_grid_block(const lqt_grid_problem& p, double* Vblock, char* ws, cudaStream_t st) {
  const GridArgs a = grid_args(p);
  const size_t GG = (size_t)p.G * p.G;
  double* C = (double*)ws;
  double* tmp = C + GG;
  grid_one_step_kernel<<<cdiv_u((int64_t)GG, 256), 256, 0, st>>>(a, C);
  count_launch();
  cudaError_t e = cudaGetLastError();
  // M_1 = C, M_{m+1} = M_m (x) C, ping-ponging between Vblock and tmp so that
  // M_substeps ends in Vblock.
  double* cur = (p.substeps & 1) ? Vblock : tmp;
  if (e == cudaSuccess) e = cudaMemcpyAsync(cur, C, GG * sizeof(double), cudaMemcpyDeviceToDevice, st);
  for (int m = 1; m < p.substeps && e == cudaSuccess; ++m) {
    double* nxt = cur == Vblock ? tmp : Vblock;
    e = launch_combine(a, cur, C, nxt, st);
    cur = nxt;
  }
  return e;
}

cudaError_t run_grid_combine(const lqt_grid_problem& p, const double* A, const double* B, double* out,
                             cudaStream_t st) {
  return launch_combine(grid_args(p), A, B, out, st);
}

cudaError_t run_grid_values(const lqt_grid_problem& p, const double* Vblock, double* V, char* ws, cudaStream_t st) {
  const GridArgs a = grid_args(p);
  const size_t GG = (size_t)p.G * p.G;
  const int L = grid_levels(p.T);
  double* pw = (double*)ws;  // P_0 .. P_{L-1}
  // their (curvature, slope) pairs, on a 16-byte boundary
  double2* tab = (double2*)(((uintptr_t)(pw + (size_t)L * GG) + 15) & ~(uintptr_t)15);
  double* X1 = (double*)(tab + (size_t)L * GG);  // second buffer of the values (V is the first)
  cudaError_t e = cudaMemcpyAsync(pw, Vblock, GG * sizeof(double), cudaMemcpyDeviceToDevice, st);
  for (int l = 1; l < L && e == cudaSuccess; ++l)
    e = launch_combine(a, pw + (l - 1) * GG, pw + (l - 1) * GG, pw + l * GG, st);
  if (e != cudaSuccess) return e;
  if (p.interp) {
    grid_curv_kernel<<<cdiv_u((int64_t)L * GG, 256), 256, 0, st>>>(a, pw, L, tab);
    count_launch();
  }
  grid_terminal_kernel<<<cdiv_u((p.T + 1) * p.G, 256), 256, 0, st>>>(a, V, X1);
  count_launch();
  for (int l = 0; l < L; ++l) {
    const int64_t nc = set_count(p.T, l);
    const dim3 grid(cdiv_u(nc, kGT), cdiv_u(p.G, kGT));
    grid_minplus_kernel<true><<<grid, kGT * kGT, 0, st>>>(a, pw + l * GG, nullptr, nullptr, V, X1, l, nc,
                                                          p.interp ? tab + l * GG : nullptr);
    count_launch();
  }
  return cudaGetLastError();
}

}  // namespace lqt
