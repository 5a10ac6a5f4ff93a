// Reverse mode of the parallel LQT solve (lqt_backward).
//
// Forward quantities (recomputed or given): elements e_k (Sec. IV-B/IV-D),
// values (S_k, v_k, zeta_k) (Sec. IV-A, eq. eJ_vS), one-sub-interval maps
// x_{k+1} = Psi_k x_k + alpha_k (Sec. IV-E), states x_k, cost
// V(x0,t0) = zeta_0 + x0'S_0x0/2 - v_0'x0.
//
// Backward, for upstream gradients gS, gv, gzeta, gx (per boundary) and g_cost:
//  1. states: xbar_T = gx_T, xbar_k = gx_k + Psi_k^T xbar_{k+1}  -- a linear
//     recurrence run as a forward affine-map scan over reversed indices.
//  2. maps: with Z = [Psi | alpha] = W^-1 R, W = I + C_k S_{k+1},
//     R = [A_k | b_k + C_k v_{k+1}] and Zbar = [xbar_{k+1} x_k^T | xbar_{k+1}]:
//     Rbar = W^-T Zbar, Wbar = -Rbar Z^T, giving Abar_k, bbar_k, Cbar_k and
//     direct terms for Sbar_{k+1}, vbar_{k+1}.
//  3. values: the value at k is the pull-back of the value at k+1 through
//     z = Psi_k x + alpha_k (envelope theorem on the min over z), so in
//     homogeneous form M = [[S, -v], [-v^T, 2 zeta]] one has
//     M_k = P_k^T M_{k+1} P_k + (element part), P_k = [[Psi_k, alpha_k], [0, 1]].
//     The adjoint Sigma = [[Sbar, -vbar/2], [-vbar^T/2, zetabar/2]] therefore
//     runs FORWARD: Sigma_{k+1} = P_k Sigma_k P_k^T + D_{k+1}, a congruence scan.
//  4. elements from the values (envelope theorem on the saddle point of the
//     dual form eq. LQT_V_form2 with lambda* = Lambda x + l, Lambda = S_{k+1}
//     Psi_k, l = S_{k+1} alpha_k - v_{k+1}):
//     Jbar += Sbar, etabar += vbar, zetabar_e += zetabar,
//     Abar += 2 Lambda Sbar - l vbar^T, bbar += -Lambda vbar + zetabar l,
//     Cbar += -Lambda Sbar Lambda^T + sym(Lambda vbar l^T) - zetabar l l^T / 2.
//  5. element build: discrete adjoint of the K classical RK4 steps of the
//     backward conditional HJB ODEs (Theorem Backward_HJB_LQT), per
//     sub-interval, about the stage inputs that this pass's element build
//     recomputed and stored, giving Fbar, Bbar (B = L U^-1 L^T), Qbar, qbar, rhobar, then
//     Xbar, rbar (Q = X, q = X r, rho = r'Xr for H = I) and, after the
//     reduction over sub-intervals, Lbar = (Bbar + Bbar^T) L U^-1 and
//     Ubar = -U^-1 L^T Bbar L U^-1.
//
// Kernels here use runtime-n loops over small local arrays (n <= 8): the
// backward is not the benchmarked path and this keeps compile time small.
#include <cuda_runtime.h>

#include "lqt_device.cuh"
#include "lqt_internal.h"

namespace lqt {

constexpr int AN = 8;            // largest n of the backward
constexpr int AH = AN + 1;       // homogeneous size
constexpr int AS = 3 * AN * AN + 2 * AN + 1;

static int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }
static size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

// ---------------------------------------------------------------------------
// small runtime-n helpers (row-major, leading dimension = n)
// ---------------------------------------------------------------------------

__device__ __forceinline__ void mm(int n, const double* a, const double* b, double* c) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int l = 0; l < n; ++l) s = fma(a[i * n + l], b[l * n + j], s);
      c[i * n + j] = s;
    }
}
// c = a^T b
__device__ __forceinline__ void mtm(int n, const double* a, const double* b, double* c) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int l = 0; l < n; ++l) s = fma(a[l * n + i], b[l * n + j], s);
      c[i * n + j] = s;
    }
}
// c = a b^T
__device__ __forceinline__ void mmt(int n, const double* a, const double* b, double* c) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int l = 0; l < n; ++l) s = fma(a[i * n + l], b[j * n + l], s);
      c[i * n + j] = s;
    }
}
__device__ __forceinline__ void mv(int n, const double* a, const double* x, double* y) {
  for (int i = 0; i < n; ++i) {
    double s = 0.0;
    for (int l = 0; l < n; ++l) s = fma(a[i * n + l], x[l], s);
    y[i] = s;
  }
}
__device__ __forceinline__ void mtv(int n, const double* a, const double* x, double* y) {
  for (int i = 0; i < n; ++i) {
    double s = 0.0;
    for (int l = 0; l < n; ++l) s = fma(a[l * n + i], x[l], s);
    y[i] = s;
  }
}
__device__ __forceinline__ void symm(int n, double* a) {
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j) {
      const double s = 0.5 * (a[i * n + j] + a[j * n + i]);
      a[i * n + j] = s;
      a[j * n + i] = s;
    }
}
// Solve W X = R (W n x n, n <= 16, R n x q, both overwritten) with partial
// pivoting; a pivot no larger than 2^-40 of its row's original scale sets the
// SINGULAR status bit (pivot_too_small).  The row scale is max_j |W_ij|, and
// at least 1 when unit_part (W = I + P: cancellation between I and P counts).
__device__ void solve_rt(int n, int q, double* W, double* R, bool unit_part) {
  unsigned long long rk[16];
  for (int i = 0; i < n; ++i) {
    rk[i] = unit_part ? mag_key(1.0) : 0ull;
    for (int j = 0; j < n; ++j) rk[i] = umax64(rk[i], mag_key(W[i * n + j]));
  }
  for (int k = 0; k < n; ++k) {
    int piv = k;
    double best = fabs(W[k * n + k]);
    for (int i = k + 1; i < n; ++i)
      if (fabs(W[i * n + k]) > best) { best = fabs(W[i * n + k]); piv = i; }
    if (pivot_too_small(best, rk[piv])) flag(kStatusSingular);
    if (piv != k) {
      for (int j = 0; j < n; ++j) { const double s = W[k * n + j]; W[k * n + j] = W[piv * n + j]; W[piv * n + j] = s; }
      for (int j = 0; j < q; ++j) { const double s = R[k * q + j]; R[k * q + j] = R[piv * q + j]; R[piv * q + j] = s; }
      const unsigned long long t = rk[k]; rk[k] = rk[piv]; rk[piv] = t;
    }
    const double inv = 1.0 / W[k * n + k];
    for (int i = k + 1; i < n; ++i) {
      const double f = W[i * n + k] * inv;
      for (int j = k + 1; j < n; ++j) W[i * n + j] = fma(-f, W[k * n + j], W[i * n + j]);
      for (int j = 0; j < q; ++j) R[i * q + j] = fma(-f, R[k * q + j], R[i * q + j]);
    }
  }
  for (int k = n - 1; k >= 0; --k) {
    const double inv = 1.0 / W[k * n + k];
    for (int j = 0; j < q; ++j) {
      double s = R[k * q + j];
      for (int l = k + 1; l < n; ++l) s = fma(-W[k * n + l], R[l * q + j], s);
      R[k * q + j] = s * inv;
    }
  }
}

// Full-layout element record: A (n^2), b (n), C (n^2), eta (n), J (n^2), zeta.
struct FE {
  double* A; double* b; double* C; double* eta; double* J; double* z;
};
__device__ __forceinline__ FE fe_view(int n, double* base) {
  FE e;
  e.A = base; e.b = e.A + n * n; e.C = e.b + n; e.eta = e.C + n * n; e.J = e.eta + n; e.z = e.J + n * n;
  return e;
}
__device__ __forceinline__ int fe_size(int n) { return 3 * n * n + 2 * n + 1; }

// ---------------------------------------------------------------------------
// 1. trajectory adjoint: reversed maps (Psi_{T-1-k'}^T, gx_{T-1-k'})
// ---------------------------------------------------------------------------

__global__ void reversed_adjoint_maps_kernel(int n, int64_t T, const double* __restrict__ maps,
                                             const double* __restrict__ gx, double* __restrict__ rmaps) {
  const int64_t kp = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (kp >= T) return;
  const int64_t k = T - 1 - kp;
  const int PM = n * n + n;
  const double* m = maps + k * PM;
  double* o = rmaps + kp * PM;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) o[i * n + j] = m[j * n + i];
  for (int i = 0; i < n; ++i) o[n * n + i] = gx ? gx[k * n + i] : 0.0;
}

// ---------------------------------------------------------------------------
// 2. map adjoint per sub-interval, and the direct value-adjoint terms
// ---------------------------------------------------------------------------

struct MapAdjArgs {
  int n;
  int64_t T;
  ElemPtrs el;
  const double *S, *v, *x, *xbar_rev;  // xbar_rev[k'] = xbar_{T-k'}
  const double *gS, *gv, *gz;           // may be null
  const double* x0;
  double g_cost;
  double* D;      // [T+1][(n+1)^2]
  double* emap;   // [T][fe_size]: element terms of the map adjoint (slot j = element j)
  double* gx0;    // [n] or null
};

__global__ void map_adjoint_kernel(MapAdjArgs a) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k > a.T) return;
  const int n = a.n, n1 = n + 1, nn = n * n;
  double Sb[AN * AN], vb[AN];
  double zb = 0.0;
  for (int i = 0; i < nn; ++i) Sb[i] = a.gS ? a.gS[k * nn + i] : 0.0;
  for (int i = 0; i < n; ++i) vb[i] = a.gv ? a.gv[k * n + i] : 0.0;
  if (a.gz) zb = a.gz[k];
  if (k == 0) {  // cost = zeta_0 + x0'S_0 x0/2 - v_0'x0
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) Sb[i * n + j] += 0.5 * a.g_cost * a.x0[i] * a.x0[j];
    for (int i = 0; i < n; ++i) vb[i] -= a.g_cost * a.x0[i];
    zb += a.g_cost;
    if (a.gx0) {  // d cost / d x0 = S_0 x0 - v_0, plus the state adjoint at 0
      const double* xb0 = a.xbar_rev + a.T * n;
      for (int i = 0; i < n; ++i) {
        double s = -a.v[i];
        for (int l = 0; l < n; ++l) s = fma(a.S[i * n + l], a.x0[l], s);
        a.gx0[i] = xb0[i] + a.g_cost * s;
      }
    }
  }
  if (k >= 1) {
    // the map of sub-interval j = k-1 uses S_k, v_k
    const int64_t j = k - 1;
    const double* A = a.el.A + j * nn;
    const double* b = a.el.b + j * n;
    const double* C = a.el.C + j * nn;
    const double* Sk = a.S + k * nn;
    const double* vk = a.v + k * n;
    const double* xj = a.x + j * n;
    const double* xbk = a.xbar_rev + (a.T - k) * n;  // xbar_{k}
    FE E = fe_view(n, a.emap + j * fe_size(n));
    double W[AN * AN], Wt[AN * AN], Z[AN * AH], Rb[AN * AH];
    const int q = n + 1;
    for (int i = 0; i < n; ++i) {
      for (int c = 0; c < n; ++c) {
        double s = (i == c) ? 1.0 : 0.0;
        for (int l = 0; l < n; ++l) s = fma(C[i * n + l], Sk[l * n + c], s);
        W[i * n + c] = s;
        Z[i * q + c] = A[i * n + c];
      }
      double s = b[i];
      for (int l = 0; l < n; ++l) s = fma(C[i * n + l], vk[l], s);
      Z[i * q + n] = s;
    }
    for (int i = 0; i < n; ++i)
      for (int c = 0; c < n; ++c) Wt[i * n + c] = W[c * n + i];
    double Wc[AN * AN];
    for (int i = 0; i < nn; ++i) Wc[i] = W[i];
    solve_rt(n, q, Wc, Z, true);  // Z = [Psi | alpha]
    // Zbar = [xbar_k x_j^T | xbar_k]; Rbar = W^-T Zbar
    for (int i = 0; i < n; ++i) {
      for (int c = 0; c < n; ++c) Rb[i * q + c] = xbk[i] * xj[c];
      Rb[i * q + n] = xbk[i];
    }
    solve_rt(n, q, Wt, Rb, true);
    // Wbar = -Rbar Z^T  (n x n)
    double Wb[AN * AN];
    for (int i = 0; i < n; ++i)
      for (int c = 0; c < n; ++c) {
        double s = 0.0;
        for (int l = 0; l < q; ++l) s = fma(-Rb[i * q + l], Z[c * q + l], s);
        Wb[i * n + c] = s;
      }
    // W = I + C S : Cbar += Wbar S^T ; Sbar_k += C^T Wbar
    // R = [A | b + C v] : Abar = Rbar_A ; bbar = Rbar_a ; Cbar += Rbar_a v^T ; vbar_k += C^T Rbar_a
    for (int i = 0; i < n; ++i)
      for (int c = 0; c < n; ++c) {
        double s = 0.0, t = 0.0;
        for (int l = 0; l < n; ++l) {
          s = fma(Wb[i * n + l], Sk[c * n + l], s);  // Wbar S^T
          t = fma(C[l * n + i], Wb[l * n + c], t);   // C^T Wbar
        }
        E.C[i * n + c] = s + Rb[i * q + n] * vk[c];
        Sb[i * n + c] += t;
        E.A[i * n + c] = Rb[i * q + c];
      }
    for (int i = 0; i < n; ++i) {
      E.b[i] = Rb[i * q + n];
      E.eta[i] = 0.0;
      double s = 0.0;
      for (int l = 0; l < n; ++l) s = fma(C[l * n + i], Rb[l * q + n], s);
      vb[i] += s;
    }
  }
  // D_k in homogeneous form: [[Sbar_sym, -vbar/2], [-vbar^T/2, zetabar/2]]
  double* Dk = a.D + k * n1 * n1;
  for (int i = 0; i < n; ++i)
    for (int c = 0; c < n; ++c) Dk[i * n1 + c] = 0.5 * (Sb[i * n + c] + Sb[c * n + i]);
  for (int i = 0; i < n; ++i) {
    Dk[i * n1 + n] = -0.5 * vb[i];
    Dk[n * n1 + i] = -0.5 * vb[i];
  }
  Dk[n * n1 + n] = 0.5 * zb;
}

// ---------------------------------------------------------------------------
// 3. congruence scan: Sigma_{k+1} = P_k Sigma_k P_k^T + D_{k+1}
// ---------------------------------------------------------------------------

// Composite of maps (P, D) over a group: (P2 P1, P2 D1 P2^T + D2).  Map k is
// (P_k from the optimal-state maps, D_{k+1}).
//
// Congruence-scan levels, one warp per group: the n1^2 entries of every
// congruence over the lanes, buffers in shared memory (a thread per group
// leaves the levels latency-bound: 2^13 threads at the first level of
// T = 2^14, far fewer above, each a chain of ~2k dependent FP64 operations).
// Level maps are stored as [P (n1^2) | D (n1^2)].
__device__ __forceinline__ void wcongruence(int lane, int n1, const double* P, const double* X, const double* D,
                                            double* y, double* tmp) {
  const int m2 = n1 * n1;
  for (int e = lane; e < m2; e += 32) {
    const int i = e / n1, c = e % n1;
    double s = 0.0;
    for (int l = 0; l < n1; ++l) s = fma(P[i * n1 + l], X[l * n1 + c], s);
    tmp[e] = s;
  }
  __syncwarp();
  for (int e = lane; e < m2; e += 32) {
    const int i = e / n1, c = e % n1;
    double s = D ? D[e] : 0.0;
    for (int l = 0; l < n1; ++l) s = fma(tmp[i * n1 + l], P[c * n1 + l], s);
    y[e] = s;
  }
  __syncwarp();
}

__device__ __forceinline__ void wload_level(int lane, int n, int level0, const double* maps0, const double* D,
                                            const double* in, int64_t k, double* Pm, double* Dm) {
  const int n1 = n + 1, m2 = n1 * n1;
  for (int e = lane; e < m2; e += 32) {
    if (level0) {
      const int i = e / n1, c = e % n1;
      const double* mapk = maps0 + k * (n * n + n);
      Pm[e] = i < n ? (c < n ? mapk[i * n + c] : mapk[n * n + i]) : (c == n ? 1.0 : 0.0);
      Dm[e] = D[(k + 1) * m2 + e];
    } else {
      Pm[e] = in[k * 2 * m2 + e];
      Dm[e] = in[k * 2 * m2 + m2 + e];
    }
  }
  __syncwarp();
}

__global__ void __launch_bounds__(32) cong_reduce_warp_kernel(int n, int64_t cnt, int G, int level0,
                                                              const double* __restrict__ maps0,
                                                              const double* __restrict__ D,
                                                              const double* __restrict__ in, double* __restrict__ out) {
  __shared__ double P[AH * AH], Dc[AH * AH], Pk[AH * AH], Dk[AH * AH], t1[AH * AH], t2[AH * AH];
  const int lane = threadIdx.x;
  const int n1 = n + 1, m2 = n1 * n1;
  for (int64_t g = blockIdx.x; g * G < cnt; g += gridDim.x) {
    const int64_t first = g * G;
    const int64_t last = (first + G < cnt ? first + G : cnt) - 1;
    wload_level(lane, n, level0, maps0, D, in, first, P, Dc);
    for (int64_t k = first + 1; k <= last; ++k) {
      wload_level(lane, n, level0, maps0, D, in, k, Pk, Dk);
      // (Pk, Dk) o (P, Dc) = (Pk P, Pk Dc Pk^T + Dk)
      wcongruence(lane, n1, Pk, Dc, Dk, t1, t2);
      for (int e = lane; e < m2; e += 32) {
        Dc[e] = t1[e];
        const int i = e / n1, c = e % n1;
        double s = 0.0;
        for (int l = 0; l < n1; ++l) s = fma(Pk[i * n1 + l], P[l * n1 + c], s);
        t2[e] = s;
      }
      __syncwarp();
      for (int e = lane; e < m2; e += 32) P[e] = t2[e];
      __syncwarp();
    }
    for (int e = lane; e < m2; e += 32) {
      out[g * 2 * m2 + e] = P[e];
      out[g * 2 * m2 + m2 + e] = Dc[e];
    }
    __syncwarp();
  }
}

__global__ void __launch_bounds__(32) cong_down_warp_kernel(int n, int64_t cnt, int G, int level0,
                                                            const double* __restrict__ maps0,
                                                            const double* __restrict__ D,
                                                            const double* __restrict__ in,
                                                            const double* __restrict__ above,
                                                            const double* __restrict__ init,
                                                            double* __restrict__ states) {
  __shared__ double X[AH * AH], P[AH * AH], Dk[AH * AH], y[AH * AH], t[AH * AH];
  const int lane = threadIdx.x;
  const int n1 = n + 1, m2 = n1 * n1;
  for (int64_t g = blockIdx.x; g * G < cnt; g += gridDim.x) {
    const int64_t first = g * G;
    const int64_t last = (first + G < cnt ? first + G : cnt) - 1;
    const double* xs = above ? above + g * m2 : init;
    for (int e = lane; e < m2; e += 32) X[e] = xs[e];
    __syncwarp();
    for (int64_t k = first; k <= last; ++k) {
      for (int e = lane; e < m2; e += 32) states[k * m2 + e] = X[e];
      wload_level(lane, n, level0, maps0, D, in, k, P, Dk);
      wcongruence(lane, n1, P, X, Dk, y, t);
      for (int e = lane; e < m2; e += 32) X[e] = y[e];
      __syncwarp();
    }
    if (last == cnt - 1)
      for (int e = lane; e < m2; e += 32) states[cnt * m2 + e] = X[e];
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// 4. element adjoint from the value adjoint
// ---------------------------------------------------------------------------

struct ElemAdjArgs {
  int n;
  int64_t T;
  const double *S, *v, *maps, *Sigma;  // Sigma [T+1][n1^2]
  const double* emap;                   // [T][fe] map-adjoint terms of element k
  double* ebar_out;                     // [T+1][fe]
  const double *Xf, *rf;                // terminal (Hf = I)
  double *gXf, *grf;                    // may be null
};

__global__ void elem_adjoint_kernel(ElemAdjArgs a) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k > a.T) return;
  const int n = a.n, n1 = n + 1, nn = n * n, fs = fe_size(n);
  const double* Sg = a.Sigma + k * n1 * n1;
  double Sb[AN * AN], vb[AN];
  for (int i = 0; i < n; ++i)
    for (int c = 0; c < n; ++c) Sb[i * n + c] = Sg[i * n1 + c];
  for (int i = 0; i < n; ++i) vb[i] = -(Sg[i * n1 + n] + Sg[n * n1 + i]);
  const double zb = 2.0 * Sg[n * n1 + n];
  double* out = a.ebar_out + k * fs;
  FE O = fe_view(n, out);
  if (k < a.T) {
    const FE Mterm = fe_view(n, const_cast<double*>(a.emap) + k * fs);
    for (int i = 0; i < nn; ++i) {
      O.A[i] = Mterm.A[i];
      O.C[i] = Mterm.C[i];
    }
    for (int i = 0; i < n; ++i) O.b[i] = Mterm.b[i];
  } else {
    for (int i = 0; i < nn; ++i) { O.A[i] = 0.0; O.C[i] = 0.0; }
    for (int i = 0; i < n; ++i) O.b[i] = 0.0;
  }
  for (int i = 0; i < nn; ++i) O.J[i] = Sb[i];
  for (int i = 0; i < n; ++i) O.eta[i] = vb[i];
  *O.z = zb;
  if (k == a.T) {
    // terminal element: J = Xf, eta = Xf rf, zeta = rf'Xf rf / 2 (Hf = I)
    if (a.gXf) {
      for (int i = 0; i < n; ++i)
        for (int c = 0; c < n; ++c) {
          double g = Sb[i * n + c];
          if (a.rf) g += vb[i] * a.rf[c] + 0.5 * zb * a.rf[i] * a.rf[c];
          a.gXf[i * n + c] = g;
        }
    }
    if (a.grf) {
      for (int i = 0; i < n; ++i) {
        double s = 0.0;
        for (int l = 0; l < n; ++l) s = fma(a.Xf[l * n + i], vb[l], s);
        if (a.rf)
          for (int l = 0; l < n; ++l) s += 0.5 * zb * (a.Xf[i * n + l] + a.Xf[l * n + i]) * a.rf[l];
        a.grf[i] = s;
      }
    }
    return;
  }
  // value-combination terms (Lambda = S_{k+1} Psi_k, l = S_{k+1} alpha_k - v_{k+1})
  const double* mk = a.maps + k * (nn + n);
  const double* S1 = a.S + (k + 1) * nn;
  const double* v1 = a.v + (k + 1) * n;
  double Lam[AN * AN], l[AN], LS[AN * AN], Lv[AN];
  mm(n, S1, mk, Lam);
  mv(n, S1, mk + nn, l);
  for (int i = 0; i < n; ++i) l[i] -= v1[i];
  mm(n, Lam, Sb, LS);
  mv(n, Lam, vb, Lv);
  for (int i = 0; i < n; ++i) {
    for (int c = 0; c < n; ++c) O.A[i * n + c] += 2.0 * LS[i * n + c] - l[i] * vb[c];
    O.b[i] += -Lv[i] + zb * l[i];
  }
  // Cbar += -Lambda Sbar Lambda^T + (Lv l^T + l Lv^T)/2 - zetabar l l^T / 2
  for (int i = 0; i < n; ++i)
    for (int c = 0; c < n; ++c) {
      double s = 0.0;
      for (int q = 0; q < n; ++q) s = fma(LS[i * n + q], Lam[c * n + q], s);
      O.C[i * n + c] += -s + 0.5 * (Lv[i] * l[c] + l[i] * Lv[c]) - 0.5 * zb * l[i] * l[c];
    }
}

// ---------------------------------------------------------------------------
// 5. discrete adjoint of the RK4 element build, per sub-interval
// ---------------------------------------------------------------------------

// Full-matrix right-hand side (c = 0):
//   G = B J, beta = B eta
//   dA = A G - A F, db = -A beta, dC = sym(-A B A^T), deta = -q - F^T eta + J beta,
//   dJ = sym(-Q - J F - F^T J + J G), dz = -rho/2 + eta^T beta / 2
// whose vector-Jacobian product the reverse sweep evaluates at every stored
// stage input; one warp per sub-interval (below).

struct RK4AdjArgs {
  int n, K, M;
  int64_t T;
  const double* t;
  Coefs cf;
  const double* X;      // X samples (H = I), CONST or PER_INTERVAL
  int32_t X_mode;
  const double* r;      // may be null
  int32_t r_mode;
  const double* ebar;   // [T+1][fe]
  int64_t j0;           // this launch covers sub-intervals j0 .. j0 + T - 1 (T counts the segment)
  double* ys;           // scratch [T][K][4][fe]: the segment's RK4 stage inputs, recomputed for it
  // per-sub-interval partials
  double *pF, *pB, *pX;  // [T][n^2]
  double* pr;            // [T][2K+1][n] (per stage sample) or null
};

// One warp per sub-interval: one thread per sub-interval would leave the FP64
// pipe mostly idle at the adjoint workload's size (2^14 sub-intervals = 512
// warps for 608 sub-partitions, each a long dependent chain with its matrices
// in local memory).  A warp owns a sub-interval: every matrix product spreads
// its n^2 outputs over the 32 lanes and all buffers live in shared memory.

namespace warp {

__device__ __forceinline__ void sync() { __syncwarp(); }

// c = a b, c = a^T b, c = a b^T  (n x n, lanes over the outputs)
__device__ __forceinline__ void mm(int lane, int n, const double* a, const double* b, double* c) {
  for (int e = lane; e < n * n; e += 32) {
    const int i = e / n, j = e % n;
    double s = 0.0;
    for (int l = 0; l < n; ++l) s = fma(a[i * n + l], b[l * n + j], s);
    c[e] = s;
  }
  sync();
}
__device__ __forceinline__ void mtm(int lane, int n, const double* a, const double* b, double* c) {
  for (int e = lane; e < n * n; e += 32) {
    const int i = e / n, j = e % n;
    double s = 0.0;
    for (int l = 0; l < n; ++l) s = fma(a[l * n + i], b[l * n + j], s);
    c[e] = s;
  }
  sync();
}
__device__ __forceinline__ void mmt(int lane, int n, const double* a, const double* b, double* c) {
  for (int e = lane; e < n * n; e += 32) {
    const int i = e / n, j = e % n;
    double s = 0.0;
    for (int l = 0; l < n; ++l) s = fma(a[i * n + l], b[j * n + l], s);
    c[e] = s;
  }
  sync();
}
// c += a b or c -= a b, with a and / or b read transposed (TA, TB): the
// product accumulated onto c's entries directly (no temporary, no separate
// pass of adds).
template <bool TA, bool TB, bool SUB>
__device__ __forceinline__ void mm_acc(int lane, int n, const double* a, const double* b, double* c) {
  for (int e = lane; e < n * n; e += 32) {
    const int i = e / n, j = e % n;
    double s = c[e];
    for (int l = 0; l < n; ++l) {
      const double av = TA ? a[l * n + i] : a[i * n + l];
      const double bv = TB ? b[j * n + l] : b[l * n + j];
      s = fma(SUB ? -av : av, bv, s);
    }
    c[e] = s;
  }
  sync();
}
// y = a x, y = a^T x (n <= 8): four lanes per output, each summing every
// fourth column, then two butterfly steps, so that the warp's FP64
// instructions run with all lanes rather than n of them.
template <bool kTrans>
__device__ __forceinline__ void mv4(int lane, int n, const double* a, const double* x, double* y) {
  const int i = lane >> 2, q = lane & 3;
  double s = 0.0;
  if (i < n)
    for (int l = q; l < n; l += 4) s = fma(kTrans ? a[l * n + i] : a[i * n + l], x[l], s);
  s += __shfl_xor_sync(0xffffffffu, s, 1);
  s += __shfl_xor_sync(0xffffffffu, s, 2);
  if (i < n && q == 0) y[i] = s;
  sync();
}
__device__ __forceinline__ void mv(int lane, int n, const double* a, const double* x, double* y) {
  mv4<false>(lane, n, a, x, y);
}
__device__ __forceinline__ void mtv(int lane, int n, const double* a, const double* x, double* y) {
  mv4<true>(lane, n, a, x, y);
}
// a <- (a + a^T) / 2  (n <= 8: at most two entries per lane; every lane runs
// the same iterations so that the warp barrier is reached by all)
__device__ __forceinline__ void symm(int lane, int n, double* a) {
  double v[(AN * AN + 31) / 32];
#pragma unroll
  for (int it = 0; it < (AN * AN + 31) / 32; ++it) {
    const int e = lane + 32 * it;
    const int i = e / n, j = e % n;
    v[it] = (e < n * n && i < j) ? 0.5 * (a[i * n + j] + a[j * n + i]) : 0.0;
  }
  sync();
#pragma unroll
  for (int it = 0; it < (AN * AN + 31) / 32; ++it) {
    const int e = lane + 32 * it;
    const int i = e / n, j = e % n;
    if (e < n * n && i < j) {
      a[i * n + j] = v[it];
      a[j * n + i] = v[it];
    }
  }
  sync();
}

// Buffers of one RHS evaluation: t1, t2, t3 (n^2 each), vectors beta, betab,
// Fe, Jb (n each), JG (n^2).
struct Tmp {
  double *t1, *t2, *t3, *JG, *beta, *betab, *v1, *v2;
};

// Vector-Jacobian product of the full-matrix right-hand side at y with output adjoint kb (its C, J
// parts symmetrised first), accumulated into yb and the coefficient adjoints;
// lanes over entries: Fb, Bb, Qb accumulate entry-wise (each lane owns the same
// entries throughout), qb, rhob by lanes < n and lane 0.
__device__ void rhs_vjp(int lane, int n, const double* y, const double* F, const double* B, double* kb, double* yb,
                        double* Fb, double* Bb, double* Qb, double* qb, double* rhob, const Tmp& t) {
  const int nn = n * n;
  FE Y = fe_view(n, const_cast<double*>(y)), Kb = fe_view(n, kb), YB = fe_view(n, yb);
  symm(lane, n, Kb.C);
  symm(lane, n, Kb.J);
  mv(lane, n, B, Y.eta, t.beta);
  if (lane < n) t.betab[lane] = 0.0;
  mm(lane, n, B, Y.J, t.t1);  // G = B J
  for (int e = lane; e < nn; e += 32) t.t2[e] = t.t1[e] - F[e];
  sync();
  mm_acc<false, true, false>(lane, n, Kb.A, t.t2, YB.A);
  mtm(lane, n, Y.A, Kb.A, t.t3);  // Gbar
  for (int e = lane; e < nn; e += 32) Fb[e] -= t.t3[e];
  sync();
  mm_acc<false, true, false>(lane, n, t.t3, Y.J, Bb);
  mm_acc<true, false, false>(lane, n, B, t.t3, YB.J);
  for (int e = lane; e < nn; e += 32) {
    const int i = e / n, c = e % n;
    YB.A[e] -= Kb.b[i] * t.beta[c];
  }
  sync();
  mtv(lane, n, Y.A, Kb.b, t.v1);
  if (lane < n) t.betab[lane] -= t.v1[lane];
  mm(lane, n, Kb.C, Y.A, t.t2);
  mm(lane, n, t.t2, B, t.t3);
  for (int e = lane; e < nn; e += 32) YB.A[e] -= 2.0 * t.t3[e];
  sync();
  mm_acc<true, false, true>(lane, n, Y.A, t.t2, Bb);
  for (int e = lane; e < nn; e += 32) {
    const int i = e / n, c = e % n;
    Fb[e] -= Y.eta[i] * Kb.eta[c];
    YB.J[e] += Kb.eta[i] * t.beta[c];
  }
  if (lane < n) qb[lane] -= Kb.eta[lane];
  sync();
  mv(lane, n, F, Kb.eta, t.v1);
  mtv(lane, n, Y.J, Kb.eta, t.v2);
  if (lane < n) {
    YB.eta[lane] -= t.v1[lane];
    t.betab[lane] += t.v2[lane];
  }
  for (int e = lane; e < nn; e += 32) Qb[e] -= Kb.J[e];
  sync();
  // Kb.J F^T + F Kb.J = X + X^T with X = Kb.J F^T (Kb.J symmetric)
  mmt(lane, n, Kb.J, F, t.t2);
  for (int e = lane; e < nn; e += 32) {
    const int i = e / n, c = e % n;
    YB.J[e] -= t.t2[i * n + c] + t.t2[c * n + i];
  }
  sync();
  mm_acc<false, true, false>(lane, n, Kb.J, t.t1, YB.J);
  // Gbar2 = J^T Kb.J, which is also J Kb.J^T term by term: the stage input's
  // J is built symmetric and Kb.J was symmetrised above
  mtm(lane, n, Y.J, Kb.J, t.t3);
  for (int e = lane; e < nn; e += 32) Fb[e] -= 2.0 * t.t3[e];
  sync();
  mm_acc<false, true, false>(lane, n, t.t3, Y.J, Bb);
  mm_acc<true, false, false>(lane, n, B, t.t3, YB.J);
  const double zb = *Kb.z;
  if (lane == 0) *rhob -= 0.5 * zb;
  if (lane < n) {
    YB.eta[lane] += 0.5 * zb * t.beta[lane];
    t.betab[lane] += 0.5 * zb * Y.eta[lane];
  }
  sync();
  for (int e = lane; e < nn; e += 32) {
    const int i = e / n, c = e % n;
    Bb[e] += t.betab[i] * Y.eta[c];
  }
  mtv(lane, n, B, t.betab, t.v1);
  if (lane < n) YB.eta[lane] += t.v1[lane];
  sync();
}

}  // namespace warp

// Shared-memory doubles of one warp of rk4_adjoint_warp_kernel: five element
// buffers, B, Fb, Bb, Qb, the temporaries, and the per-sample q, rho adjoints.
__host__ __device__ constexpr int rk4w_smem_doubles() {
  return 5 * AS + 8 * AN * AN + 4 * AN + (2 * 8 + 1) * AN + (2 * 8 + 1) + 8;
}

__global__ void __launch_bounds__(32, 15) rk4_adjoint_warp_kernel(RK4AdjArgs a) {
  extern __shared__ double sm[];
  const int lane = threadIdx.x;
  const int n = a.n, nn = n * n, fs = fe_size(n), K = a.K, M = a.M;
  // y (a stage input), yb (the state adjoint), kb (one stage's output
  // adjoint), acc (its input adjoint), kbs (the step's output adjoint)
  double* y = sm;
  double* yb = y + AS;
  double* kb = yb + AS;
  double* acc = kb + AS;
  double* kbs = acc + AS;
  double* B = kbs + AS;
  double* Fb = B + AN * AN;
  double* Bb = Fb + AN * AN;
  double* Qb = Bb + AN * AN;
  warp::Tmp tmp;
  tmp.t1 = Qb + AN * AN;
  tmp.t2 = tmp.t1 + AN * AN;
  tmp.t3 = tmp.t2 + AN * AN;
  tmp.JG = tmp.t3 + AN * AN;
  tmp.beta = tmp.JG + AN * AN;
  tmp.betab = tmp.beta + AN;
  tmp.v1 = tmp.betab + AN;
  tmp.v2 = tmp.v1 + AN;
  double* qb = tmp.v2 + AN;          // [(2K+1) n]
  double* rhob = qb + (2 * 8 + 1) * AN;  // [2K+1]
  for (int64_t jj = blockIdx.x; jj < a.T; jj += gridDim.x) {
    const int64_t j = a.j0 + jj;
    const double h = (a.t[j + 1] - a.t[j]) / K;
    const double* F = a.cf.F.ptr + sample_index(a.cf.F.mode, j, 0, K) * nn;
    const double* Lt = a.cf.Lt.ptr + sample_index(a.cf.Lt.mode, j, 0, K) * n * M;
    const double* Q = a.X + sample_index(a.X_mode, j, 0, K) * nn;
    for (int e = lane; e < nn; e += 32) {
      const int i = e / n, c = e % n;
      double s = 0.0;
      for (int l = 0; l < M; ++l) s = fma(Lt[i * M + l], Lt[c * M + l], s);
      B[e] = s;
      Fb[e] = 0.0;
      Bb[e] = 0.0;
      Qb[e] = 0.0;
    }
    for (int e = lane; e < (2 * K + 1) * n; e += 32) qb[e] = 0.0;
    for (int e = lane; e <= 2 * K; e += 32) rhob[e] = 0.0;
    warp::sync();
    // the four stage inputs of every RK4 step, recomputed for this segment
    // (build_stages_kernel) from the sub-interval's fixed initial condition
    const double* ysj = a.ys + jj * (int64_t)K * 4 * fs;
    // adjoint
    const double* eb = a.ebar + j * fs;
    for (int e = lane; e < fs; e += 32) yb[e] = eb[e];
    warp::sync();
    auto load_stage = [&](const double* src) {
      for (int e = lane; e < fs; e += 32) y[e] = src[e];
      warp::sync();
    };
    for (int i = 0; i < K; ++i) {
      const double* st = ysj + (int64_t)i * 4 * fs;
      const int p1 = 2 * i + 2, p2 = 2 * i + 1, p3 = 2 * i;
      // y_new = y - h/6 (k1 + 2 k2 + 2 k3 + k4): stage output adjoints
      // kb4 = -h/6 yb, kb3 = -h/3 yb (+ -h acc4), kb2 = -h/3 yb (+ -h/2 acc3),
      // kb1 = -h/6 yb (+ -h/2 acc2)
      for (int e = lane; e < fs; e += 32) {
        kbs[e] = yb[e];
        kb[e] = -(h / 6.0) * yb[e];
        acc[e] = 0.0;
      }
      load_stage(st + 3 * fs);
      warp::rhs_vjp(lane, n, y, F, B, kb, acc, Fb, Bb, Qb, qb + p3 * n, rhob + p3, tmp);
      for (int e = lane; e < fs; e += 32) {
        yb[e] += acc[e];
        kb[e] = -(h / 3.0) * kbs[e] - h * acc[e];
        acc[e] = 0.0;
      }
      load_stage(st + 2 * fs);
      warp::rhs_vjp(lane, n, y, F, B, kb, acc, Fb, Bb, Qb, qb + p2 * n, rhob + p2, tmp);
      for (int e = lane; e < fs; e += 32) {
        yb[e] += acc[e];
        kb[e] = -(h / 3.0) * kbs[e] - 0.5 * h * acc[e];
        acc[e] = 0.0;
      }
      load_stage(st + fs);
      warp::rhs_vjp(lane, n, y, F, B, kb, acc, Fb, Bb, Qb, qb + p2 * n, rhob + p2, tmp);
      for (int e = lane; e < fs; e += 32) {
        yb[e] += acc[e];
        kb[e] = -(h / 6.0) * kbs[e] - 0.5 * h * acc[e];
        acc[e] = 0.0;
      }
      load_stage(st);
      warp::rhs_vjp(lane, n, y, F, B, kb, acc, Fb, Bb, Qb, qb + p1 * n, rhob + p1, tmp);
      for (int e = lane; e < fs; e += 32) yb[e] += acc[e];
      warp::sync();
    }
    // coefficient adjoints of this sub-interval:
    //   Xbar = sym(Qbar) + sum_p (qbar_p r_p^T + rhobar_p r_p r_p^T)
    //   rbar_p = X^T qbar_p + rhobar_p (X + X^T) r_p
    double* oF = a.pF + j * nn;
    double* oB = a.pB + j * nn;
    double* oX = a.pX + j * nn;
    for (int e = lane; e < nn; e += 32) {
      const int i = e / n, c = e % n;
      oF[e] = Fb[e];
      oB[e] = Bb[e];
      double x = 0.5 * (Qb[i * n + c] + Qb[c * n + i]);
      for (int p = 0; p <= 2 * K; ++p) {
        const double* rp = a.r ? a.r + sample_index(a.r_mode, j, p, K) * n : nullptr;
        if (rp) x += qb[p * n + i] * rp[c] + rhob[p] * rp[i] * rp[c];
      }
      oX[e] = x;
    }
    if (a.pr) {
      for (int e = lane; e < (2 * K + 1) * n; e += 32) {
        const int p = e / n, i = e % n;
        const double* rp = a.r ? a.r + sample_index(a.r_mode, j, p, K) * n : nullptr;
        double s = 0.0;
        for (int l = 0; l < n; ++l) s = fma(Q[l * n + i], qb[p * n + l], s);
        if (rp)
          for (int l = 0; l < n; ++l) s += rhob[p] * (Q[i * n + l] + Q[l * n + i]) * rp[l];
        a.pr[(j * (2 * K + 1) + p) * n + i] = s;
      }
    }
    warp::sync();
  }
}

// ---------------------------------------------------------------------------
// 6. reductions into the coefficient layouts
// ---------------------------------------------------------------------------

// out[s][e] = sum over sub-intervals j mapped to sample s of part[j][e]
// (mode CONST: all j; PER_INTERVAL: j = s).  One thread per (s, e); the sum
// over j runs in a fixed order (deterministic).
__global__ void reduce_partials_kernel(const double* __restrict__ part, int64_t T, int size, int32_t mode,
                                       double* __restrict__ out) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (mode == kConst) {
    // one block per entry e: tree over j
    __shared__ double red[256];
    const int e = blockIdx.x;
    if (e >= size) return;
    double s = 0.0;
    for (int64_t j = threadIdx.x; j < T; j += blockDim.x) s += part[j * size + e];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
      if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[e] = red[0];
    return;
  }
  if (idx >= T * size) return;
  out[idx] = part[idx];
}

// r per stage sample: sample s = 2Kj + p gets block j's p and, at shared
// ends, block j-1's 2K.
__global__ void reduce_stage_r_kernel(const double* __restrict__ pr, int64_t T, int K, int n, int32_t r_mode,
                                      double* __restrict__ gr) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int P = 2 * K + 1;
  if (r_mode == kPerStage) {
    const int64_t cnt = 2 * (int64_t)K * T + 1;
    if (idx >= cnt * n) return;
    const int64_t s = idx / n;
    const int i = (int)(idx % n);
    const int64_t j = s / (2 * K);
    const int p = (int)(s % (2 * K));
    double v = 0.0;
    if (j < T) v += pr[(j * P + p) * n + i];
    if (p == 0 && j >= 1) v += pr[((j - 1) * P + 2 * K) * n + i];
    gr[idx] = v;
  } else if (r_mode == kPerInterval) {
    if (idx >= T * n) return;
    const int64_t j = idx / n;
    const int i = (int)(idx % n);
    double v = 0.0;
    for (int p = 0; p < P; ++p) v += pr[(j * P + p) * n + i];
    gr[idx] = v;
  }
}

// Lbar = (Bbar + Bbar^T) L U^-1, Ubar = -U^-1 L^T sym(Bbar) L U^-1 per sample of the
// B layout (CONST or PER_INTERVAL, L and U in that same layout or CONST).
__global__ void b_to_lu_kernel(int n, int m, int64_t cnt, const double* __restrict__ Bb, const double* __restrict__ L,
                               int32_t L_mode, const double* __restrict__ U, int32_t U_mode, int K,
                               double* __restrict__ gL, double* __restrict__ gU) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= cnt) return;
  const double* Ls = L + sample_index(L_mode, s, 0, K) * n * m;
  const double* Us = U + sample_index(U_mode, s, 0, K) * m * m;
  const double* Bs = Bb + s * n * n;
  // G = L U^-1  (n x m): solve U^T G^T = L^T, U symmetric -> G^T = U^-1 L^T
  double W[16 * 16], R[16 * AN];
  for (int i = 0; i < m * m; ++i) W[i] = Us[i];
  for (int i = 0; i < m; ++i)
    for (int c = 0; c < n; ++c) R[i * n + c] = Ls[c * m + i];
  solve_rt(m, n, W, R, false);  // R = U^-1 L^T  (m x n)
  // Lbar = (Bbar + Bbar^T) G, G = R^T (n x m)
  for (int i = 0; i < n; ++i)
    for (int c = 0; c < m; ++c) {
      double sum = 0.0;
      for (int l = 0; l < n; ++l) sum = fma(Bs[i * n + l] + Bs[l * n + i], R[c * n + l], sum);
      gL[s * n * m + i * m + c] = sum;
    }
  // Ubar = -R sym(Bbar) R^T
  for (int i = 0; i < m; ++i)
    for (int c = 0; c < m; ++c) {
      double sum = 0.0;
      for (int l = 0; l < n; ++l) {
        double t = 0.0;
        for (int q = 0; q < n; ++q) t = fma(0.5 * (Bs[l * n + q] + Bs[q * n + l]), R[c * n + q], t);
        sum = fma(R[i * n + l], t, sum);
      }
      gU[s * m * m + i * m + c] = -sum;
    }
}

// ---------------------------------------------------------------------------
// host driver
// ---------------------------------------------------------------------------

// Congruence scan Sigma_{k+1} = P_k Sigma_k P_k^T + D_{k+1}, k = 0..T-1, from
// Sigma_0 = D_0: level 0 reads P_k from the optimal-state maps, upper levels
// hold composites; pairs above level 0.
static void cong_scan(int n, int64_t T, const double* maps0, const double* D, double* Sigma, char* ws, size_t& off,
                      cudaStream_t st) {
  const int m2 = (n + 1) * (n + 1);
  const int G = 2;
  int nlev = 0;
  int64_t c[64];
  double* lv[64];
  double* sv[64];
  int64_t mc = T;
  while (mc > G) {
    const int64_t nc = cdiv(mc, G);
    double* out = (double*)(ws + off);
    off = al(off + nc * 2 * m2 * sizeof(double));
    cong_reduce_warp_kernel<<<(unsigned)(nc < 152 * 32 ? nc : 152 * 32), 32, 0, st>>>(
        n, mc, G, nlev == 0, maps0, D, nlev ? lv[nlev - 1] : nullptr, out);
    count_launch();
    c[nlev] = nc;
    lv[nlev] = out;
    sv[nlev] = (double*)(ws + off);
    off = al(off + (nc + 1) * m2 * sizeof(double));
    mc = nc;
    ++nlev;
  }
  // top level: one group
  {
    const int64_t tc = nlev ? c[nlev - 1] : T;
    double* tst = nlev ? sv[nlev - 1] : Sigma;
    cong_down_warp_kernel<<<1, 32, 0, st>>>(n, tc, (int)tc, nlev == 0, maps0, D, nlev ? lv[nlev - 1] : nullptr,
                                            nullptr, D, tst);
    count_launch();
  }
  for (int l = nlev - 1; l >= 0; --l) {
    const int64_t cnt = (l == 0) ? T : c[l - 1];
    double* out = (l == 0) ? Sigma : sv[l - 1];
    const int64_t groups = cdiv(cnt, G);
    cong_down_warp_kernel<<<(unsigned)(groups < 152 * 32 ? groups : 152 * 32), 32, 0, st>>>(
        n, cnt, G, l == 0, maps0, D, l == 0 ? nullptr : lv[l - 1], sv[l], D, out);
    count_launch();
  }
}

struct BackwardPlan {
  size_t coef, elems, maps, rmaps, ystates, affine, D, emap, Sigma, cong, ebar, ys, pF, pB, pX, pr, gB, gLt, gUt,
      end;
};

// The RK4 adjoint runs over segments of sub-intervals: the stage inputs it
// differentiates are recomputed per segment from every sub-interval's fixed
// initial condition (A = I, the rest 0; Theorem Backward_HJB_LQT's boundary,
// eq. abcej_boundary), so their storage is one segment's, not T's.  A segment
// of 2^15 sub-intervals keeps the stage-recording build (one thread per
// sub-interval: 1024 warps) filling every sub-partition; a shorter one left
// most of them idle (2280 sub-intervals per segment made the backward pass
// 2.5x slower at T = 2^14).  Up to one segment, the stages come from the same
// build as the elements.
constexpr int64_t kAdjSegment = 1 << 15;
static int64_t adjoint_segment(int64_t T) { return T < kAdjSegment ? T : kAdjSegment; }

static BackwardPlan backward_plan(const lqt_problem& p, const Layout& L, size_t elem_bytes) {
  BackwardPlan b{};
  const size_t n = p.n, T = p.T, T1 = T + 1, K = p.K, m = p.m, fs = 3 * n * n + 2 * n + 1, m2 = (n + 1) * (n + 1);
  size_t off = 0;
  b.coef = off; off = al(off + L.coef_bytes);
  b.elems = off; off = al(off + elem_bytes);
  b.maps = off; off = al(off + T * (n * n + n) * 8);
  b.rmaps = off; off = al(off + T * (n * n + n) * 8);
  b.ystates = off; off = al(off + T1 * n * 8);
  b.affine = off; off = al(off + affine_scan_bytes(p.n, T) + 256);
  b.D = off; off = al(off + T1 * m2 * 8);
  b.emap = off; off = al(off + T * fs * 8);
  b.Sigma = off; off = al(off + T1 * m2 * 8);
  b.cong = off;
  {
    int64_t mc = T;
    size_t c = 0;
    while (mc > 2) { const int64_t nc = cdiv(mc, 2); c = al(c + nc * 2 * m2 * 8); c = al(c + (nc + 1) * m2 * 8); mc = nc; }
    off = al(off + c);
  }
  b.ebar = off; off = al(off + T1 * fs * 8);
  b.ys = off; off = al(off + (size_t)adjoint_segment(p.T) * K * 4 * fs * 8);
  b.pF = off; off = al(off + T * n * n * 8);
  b.pB = off; off = al(off + T * n * n * 8);
  b.pX = off; off = al(off + T * n * n * 8);
  b.pr = off; off = al(off + T * (2 * K + 1) * n * 8);
  const size_t nLt = (size_t)sample_count(L.mode_Lt, p.T, p.K);
  b.gB = off; off = al(off + nLt * n * n * 8);
  b.gLt = off; off = al(off + nLt * n * m * 8);
  b.gUt = off; off = al(off + nLt * m * m * 8);
  b.end = off;
  return b;
}

size_t backward_workspace_bytes(const lqt_problem& p, const Layout& L, size_t elem_bytes) {
  return backward_plan(p, L, elem_bytes).end;
}

static unsigned nb(int64_t threads, int bs) { return (unsigned)cdiv(threads > 0 ? threads : 1, bs); }

cudaError_t run_backward(const lqt_problem& p, const Layout& L, size_t elem_bytes, const double* x0, const double* S,
                         const double* v, const double* x, const double* gS, const double* gv, const double* gz,
                         const double* gx, double g_cost, double* gF, double* gL, double* gX, double* gU, double* gr,
                         double* gXf, double* grf, double* gx0, char* ws, cudaStream_t st) {
  const BackwardPlan b = backward_plan(p, L, elem_bytes);
  const int n = p.n, K = p.K, m = p.m;
  const int64_t T = p.T;
  const int fs = 3 * n * n + 2 * n + 1, m2 = (n + 1) * (n + 1);
  Coefs cf;
  cudaError_t e = launch_prepare_coefs(p, L, ws + b.coef, cf, st);
  if (e != cudaSuccess) return e;
  ElemPtrs el = carve_elements_at(p, ws + b.elems);
  // the elements; with T beyond one segment the RK4 stage inputs for step 5
  // are recomputed there, segment by segment
  const bool one_segment = T <= adjoint_segment(T) && T <= kAdjSegment;
  if (one_segment) {
    e = launch_build_stages_range(p, L, cf, 0, T, (double*)(ws + b.ys), st, el);
    if (e == cudaSuccess) e = launch_terminal_element(p, el, st);
  } else {
    e = launch_build(p, L, cf, el, st);
  }
  if (e != cudaSuccess) return e;
  double* maps = (double*)(ws + b.maps);
  e = launch_maps_from_values(p, el, S, v, maps, st);
  if (e != cudaSuccess) return e;
  // 1. state adjoint
  double* rmaps = (double*)(ws + b.rmaps);
  double* ystates = (double*)(ws + b.ystates);
  reversed_adjoint_maps_kernel<<<nb(T, 128), 128, 0, st>>>(n, T, maps, gx, rmaps);
  count_launch();
  size_t aoff = b.affine;
  const double* x_in = gx ? gx + T * n : nullptr;
  if (!x_in) {  // no state gradient: start the recurrence from a zero vector
    double* zero = (double*)(ws + aoff);
    aoff = al(aoff + n * sizeof(double));
    if (cudaMemsetAsync(zero, 0, n * sizeof(double), st) != cudaSuccess) return cudaGetLastError();
    x_in = zero;
  }
  e = affine_scan_states(n, rmaps, T, x_in, ystates, ws, aoff, st);
  if (e != cudaSuccess) return e;
  // 2. map adjoint + direct value terms
  MapAdjArgs ma;
  ma.n = n; ma.T = T; ma.el = el; ma.S = S; ma.v = v; ma.x = x; ma.xbar_rev = ystates;
  ma.gS = gS; ma.gv = gv; ma.gz = gz; ma.x0 = x0; ma.g_cost = g_cost;
  ma.D = (double*)(ws + b.D); ma.emap = (double*)(ws + b.emap); ma.gx0 = gx0;
  map_adjoint_kernel<<<nb(T + 1, 64), 64, 0, st>>>(ma);
  count_launch();
  // 3. value adjoint (congruence scan)
  double* Sigma = (double*)(ws + b.Sigma);
  size_t coff = b.cong;
  cong_scan(n, T, maps, ma.D, Sigma, ws, coff, st);
  // 4. element adjoint
  ElemAdjArgs ea;
  ea.n = n; ea.T = T; ea.S = S; ea.v = v; ea.maps = maps; ea.Sigma = Sigma; ea.emap = ma.emap;
  ea.ebar_out = (double*)(ws + b.ebar); ea.Xf = p.Xf; ea.rf = p.rf; ea.gXf = gXf; ea.grf = grf;
  elem_adjoint_kernel<<<nb(T + 1, 64), 64, 0, st>>>(ea);
  count_launch();
  // 5. RK4 adjoint
  RK4AdjArgs ra;
  ra.n = n; ra.K = K; ra.M = cf.M; ra.T = T; ra.t = p.t; ra.cf = cf; ra.X = p.X.ptr; ra.X_mode = p.X.mode;
  ra.r = p.r.ptr; ra.r_mode = p.r.mode; ra.ebar = ea.ebar_out; ra.ys = (double*)(ws + b.ys);
  ra.pF = (double*)(ws + b.pF); ra.pB = (double*)(ws + b.pB); ra.pX = (double*)(ws + b.pX);
  ra.pr = (double*)(ws + b.pr);
  {
    const size_t smem = rk4w_smem_doubles() * sizeof(double);
    cudaFuncSetAttribute(rk4_adjoint_warp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    // 14 KB of shared memory per warp (+1 KB reserved per CTA): 15 warps per
    // SM, one segment per wave
    const int64_t seg = adjoint_segment(T);
    for (int64_t j0 = 0; j0 < T; j0 += seg) {
      const int64_t cnt = T - j0 < seg ? T - j0 : seg;
      if (!one_segment) {
        e = launch_build_stages_range(p, L, cf, j0, cnt, ra.ys, st, ElemPtrs{});
        if (e != cudaSuccess) return e;
      }
      ra.j0 = j0;
      ra.T = cnt;
      const int64_t grid = cnt < 152 * 15 ? cnt : 152 * 15;
      rk4_adjoint_warp_kernel<<<(unsigned)grid, 32, smem, st>>>(ra);
      count_launch();
    }
    ra.T = T;
  }
  // 6. reductions
  auto reduce = [&](const double* part, int64_t rows, int size, int32_t mode, double* out) {
    if (!out) return;
    if (mode == kConst) {
      reduce_partials_kernel<<<size, 256, 0, st>>>(part, rows, size, kConst, out);
    } else {
      reduce_partials_kernel<<<nb(rows * size, 256), 256, 0, st>>>(part, rows, size, mode, out);
    }
    count_launch();
  };
  reduce(ra.pF, T, n * n, p.F.mode, gF);
  reduce(ra.pX, T, n * n, p.X.mode, gX);
  if (gr && p.r.ptr) {
    if (p.r.mode == kConst) {
      reduce(ra.pr, T * (2 * K + 1), n, kConst, gr);
    } else {
      const int64_t cnt = (p.r.mode == kPerStage ? 2 * (int64_t)K * T + 1 : T) * n;
      reduce_stage_r_kernel<<<nb(cnt, 256), 256, 0, st>>>(ra.pr, T, K, n, p.r.mode, gr);
      count_launch();
    }
  }
  if (gL || gU) {
    const int64_t nLt = sample_count(L.mode_Lt, T, K);
    double* gB = (double*)(ws + b.gB);
    reduce(ra.pB, T, n * n, L.mode_Lt, gB);
    double* gLt = (double*)(ws + b.gLt);
    double* gUt = (double*)(ws + b.gUt);
    b_to_lu_kernel<<<nb(nLt, 64), 64, 0, st>>>(n, m, nLt, gB, p.L.ptr, p.L.mode, p.U.ptr, p.U.mode, K, gLt, gUt);
    count_launch();
    reduce(gLt, nLt, n * m, p.L.mode == L.mode_Lt ? kPerInterval : kConst, gL);
    reduce(gUt, nLt, m * m, p.U.mode == L.mode_Lt ? kPerInterval : kConst, gU);
  }
  (void)fs;
  (void)m2;
  return cudaGetLastError();
}

}  // namespace lqt
