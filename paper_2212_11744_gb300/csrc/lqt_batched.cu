// Batches of independent LQT problems of one state dimension in one call.
//
// The problems are laid end to end: problem b's T_b + 1 elements (its
// sub-intervals and its terminal element) occupy boundaries
// [off_b, off_b + T_b] of one long sequence.  One value scan over the whole
// sequence then solves every problem at once, because a terminal element has
// A = b = C = 0 (Sec. IV-D, eq. LQT_final_initialisation): combining it with
// whatever lies to its right gives its own J and eta exactly, so S and v never
// leak across problems.  Only the state-free term zeta does leak, additively
// (the combination adds zeta_1 + zeta_2 when z0 = 0): the scan's running zeta
// at a boundary of problem b carries the zeta of every later problem, and
// removing that sum by a subtraction would leave its rounding (~1e-12 of a
// batch's total) in values that are small near a problem's end.  So the
// level-0 down-sweep of a batch writes each boundary's own share of zeta
// (zeta_k - zeta_{k+1}, as the combination forms it, without a subtraction)
// and a segmented suffix sum per problem adds them up.  For the states, the
// map at each problem's last boundary is replaced by x -> x0 of the next
// problem before the affine scan.  The controls and per-problem costs are
// evaluated last, with each problem's own U^-1 L^T.
#include <cstring>
#include <vector>

#include <cuda_runtime.h>

#include "lqt_internal.h"

namespace lqt {

static size_t bal(size_t x) { return (x + 255) & ~(size_t)255; }

// zeta_k = sum over j >= k of problem b of the shares left in zeta by the
// level-0 down-sweep: one warp per problem, 32 boundaries at a time from the
// problem's end (lane l holds boundary hi - l), a warp prefix sum over the
// lanes plus the carry from the boundaries after them.
__global__ void zeta_suffix_kernel(BatchDev bd, double* zeta) {
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= bd.B) return;  // uniform over the warp
  const int64_t first = bd.off[w], last = bd.off[w + 1] - 1;
  double carry = 0.0;
  for (int64_t hi = last; hi >= first; hi -= 32) {
    const int64_t k = hi - lane;
    double x = (k >= first) ? zeta[k] : 0.0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const double y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    x += carry;
    if (k >= first) zeta[k] = x;
    carry = __shfl_sync(0xffffffffu, x, 31);
  }
}

// The same with one warp per boundary (8 <= n <= 32): lane i < n forms row i of
// e = v - S x (consecutive lanes read consecutive entries of S's rows as the
// loop runs over the columns), then lane q < m forms u_q from e by shuffles;
// one thread per boundary would read S_g with a 2 KB stride between lanes.
__global__ void controls_cost_warp_kernel(BatchDev bd, const double* S, const double* v, const double* zeta,
                                          const double* x, double* u, double* cost) {
  const int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (g >= bd.total) return;  // uniform over the warp
  const int n = bd.n, m = bd.m;
  const int32_t b = batch_find(bd.off, bd.B, g);
  const BatchProb& P = bd.probs[b];
  const double* Sg = S + g * n * n;
  const double* vg = v + g * n;
  const double* xg = x + g * n;
  double sx = 0.0;
  if (lane < n)
    for (int l = 0; l < n; ++l) sx = fma(Sg[lane * n + l], xg[l], sx);
  const double xi = lane < n ? xg[lane] : 0.0;
  const double vi = lane < n ? vg[lane] : 0.0;
  const double e = vi - sx;
  if (u) {
    const double* Ku = P.cf.Ku;
    double s = 0.0;
    for (int i = 0; i < n; ++i) {
      const double ei = __shfl_sync(0xffffffffu, e, i);
      if (lane < m) s = fma(Ku[lane * n + i], ei, s);
    }
    if (lane < m) u[g * m + lane] = s;
  }
  if (cost && g == P.off) {
    double c = lane < n ? xi * fma(0.5, sx, -vi) : 0.0;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) cost[b] = zeta[g] + c;
  }
}

// u_g = U_b^-1 L_b^T (v_g - S_g x_g); cost_b at the first boundary of b.
__global__ void controls_cost_kernel(BatchDev bd, const double* S, const double* v, const double* zeta,
                                     const double* x, double* u, double* cost) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= bd.total) return;
  const int n = bd.n, m = bd.m;
  const int32_t b = batch_find(bd.off, bd.B, g);
  const BatchProb& P = bd.probs[b];
  const double* Sg = S + g * n * n;
  const double* vg = v + g * n;
  const double* xg = x + g * n;
  if (u) {
    const double* Ku = P.cf.Ku;
    for (int q = 0; q < m; ++q) {
      double s = 0.0;
      for (int i = 0; i < n; ++i) {
        double e = vg[i];
        for (int l = 0; l < n; ++l) e = fma(-Sg[i * n + l], xg[l], e);
        s = fma(Ku[q * n + i], e, s);
      }
      u[g * m + q] = s;
    }
  }
  if (cost && g == P.off) {
    double c = zeta[g];
    for (int i = 0; i < n; ++i) {
      double s = 0.0;
      for (int l = 0; l < n; ++l) s = fma(Sg[i * n + l], xg[l], s);
      c = fma(xg[i], fma(0.5, s, -vg[i]), c);
    }
    cost[b] = c;
  }
}

// Workspace layout of a batch.
struct BatchLayout {
  int32_t B, n, m, K, M;
  int64_t total, total_qr;
  size_t off_probs, off_off, off_offqr, off_Lt, off_Ku, off_qr, off_el, off_team, off_inv, off_scan, bytes;
};

static int32_t batch_factor_width(int n, int m) {
  if (n == 64) return 16;
  return padded_M(m);
}

static lqt_status batch_validate(const lqt_batch* bt, BatchLayout& L) {
  if (!bt || bt->count < 1 || !bt->problems || !bt->x0) return LQT_EINVAL;
  const lqt_problem& p0 = bt->problems[0];
  const int n = p0.n;
  if (!(n == 1 || n == 2 || n == 3 || n == 4 || n == 8 || n == 16 || n == 64)) return LQT_EUNSUPPORTED;
  if (p0.m < 1 || p0.m > 16 || p0.K < 1) return LQT_EINVAL;
  L.B = bt->count;
  L.n = n;
  L.m = p0.m;
  L.K = p0.K;
  L.M = batch_factor_width(n, p0.m);
  const int maxM = n == 1 ? 1 : n == 2 ? 2 : n <= 4 ? 4 : n == 8 ? 8 : 16;
  if (L.M > maxM) return LQT_EUNSUPPORTED;
  int64_t total = 0, total_qr = 0;
  for (int32_t b = 0; b < bt->count; ++b) {
    const lqt_problem& p = bt->problems[b];
    if (p.n != n || p.m != p0.m || p.nr != n || p.K != p0.K || p.T < 1) return LQT_EINVAL;
    if (p.H.ptr || p.Hf || !p.t || !p.F.ptr || !p.L.ptr || !p.X.ptr || !p.U.ptr || !p.Xf) return LQT_EINVAL;
    if (p.F.mode != LQT_CONST || p.L.mode != LQT_CONST || p.X.mode != LQT_CONST || p.U.mode != LQT_CONST)
      return LQT_EUNSUPPORTED;
    if (p.c.ptr && p.c.mode != LQT_CONST) return LQT_EUNSUPPORTED;
    const int32_t rm = p.r.ptr ? p.r.mode : LQT_CONST;
    const int32_t rm0 = p0.r.ptr ? p0.r.mode : LQT_CONST;
    if (rm != rm0 || (rm != LQT_CONST && rm != LQT_PER_INTERVAL && rm != LQT_PER_STAGE)) return LQT_EINVAL;
    if (!bt->x0[b]) return LQT_EINVAL;
    total += p.T + 1;
    total_qr += p.r.ptr ? sample_count(rm, p.T, p.K) : 1;
  }
  L.total = total;
  L.total_qr = total_qr;
  size_t off = 0;
  L.off_probs = off; off = bal(off + (size_t)L.B * sizeof(BatchProb));
  L.off_off = off; off = bal(off + ((size_t)L.B + 1) * sizeof(int64_t));
  L.off_offqr = off; off = bal(off + ((size_t)L.B + 1) * sizeof(int64_t));
  L.off_Lt = off; off = bal(off + (size_t)L.B * n * L.M * 8);
  L.off_Ku = off; off = bal(off + (size_t)L.B * L.m * n * 8);
  L.off_qr = off; off = bal(off + (size_t)total_qr * (n + 1) * 8);
  L.off_el = off;
  const size_t T1 = (size_t)total;
  off = bal(off + bal(T1 * n * n * 8) * 3 + bal(T1 * n * 8) * 2 + bal(T1 * 8));
  L.off_team = off; off = bal(off + team_build_scratch_bytes(n));
  // per-problem tables of the time-invariant build (when it supports n)
  L.off_inv = off;
  if (invariant_supported(n, L.M)) off = bal(off + (size_t)L.B * invariant_table_bytes(n, L.M, L.K));
  // The scans may run with any first-level chunk the caller's tuning picks;
  // the shortest chunk (2) needs the most level storage, so size for it.
  const int prev = scan_chunk_override();
  set_scan_chunk(2);
  const size_t scan_bytes = concat_workspace_bytes(n, total - 1);
  set_scan_chunk(prev);
  L.off_scan = off; off = bal(off + scan_bytes);
  L.bytes = off;
  return LQT_OK;
}

static BatchDev batch_dev(const BatchLayout& L, char* ws) {
  BatchDev d{};
  d.B = L.B; d.n = L.n; d.m = L.m; d.K = L.K; d.M = L.M;
  d.probs = (const BatchProb*)(ws + L.off_probs);
  d.off = (const int64_t*)(ws + L.off_off);
  d.off_qr = (const int64_t*)(ws + L.off_offqr);
  d.total = L.total;
  d.total_qr = L.total_qr;
  return d;
}

static ElemPtrs batch_elements(const BatchLayout& L, char* ws) {
  const size_t n = L.n, T1 = (size_t)L.total;
  char* c = ws + L.off_el;
  ElemPtrs e;
  e.A = (double*)c; c += bal(T1 * n * n * 8);
  e.C = (double*)c; c += bal(T1 * n * n * 8);
  e.J = (double*)c; c += bal(T1 * n * n * 8);
  e.b = (double*)c; c += bal(T1 * n * 8);
  e.eta = (double*)c; c += bal(T1 * n * 8);
  e.zeta = (double*)c;
  return e;
}

}  // namespace lqt

using namespace lqt;

extern "C" {

size_t lqt_batch_workspace_size(const lqt_batch* bt) {
  BatchLayout L;
  if (batch_validate(bt, L) != LQT_OK) return 0;
  return L.bytes;
}

int64_t lqt_batch_boundaries(const lqt_batch* bt) {
  BatchLayout L;
  if (batch_validate(bt, L) != LQT_OK) return 0;
  return L.total;
}

lqt_status lqt_batch_plan(const lqt_batch* bt, void* ws, size_t ws_bytes, void* stream) {
  BatchLayout L;
  lqt_status s = batch_validate(bt, L);
  if (s != LQT_OK) return s;
  if (!ws || ws_bytes < L.bytes) return LQT_EWORKSPACE;
  char* w = (char*)ws;
  std::vector<BatchProb> probs((size_t)L.B);
  std::vector<int64_t> off((size_t)L.B + 1), offqr((size_t)L.B + 1);
  int64_t o = 0, oq = 0;
  for (int32_t b = 0; b < L.B; ++b) {
    const lqt_problem& p = bt->problems[b];
    BatchProb& P = probs[b];
    std::memset(&P, 0, sizeof(P));
    P.T = p.T;
    P.off = o;
    P.t = p.t;
    P.Xf = p.Xf;
    P.rf = p.rf;
    P.x0 = bt->x0[b];
    P.L = p.L.ptr;
    P.U = p.U.ptr;
    P.X = p.X.ptr;
    P.r = p.r.ptr;
    P.r_mode = p.r.ptr ? p.r.mode : LQT_CONST;
    P.off_qr = oq;
    P.cf.F = {p.F.ptr, kConst};
    P.cf.c = {p.c.ptr, kConst};
    P.cf.Lt = {(const double*)(w + L.off_Lt) + (size_t)b * L.n * L.M, kConst};
    P.cf.Q = {p.X.ptr, kConst};
    P.cf.qr = {(const double*)(w + L.off_qr) + (size_t)oq * (L.n + 1), p.r.ptr ? p.r.mode : kConst};
    P.cf.Ku = (const double*)(w + L.off_Ku) + (size_t)b * L.m * L.n;
    P.cf.Ku_per_boundary = 0;
    P.cf.M = L.M;
    off[b] = o;
    offqr[b] = oq;
    o += p.T + 1;
    oq += p.r.ptr ? sample_count(p.r.mode, p.T, p.K) : 1;
  }
  off[L.B] = o;
  offqr[L.B] = oq;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(w + L.off_probs, probs.data(), probs.size() * sizeof(BatchProb),
                                  cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(w + L.off_off, off.data(), off.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(w + L.off_offqr, offqr.data(), offqr.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // host tables go out of scope
  return e == cudaSuccess ? LQT_OK : LQT_ECUDA;
}

lqt_status lqt_solve_batched(const lqt_batch* bt, const lqt_tuning* tune, double* S, double* v, double* zeta,
                             double* x, double* u, double* cost, void* ws, size_t ws_bytes, void* stream) {
  reset_launch_count();
  BatchLayout L;
  lqt_status s = batch_validate(bt, L);
  if (s != LQT_OK) return s;
  if (!S || !v || !zeta || !x) return LQT_EINVAL;
  if (!ws || ws_bytes < L.bytes) return LQT_EWORKSPACE;
  const int chunk = tune ? tune->chunk : 0;
  if (!(chunk == 0 || chunk == 2 || chunk == 4 || chunk == 8 || chunk == 16 || chunk == 32)) return LQT_EINVAL;
  const int flags = tune ? tune->flags : 0;
  if (flags & ~LQT_TUNE_INVARIANT_BUILD) return LQT_EINVAL;
  const bool invariant = (flags & LQT_TUNE_INVARIANT_BUILD) != 0;
  if (invariant && !invariant_supported(L.n, L.M)) return LQT_EUNSUPPORTED;
  cudaStream_t st = (cudaStream_t)stream;
  char* w = (char*)ws;
  const BatchDev bd = batch_dev(L, w);
  set_scan_chunk(chunk);
  cudaError_t e = batch_prepare(bd, st);
  const ElemPtrs el = batch_elements(L, w);
  if (e == cudaSuccess)
    e = invariant ? batch_build_invariant(bd, el, (double*)(w + L.off_inv), st)
                  : batch_build(bd, el, w + L.off_team, st);
  BoundaryPatch patch{L.B, bd.off, bd.probs};
  if (e == cudaSuccess)
    e = concat_scan(L.n, L.total - 1, el, S, v, zeta, bt->x0[0], x, patch, w + L.off_scan, st);
  set_scan_chunk(0);
  if (e != cudaSuccess) return LQT_ECUDA;
  zeta_suffix_kernel<<<(unsigned)((L.B + 3) / 4), 128, 0, st>>>(bd, zeta);
  if (L.n >= 8 && L.n <= 32)
    controls_cost_warp_kernel<<<(unsigned)((L.total + 3) / 4), 128, 0, st>>>(bd, S, v, zeta, x, u, cost);
  else
    controls_cost_kernel<<<(unsigned)((L.total + 127) / 128), 128, 0, st>>>(bd, S, v, zeta, x, u, cost);
  count_launch(2);
  return cudaGetLastError() == cudaSuccess ? LQT_OK : LQT_ECUDA;
}

}  // extern "C"
