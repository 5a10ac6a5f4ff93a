// Solve path for state dimensions 16 and 64: the same three stages as the
// one-thread-per-element kernels (lqt_build.cu, lqt_scan.cu) with a team of
// threads per element (lqt_team.cuh).  n = 16: one warp per element, every
// buffer in shared memory (the combinations: lqt_warp16.cuh).  n = 64: one CTA
// of 256 threads per element, the element-sized buffers in a per-CTA slot of
// the workspace (they stay in L2) and the combinations' scratch in shared
// memory, grid = one CTA per SM looping over the work.  Also here: Method 2
// (forward-ODE elements, prefix scan, states) for n = 16 and 64, the
// warp-per-element build of n = 4 and 8 at short horizons, and the warp-per-pair
// upper scan levels of n = 4 and 8 (lqt_warp8.cuh).
#include <cuda_runtime.h>

#include "lqt_device.cuh"
#include "lqt_internal.h"
#include "lqt_team.cuh"
#include "lqt_warp16.cuh"
#include "lqt_warp8.cuh"

namespace lqt {

using team::Rec;

__host__ __device__ __forceinline__ int64_t tdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }
static size_t tal(size_t x) { return (x + 255) & ~(size_t)255; }

template <int N>
struct TeamCfg;
template <>
struct TeamCfg<16> {
  static constexpr int TEAM = 32;
  static constexpr bool SMEM = true;
  static constexpr int SLOTS = 152 * 8;
  // the build: 21.3 KB of shared memory per warp (one full record and three
  // flow records) and at most 204 registers: 10 warps per SM
  static constexpr int BUILD_MIN = 10;
  static constexpr int BUILD_SLOTS = 152 * 10;
  // the scan's combinations: <= 21.7 KB and <= 146 registers per warp
  static constexpr int SCAN_MIN = 10;
  static constexpr int SCAN_SLOTS = 152 * 10;
};
// n <= 8: the thread-per-element kernels do level 0 of the scans; these
// warp-per-combination instances run the pairwise upper levels.
template <int N>
struct TeamCfgSmall {
  static constexpr int TEAM = 32;
  static constexpr bool SMEM = true;
  static constexpr int SLOTS = 152 * 8;
  static constexpr int BUILD_MIN = 1;
  static constexpr int BUILD_SLOTS = SLOTS;
  static constexpr int SCAN_MIN = 1;
  static constexpr int SCAN_SLOTS = SLOTS;
};
template <>
struct TeamCfg<1> : TeamCfgSmall<1> {};
template <>
struct TeamCfg<2> : TeamCfgSmall<2> {};
template <>
struct TeamCfg<3> : TeamCfgSmall<3> {};
template <>
struct TeamCfg<4> : TeamCfgSmall<4> {};
template <>
struct TeamCfg<8> : TeamCfgSmall<8> {};
template <>
struct TeamCfg<64> {
  static constexpr int TEAM = 256;
  static constexpr bool SMEM = false;
  static constexpr int SLOTS = 152;
  static constexpr int BUILD_MIN = 1;
  static constexpr int BUILD_SLOTS = SLOTS;  // one global scratch slot per CTA
  static constexpr int SCAN_MIN = 1;
  static constexpr int SCAN_SLOTS = SLOTS;
};

// Doubles of per-slot scratch of each kernel.
template <int N, int M>
constexpr int build_slot_doubles() { return Rec<N>::SIZE + 3 * Rec<N>::FLOW + 2 * N * M + M + 8; }
template <int N>
constexpr int reduce_slot_doubles() { return 2 * Rec<N>::SIZE + team::combine_scratch_doubles<N>() + 8; }
template <int N>
constexpr int down_slot_doubles() {
  return 2 * team::val_doubles<N>() + team::value_scratch_doubles<N>() + 3 * (N * N + N) + N * N + N + 8;
}
template <int N>
constexpr int maps_slot_doubles() { return 3 * (N * N + N) + 2 * N + 8; }

template <int N>
constexpr int max_slot_doubles() {
  int a = build_slot_doubles<N, N>();
  if (reduce_slot_doubles<N>() > a) a = reduce_slot_doubles<N>();
  if (down_slot_doubles<N>() > a) a = down_slot_doubles<N>();
  if (maps_slot_doubles<N>() > a) a = maps_slot_doubles<N>();
  return a;
}

// Buffer base of this CTA: dynamic shared memory, or its workspace slot.
template <int N>
__device__ __forceinline__ double* slot_base(double* gscratch, int slot_doubles) {
  extern __shared__ double dyn_smem[];
  if constexpr (TeamCfg<N>::SMEM) {
    (void)gscratch;
    (void)slot_doubles;
    return dyn_smem;
  } else {
    return gscratch + (size_t)blockIdx.x * slot_doubles;
  }
}

// ---------------------------------------------------------------------------
// stage (a)
// ---------------------------------------------------------------------------

struct TeamBuildArgs {
  int64_t T;
  int32_t K;
  const double* t;
  Coefs cf;
  ElemPtrs out;
  double* gscratch;
};

// One RK4 stage input in the full layout (A, b, C, eta, J, zeta) at dst: a
// packed record whole, a flow record's A, eta, J with b, C, zeta as zero (the
// discrete adjoint reads only A, eta, J of a stage input).
template <int N, int TEAM>
__device__ void store_stage(int lane, double* dst, Rec<N> src, bool full) {
  for (int e = lane; e < Rec<N>::SIZE; e += TEAM) {
    double v;
    if (e < N * N) v = src.A()[e];
    else if (e < N * N + N) v = full ? src.b()[e - N * N] : 0.0;
    else if (e < 2 * N * N + N) v = full ? src.C()[e - N * N - N] : 0.0;
    else if (e < 2 * N * N + 2 * N) v = src.eta()[e - 2 * N * N - N];
    else if (e < 3 * N * N + 2 * N) v = src.J()[e - 2 * N * N - 2 * N];
    else v = full ? *src.zeta() : 0.0;
    dst[e] = v;
  }
  team::sync<TEAM>();
}

// Element j of a problem (coefficients cf, grid t) into the packed record at
// yb; the other buffers are scratch.  With `stages`, the four stage inputs of
// RK4 step i go to stages + (i 4 + s) (3N^2 + 2N + 1), s = 0..3, in the full
// layout.
template <int N, int M>
__device__ void team_build_one(int lane, const Coefs& cf, const double* t, int64_t j, int32_t K, double* yb,
                               double* ynb, double* ytb, double* kb, double* AL, double* P, double* w,
                               double* stages = nullptr) {
  constexpr int TEAM = TeamCfg<N>::TEAM;
  constexpr int FS = Rec<N>::SIZE;
  const Rec<N> y = Rec<N>::packed(yb), yn = Rec<N>::flow(ynb), yt = Rec<N>::flow(ytb), k = Rec<N>::flow(kb);
  const double h = (t[j + 1] - t[j]) / K;
  for (int e = lane; e < Rec<N>::SIZE; e += TEAM) yb[e] = (e < N * N && e % (N + 1) == 0) ? 1.0 : 0.0;
  team::sync<TEAM>();
  for (int32_t i = K - 1; i >= 0; --i) {
    double* st = stages ? stages + (int64_t)i * 4 * FS : nullptr;
    const int32_t ps[3] = {2 * i + 2, 2 * i + 1, 2 * i};
    const double *F[3], *c[3], *Lt[3], *Q[3], *qr[3];
    for (int q = 0; q < 3; ++q) {
      F[q] = cf.F.ptr + sample_index(cf.F.mode, j, ps[q], K) * N * N;
      c[q] = cf.c.ptr ? cf.c.ptr + sample_index(cf.c.mode, j, ps[q], K) * N : nullptr;
      Lt[q] = cf.Lt.ptr + sample_index(cf.Lt.mode, j, ps[q], K) * N * M;
      Q[q] = cf.Q.ptr + sample_index(cf.Q.mode, j, ps[q], K) * N * N;
      qr[q] = cf.qr.ptr + sample_index(cf.qr.mode, j, ps[q], K) * (N + 1);
    }
    // (A, eta, J) by classical RK4 through yn and yt; b, C, zeta accumulated
    // into y by the right-hand side
    if (st) store_stage<N, TEAM>(lane, st, y, true);
    team::rhs<N, M, TEAM>(lane, y, k, F[0], c[0], Lt[0], Q[0], qr[0], AL, P, w, -h / 6.0, y);
    team::axpy_flow<N, TEAM>(lane, yn, y, -h / 6.0, k);
    team::axpy_flow<N, TEAM>(lane, yt, y, -0.5 * h, k);
    if (st) store_stage<N, TEAM>(lane, st + FS, yt, false);
    team::rhs<N, M, TEAM>(lane, yt, k, F[1], c[1], Lt[1], Q[1], qr[1], AL, P, w, -h / 3.0, y);
    team::axpy_flow<N, TEAM>(lane, yn, yn, -h / 3.0, k);
    team::axpy_flow<N, TEAM>(lane, yt, y, -0.5 * h, k);
    if (st) store_stage<N, TEAM>(lane, st + 2 * FS, yt, false);
    team::rhs<N, M, TEAM>(lane, yt, k, F[1], c[1], Lt[1], Q[1], qr[1], AL, P, w, -h / 3.0, y);
    team::axpy_flow<N, TEAM>(lane, yn, yn, -h / 3.0, k);
    team::axpy_flow<N, TEAM>(lane, yt, y, -h, k);
    if (st) store_stage<N, TEAM>(lane, st + 3 * FS, yt, false);
    team::rhs<N, M, TEAM>(lane, yt, k, F[2], c[2], Lt[2], Q[2], qr[2], AL, P, w, -h / 6.0, y);
    team::axpy_flow<N, TEAM>(lane, y, yn, -h / 6.0, k);
  }
}

template <int N, int M>
__global__ void __launch_bounds__(TeamCfg<N>::TEAM, TeamCfg<N>::BUILD_MIN) build_team_kernel(TeamBuildArgs a) {
  constexpr int TEAM = TeamCfg<N>::TEAM;
  constexpr int SD = build_slot_doubles<N, M>();
  const int lane = threadIdx.x;
  double* base = slot_base<N>(a.gscratch, SD);
  double* yb = base;
  double* ynb = yb + Rec<N>::SIZE;
  double* ytb = ynb + Rec<N>::FLOW;
  double* kb = ytb + Rec<N>::FLOW;
  double* AL = kb + Rec<N>::FLOW;
  double* P = AL + N * M;
  double* w = P + N * M;
  for (int64_t j = blockIdx.x; j < a.T; j += gridDim.x) {
    team_build_one<N, M>(lane, a.cf, a.t, j, a.K, yb, ynb, ytb, kb, AL, P, w);
    double zz = 0.0;
    Rec<N> dst = Rec<N>::pub(a.out, j, &zz);
    team::copy_rec<N, TEAM>(lane, dst, Rec<N>::packed(yb));
  }
}

// Elements j0 .. j0 + a.T - 1 with one warp each, for n = 4 and 8 at short
// horizons: one thread per element then leaves most sub-partitions without a
// warp, and each warp's chain of FP64 instructions (64 cycles apiece) is a
// whole element's; a warp per element spreads each right-hand side over its
// lanes.  With `stages`, the stage inputs of element j0 + jj go to
// stages + jj K 4 (3N^2 + 2N + 1); the element is stored when a.out.A is set.
template <int N, int M>
__global__ void __launch_bounds__(TeamCfg<N>::TEAM) build_team_range_kernel(TeamBuildArgs a, int64_t j0,
                                                                            double* stages) {
  constexpr int TEAM = TeamCfg<N>::TEAM;
  constexpr int SD = build_slot_doubles<N, M>();
  const int lane = threadIdx.x;
  double* base = slot_base<N>(a.gscratch, SD);
  double* yb = base;
  double* ynb = yb + Rec<N>::SIZE;
  double* ytb = ynb + Rec<N>::FLOW;
  double* kb = ytb + Rec<N>::FLOW;
  double* AL = kb + Rec<N>::FLOW;
  double* P = AL + N * M;
  double* w = P + N * M;
  for (int64_t jj = blockIdx.x; jj < a.T; jj += gridDim.x) {
    team_build_one<N, M>(lane, a.cf, a.t, j0 + jj, a.K, yb, ynb, ytb, kb, AL, P, w,
                         stages ? stages + jj * (int64_t)a.K * 4 * Rec<N>::SIZE : nullptr);
    if (a.out.A) {
      double zz = 0.0;
      team::copy_rec<N, TEAM>(lane, Rec<N>::pub(a.out, j0 + jj, &zz), Rec<N>::packed(yb));
    }
  }
}

// Batches: one team per boundary of the concatenation (element or terminal).
template <int N, int M>
__global__ void __launch_bounds__(TeamCfg<N>::TEAM, TeamCfg<N>::BUILD_MIN)
    batch_build_team_kernel(BatchDev bd, ElemPtrs out, double* gscratch) {
  constexpr int TEAM = TeamCfg<N>::TEAM;
  constexpr int SD = build_slot_doubles<N, M>();
  const int lane = threadIdx.x;
  double* base = slot_base<N>(gscratch, SD);
  double* yb = base;
  double* ynb = yb + Rec<N>::SIZE;
  double* ytb = ynb + Rec<N>::FLOW;
  double* kb = ytb + Rec<N>::FLOW;
  double* AL = kb + Rec<N>::FLOW;
  double* P = AL + N * M;
  double* w = P + N * M;
  for (int64_t g = blockIdx.x; g < bd.total; g += gridDim.x) {
    const int32_t b = batch_find(bd.off, bd.B, g);
    const BatchProb& pb = bd.probs[b];
    const int64_t j = g - pb.off;
    if (j < pb.T) {
      team_build_one<N, M>(lane, pb.cf, pb.t, j, bd.K, yb, ynb, ytb, kb, AL, P, w);
    } else {
      const Rec<N> y = Rec<N>::packed(yb);
      for (int e = lane; e < Rec<N>::SIZE; e += TEAM) yb[e] = 0.0;
      team::sync<TEAM>();
      for (int e = lane; e < N * N + N + 1; e += TEAM) {
        if (e < N * N) {
          const int i = e / N, c = e % N;
          y.J()[e] = 0.5 * (pb.Xf[i * N + c] + pb.Xf[c * N + i]);
        } else if (e < N * N + N) {
          const int i = e - N * N;
          double v = 0.0;
          if (pb.rf)
            for (int l = 0; l < N; ++l) v = fma(pb.Xf[i * N + l], pb.rf[l], v);
          y.eta()[i] = v;
        } else {
          double z = 0.0;
          if (pb.rf)
            for (int i = 0; i < N; ++i) {
              double v = 0.0;
              for (int l = 0; l < N; ++l) v = fma(pb.Xf[i * N + l], pb.rf[l], v);
              z = fma(pb.rf[i], v, z);
            }
          *y.zeta() = 0.5 * z;
        }
      }
      team::sync<TEAM>();
    }
    double zz = 0.0;
    Rec<N> dst = Rec<N>::pub(out, g, &zz);
    team::copy_rec<N, TEAM>(lane, dst, Rec<N>::packed(yb));
  }
}

// Elements of the forward conditional ODEs (Sec. IV-C, Theorem
// Forward_HJB_LQT) for Method 2: element j by K classical RK4 steps in tau
// from A = I, b = C = eta = J = 0, zeta = 0 at tau = t_j (eq.
// abcej_boundary) to t_{j+1}, stage samples at half-steps 2i, 2i+1, 2i+2 of
// step i.  One team per element; records y (state), yn (the four-stage sum),
// yt (stage input), k (rate), all packed.
template <int N>
constexpr int forward_slot_doubles() { return 4 * Rec<N>::SIZE + 2 * N * N + N + 8; }

template <int N, int M>
__global__ void __launch_bounds__(TeamCfg<N>::TEAM) build_forward_team_kernel(TeamBuildArgs a) {
  constexpr int TEAM = TeamCfg<N>::TEAM;
  constexpr int RS = Rec<N>::SIZE;
  const int lane = threadIdx.x;
  double* y = slot_base<N>(a.gscratch, forward_slot_doubles<N>());
  double* yn = y + RS;
  double* yt = yn + RS;
  double* k = yt + RS;
  double* QA = k + RS;
  double* CQ = QA + N * N;
  double* w = CQ + N * N;
  const Coefs& cf = a.cf;
  for (int64_t j = blockIdx.x; j < a.T; j += gridDim.x) {
    const double h = (a.t[j + 1] - a.t[j]) / a.K;
    for (int e = lane; e < RS; e += TEAM) y[e] = (e < N * N && e % (N + 1) == 0) ? 1.0 : 0.0;
    team::sync<TEAM>();
    for (int32_t i = 0; i < a.K; ++i) {
      const int32_t ps[3] = {2 * i, 2 * i + 1, 2 * i + 2};
      const double *F[3], *c[3], *Lt[3], *Q[3], *qr[3];
      for (int q = 0; q < 3; ++q) {
        F[q] = cf.F.ptr + sample_index(cf.F.mode, j, ps[q], a.K) * N * N;
        c[q] = cf.c.ptr ? cf.c.ptr + sample_index(cf.c.mode, j, ps[q], a.K) * N : nullptr;
        Lt[q] = cf.Lt.ptr + sample_index(cf.Lt.mode, j, ps[q], a.K) * N * M;
        Q[q] = cf.Q.ptr + sample_index(cf.Q.mode, j, ps[q], a.K) * N * N;
        qr[q] = cf.qr.ptr + sample_index(cf.qr.mode, j, ps[q], a.K) * (N + 1);
      }
      const Rec<N> Ry = Rec<N>::packed(y), Rt = Rec<N>::packed(yt), Rk = Rec<N>::packed(k);
      team::forward_rhs<N, M, TEAM>(lane, Ry, Rk, F[0], c[0], Lt[0], Q[0], qr[0], QA, CQ, w);
      team::axpy2_rec<N, TEAM>(lane, yn, y, h / 6.0, yt, y, 0.5 * h, k);
      team::forward_rhs<N, M, TEAM>(lane, Rt, Rk, F[1], c[1], Lt[1], Q[1], qr[1], QA, CQ, w);
      team::axpy2_rec<N, TEAM>(lane, yn, yn, h / 3.0, yt, y, 0.5 * h, k);
      team::forward_rhs<N, M, TEAM>(lane, Rt, Rk, F[1], c[1], Lt[1], Q[1], qr[1], QA, CQ, w);
      team::axpy2_rec<N, TEAM>(lane, yn, yn, h / 3.0, yt, y, h, k);
      team::forward_rhs<N, M, TEAM>(lane, Rt, Rk, F[2], c[2], Lt[2], Q[2], qr[2], QA, CQ, w);
      team::axpy2_rec<N, TEAM>(lane, y, yn, h / 6.0, nullptr, nullptr, 0.0, k);
    }
    double zz = 0.0;
    team::copy_rec<N, TEAM>(lane, Rec<N>::pub(a.out, j, &zz), Rec<N>::packed(y));
  }
}

// ---------------------------------------------------------------------------
// stage (b): reduce / down-sweep of the value scan
// ---------------------------------------------------------------------------

// The FP32 products of the n = 64 combinations run on the tensor core.
template <int N, typename GT>
constexpr bool kTensorProducts = (N == 64 && std::is_same<GT, float>::value);
// The FP64 n = 64 combinations keep their scratch (W, R = [K1 | MC1 | z0],
// T1, vectors; 131 KB) in dynamic shared memory: the 64 dependent pivot steps
// of the LU then wait on shared memory instead of L2.
template <int N, typename GT>
constexpr bool kSharedScratch = (N == 64 && !kTensorProducts<N, GT>);
// After the scratch: the A and C blocks of the element being combined, staged
// by the TMA unit at level 0 (stage_ac).
template <int N>
constexpr size_t kReduceSmemBytes = sizeof(double) * (team::combine_scratch_doubles<N>() + 2 * N * N);
template <int N>
constexpr size_t kDownSmemBytes = sizeof(double) * (team::value_scratch_doubles<N>() + N * N + N + 2 * N * N);
// The tensor-core instances: the operand tiles, then W, R and the vectors
// (and the map Psi, alpha in the down-sweep); T1 stays in the slot.
template <int N>
constexpr int kTcReduceScr = N * N + N * (2 * N + 1) + 4 * N;
template <int N>
constexpr int kTcDownScr = N * N + N * (N + 1) + 3 * N + N * N + N;
template <int N>
constexpr size_t kTcReduceSmemBytes = tc::kSmemBytes + sizeof(double) * kTcReduceScr<N>;
template <int N>
constexpr size_t kTcDownSmemBytes = tc::kSmemBytes + sizeof(double) * kTcDownScr<N>;

struct TeamScanArgs {
  ElemPtrs el;           // level-0 elements (public layout)
  const double* src;     // packed elements of the level (levels >= 1), or null at level 0
  int64_t cnt;           // elements at this level
  int G;                 // group length
  double* agg;           // reduce output (packed)
  const double* above;   // packed values of the level above (down), or null
  int64_t cnt_above;
  double* vals;          // packed values out (levels >= 1)
  double *S, *v, *zeta;  // level-0 outputs
  double *maps, *comp;   // level-0 maps [T][N^2+N] and chunk composites
  int64_t T;
  double* gscratch;
  int zeta_inc;          // level 0 of a batch: zeta[k] receives the element's own share (see DownOut)
  int bulk;              // FP64 n = 64, level 0: stage A, C of each element by TMA
};

template <int N>
__device__ __forceinline__ Rec<N> level_elem(const TeamScanArgs& a, int64_t k, double* zero) {
  if (a.src) return Rec<N>::packed(const_cast<double*>(a.src) + k * Rec<N>::SIZE);
  return Rec<N>::pub(a.el, k, zero);
}

// Element k of the public arrays with its A and C blocks (N x N each, 32 KB at
// n = 64) copied into shared memory sA, sC by the TMA unit (cp.async.bulk,
// completion on the mbarrier `bar` with a bounded wait); every thread of the
// CTA calls it after its last read of sA, sC.  The arrays must be 16-byte
// aligned (bulk_ok).
template <int N>
__device__ __forceinline__ Rec<N> stage_ac(const ElemPtrs& el, int64_t k, double* sA, double* sC,
                                           unsigned long long* bar, unsigned& phase, double* zero) {
  constexpr unsigned kBytes = N * N * sizeof(double);
  w16::fence_proxy_async();  // this thread's reads of sA, sC before the copies' writes
  __syncthreads();
  if (threadIdx.x == 0) {
    w16::mbar_expect_tx(bar, 2 * kBytes);
    w16::bulk_g2s(sA, el.A + k * N * N, kBytes, bar);
    w16::bulk_g2s(sC, el.C + k * N * N, kBytes, bar);
  }
  w16::mbar_wait_bounded(bar, phase);
  phase ^= 1u;
  Rec<N> e = Rec<N>::pub(el, k, zero);
  e.a_ = sA;
  e.c_ = sC;
  return e;
}

template <int N, typename GT = double>
__global__ void __launch_bounds__(TeamCfg<N>::TEAM, TeamCfg<N>::SCAN_MIN) reduce_team_kernel(TeamScanArgs a) {
  constexpr int TEAM = TeamCfg<N>::TEAM;
  constexpr int SD = reduce_slot_doubles<N>();
  __shared__ double fs[2 * TEAM];
  __shared__ int is[TEAM];
  __shared__ double zero;
  const int lane = threadIdx.x;
  if (lane == 0) zero = 0.0;
  double* base = slot_base<N>(a.gscratch, SD);
  double* bufA = base;
  double* bufB = bufA + Rec<N>::SIZE;
  double* scr = bufB + Rec<N>::SIZE;
  double* t1 = nullptr;
  double *sA = nullptr, *sC = nullptr;
  __shared__ unsigned long long st_bar;
  unsigned st_phase = 0;
  if constexpr (kSharedScratch<N, GT>) {
    extern __shared__ __align__(16) double scr_smem[];
    scr = scr_smem;
    sA = scr + team::combine_scratch_doubles<N>();
    sC = sA + N * N;
    if (lane == 0) w16::mbar_init(&st_bar, 1);
  }
  tc::Ctx* tcx = nullptr;
  tc::Ctx tc_ctx;
  if constexpr (kTensorProducts<N, GT>) {
    extern __shared__ __align__(16) unsigned char tc_smem[];
    __shared__ uint32_t tmem_slot;
    __shared__ unsigned long long tc_bar;
    tc::init(tc_ctx, &tmem_slot, &tc_bar, tc_smem);
    tcx = &tc_ctx;
    t1 = scr + N * N + N * (2 * N + 1);
    scr = reinterpret_cast<double*>(tc_smem + tc::kSmemBytes);
  }
  team::sync<TEAM>();
  const int64_t groups = tdiv(a.cnt, a.G);
  for (int64_t g = blockIdx.x; g < groups; g += gridDim.x) {
    const int64_t first = g * a.G;
    const int64_t last = (first + a.G < a.cnt ? first + a.G : a.cnt) - 1;
    Rec<N> acc = Rec<N>::packed(bufA), nxt = Rec<N>::packed(bufB);
    team::copy_rec<N, TEAM>(lane, acc, level_elem<N>(a, last, &zero));
    for (int64_t k = last - 1; k >= first; --k) {
      Rec<N> e1 = level_elem<N>(a, k, &zero);
      if constexpr (kSharedScratch<N, GT>)
        if (a.bulk) e1 = stage_ac<N>(a.el, k, sA, sC, &st_bar, st_phase, &zero);
      team::combine<N, TEAM, GT>(lane, e1, acc, nxt, scr, fs, is, tcx, t1);
      const Rec<N> t = acc;
      acc = nxt;
      nxt = t;
    }
    team::copy_rec<N, TEAM>(lane, Rec<N>::packed(a.agg + g * Rec<N>::SIZE), acc);
  }
  if constexpr (kTensorProducts<N, GT>) tc::release(tc_ctx);
}

template <int N, bool Level0, typename GT = double>
__global__ void __launch_bounds__(TeamCfg<N>::TEAM, TeamCfg<N>::SCAN_MIN) down_team_kernel(TeamScanArgs a) {
  constexpr int TEAM = TeamCfg<N>::TEAM;
  constexpr int SD = down_slot_doubles<N>();
  constexpr int VS = team::val_doubles<N>();
  constexpr int PM = N * N + N;
  __shared__ double fs[2 * TEAM];
  __shared__ int is[TEAM];
  __shared__ double zero;
  __shared__ double zinc;
  const int lane = threadIdx.x;
  if (lane == 0) zero = 0.0;
  double* base = slot_base<N>(a.gscratch, SD);
  double* c0 = base;
  double* c1 = c0 + VS;
  double* scr = c1 + VS;
  double* Psi = scr + team::value_scratch_doubles<N>();
  double* alpha = Psi + N * N;
  double* P = alpha + N;
  double* pv = P + N * N;
  double* Tm = pv + N;
  double* t1 = nullptr;
  double *sA = nullptr, *sC = nullptr;
  __shared__ unsigned long long st_bar;
  unsigned st_phase = 0;
  if constexpr (kSharedScratch<N, GT>) {
    // the combination's scratch, its map (Psi, alpha) and the staged A, C in
    // shared memory; the chunk composite (P, pv, Tm) stays in the slot
    extern __shared__ __align__(16) double scr_smem[];
    scr = scr_smem;
    Psi = scr + team::value_scratch_doubles<N>();
    alpha = Psi + N * N;
    sA = alpha + N;
    sC = sA + N * N;
    if (lane == 0) w16::mbar_init(&st_bar, 1);
  }
  tc::Ctx* tcx = nullptr;
  tc::Ctx tc_ctx;
  if constexpr (kTensorProducts<N, GT>) {
    extern __shared__ __align__(16) unsigned char tc_smem[];
    __shared__ uint32_t tmem_slot;
    __shared__ unsigned long long tc_bar;
    tc::init(tc_ctx, &tmem_slot, &tc_bar, tc_smem);
    tcx = &tc_ctx;
    t1 = scr + N * N + N * (N + 1);
    scr = reinterpret_cast<double*>(tc_smem + tc::kSmemBytes);
    Psi = scr + N * N + N * (N + 1) + 3 * N;
    alpha = Psi + N * N;
  }
  team::sync<TEAM>();
  const int64_t groups = tdiv(a.cnt, a.G);
  for (int64_t g = blockIdx.x; g < groups; g += gridDim.x) {
    const int64_t first = g * a.G;
    const int64_t last = (first + a.G < a.cnt ? first + a.G : a.cnt) - 1;
    double* carry = c0;
    double* nv = c1;
    for (int e = lane; e < VS; e += TEAM)
      carry[e] = (a.above != nullptr && g + 1 < a.cnt_above) ? a.above[(g + 1) * VS + e] : 0.0;
    if (Level0)
      for (int e = lane; e < PM; e += TEAM) {
        if (e < N * N) P[e] = (e % (N + 1) == 0) ? 1.0 : 0.0;
        else pv[e - N * N] = 0.0;
      }
    team::sync<TEAM>();
    for (int64_t k = last; k >= first; --k) {
      Rec<N> e = level_elem<N>(a, k, &zero);
      if constexpr (kSharedScratch<N, GT>)
        if (a.bulk) e = stage_ac<N>(a.el, k, sA, sC, &st_bar, st_phase, &zero);
      team::combine_value<N, TEAM, GT>(lane, e, carry, nv, Psi, alpha, scr, fs, is, &zinc, tcx, t1);
      if (Level0) {
        bool ok = true;
        for (int e = lane; e < VS; e += TEAM) {
          const double x = nv[e];
          ok = ok && isfinite(x);
          if (e < N * N) a.S[k * N * N + e] = x;
          else if (e < N * N + N) a.v[k * N + e - N * N] = x;
          else if (a.zeta) a.zeta[k] = a.zeta_inc ? zinc : x;
        }
        if (!ok) flag(kStatusNonFinite);
        if (a.maps != nullptr && k < a.T) {
          for (int e = lane; e < PM; e += TEAM) a.maps[k * PM + e] = e < N * N ? Psi[e] : alpha[e - N * N];
          team::compose_right<N, TEAM>(lane, P, pv, Psi, alpha, Tm);
        }
      } else {
        for (int e = lane; e < VS; e += TEAM) a.vals[k * VS + e] = nv[e];
      }
      team::sync<TEAM>();
      double* t = carry;
      carry = nv;
      nv = t;
    }
    if (Level0 && a.comp != nullptr && last + 1 <= a.T)
      for (int e = lane; e < PM; e += TEAM) a.comp[g * PM + e] = e < N * N ? P[e] : pv[e - N * N];
    team::sync<TEAM>();
  }
  if constexpr (kTensorProducts<N, GT>) tc::release(tc_ctx);
}

// n = 16: one warp per combination with the register Gauss-Jordan solve and
// TMA-staged element operands (lqt_warp16.cuh).  Same levels, groups and
// records as the kernels above.
constexpr int kW16ReduceSmem = 2 * w16::kRecPad + w16::kScratch;
constexpr int kW16DownSmem = 2 * 276 + w16::kRecPad + w16::kVScratch + 256 + 16 + 256 + 16 + 16 * w16::kWld;

__device__ __forceinline__ bool finite_bits(double x) {
  return (__double_as_longlong(x) & 0x7ff0000000000000ll) != 0x7ff0000000000000ll;
}

template <typename GT>
__global__ void __launch_bounds__(32, 10) reduce_w16_kernel(TeamScanArgs a, int bulk) {
  extern __shared__ __align__(16) double w16_smem[];
  __shared__ unsigned long long bar;
  __shared__ double zero;
  const int lane = threadIdx.x;
  double* bufA = w16_smem;
  double* bufB = bufA + w16::kRecPad;
  double* scr = bufB + w16::kRecPad;
  if (lane == 0) {
    zero = 0.0;
    w16::mbar_init(&bar, 1);
  }
  __syncwarp();
  unsigned phase = 0;
  const w16::ElemSrc src{a.el, a.src, bulk != 0};
  const int64_t groups = tdiv(a.cnt, a.G);
  for (int64_t g = blockIdx.x; g < groups; g += gridDim.x) {
    const int64_t first = g * a.G;
    const int64_t last = (first + a.G < a.cnt ? first + a.G : a.cnt) - 1;
    double* acc = bufA;
    double* nxt = bufB;
    w16::stage(lane, src, last, acc, &bar, phase, &zero);
    for (int64_t k = last - 1; k >= first; --k) {
      w16::stage(lane, src, k, nxt, &bar, phase, &zero);
      w16::combine<GT>(lane, nxt, acc, scr);
      double* t = acc;
      acc = nxt;
      nxt = t;
    }
    double* out = a.agg + g * w16::kRec;
    for (int e = lane; e < w16::kRec; e += 32) out[e] = acc[e];
    __syncwarp();
  }
}

template <bool Level0, typename GT>
__global__ void __launch_bounds__(32, 10) down_w16_kernel(TeamScanArgs a, int bulk) {
  extern __shared__ __align__(16) double w16_smem[];
  __shared__ unsigned long long bar;
  __shared__ double zero;
  __shared__ double zinc;
  constexpr int VS = w16::kVal;
  const int lane = threadIdx.x;
  double* c0 = w16_smem;
  double* c1 = c0 + 276;
  double* E = c1 + 276;
  double* scr = E + w16::kRecPad;
  double* Psi = scr + w16::kVScratch;
  double* alpha = Psi + 256;
  double* P = alpha + 16;
  double* pv = P + 256;
  double* Tm = pv + 16;
  if (lane == 0) {
    zero = 0.0;
    w16::mbar_init(&bar, 1);
  }
  __syncwarp();
  unsigned phase = 0;
  const w16::ElemSrc src{a.el, a.src, bulk != 0};
  const int64_t groups = tdiv(a.cnt, a.G);
  for (int64_t g = blockIdx.x; g < groups; g += gridDim.x) {
    const int64_t first = g * a.G;
    const int64_t last = (first + a.G < a.cnt ? first + a.G : a.cnt) - 1;
    double* carry = c0;
    double* nv = c1;
    for (int e = lane; e < VS; e += 32)
      carry[e] = (a.above != nullptr && g + 1 < a.cnt_above) ? a.above[(g + 1) * VS + e] : 0.0;
    if (Level0) {
      for (int e = lane; e < 256; e += 32) P[e] = ((e >> 4) == (e & 15)) ? 1.0 : 0.0;
      if (lane < 16) pv[lane] = 0.0;
    }
    __syncwarp();
    for (int64_t k = last; k >= first; --k) {
      w16::stage(lane, src, k, E, &bar, phase, &zero);
      w16::combine_value<GT>(lane, E, carry, nv, Psi, alpha, scr, &zinc);
      if (Level0) {
        bool ok = true;
        for (int e = lane; e < VS; e += 32) {
          const double x = nv[e];
          ok = ok && finite_bits(x);
          if (e < 256) a.S[k * 256 + e] = x;
          else if (e < 272) a.v[k * 16 + e - 256] = x;
          else if (a.zeta) a.zeta[k] = a.zeta_inc ? zinc : x;
        }
        if (!ok) flag(kStatusNonFinite);
        if (a.maps != nullptr && k < a.T) {
          for (int e = lane; e < 272; e += 32) a.maps[k * 272 + e] = e < 256 ? Psi[e] : alpha[e - 256];
          w16::compose_right(lane, P, pv, Psi, alpha, Tm);
        }
      } else {
        for (int e = lane; e < VS; e += 32) a.vals[k * VS + e] = nv[e];
      }
      __syncwarp();
      double* t = carry;
      carry = nv;
      nv = t;
    }
    if (Level0 && a.comp != nullptr && last + 1 <= a.T)
      for (int e = lane; e < 272; e += 32) a.comp[g * 272 + e] = e < 256 ? P[e] : pv[e - 256];
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// stage (c): affine-map scan and the final pass
// ---------------------------------------------------------------------------

struct TeamMapArgs {
  const double* maps;  // [cnt][N^2+N]
  int64_t cnt;
  int G;
  double* comp;         // reduce output
  const double* above;  // starts of the level above (down), or null -> x_in
  const double* x_in;
  double* starts;       // [cnt+1][N]
  double* gscratch;
};

template <int N>
__global__ void __launch_bounds__(TeamCfg<N>::TEAM) reduce_maps_team_kernel(TeamMapArgs a) {
  constexpr int TEAM = TeamCfg<N>::TEAM;
  constexpr int PM = N * N + N;
  const int lane = threadIdx.x;
  double* base = slot_base<N>(a.gscratch, maps_slot_doubles<N>());
  double* P = base;
  double* p = P + N * N;
  double* Tm = p + N;
  const int64_t groups = tdiv(a.cnt, a.G);
  for (int64_t g = blockIdx.x; g < groups; g += gridDim.x) {
    const int64_t first = g * a.G;
    const int64_t last = (first + a.G < a.cnt ? first + a.G : a.cnt) - 1;
    for (int e = lane; e < PM; e += TEAM) (e < N * N ? P[e] : p[e - N * N]) = a.maps[first * PM + e];
    team::sync<TEAM>();
    for (int64_t k = first + 1; k <= last; ++k)
      team::compose_left<N, TEAM>(lane, P, p, a.maps + k * PM, a.maps + k * PM + N * N, Tm);
    for (int e = lane; e < PM; e += TEAM) a.comp[g * PM + e] = e < N * N ? P[e] : p[e - N * N];
    team::sync<TEAM>();
  }
}

template <int N>
__global__ void __launch_bounds__(TeamCfg<N>::TEAM) down_maps_team_kernel(TeamMapArgs a) {
  constexpr int TEAM = TeamCfg<N>::TEAM;
  constexpr int PM = N * N + N;
  const int lane = threadIdx.x;
  double* base = slot_base<N>(a.gscratch, maps_slot_doubles<N>());
  double* x = base;
  double* y = x + N;
  const int64_t groups = tdiv(a.cnt, a.G);
  for (int64_t g = blockIdx.x; g < groups; g += gridDim.x) {
    const int64_t first = g * a.G;
    const int64_t last = (first + a.G < a.cnt ? first + a.G : a.cnt) - 1;
    const double* xs = a.above ? a.above + g * N : a.x_in;
    for (int e = lane; e < N; e += TEAM) x[e] = xs[e];
    team::sync<TEAM>();
    for (int64_t k = first; k <= last; ++k) {
      for (int e = lane; e < N; e += TEAM) a.starts[k * N + e] = x[e];
      team::apply_map<N, TEAM>(lane, a.maps + k * PM, a.maps + k * PM + N * N, x, y);
      for (int e = lane; e < N; e += TEAM) x[e] = y[e];
      team::sync<TEAM>();
    }
    if (last == a.cnt - 1)
      for (int e = lane; e < N; e += TEAM) a.starts[a.cnt * N + e] = x[e];
    team::sync<TEAM>();
  }
}

struct TeamFinalArgs {
  const double* maps;
  int64_t T;
  int G;
  const double *starts1, *x0, *S, *v, *zeta, *Ku;
  int32_t Ku_per_boundary, m;
  double *x, *u, *cost;
  double* gscratch;
};

template <int N>
__global__ void __launch_bounds__(TeamCfg<N>::TEAM) final_team_kernel(TeamFinalArgs a) {
  constexpr int TEAM = TeamCfg<N>::TEAM;
  constexpr int PM = N * N + N;
  const int lane = threadIdx.x;
  double* base = slot_base<N>(a.gscratch, maps_slot_doubles<N>());
  double* x = base;
  double* y = x + N;
  const int64_t groups = tdiv(a.T + 1, a.G);
  for (int64_t g = blockIdx.x; g < groups; g += gridDim.x) {
    const int64_t first = g * a.G;
    const int64_t last = (first + a.G < a.T + 1 ? first + a.G : a.T + 1) - 1;
    const double* xs = a.starts1 ? a.starts1 + g * N : a.x0;
    for (int e = lane; e < N; e += TEAM) x[e] = xs[e];
    team::sync<TEAM>();
    for (int64_t k = first; k <= last; ++k) {
      for (int e = lane; e < N; e += TEAM) a.x[k * N + e] = x[e];
      if (a.u) {
        // y = v_k - S_k x_k, then u = Ku y
        const double* Sk = a.S + k * N * N;
        for (int i = lane; i < N; i += TEAM) {
          double s = a.v[k * N + i];
          for (int l = 0; l < N; ++l) s = fma(-Sk[i * N + l], x[l], s);
          y[i] = s;
        }
        team::sync<TEAM>();
        const double* Kk = a.Ku + (a.Ku_per_boundary ? k * a.m * N : 0);
        for (int q = lane; q < a.m; q += TEAM) {
          double s = 0.0;
          for (int l = 0; l < N; ++l) s = fma(Kk[q * N + l], y[l], s);
          a.u[k * a.m + q] = s;
        }
        team::sync<TEAM>();
      }
      if (k < a.T) {
        team::apply_map<N, TEAM>(lane, a.maps + k * PM, a.maps + k * PM + N * N, x, y);
        for (int e = lane; e < N; e += TEAM) x[e] = y[e];
        team::sync<TEAM>();
      }
    }
    if (g == 0 && a.cost && lane == 0) {
      double c = a.zeta ? a.zeta[0] : 0.0;
      for (int i = 0; i < N; ++i) {
        double s = 0.0;
        for (int l = 0; l < N; ++l) s = fma(a.S[i * N + l], a.x0[l], s);
        c = fma(a.x0[i], fma(0.5, s, -a.v[i]), c);
      }
      *a.cost = c;
    }
    team::sync<TEAM>();
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

template <int N>
static int team_group0(int64_t T) {
  if (scan_chunk_override() >= 2) return scan_chunk_override();
  const int64_t want = TeamCfg<N>::SLOTS;  // chunks that keep every slot busy
  int g = 2;
  while (g < 32 && (T + 1) / (2 * g) >= want) g *= 2;
  return g;
}

template <int N>
struct TeamPlan {
  int G0;
  int nlev;
  int64_t cnt[64];
  size_t off_agg[64], off_val[64];
  size_t off_maps;
  int tlev;
  int64_t tcnt[64];
  size_t off_tmap[64], off_tstart[64];
  size_t off_scratch;
  size_t bytes;
};

template <int N>
static TeamPlan<N> team_plan(int64_t T, bool with_traj) {
  TeamPlan<N> pl{};
  pl.G0 = team_group0<N>(T);
  size_t off = 0;
  const size_t PE = sizeof(double) * Rec<N>::SIZE;
  const size_t PV = sizeof(double) * team::val_doubles<N>();
  const size_t PM = sizeof(double) * (N * N + N);
  int64_t c = T + 1;
  int G = pl.G0;
  while (c > G) {
    const int64_t nc = tdiv(c, G);
    pl.cnt[pl.nlev] = nc;
    pl.off_agg[pl.nlev] = off;
    off = tal(off + nc * PE);
    pl.off_val[pl.nlev] = off;
    off = tal(off + nc * PV);
    ++pl.nlev;
    c = nc;
    G = 2;
  }
  pl.off_maps = off;
  if (with_traj) {
    off = tal(off + (size_t)T * PM);
    int64_t mc = tdiv(T + 1, pl.G0) - 1;
    while (mc > 0) {
      pl.tcnt[pl.tlev] = mc;
      pl.off_tmap[pl.tlev] = off;
      off = tal(off + mc * PM);
      pl.off_tstart[pl.tlev] = off;
      off = tal(off + (mc + 1) * sizeof(double) * N);
      ++pl.tlev;
      if (mc <= 2) break;
      mc = tdiv(mc, 2);
    }
  }
  pl.off_scratch = off;
  if (!TeamCfg<N>::SMEM) off = tal(off + (size_t)TeamCfg<N>::SLOTS * max_slot_doubles<N>() * sizeof(double));
  pl.bytes = tal(off);
  return pl;
}

template <int N>
static unsigned team_grid(int64_t work, int64_t s = TeamCfg<N>::SLOTS) {
  return (unsigned)(work < s ? (work > 0 ? work : 1) : s);
}

template <int N, class Kern, class Args, class... More>
static void team_launch(Kern k, int64_t work, size_t smem_doubles, const Args& a, cudaStream_t st,
                        int64_t slots = TeamCfg<N>::SLOTS, More... more) {
  const size_t smem = TeamCfg<N>::SMEM ? smem_doubles * sizeof(double) : 0;
  if (smem > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k<<<team_grid<N>(work, slots), TeamCfg<N>::TEAM, smem, st>>>(a, more...);
  count_launch();
}

// Elements of the public layout can be staged by TMA when every array is
// 16-byte aligned.
static int bulk_ok(const ElemPtrs& el) {
  const uintptr_t m = (uintptr_t)el.A | (uintptr_t)el.b | (uintptr_t)el.C | (uintptr_t)el.eta | (uintptr_t)el.J;
  return (m & 15) == 0 ? 1 : 0;
}

template <int N, typename GT>
static void launch_reduce(const TeamScanArgs& a, int64_t groups, cudaStream_t st) {
  if constexpr (N == 16) {
    reduce_w16_kernel<GT><<<(unsigned)(groups < TeamCfg<16>::SCAN_SLOTS ? (groups > 0 ? groups : 1)
                                                                         : TeamCfg<16>::SCAN_SLOTS),
                            32, kW16ReduceSmem * sizeof(double), st>>>(a, a.src == nullptr ? bulk_ok(a.el) : 0);
    count_launch();
  } else if constexpr (kTensorProducts<N, GT> || kSharedScratch<N, GT>) {
    const size_t smem = kTensorProducts<N, GT> ? kTcReduceSmemBytes<N> : kReduceSmemBytes<N>;
    TeamScanArgs b = a;
    b.bulk = (kSharedScratch<N, GT> && a.src == nullptr) ? bulk_ok(a.el) : 0;
    cudaFuncSetAttribute(reduce_team_kernel<N, GT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    reduce_team_kernel<N, GT><<<team_grid<N>(groups, TeamCfg<N>::SCAN_SLOTS), TeamCfg<N>::TEAM, smem, st>>>(b);
    count_launch();
  } else {
    team_launch<N>(reduce_team_kernel<N, GT>, groups, reduce_slot_doubles<N>(), a, st, TeamCfg<N>::SCAN_SLOTS);
  }
}

template <int N, bool Level0, typename GT>
static void launch_down(const TeamScanArgs& a, int64_t groups, cudaStream_t st) {
  if constexpr (N == 16) {
    down_w16_kernel<Level0, GT><<<(unsigned)(groups < TeamCfg<16>::SCAN_SLOTS ? (groups > 0 ? groups : 1)
                                                                              : TeamCfg<16>::SCAN_SLOTS),
                                  32, kW16DownSmem * sizeof(double), st>>>(a, a.src == nullptr ? bulk_ok(a.el) : 0);
    count_launch();
  } else if constexpr (kTensorProducts<N, GT> || kSharedScratch<N, GT>) {
    const size_t smem = kTensorProducts<N, GT> ? kTcDownSmemBytes<N> : kDownSmemBytes<N>;
    TeamScanArgs b = a;
    b.bulk = (kSharedScratch<N, GT> && a.src == nullptr) ? bulk_ok(a.el) : 0;
    cudaFuncSetAttribute(down_team_kernel<N, Level0, GT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    down_team_kernel<N, Level0, GT><<<team_grid<N>(groups, TeamCfg<N>::SCAN_SLOTS), TeamCfg<N>::TEAM, smem, st>>>(b);
    count_launch();
  } else {
    team_launch<N>(down_team_kernel<N, Level0, GT>, groups, down_slot_doubles<N>(), a, st, TeamCfg<N>::SCAN_SLOTS);
  }
}

template <int N, int M>
static cudaError_t team_build_nm(const lqt_problem& p, const Coefs& cf, const ElemPtrs& out, double* gscratch,
                                 cudaStream_t st) {
  TeamBuildArgs a{p.T, p.K, p.t, cf, out, gscratch};
  team_launch<N>(build_team_kernel<N, M>, p.T, build_slot_doubles<N, M>(), a, st, TeamCfg<N>::BUILD_SLOTS);
  return cudaGetLastError();
}

template <int N, typename GT>
static cudaError_t team_run_g(const lqt_problem& p, const Coefs& cf, const ElemPtrs& el, double* S, double* v,
                            double* zeta, const double* x0, double* x, double* u, double* cost, bool do_value,
                            bool do_traj, char* ws, cudaStream_t st) {
  const TeamPlan<N> pl = team_plan<N>(p.T, do_traj);
  double* gs = TeamCfg<N>::SMEM ? nullptr : (double*)(ws + pl.off_scratch);
  double* maps0 = (double*)(ws + pl.off_maps);
  double* comp1 = pl.tlev > 0 ? (double*)(ws + pl.off_tmap[0]) : nullptr;
  if (do_value) {
    int64_t c = p.T + 1;
    int G = pl.G0;
    for (int l = 0; l < pl.nlev; ++l) {
      TeamScanArgs a{};
      a.el = el; a.src = l ? (const double*)(ws + pl.off_agg[l - 1]) : nullptr; a.cnt = c; a.G = G;
      a.agg = (double*)(ws + pl.off_agg[l]); a.T = p.T; a.gscratch = gs;
      launch_reduce<N, GT>(a, pl.cnt[l], st);
      c = pl.cnt[l];
      G = 2;
    }
    for (int l = pl.nlev; l >= 0; --l) {
      TeamScanArgs a{};
      a.el = el;
      a.src = l ? (const double*)(ws + pl.off_agg[l - 1]) : nullptr;
      a.cnt = l ? pl.cnt[l - 1] : p.T + 1;
      a.G = l ? 2 : pl.G0;
      a.above = l < pl.nlev ? (const double*)(ws + pl.off_val[l]) : nullptr;
      a.cnt_above = l < pl.nlev ? pl.cnt[l] : 0;
      a.T = p.T;
      a.gscratch = gs;
      const int64_t groups = tdiv(a.cnt, a.G);
      if (l == 0) {
        a.S = S; a.v = v; a.zeta = zeta;
        a.maps = do_traj ? maps0 : nullptr;
        a.comp = do_traj ? comp1 : nullptr;
        launch_down<N, true, GT>(a, groups, st);
      } else {
        a.vals = (double*)(ws + pl.off_val[l - 1]);
        launch_down<N, false, GT>(a, groups, st);
      }
    }
  } else if (do_traj) {
    return cudaErrorNotSupported;
  }
  if (!do_traj) return cudaGetLastError();
  for (int l = 1; l < pl.tlev; ++l) {
    TeamMapArgs a{};
    a.maps = (const double*)(ws + pl.off_tmap[l - 1]); a.cnt = pl.tcnt[l - 1]; a.G = 2;
    a.comp = (double*)(ws + pl.off_tmap[l]); a.gscratch = gs;
    team_launch<N>(reduce_maps_team_kernel<N>, pl.tcnt[l], maps_slot_doubles<N>(), a, st);
  }
  for (int l = pl.tlev - 1; l >= 0; --l) {
    TeamMapArgs a{};
    a.maps = (const double*)(ws + pl.off_tmap[l]); a.cnt = pl.tcnt[l];
    a.G = (l + 1 < pl.tlev) ? 2 : (int)pl.tcnt[l];
    a.above = (l + 1 < pl.tlev) ? (const double*)(ws + pl.off_tstart[l + 1]) : nullptr;
    a.x_in = x0; a.starts = (double*)(ws + pl.off_tstart[l]); a.gscratch = gs;
    team_launch<N>(down_maps_team_kernel<N>, tdiv(pl.tcnt[l], a.G), maps_slot_doubles<N>(), a, st);
  }
  TeamFinalArgs f{};
  f.maps = maps0; f.T = p.T; f.G = pl.G0;
  f.starts1 = pl.tlev > 0 ? (const double*)(ws + pl.off_tstart[0]) : nullptr;
  f.x0 = x0; f.S = S; f.v = v; f.zeta = zeta; f.Ku = cf.Ku; f.Ku_per_boundary = cf.Ku_per_boundary; f.m = p.m;
  f.x = x; f.u = u; f.cost = cost; f.gscratch = gs;
  team_launch<N>(final_team_kernel<N>, tdiv(p.T + 1, pl.G0), maps_slot_doubles<N>(), f, st);
  return cudaGetLastError();
}

// Upper levels of the thread-per-element scans (lqt_scan.cu), n = 4 and 8:
// one warp per pair with the register Gauss-Jordan combinations of
// lqt_warp8.cuh, records in the full-matrix layout (full_elem_doubles,
// full_val_doubles), staged in shared memory by coalesced loads.
template <int N, typename GT>
__global__ void __launch_bounds__(32) reduce_w8_kernel(const double* __restrict__ src, int64_t cnt,
                                                       double* __restrict__ agg) {
  using L = w8::Lay<N>;
  __shared__ double e1[L::REC], e2[L::REC], out[L::REC], scr[L::SCRATCH];
  const int lane = threadIdx.x;
  const int64_t groups = tdiv(cnt, 2);
  for (int64_t g = blockIdx.x; g < groups; g += gridDim.x) {
    const int64_t first = 2 * g;
    double* dst = agg + g * L::REC;
    if (first + 1 >= cnt) {
      for (int e = lane; e < L::REC; e += 32) dst[e] = src[first * L::REC + e];
      continue;
    }
    for (int e = lane; e < L::REC; e += 32) {
      e1[e] = src[first * L::REC + e];
      e2[e] = src[(first + 1) * L::REC + e];
    }
    __syncwarp();
    w8::combine<N, GT>(lane, e1, e2, out, scr);
    for (int e = lane; e < L::REC; e += 32) dst[e] = out[e];
    __syncwarp();
  }
}

template <int N, typename GT>
__global__ void __launch_bounds__(32) down_w8_kernel(const double* __restrict__ src, int64_t cnt,
                                                     const double* __restrict__ above, int64_t cnt_above,
                                                     double* __restrict__ vals) {
  using L = w8::Lay<N>;
  __shared__ double e[L::REC], c0[L::VAL], c1[L::VAL], scr[L::SCRATCH];
  const int lane = threadIdx.x;
  const int64_t groups = tdiv(cnt, 2);
  for (int64_t g = blockIdx.x; g < groups; g += gridDim.x) {
    const int64_t first = 2 * g;
    const int64_t last = (first + 2 < cnt ? first + 2 : cnt) - 1;
    double* carry = c0;
    double* nv = c1;
    for (int q = lane; q < L::VAL; q += 32)
      carry[q] = (above != nullptr && g + 1 < cnt_above) ? above[(g + 1) * L::VAL + q] : 0.0;
    for (int64_t k = last; k >= first; --k) {
      for (int q = lane; q < L::REC; q += 32) e[q] = src[k * L::REC + q];
      __syncwarp();
      w8::combine_value<N, GT>(lane, e, carry, nv, scr);
      for (int q = lane; q < L::VAL; q += 32) vals[k * L::VAL + q] = nv[q];
      __syncwarp();
      double* t = carry;
      carry = nv;
      nv = t;
    }
  }
}

template <int N, typename GT>
void team_upper_reduce(const double* src, int64_t cnt, double* agg, cudaStream_t st) {
  static_assert(Rec<N>::SIZE == full_elem_doubles<N>(), "record layouts differ");
  if constexpr (N == 4 || N == 8) {
    team_launch<N>(reduce_w8_kernel<N, GT>, tdiv(cnt, 2), 0, src, st, TeamCfg<N>::SLOTS, cnt, agg);
  } else {
    TeamScanArgs a{};
    a.src = src; a.cnt = cnt; a.G = 2; a.agg = agg;
    team_launch<N>(reduce_team_kernel<N, GT>, tdiv(cnt, 2), reduce_slot_doubles<N>(), a, st);
  }
}

template <int N, typename GT>
void team_upper_down(const double* src, int64_t cnt, const double* above, int64_t cnt_above, double* vals,
                     cudaStream_t st) {
  static_assert(team::val_doubles<N>() == full_val_doubles<N>(), "value layouts differ");
  if constexpr (N == 4 || N == 8) {
    team_launch<N>(down_w8_kernel<N, GT>, tdiv(cnt, 2), 0, src, st, TeamCfg<N>::SLOTS, cnt, above, cnt_above,
                   vals);
  } else {
    TeamScanArgs a{};
    a.src = src; a.cnt = cnt; a.G = 2; a.above = above; a.cnt_above = cnt_above; a.vals = vals;
    team_launch<N>(down_team_kernel<N, false, GT>, tdiv(cnt, 2), down_slot_doubles<N>(), a, st);
  }
}

template <int N>
void team_maps_reduce(const double* maps, int64_t cnt, int G, double* comp, cudaStream_t st) {
  TeamMapArgs a{};
  a.maps = maps; a.cnt = cnt; a.G = G; a.comp = comp;
  team_launch<N>(reduce_maps_team_kernel<N>, tdiv(cnt, G), maps_slot_doubles<N>(), a, st);
}

template <int N>
void team_maps_down(const double* maps, int64_t cnt, int G, const double* above, const double* x_in, double* starts,
                    cudaStream_t st) {
  TeamMapArgs a{};
  a.maps = maps; a.cnt = cnt; a.G = G; a.above = above; a.x_in = x_in; a.starts = starts;
  team_launch<N>(down_maps_team_kernel<N>, tdiv(cnt, G), maps_slot_doubles<N>(), a, st);
}

// Exclusive prefixes of the level-l aggregates of the Method 2 prefix scan:
// pre[2g] = pre_up[g], pre[2g+1] = pre_up[g] (x) agg[2g] (pre_up = the level
// above; at the top level, the identity element).  One warp per pair.
struct TeamPrefixArgs {
  const double* agg;     // level-l aggregates, full records
  int64_t cnt;           // entries at level l
  const double* pre_up;  // prefixes of level l+1 (full records), or null at the top
  double* pre;           // out: prefixes of level l
  double* gscratch;      // per-CTA slots (teams whose buffers live in global memory)
};

template <int N>
constexpr int prefix_slot_doubles() { return Rec<N>::SIZE + team::combine_scratch_doubles<N>() + 8; }

template <int N>
__global__ void __launch_bounds__(TeamCfg<N>::TEAM) prefix_down_team_kernel(TeamPrefixArgs a) {
  constexpr int TEAM = TeamCfg<N>::TEAM;
  __shared__ double fs[2 * TEAM];
  __shared__ int is[TEAM];
  const int lane = threadIdx.x;
  double* base = slot_base<N>(a.gscratch, prefix_slot_doubles<N>());
  double* ident = base;
  double* scr = ident + Rec<N>::SIZE;
  for (int e = lane; e < Rec<N>::SIZE; e += TEAM) ident[e] = (e < N * N && e % (N + 1) == 0) ? 1.0 : 0.0;
  team::sync<TEAM>();
  const int64_t groups = tdiv(a.cnt, 2);
  for (int64_t g = blockIdx.x; g < groups; g += gridDim.x) {
    const Rec<N> left = a.pre_up ? Rec<N>::packed(const_cast<double*>(a.pre_up) + g * Rec<N>::SIZE)
                                 : Rec<N>::packed(ident);
    team::copy_rec<N, TEAM>(lane, Rec<N>::packed(a.pre + 2 * g * Rec<N>::SIZE), left);
    if (2 * g + 1 < a.cnt)
      team::combine<N, TEAM>(lane, left, Rec<N>::packed(const_cast<double*>(a.agg) + 2 * g * Rec<N>::SIZE),
                             Rec<N>::packed(a.pre + (2 * g + 1) * Rec<N>::SIZE), scr, fs, is);
    team::sync<TEAM>();
  }
}

template <int N>
void team_prefix_down(const double* agg, int64_t cnt, const double* pre_up, double* pre, cudaStream_t st,
                      double* gscratch) {
  TeamPrefixArgs a{agg, cnt, pre_up, pre, gscratch};
  team_launch<N>(prefix_down_team_kernel<N>, tdiv(cnt, 2), prefix_slot_doubles<N>(), a, st);
}

// ---------------------------------------------------------------------------
// Method 2 of the trajectory recovery (Sec. IV-E, eq.
// Opt_trajectory_method2), n = 16 and 64
// ---------------------------------------------------------------------------

// The forward elements' prefixes V(., t_0; ., t_k) = a_0 (x) ... (x) a_{k-1}:
// chunk aggregates by the value scan's reduce kernels (the same combination,
// Sec. IV-A eq. lqt_comb), their exclusive prefixes by prefix_down_team_kernel,
// and in each level-0 chunk a team folds the chunk's elements onto the chunk's
// prefix left to right, emitting at every boundary k
//   x_k = (I + C_k S_k)^-1 (A_k x0 + b_k + C_k v_k),  u_k = Ku (v_k - S_k x_k).
struct TeamM2Args {
  ElemPtrs el;         // forward-ODE elements, T of them
  int64_t T;
  int G;               // level-0 chunk length
  const double* pre0;  // exclusive prefixes of the level-0 chunks (packed), or null (one chunk)
  const double *S, *v, *zeta, *x0, *Ku;
  int32_t Ku_per_boundary, m;
  double *x, *u, *cost;
  double* gscratch;
  int bulk;            // n = 16: stage the elements by TMA
};

// Per-team buffers: the prefix P and (n = 16) the staged element or (n = 64)
// the prefix's successor, the combination's scratch, then W (N x N), r, e (N).
template <int N>
constexpr int m2_rec_doubles() { return N == 16 ? w16::kRecPad : Rec<N>::SIZE; }
template <int N>
constexpr int m2_scratch_doubles() { return N == 16 ? w16::kScratch : team::combine_scratch_doubles<N>(); }
template <int N>
constexpr int m2_slot_doubles() { return 2 * m2_rec_doubles<N>() + m2_scratch_doubles<N>() + N * N + 2 * N + 8; }

// State and control at boundary k from the prefix P (packed record).
template <int N, int TEAM>
__device__ void m2_state(int lane, const TeamM2Args& a, int64_t k, const double* P, double* W, double* r,
                         double* ev, double* fs, int* is) {
  const double* PA = P;
  const double* Pb = P + N * N;
  const double* PC = P + N * N + N;
  const double* Sk = a.S + k * N * N;
  const double* vk = a.v + k * N;
  team::gemm<N, N, N, TEAM, double>(
      lane, [&](int i, int l) { return PC[i * N + l]; }, [&](int l, int j) { return Sk[l * N + j]; },
      [&](int i, int j, double s) { W[i * N + j] = s + (i == j ? 1.0 : 0.0); });
  for (int i = lane; i < N; i += TEAM) {
    double s = Pb[i];
    for (int l = 0; l < N; ++l) {
      s = fma(PA[i * N + l], a.x0[l], s);
      s = fma(PC[i * N + l], vk[l], s);
    }
    r[i] = s;
  }
  team::sync<TEAM>();
  team::lu_solve<N, TEAM, 1>(lane, W, r, fs, is);
  for (int i = lane; i < N; i += TEAM) {
    a.x[k * N + i] = r[i];
    if (!isfinite(r[i])) flag(kStatusNonFinite);
  }
  if (a.u) {
    for (int i = lane; i < N; i += TEAM) {
      double s = vk[i];
      for (int l = 0; l < N; ++l) s = fma(-Sk[i * N + l], r[l], s);
      ev[i] = s;
    }
    team::sync<TEAM>();
    const double* Kk = a.Ku + (a.Ku_per_boundary ? k * a.m * N : 0);
    for (int q = lane; q < a.m; q += TEAM) {
      double s = 0.0;
      for (int l = 0; l < N; ++l) s = fma(Kk[q * N + l], ev[l], s);
      a.u[k * a.m + q] = s;
    }
  }
  team::sync<TEAM>();
}

template <int N>
__global__ void __launch_bounds__(TeamCfg<N>::TEAM) method2_team_kernel(TeamM2Args a) {
  constexpr int TEAM = TeamCfg<N>::TEAM;
  constexpr int RS = Rec<N>::SIZE;
  __shared__ double fs[2 * TEAM];
  __shared__ int is[TEAM];
  __shared__ unsigned long long bar;
  __shared__ double zero;
  const int lane = threadIdx.x;
  extern __shared__ __align__(16) double m2_smem[];
  double *P, *Pn, *scr;
  if constexpr (N == 16) {
    P = m2_smem;
    Pn = P + m2_rec_doubles<N>();
    scr = Pn + m2_rec_doubles<N>();
  } else {
    // the records in the slot, the scratch (W, r, e included) in shared memory
    P = slot_base<N>(a.gscratch, m2_slot_doubles<N>());
    Pn = P + m2_rec_doubles<N>();
    scr = m2_smem;
  }
  double* W = scr + m2_scratch_doubles<N>();
  double* r = W + N * N;
  double* ev = r + N;
  if (lane == 0) {
    zero = 0.0;
    if constexpr (N == 16) w16::mbar_init(&bar, 1);
  }
  team::sync<TEAM>();
  unsigned phase = 0;
  const int64_t groups = tdiv(a.T, a.G);
  for (int64_t g = blockIdx.x; g < groups; g += gridDim.x) {
    const int64_t first = g * a.G;
    const int64_t last = (first + a.G < a.T ? first + a.G : a.T) - 1;
    for (int e = lane; e < RS; e += TEAM)
      P[e] = a.pre0 ? a.pre0[g * RS + e] : ((e < N * N && e % (N + 1) == 0) ? 1.0 : 0.0);
    team::sync<TEAM>();
    for (int64_t k = first; k <= last; ++k) {
      m2_state<N, TEAM>(lane, a, k, P, W, r, ev, fs, is);
      if constexpr (N == 16) {
        w16::stage(lane, w16::ElemSrc{a.el, nullptr, a.bulk != 0}, k, Pn, &bar, phase, &zero);
        w16::combine<double>(lane, P, Pn, scr);
      } else {
        team::combine<N, TEAM>(lane, Rec<N>::packed(P), Rec<N>::pub(a.el, k, &zero), Rec<N>::packed(Pn), scr, fs,
                               is);
        double* t = P;
        P = Pn;
        Pn = t;
      }
    }
    if (last == a.T - 1) m2_state<N, TEAM>(lane, a, a.T, P, W, r, ev, fs, is);
    if (g == 0 && a.cost != nullptr && lane == 0) {
      double c = a.zeta ? a.zeta[0] : 0.0;
      for (int i = 0; i < N; ++i) {
        double s = 0.0;
        for (int l = 0; l < N; ++l) s = fma(a.S[i * N + l], a.x0[l], s);
        c = fma(a.x0[i], fma(0.5, s, -a.v[i]), c);
      }
      *a.cost = c;
    }
    team::sync<TEAM>();
  }
}

template <int N>
struct TeamPrefixPlan {
  int G0;
  int nlev;
  int64_t cnt[64];
  size_t off_agg[64], off_pre[64];
  size_t off_scratch;
  size_t bytes;
};

template <int N>
static TeamPrefixPlan<N> team_prefix_plan(int64_t T) {
  TeamPrefixPlan<N> pl{};
  pl.G0 = team_group0<N>(T - 1);
  const size_t PE = sizeof(double) * Rec<N>::SIZE;
  size_t off = 0;
  int64_t c = T;
  int G = pl.G0;
  while (c > G) {
    const int64_t nc = tdiv(c, G);
    pl.cnt[pl.nlev] = nc;
    pl.off_agg[pl.nlev] = off;
    off = tal(off + nc * PE);
    pl.off_pre[pl.nlev] = off;
    off = tal(off + nc * PE);
    ++pl.nlev;
    c = nc;
    G = 2;
  }
  pl.off_scratch = off;
  if (!TeamCfg<N>::SMEM) {
    size_t sd = m2_slot_doubles<N>();
    if ((size_t)reduce_slot_doubles<N>() > sd) sd = reduce_slot_doubles<N>();
    if ((size_t)prefix_slot_doubles<N>() > sd) sd = prefix_slot_doubles<N>();
    off = tal(off + (size_t)TeamCfg<N>::SLOTS * sd * sizeof(double));
  }
  pl.bytes = tal(off);
  return pl;
}

template <int N>
static cudaError_t team_method2_n(const lqt_problem& p, const Coefs& cf, const ElemPtrs& fwd, const double* S,
                                 const double* v, const double* zeta, const double* x0, double* x, double* u,
                                 double* cost, char* ws, cudaStream_t st) {
  const TeamPrefixPlan<N> pl = team_prefix_plan<N>(p.T);
  double* gs = TeamCfg<N>::SMEM ? nullptr : (double*)(ws + pl.off_scratch);
  int64_t c = p.T;
  int G = pl.G0;
  for (int l = 0; l < pl.nlev; ++l) {
    TeamScanArgs a{};
    a.el = fwd; a.src = l ? (const double*)(ws + pl.off_agg[l - 1]) : nullptr; a.cnt = c; a.G = G;
    a.agg = (double*)(ws + pl.off_agg[l]); a.T = p.T; a.gscratch = gs;
    launch_reduce<N, double>(a, pl.cnt[l], st);
    c = pl.cnt[l];
    G = 2;
  }
  for (int l = pl.nlev - 1; l >= 0; --l) {
    const double* up = l + 1 < pl.nlev ? (const double*)(ws + pl.off_pre[l + 1]) : nullptr;
    team_prefix_down<N>((const double*)(ws + pl.off_agg[l]), pl.cnt[l], up, (double*)(ws + pl.off_pre[l]), st, gs);
  }
  TeamM2Args a{};
  a.el = fwd; a.T = p.T; a.G = pl.G0;
  a.pre0 = pl.nlev > 0 ? (const double*)(ws + pl.off_pre[0]) : nullptr;
  a.S = S; a.v = v; a.zeta = zeta; a.x0 = x0;
  a.Ku = cf.Ku; a.Ku_per_boundary = cf.Ku_per_boundary; a.m = p.m;
  a.x = x; a.u = u; a.cost = cost; a.gscratch = gs; a.bulk = bulk_ok(fwd);
  if constexpr (N == 64) {
    const size_t smem = sizeof(double) * (m2_scratch_doubles<N>() + N * N + 2 * N);
    cudaFuncSetAttribute(method2_team_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    method2_team_kernel<N><<<team_grid<N>(tdiv(p.T, pl.G0)), TeamCfg<N>::TEAM, smem, st>>>(a);
    count_launch();
  } else {
    team_launch<N>(method2_team_kernel<N>, tdiv(p.T, pl.G0), m2_slot_doubles<N>(), a, st);
  }
  return cudaGetLastError();
}

size_t team_prefix_workspace_bytes(int n, int64_t T) {
  switch (n) {
    case 16: return team_prefix_plan<16>(T).bytes;
    case 64: return team_prefix_plan<64>(T).bytes;
    default: return 0;
  }
}

cudaError_t team_run_method2(const lqt_problem& p, const Coefs& cf, const ElemPtrs& fwd, const double* S,
                             const double* v, const double* zeta, const double* x0, double* x, double* u,
                             double* cost, char* ws, cudaStream_t st) {
  switch (p.n) {
    case 16: return team_method2_n<16>(p, cf, fwd, S, v, zeta, x0, x, u, cost, ws, st);
    case 64: return team_method2_n<64>(p, cf, fwd, S, v, zeta, x0, x, u, cost, ws, st);
    default: return cudaErrorInvalidValue;
  }
}

template <int N, int M>
static cudaError_t team_fwd_nm(const lqt_problem& p, const Coefs& cf, const ElemPtrs& out, double* gscratch,
                               cudaStream_t st) {
  TeamBuildArgs a{p.T, p.K, p.t, cf, out, gscratch};
  // n = 16: 29.9 KB of shared memory per warp, 7 warps per SM
  team_launch<N>(build_forward_team_kernel<N, M>, p.T, forward_slot_doubles<N>(), a, st,
                 N == 16 ? 152 * 7 : TeamCfg<N>::SLOTS);
  return cudaGetLastError();
}

cudaError_t team_launch_build_forward(const lqt_problem& p, const Layout& lay, const Coefs& cf, const ElemPtrs& out,
                                      double* gscratch, cudaStream_t st) {
  switch (p.n) {
    case 16:
      switch (lay.M) {
        case 1: return team_fwd_nm<16, 1>(p, cf, out, gscratch, st);
        case 2: return team_fwd_nm<16, 2>(p, cf, out, gscratch, st);
        case 4: return team_fwd_nm<16, 4>(p, cf, out, gscratch, st);
        case 8: return team_fwd_nm<16, 8>(p, cf, out, gscratch, st);
        case 16: return team_fwd_nm<16, 16>(p, cf, out, gscratch, st);
        default: return cudaErrorInvalidValue;
      }
    case 64:
      switch (lay.M) {
        case 16: return team_fwd_nm<64, 16>(p, cf, out, gscratch, st);
        default: return cudaErrorInvalidValue;
      }
    default: return cudaErrorInvalidValue;
  }
}

// Time-invariant element build (lqt_invariant.cu), n = 16 and 64: the shared
// A, C, J integration by one team per problem.  The full element is integrated
// with zero r and c (the b, eta, zeta parts are unused here and cost O(n^2));
// after every right-hand side the stage's AL = A Lt, P = J Lt (the RHS's own
// scratch) and its input A, J are recorded into the problem's table, laid out
// as the thread integrator's (inv_table_doubles).
struct InvTeamMasterArgs {
  int32_t K, B;
  const BatchProb* probs;  // batch descriptors, or null (single problem: t, cf)
  const double* t;
  Coefs cf;
  double* tables;
  int64_t table_doubles;
};

template <int N, int M>
__global__ void __launch_bounds__(TeamCfg<N>::TEAM) inv_master_team_kernel(InvTeamMasterArgs a) {
  constexpr int TEAM = TeamCfg<N>::TEAM;
  constexpr int SZ = Rec<N>::SIZE;
  constexpr int64_t SD = 2 * N * M + 2 * N * N;
  const int lane = threadIdx.x;
  const int K = a.K;
  for (int64_t b = blockIdx.x; b < a.B; b += gridDim.x) {
    const Coefs& cf = a.probs ? a.probs[b].cf : a.cf;
    const double* t = a.probs ? a.probs[b].t : a.t;
    double* table = a.tables + b * a.table_doubles;
    double* fin = table + 4 * (int64_t)K * SD;
    double* yb = fin + 3 * N * N;
    double* ynb = yb + SZ;
    double* ytb = ynb + SZ;
    double* kb = ytb + SZ;
    double* AL = kb + SZ;
    double* P = AL + N * M;
    double* w = P + N * M;
    double* JF = w + M;
    double* zq = JF + N * N;  // N + 1 zeros: q = 0, rho = 0
    const Rec<N> y = Rec<N>::packed(yb), yn = Rec<N>::flow(ynb), yt = Rec<N>::flow(ytb), k = Rec<N>::flow(kb);
    for (int e = lane; e < SZ; e += TEAM) yb[e] = (e < N * N && e % (N + 1) == 0) ? 1.0 : 0.0;
    for (int e = lane; e <= N; e += TEAM) zq[e] = 0.0;
    team::sync<TEAM>();
    const double h = (t[1] - t[0]) / K;
    const double* F = cf.F.ptr;
    const double* Lt = cf.Lt.ptr;
    const double* Q = cf.Q.ptr;
    auto record = [&](double* rec, const Rec<N>& st) {
      for (int e = lane; e < N * M; e += TEAM) {
        rec[e] = AL[e];
        rec[N * M + e] = P[e];
      }
      for (int e = lane; e < N * N; e += TEAM) {
        rec[2 * N * M + e] = st.A()[e];
        rec[2 * N * M + N * N + e] = st.J()[e];
      }
    };
    for (int32_t i = K - 1; i >= 0; --i) {
      double* rec = table + 4 * (int64_t)i * SD;
      team::rhs<N, M, TEAM>(lane, y, k, F, nullptr, Lt, Q, zq, AL, P, w, -h / 6.0, y);
      record(rec, y);
      team::axpy_flow<N, TEAM>(lane, yn, y, -h / 6.0, k);
      team::axpy_flow<N, TEAM>(lane, yt, y, -0.5 * h, k);
      team::rhs<N, M, TEAM>(lane, yt, k, F, nullptr, Lt, Q, zq, AL, P, w, -h / 3.0, y);
      record(rec + SD, yt);
      team::axpy_flow<N, TEAM>(lane, yn, yn, -h / 3.0, k);
      team::axpy_flow<N, TEAM>(lane, yt, y, -0.5 * h, k);
      team::rhs<N, M, TEAM>(lane, yt, k, F, nullptr, Lt, Q, zq, AL, P, w, -h / 3.0, y);
      record(rec + 2 * SD, yt);
      team::axpy_flow<N, TEAM>(lane, yn, yn, -h / 3.0, k);
      team::axpy_flow<N, TEAM>(lane, yt, y, -h, k);
      team::rhs<N, M, TEAM>(lane, yt, k, F, nullptr, Lt, Q, zq, AL, P, w, -h / 6.0, y);
      record(rec + 3 * SD, yt);
      team::axpy_flow<N, TEAM>(lane, y, yn, -h / 6.0, k);
    }
    for (int e = lane; e < N * N; e += TEAM) {
      fin[e] = y.A()[e];
      fin[N * N + e] = y.C()[e];
      fin[2 * N * N + e] = y.J()[e];
    }
    team::sync<TEAM>();
  }
}

template <int N, int M>
void launch_inv_master_team(int32_t K, int32_t B, const BatchProb* probs, const double* t, const Coefs& cf,
                            double* tables, int64_t table_doubles, cudaStream_t st) {
  InvTeamMasterArgs a{K, B, probs, t, cf, tables, table_doubles};
  const unsigned grid = (unsigned)(B < TeamCfg<N>::SLOTS ? B : TeamCfg<N>::SLOTS);
  inv_master_team_kernel<N, M><<<grid, TeamCfg<N>::TEAM, 0, st>>>(a);
  count_launch();
}
template void launch_inv_master_team<16, 8>(int32_t, int32_t, const BatchProb*, const double*, const Coefs&, double*,
                                            int64_t, cudaStream_t);
template void launch_inv_master_team<64, 16>(int32_t, int32_t, const BatchProb*, const double*, const Coefs&,
                                             double*, int64_t, cudaStream_t);

#define LQT_TEAM_UPPER(N)                                                                                 \
  template void team_upper_reduce<N, double>(const double*, int64_t, double*, cudaStream_t);             \
  template void team_upper_reduce<N, float>(const double*, int64_t, double*, cudaStream_t);              \
  template void team_upper_down<N, double>(const double*, int64_t, const double*, int64_t, double*,      \
                                           cudaStream_t);                                                \
  template void team_upper_down<N, float>(const double*, int64_t, const double*, int64_t, double*,       \
                                          cudaStream_t);                                                 \
  template void team_maps_reduce<N>(const double*, int64_t, int, double*, cudaStream_t);                 \
  template void team_maps_down<N>(const double*, int64_t, int, const double*, const double*, double*,    \
                                  cudaStream_t);                                                         \
  template void team_prefix_down<N>(const double*, int64_t, const double*, double*, cudaStream_t, double*);
LQT_TEAM_UPPER(1)
LQT_TEAM_UPPER(2)
LQT_TEAM_UPPER(3)
LQT_TEAM_UPPER(4)
LQT_TEAM_UPPER(8)
#undef LQT_TEAM_UPPER

template <int N>
static cudaError_t team_concat(int64_t Tcat, const ElemPtrs& el, double* S, double* v, double* zeta,
                               const double* x0_first, double* x, const BoundaryPatch& patch, char* ws,
                               cudaStream_t st) {
  const TeamPlan<N> pl = team_plan<N>(Tcat, true);
  double* gs = TeamCfg<N>::SMEM ? nullptr : (double*)(ws + pl.off_scratch);
  double* maps0 = (double*)(ws + pl.off_maps);
  // value scan with the level-0 maps
  int64_t c = Tcat + 1;
  int G = pl.G0;
  for (int l = 0; l < pl.nlev; ++l) {
    TeamScanArgs a{};
    a.el = el; a.src = l ? (const double*)(ws + pl.off_agg[l - 1]) : nullptr; a.cnt = c; a.G = G;
    a.agg = (double*)(ws + pl.off_agg[l]); a.T = Tcat; a.gscratch = gs;
    launch_reduce<N, double>(a, pl.cnt[l], st);
    c = pl.cnt[l];
    G = 2;
  }
  for (int l = pl.nlev; l >= 0; --l) {
    TeamScanArgs a{};
    a.el = el;
    a.src = l ? (const double*)(ws + pl.off_agg[l - 1]) : nullptr;
    a.cnt = l ? pl.cnt[l - 1] : Tcat + 1;
    a.G = l ? 2 : pl.G0;
    a.above = l < pl.nlev ? (const double*)(ws + pl.off_val[l]) : nullptr;
    a.cnt_above = l < pl.nlev ? pl.cnt[l] : 0;
    a.T = Tcat;
    a.gscratch = gs;
    const int64_t groups = tdiv(a.cnt, a.G);
    if (l == 0) {
      a.S = S; a.v = v; a.zeta = zeta; a.maps = maps0; a.comp = nullptr; a.zeta_inc = 1;
      launch_down<N, true, double>(a, groups, st);
    } else {
      a.vals = (double*)(ws + pl.off_val[l - 1]);
      launch_down<N, false, double>(a, groups, st);
    }
  }
  launch_boundary_patch(N, maps0, patch, st);
  // chunk composites of the patched maps, then the state scan
  if (pl.tlev > 0) {
    TeamMapArgs a{};
    a.maps = maps0;
    a.cnt = pl.tcnt[0] * pl.G0 < Tcat ? pl.tcnt[0] * pl.G0 : Tcat;
    a.G = pl.G0;
    a.comp = (double*)(ws + pl.off_tmap[0]);
    a.gscratch = gs;
    team_launch<N>(reduce_maps_team_kernel<N>, pl.tcnt[0], maps_slot_doubles<N>(), a, st);
  }
  for (int l = 1; l < pl.tlev; ++l) {
    TeamMapArgs a{};
    a.maps = (const double*)(ws + pl.off_tmap[l - 1]); a.cnt = pl.tcnt[l - 1]; a.G = 2;
    a.comp = (double*)(ws + pl.off_tmap[l]); a.gscratch = gs;
    team_launch<N>(reduce_maps_team_kernel<N>, pl.tcnt[l], maps_slot_doubles<N>(), a, st);
  }
  for (int l = pl.tlev - 1; l >= 0; --l) {
    TeamMapArgs a{};
    a.maps = (const double*)(ws + pl.off_tmap[l]); a.cnt = pl.tcnt[l];
    a.G = (l + 1 < pl.tlev) ? 2 : (int)pl.tcnt[l];
    a.above = (l + 1 < pl.tlev) ? (const double*)(ws + pl.off_tstart[l + 1]) : nullptr;
    a.x_in = x0_first; a.starts = (double*)(ws + pl.off_tstart[l]); a.gscratch = gs;
    team_launch<N>(down_maps_team_kernel<N>, tdiv(pl.tcnt[l], a.G), maps_slot_doubles<N>(), a, st);
  }
  TeamFinalArgs f{};
  f.maps = maps0; f.T = Tcat; f.G = pl.G0;
  f.starts1 = pl.tlev > 0 ? (const double*)(ws + pl.off_tstart[0]) : nullptr;
  f.x0 = x0_first; f.S = S; f.v = v; f.zeta = zeta; f.Ku = nullptr; f.m = 0;
  f.x = x; f.u = nullptr; f.cost = nullptr; f.gscratch = gs;
  team_launch<N>(final_team_kernel<N>, tdiv(Tcat + 1, pl.G0), maps_slot_doubles<N>(), f, st);
  return cudaGetLastError();
}

size_t team_concat_workspace_bytes(int32_t n, int64_t Tcat) { return team_scan_workspace_bytes(n, Tcat, true); }

cudaError_t team_concat_scan(int32_t n, int64_t Tcat, const ElemPtrs& el, double* S, double* v, double* zeta,
                             const double* x0_first, double* x, const BoundaryPatch& patch, char* ws,
                             cudaStream_t st) {
  switch (n) {
    case 16: return team_concat<16>(Tcat, el, S, v, zeta, x0_first, x, patch, ws, st);
    case 64: return team_concat<64>(Tcat, el, S, v, zeta, x0_first, x, patch, ws, st);
    default: return cudaErrorInvalidValue;
  }
}

template <int N, int M>
static void batch_build_team_nm(const BatchDev& bd, const ElemPtrs& el, double* gs, cudaStream_t st) {
  const size_t smem = TeamCfg<N>::SMEM ? build_slot_doubles<N, M>() * sizeof(double) : 0;
  batch_build_team_kernel<N, M><<<team_grid<N>(bd.total, TeamCfg<N>::BUILD_SLOTS), TeamCfg<N>::TEAM, smem, st>>>(
      bd, el, gs);
  count_launch();
}

cudaError_t batch_build_team(const BatchDev& bd, const ElemPtrs& el, double* gscratch, cudaStream_t st) {
  if (bd.n == 16) {
    switch (bd.M) {
      case 1: batch_build_team_nm<16, 1>(bd, el, gscratch, st); break;
      case 2: batch_build_team_nm<16, 2>(bd, el, gscratch, st); break;
      case 4: batch_build_team_nm<16, 4>(bd, el, gscratch, st); break;
      case 8: batch_build_team_nm<16, 8>(bd, el, gscratch, st); break;
      case 16: batch_build_team_nm<16, 16>(bd, el, gscratch, st); break;
      default: return cudaErrorInvalidValue;
    }
  } else if (bd.n == 64) {
    batch_build_team_nm<64, 16>(bd, el, gscratch, st);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <int N>
static cudaError_t team_run(const lqt_problem& p, const Coefs& cf, const ElemPtrs& el, double* S, double* v,
                            double* zeta, const double* x0, double* x, double* u, double* cost, bool do_value,
                            bool do_traj, char* ws, cudaStream_t st) {
  if (mixed_precision())
    return team_run_g<N, float>(p, cf, el, S, v, zeta, x0, x, u, cost, do_value, do_traj, ws, st);
  return team_run_g<N, double>(p, cf, el, S, v, zeta, x0, x, u, cost, do_value, do_traj, ws, st);
}

// Build scratch for n = 64: per-slot element buffers of the backward-ODE build
// and of the forward-ODE build of Method 2.
size_t team_build_scratch_bytes(int n) {
  if (n == 64) {
    const size_t sd = build_slot_doubles<64, 16>() > forward_slot_doubles<64>() ? build_slot_doubles<64, 16>()
                                                                                : forward_slot_doubles<64>();
    return tal((size_t)TeamCfg<64>::SLOTS * sd * sizeof(double));
  }
  return 0;
}

bool team_build_preferred(int n, int64_t count) {
  // where one warp per element beats one thread (measured crossing points)
  return (n == 4 && count < 4096) || (n == 8 && count < 24576);
}

template <int N, int M>
static cudaError_t team_range_nm(const lqt_problem& p, const Coefs& cf, int64_t j0, int64_t cnt, double* stages,
                                 const ElemPtrs& out, cudaStream_t st) {
  TeamBuildArgs a{cnt, p.K, p.t, cf, out, nullptr};
  // <= 120 registers and <= 6 KB of shared memory per warp: four warps per
  // sub-partition
  team_launch<N>(build_team_range_kernel<N, M>, cnt, build_slot_doubles<N, M>(), a, st, (int64_t)152 * 16, j0,
                 stages);
  return cudaGetLastError();
}

cudaError_t team_launch_build_small(const lqt_problem& p, const Layout& lay, const Coefs& cf, int64_t j0,
                                    int64_t cnt, double* stages, const ElemPtrs& out, cudaStream_t st) {
  if (cnt <= 0) return cudaSuccess;
  switch (p.n) {
    case 4:
      switch (lay.M) {
        case 1: return team_range_nm<4, 1>(p, cf, j0, cnt, stages, out, st);
        case 2: return team_range_nm<4, 2>(p, cf, j0, cnt, stages, out, st);
        case 4: return team_range_nm<4, 4>(p, cf, j0, cnt, stages, out, st);
        default: return cudaErrorInvalidValue;
      }
    case 8:
      switch (lay.M) {
        case 1: return team_range_nm<8, 1>(p, cf, j0, cnt, stages, out, st);
        case 2: return team_range_nm<8, 2>(p, cf, j0, cnt, stages, out, st);
        case 4: return team_range_nm<8, 4>(p, cf, j0, cnt, stages, out, st);
        case 8: return team_range_nm<8, 8>(p, cf, j0, cnt, stages, out, st);
        default: return cudaErrorInvalidValue;
      }
    default: return cudaErrorInvalidValue;
  }
}

size_t team_scan_workspace_bytes(int32_t n, int64_t T, bool with_traj) {
  switch (n) {
    case 16: return team_plan<16>(T, with_traj).bytes;
    case 64: return team_plan<64>(T, with_traj).bytes;
    default: return 0;
  }
}

cudaError_t team_launch_build(const lqt_problem& p, const Layout& lay, const Coefs& cf, const ElemPtrs& out,
                              double* gscratch, cudaStream_t st) {
  switch (p.n) {
    case 16:
      switch (lay.M) {
        case 1: return team_build_nm<16, 1>(p, cf, out, gscratch, st);
        case 2: return team_build_nm<16, 2>(p, cf, out, gscratch, st);
        case 4: return team_build_nm<16, 4>(p, cf, out, gscratch, st);
        case 8: return team_build_nm<16, 8>(p, cf, out, gscratch, st);
        case 16: return team_build_nm<16, 16>(p, cf, out, gscratch, st);
        default: return cudaErrorInvalidValue;
      }
    case 64:
      switch (lay.M) {
        case 16: return team_build_nm<64, 16>(p, cf, out, gscratch, st);
        default: return cudaErrorInvalidValue;
      }
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t team_run_value_and_traj(const lqt_problem& p, const Coefs& cf, const ElemPtrs& el, double* S, double* v,
                                    double* zeta, const double* x0, double* x, double* u, double* cost, bool do_value,
                                    bool do_traj, char* ws, cudaStream_t st) {
  switch (p.n) {
    case 16: return team_run<16>(p, cf, el, S, v, zeta, x0, x, u, cost, do_value, do_traj, ws, st);
    case 64: return team_run<64>(p, cf, el, S, v, zeta, x0, x, u, cost, do_value, do_traj, ws, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace lqt
