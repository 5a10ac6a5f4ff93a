// Internal declarations shared by the CUDA translation units of the LQT
// library (not part of the C ABI).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/lqt.h"

namespace lqt {

// Device status word bits (read and cleared by lqt_get_status).
constexpr unsigned kStatusNonFinite = 1u;
constexpr unsigned kStatusSingular = 2u;
constexpr unsigned kStatusNonUniform = 4u;  // a time-invariant build met sub-intervals of different lengths
constexpr unsigned kStatusTimeout = 8u;     // a kernel's bounded wait (a TMA copy) gave up

extern __device__ unsigned g_status_word;

// Internal sampling modes of derived coefficients.  The public ones keep their
// values; STAGE_BLOCK holds (2K+1) samples per sub-interval without sharing
// the end points (needed when a per-stage input is combined with a
// per-interval one).
enum : int32_t { kConst = 0, kPerInterval = 1, kPerStage = 2, kStageBlock = 3 };

__host__ __device__ __forceinline__ int64_t sample_index(int32_t mode, int64_t j, int32_t p, int32_t K) {
  switch (mode) {
    case kConst: return 0;
    case kPerInterval: return j;
    case kPerStage: return 2 * (int64_t)K * j + p;
    default: return (2 * (int64_t)K + 1) * j + p;
  }
}

// Number of samples a mode holds.
__host__ __device__ __forceinline__ int64_t sample_count(int32_t mode, int64_t T, int32_t K) {
  switch (mode) {
    case kConst: return 1;
    case kPerInterval: return T;
    case kPerStage: return 2 * (int64_t)K * T + 1;
    default: return (2 * (int64_t)K + 1) * T;
  }
}

struct Coef {
  const double* ptr;
  int32_t mode;
};

// Coefficients in the form the kernels consume (all device pointers):
//   F   n x n                       (input)
//   c   n, NULL = 0                 (input)
//   Lt  n x M: B = L U^-1 L^T = Lt Lt^T (Lt = L R^-T, U = R R^T), zero-padded
//       to M columns                (derived)
//   Q   H^T X H, full n x n (derived; X itself when H is the identity)
//   qr  [H^T X r (n), r^T X r]      (derived, n+1 per sample)
//   Ku  U^-1 L^T (m x n) at the T+1 boundaries (derived; CONST or T+1)
struct Coefs {
  Coef F, c, Lt, Q, qr;
  const double* Ku;
  int32_t Ku_per_boundary;
  int32_t M;  // padded column count of Lt
};

struct ElemPtrs {
  double *A, *b, *C, *eta, *J, *zeta;
};

// Sizes of the internal arrays of one problem.
struct Layout {
  int32_t n, m, nr, K, M;
  int64_t T;
  int32_t mode_Lt, mode_Q, mode_qr;
  // byte offsets inside the workspace
  size_t off_Lt, off_Q, off_qr, off_Ku, off_status;
  size_t coef_bytes;  // end of the coefficient region
};

// Padded factor width for m.
inline int32_t padded_M(int32_t m) { return m <= 1 ? 1 : m <= 2 ? 2 : m <= 4 ? 4 : m <= 8 ? 8 : m <= 16 ? 16 : 64; }

// Combined sampling mode of a derived coefficient from its inputs' modes.
inline int32_t combine_modes(int32_t a, int32_t b) {
  if (a == kConst) return b;
  if (b == kConst) return a;
  if (a == b) return a;
  return kStageBlock;  // one per-interval, one per-stage (or already block)
}

// Launch-count accounting (per host thread).
void count_launch(int k = 1);
void reset_launch_count();

// -------------------------------------------------------------------------
// launchers (defined in the .cu files, dispatched on n)
// -------------------------------------------------------------------------
cudaError_t launch_prepare_coefs(const lqt_problem& p, const Layout& lay, char* ws, Coefs& out, cudaStream_t s);
cudaError_t launch_prepare_into(const lqt_problem& p, const Layout& lay, double* Lt, double* Q, double* qr,
                                double* Ku, Coefs& cf, cudaStream_t st);
Coefs coefs_view(const lqt_problem& p, const Layout& lay, double* Lt, double* Q, double* qr, double* Ku);
cudaError_t launch_build_range(const lqt_problem& p, const Layout& lay, const Coefs& cf, const ElemPtrs& out,
                               cudaStream_t st);
cudaError_t launch_build_stages_range(const lqt_problem& p, const Layout& lay, const Coefs& cf, int64_t j0,
                                      int64_t cnt, double* stages, cudaStream_t st, const ElemPtrs& out);
cudaError_t launch_terminal_element(const lqt_problem& p, const ElemPtrs& out, cudaStream_t st);
cudaError_t launch_build(const lqt_problem& p, const Layout& lay, const Coefs& cf, const ElemPtrs& out,
                         cudaStream_t s, double* team_scratch = nullptr);
// n = 16, 64 (team kernels, lqt_team.cu)
size_t team_build_scratch_bytes(int n);
// n = 4, 8 at short horizons: one warp per element (elements j0 .. j0 + cnt - 1,
// optional RK4 stage inputs as launch_build_stages_range); where it pays
bool team_build_preferred(int n, int64_t count);
cudaError_t team_launch_build_small(const lqt_problem& p, const Layout& lay, const Coefs& cf, int64_t j0,
                                    int64_t cnt, double* stages, const ElemPtrs& out, cudaStream_t st);
size_t team_scan_workspace_bytes(int32_t n, int64_t T, bool with_traj);
cudaError_t team_launch_build(const lqt_problem& p, const Layout& lay, const Coefs& cf, const ElemPtrs& out,
                              double* gscratch, cudaStream_t st);
cudaError_t team_run_value_and_traj(const lqt_problem& p, const Coefs& cf, const ElemPtrs& el, double* S, double* v,
                                    double* zeta, const double* x0, double* x, double* u, double* cost, bool do_value,
                                    bool do_traj, char* ws, cudaStream_t st);
cudaError_t launch_terminal_values(const lqt_problem& p, double* J, double* eta, double* zeta, cudaStream_t s);

size_t scan_workspace_bytes(int32_t n, int64_t T, bool with_traj);
cudaError_t run_value_and_traj(const lqt_problem& p, const Layout& lay, const Coefs& cf, const ElemPtrs& el,
                               double* S, double* v, double* zeta, const double* x0, double* x, double* u,
                               double* cost, bool do_value, bool do_traj, const double* S_in, const double* v_in,
                               char* ws, size_t ws_bytes, cudaStream_t s);
size_t affine_scan_bytes(int n, int64_t cnt);
cudaError_t affine_scan_states(int n, const double* maps, int64_t cnt, const double* x_in, double* states, char* ws,
                               size_t& off, cudaStream_t st);
cudaError_t launch_maps_from_values(const lqt_problem& p, const ElemPtrs& el, const double* S, const double* v,
                                    double* maps, cudaStream_t st);
ElemPtrs carve_elements_at(const lqt_problem& p, char* base);
size_t element_region_bytes(const lqt_problem& p);
size_t backward_workspace_bytes(const lqt_problem& p, const Layout& L, size_t elem_bytes);
cudaError_t run_backward(const lqt_problem& p, const Layout& L, size_t elem_bytes, const double* x0, const double* S,
                         const double* v, const double* x, const double* gS, const double* gv, const double* gz,
                         const double* gx, double g_cost, double* gF, double* gL, double* gX, double* gU, double* gr,
                         double* gXf, double* grf, double* gx0, char* ws, cudaStream_t st);
// Pairwise upper levels of the n <= 8 scans, one warp per combination
// (lqt_team.cu); records in the full-matrix layout (full_elem_doubles /
// full_val_doubles of lqt_device.cuh).
template <int N, typename GT>
void team_upper_reduce(const double* src, int64_t cnt, double* agg, cudaStream_t st);
template <int N, typename GT>
void team_upper_down(const double* src, int64_t cnt, const double* above, int64_t cnt_above, double* vals,
                     cudaStream_t st);
template <int N>
void team_maps_reduce(const double* maps, int64_t cnt, int G, double* comp, cudaStream_t st);
template <int N>
void team_maps_down(const double* maps, int64_t cnt, int G, const double* above, const double* x_in, double* starts,
                    cudaStream_t st);

template <int N>
void team_prefix_down(const double* agg, int64_t cnt, const double* pre_up, double* pre, cudaStream_t st,
                      double* gscratch = nullptr);

// Method 2 (lqt_forward.cu, lqt_scan.cu): forward-ODE elements, prefix scan
// and the optimal states from the prefixes and the values.
cudaError_t launch_build_forward(const lqt_problem& p, const Layout& lay, const Coefs& cf, const ElemPtrs& out,
                                 cudaStream_t st, double* team_scratch = nullptr);
size_t prefix_workspace_bytes(int n, int64_t T);
// n = 16, 64 (team kernels, lqt_team.cu); the forward build's scratch is
// team_build_scratch_bytes(n)
cudaError_t team_launch_build_forward(const lqt_problem& p, const Layout& lay, const Coefs& cf, const ElemPtrs& out,
                                      double* gscratch, cudaStream_t st);
size_t team_prefix_workspace_bytes(int n, int64_t T);
cudaError_t team_run_method2(const lqt_problem& p, const Coefs& cf, const ElemPtrs& fwd, const double* S,
                             const double* v, const double* zeta, const double* x0, double* x, double* u,
                             double* cost, char* ws, cudaStream_t st);
cudaError_t run_method2(const lqt_problem& p, const Coefs& cf, const ElemPtrs& fwd, const double* S,
                        const double* v, const double* zeta, const double* x0, double* x, double* u, double* cost,
                        char* ws, cudaStream_t st);

// Time-invariant specialisation of the element build (lqt_invariant.cu).
bool invariant_supported(int n, int M);
size_t invariant_table_bytes(int n, int M, int K);
cudaError_t launch_build_invariant(const lqt_problem& p, const Layout& lay, const Coefs& cf, const ElemPtrs& out,
                                   double* table, cudaStream_t st);

bool densify_supported(const lqt_problem& p);
cudaError_t launch_densify(const lqt_problem& p, const Layout& lay, const Coefs& cf, const double* S, const double* v,
                           const double* zeta, const double* x, double* Sd, double* vd, double* zd, double* xd,
                           double* ud, cudaStream_t st);
size_t sequential_workspace_bytes(int32_t n, int64_t T, int32_t K);
cudaError_t launch_sequential(const lqt_problem& p, const Layout& lay, const Coefs& cf, const double* x0,
                              double* S, double* v, double* zeta, double* x, double* u, double* cost, char* ws,
                              cudaStream_t s);

// -------------------------------------------------------------------------
// batches of independent problems of one state dimension (lqt_batched.cu)
// -------------------------------------------------------------------------

// One problem of a batch, as the kernels see it.
struct BatchProb {
  int64_t T;    // sub-intervals
  int64_t off;  // its first boundary in the concatenation
  const double* t;
  Coefs cf;     // coefficients in kernel form (derived ones in the workspace)
  const double *Xf, *rf, *x0;
  // inputs of the coefficient preparation
  const double *L, *U, *X, *r;
  int32_t r_mode;
  int64_t off_qr;  // first qr sample of this problem in the concatenated qr array
};

struct BatchDev {
  int32_t B, n, m, K, M;
  const BatchProb* probs;  // device [B]
  const int64_t* off;      // device [B+1]: boundary offsets, off[B] = total boundaries
  const int64_t* off_qr;   // device [B+1]: qr sample offsets
  int64_t total;           // sum of (T_b + 1)
  int64_t total_qr;
};

__host__ __device__ __forceinline__ int32_t batch_find(const int64_t* off, int32_t B, int64_t g) {
  int32_t lo = 0, hi = B;  // off[lo] <= g < off[hi]
  while (hi - lo > 1) {
    const int32_t mid = (lo + hi) >> 1;
    if (off[mid] <= g) lo = mid;
    else hi = mid;
  }
  return lo;
}

cudaError_t batch_prepare(const BatchDev& bd, cudaStream_t st);
cudaError_t batch_build(const BatchDev& bd, const ElemPtrs& el, char* team_scratch, cudaStream_t st);
cudaError_t batch_build_team(const BatchDev& bd, const ElemPtrs& el, double* gscratch, cudaStream_t st);
cudaError_t batch_build_invariant(const BatchDev& bd, const ElemPtrs& el, double* tables, cudaStream_t st);
void launch_inv_batch_build_warp(const BatchDev& bd, const double* tables, const ElemPtrs& out, cudaStream_t st);
template <int N, int M>
void launch_inv_master_team(int32_t K, int32_t B, const BatchProb* probs, const double* t, const Coefs& cf,
                            double* tables, int64_t table_doubles, cudaStream_t st);
template <int N, int M>
void launch_inv_batch_build(const BatchDev& bd, const double* tables, const ElemPtrs& out, cudaStream_t st);

// Concatenated scan: value scan over `Tcat + 1` elements, then the boundary maps
// of every problem but the last replaced by x -> x0 of the next problem, then
// the state scan from x0 of the first problem (controls not computed).
struct BoundaryPatch {
  int32_t B;
  const int64_t* off;       // device [B+1]
  const BatchProb* probs;   // device [B] (x0 of each problem)
};
size_t concat_workspace_bytes(int32_t n, int64_t Tcat);
cudaError_t concat_scan(int32_t n, int64_t Tcat, const ElemPtrs& el, double* S, double* v, double* zeta,
                        const double* x0_first, double* x, const BoundaryPatch& patch, char* ws, cudaStream_t st);
size_t team_concat_workspace_bytes(int32_t n, int64_t Tcat);
cudaError_t team_concat_scan(int32_t n, int64_t Tcat, const ElemPtrs& el, double* S, double* v, double* zeta,
                             const double* x0_first, double* x, const BoundaryPatch& patch, char* ws,
                             cudaStream_t st);
void launch_boundary_patch(int n, double* maps, const BoundaryPatch& patch, cudaStream_t st);

// Level-0 chunk length override for the scans (0 = built-in heuristic); set by
// the batched entry point from its tuning argument.
void set_scan_chunk(int g);
int scan_chunk_override();
// Mixed precision for the scans: matrix products of the combinations in FP32,
// the LU solves of I + C J in FP64 (set by lqt_solve_mixed for one call).
void set_mixed_precision(bool on);
bool mixed_precision();

// grid method for the nonlinear scalar example (lqt_grid.cu)
size_t grid_workspace_bytes(const lqt_grid_problem& p, int which);  // 0: block, 1: values
cudaError_t run_grid_block(const lqt_grid_problem& p, double* Vblock, char* ws, cudaStream_t st);
cudaError_t run_grid_combine(const lqt_grid_problem& p, const double* A, const double* B, double* out,
                             cudaStream_t st);
cudaError_t run_grid_values(const lqt_grid_problem& p, const double* Vblock, double* V, char* ws, cudaStream_t st);

}  // namespace lqt
