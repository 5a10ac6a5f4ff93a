// C ABI entry points of the LQT library (declared in include/lqt.h): host-side
// argument validation, workspace layout, dispatch to the kernels, the device
// status word and the host-buffer convenience call.
#include <chrono>
#include <cmath>
#include <cstring>
#include <thread>

#include <cuda_runtime.h>

#include "lqt_internal.h"

namespace lqt {

__device__ unsigned g_status_word = 0;

static thread_local int32_t t_launches = 0;
void count_launch(int k) { t_launches += k; }
void reset_launch_count() { t_launches = 0; }

static size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

static bool supported_n(int n) { return n == 1 || n == 2 || n == 3 || n == 4 || n == 8 || n == 16 || n == 64; }

// Largest padded factor width compiled for each n.
static int max_M(int n) { return n == 1 ? 1 : n == 2 ? 2 : n <= 4 ? 4 : n == 8 ? 8 : 16; }

// Factor width used by the kernels (n = 64 is compiled for 16 columns only;
// zero columns do not change B = Lt Lt^T).
static int32_t factor_width(int n, int m) { return n == 64 ? 16 : padded_M(m); }

static bool valid_mode(int32_t m) { return m == LQT_CONST || m == LQT_PER_INTERVAL || m == LQT_PER_STAGE; }

static bool aligned8(const void* p) { return ((uintptr_t)p & 7u) == 0; }

// Structural validation shared by every call.  Returns LQT_OK or an error.
static lqt_status validate(const lqt_problem* p) {
  if (!p) return LQT_EINVAL;
  if (p->n < 1 || p->m < 1 || p->nr < 1 || p->T < 1 || p->K < 1) return LQT_EINVAL;
  if (!supported_n(p->n)) return LQT_EUNSUPPORTED;
  if (p->m > 16 || p->nr > 64) return LQT_EUNSUPPORTED;
  if (padded_M(p->m) > max_M(p->n)) return LQT_EUNSUPPORTED;
  if (!p->t || !p->F.ptr || !p->L.ptr || !p->X.ptr || !p->U.ptr || !p->Xf) return LQT_EINVAL;
  if (!p->H.ptr && p->nr != p->n) return LQT_EINVAL;
  if (!p->Hf && p->nr != p->n) return LQT_EINVAL;
  const lqt_coef* cs[7] = {&p->F, &p->L, &p->c, &p->H, &p->X, &p->U, &p->r};
  for (const lqt_coef* c : cs) {
    if (c->ptr && !valid_mode(c->mode)) return LQT_EINVAL;
    if (c->ptr && !aligned8(c->ptr)) return LQT_EINVAL;
  }
  if (!aligned8(p->t) || !aligned8(p->Xf) || (p->Hf && !aligned8(p->Hf)) || (p->rf && !aligned8(p->rf)))
    return LQT_EINVAL;
  return LQT_OK;
}

static Layout make_layout(const lqt_problem& p) {
  Layout L{};
  L.n = p.n; L.m = p.m; L.nr = p.nr; L.K = p.K; L.T = p.T;
  L.M = factor_width(p.n, p.m);
  const int32_t mH = p.H.ptr ? p.H.mode : kConst;
  const int32_t mr = p.r.ptr ? p.r.mode : kConst;
  L.mode_Lt = combine_modes(p.L.mode, p.U.mode);
  L.mode_Q = combine_modes(mH, p.X.mode);
  L.mode_qr = combine_modes(L.mode_Q, mr);
  size_t off = 0;
  L.off_Lt = off;
  off = align_up(off + sample_count(L.mode_Lt, p.T, p.K) * (size_t)p.n * L.M * sizeof(double));
  L.off_Q = off;
  if (p.H.ptr)  // H^T X H is derived only when H is given (otherwise X is used directly)
    off = align_up(off + sample_count(L.mode_Q, p.T, p.K) * (size_t)p.n * p.n * sizeof(double));
  L.off_qr = off;
  off = align_up(off + sample_count(L.mode_qr, p.T, p.K) * (size_t)(p.n + 1) * sizeof(double));
  L.off_Ku = off;
  const bool ku_const = p.L.mode == LQT_CONST && p.U.mode == LQT_CONST;
  off = align_up(off + (ku_const ? 1 : (size_t)p.T + 1) * (size_t)p.m * p.n * sizeof(double));
  L.coef_bytes = off;
  return L;
}

static size_t element_bytes(const lqt_problem& p) {
  const size_t n = p.n, T1 = (size_t)p.T + 1;
  return align_up(T1 * n * n * 8) * 3 + align_up(T1 * n * 8) * 2 + align_up(T1 * 8);
}

static ElemPtrs carve_elements(const lqt_problem& p, char* base) {
  const size_t n = p.n, T1 = (size_t)p.T + 1;
  ElemPtrs e;
  char* c = base;
  e.A = (double*)c; c += align_up(T1 * n * n * 8);
  e.C = (double*)c; c += align_up(T1 * n * n * 8);
  e.J = (double*)c; c += align_up(T1 * n * n * 8);
  e.b = (double*)c; c += align_up(T1 * n * 8);
  e.eta = (double*)c; c += align_up(T1 * n * 8);
  e.zeta = (double*)c;
  return e;
}

ElemPtrs carve_elements_at(const lqt_problem& p, char* base) { return carve_elements(p, base); }
size_t element_region_bytes(const lqt_problem& p) { return element_bytes(p); }

static lqt_status from_cuda(cudaError_t e) { return e == cudaSuccess ? LQT_OK : LQT_ECUDA; }

}  // namespace lqt

using namespace lqt;

extern "C" {

size_t lqt_workspace_size(const lqt_problem* p, int32_t which) {
  if (validate(p) != LQT_OK) return 0;
  const Layout L = make_layout(*p);
  const size_t T1 = (size_t)p->T + 1;
  switch (which) {
    case LQT_WS_BUILD: return L.coef_bytes + team_build_scratch_bytes(p->n);
    case LQT_WS_VALUE: {
      // a scan that fits one chunk needs no scratch; 0 is reserved for "invalid"
      const size_t b = scan_workspace_bytes(p->n, p->T, false);
      return b ? b : 256;
    }
    case LQT_WS_TRAJ: return L.coef_bytes + scan_workspace_bytes(p->n, p->T, true);
    case LQT_WS_SOLVE:
      return L.coef_bytes + element_bytes(*p) + align_up(T1 * 8) + team_build_scratch_bytes(p->n) +
             scan_workspace_bytes(p->n, p->T, true);
    case LQT_WS_SEQUENTIAL: return L.coef_bytes + align_up(sequential_workspace_bytes(p->n, p->T, p->K));
    case LQT_WS_BACKWARD: return backward_workspace_bytes(*p, L, element_bytes(*p)) + 4096;
    case LQT_WS_DENSIFY: return L.coef_bytes;
    case LQT_WS_METHOD2: return L.coef_bytes + prefix_workspace_bytes(p->n, p->T);
    case LQT_WS_INVARIANT:
      return invariant_supported(p->n, L.M) ? L.coef_bytes + align_up(invariant_table_bytes(p->n, L.M, p->K)) : 0;
    case LQT_WS_SOLVE_INVARIANT:
      return invariant_supported(p->n, L.M)
                 ? L.coef_bytes + element_bytes(*p) + align_up(T1 * 8) + team_build_scratch_bytes(p->n) +
                       scan_workspace_bytes(p->n, p->T, true) + align_up(invariant_table_bytes(p->n, L.M, p->K))
                 : 0;
    case LQT_WS_SOLVE_METHOD2:
      return L.coef_bytes + 2 * element_bytes(*p) + align_up(T1 * 8) + team_build_scratch_bytes(p->n) +
             scan_workspace_bytes(p->n, p->T, false) + prefix_workspace_bytes(p->n, p->T);
    default: return 0;
  }
}

lqt_status lqt_build_elements(const lqt_problem* p, const lqt_elements* out, void* ws, size_t ws_bytes,
                              void* stream) {
  t_launches = 0;
  lqt_status s = validate(p);
  if (s != LQT_OK) return s;
  if (!out || !out->A || !out->b || !out->C || !out->eta || !out->J) return LQT_EINVAL;
  const size_t need = lqt_workspace_size(p, LQT_WS_BUILD);
  if (!ws || ws_bytes < need) return LQT_EWORKSPACE;
  cudaStream_t st = (cudaStream_t)stream;
  const Layout L = make_layout(*p);
  Coefs cf;
  cudaError_t e = launch_prepare_coefs(*p, L, (char*)ws, cf, st);
  if (e != cudaSuccess) return LQT_ECUDA;
  ElemPtrs el{out->A, out->b, out->C, out->eta, out->J, out->zeta};
  return from_cuda(launch_build(*p, L, cf, el, st, (double*)((char*)ws + L.coef_bytes)));
}

lqt_status lqt_scan_value(const lqt_problem* p, const lqt_elements* el, double* S, double* v, double* zeta,
                          void* ws, size_t ws_bytes, void* stream) {
  t_launches = 0;
  lqt_status s = validate(p);
  if (s != LQT_OK) return s;
  if (!el || !el->A || !el->b || !el->C || !el->eta || !el->J || !S || !v) return LQT_EINVAL;
  const size_t need = lqt_workspace_size(p, LQT_WS_VALUE);
  if (!ws || ws_bytes < need) return LQT_EWORKSPACE;
  const Layout L = make_layout(*p);
  Coefs cf{};
  ElemPtrs e{el->A, el->b, el->C, el->eta, el->J, el->zeta};
  return from_cuda(run_value_and_traj(*p, L, cf, e, S, v, zeta, nullptr, nullptr, nullptr, nullptr, true, false,
                                      nullptr, nullptr, (char*)ws, ws_bytes, (cudaStream_t)stream));
}

lqt_status lqt_scan_trajectory(const lqt_problem* p, const lqt_elements* el, const double* S, const double* v,
                               const double* x0, double* x, double* u, void* ws, size_t ws_bytes, void* stream) {
  t_launches = 0;
  lqt_status s = validate(p);
  if (s != LQT_OK) return s;
  if (p->n > 8) return LQT_EUNSUPPORTED;
  if (!el || !el->A || !el->b || !el->C || !el->eta || !el->J || !S || !v || !x0 || !x) return LQT_EINVAL;
  const size_t need = lqt_workspace_size(p, LQT_WS_TRAJ);
  if (!ws || ws_bytes < need) return LQT_EWORKSPACE;
  cudaStream_t st = (cudaStream_t)stream;
  const Layout L = make_layout(*p);
  Coefs cf;
  if (launch_prepare_coefs(*p, L, (char*)ws, cf, st) != cudaSuccess) return LQT_ECUDA;
  ElemPtrs e{el->A, el->b, el->C, el->eta, el->J, el->zeta};
  return from_cuda(run_value_and_traj(*p, L, cf, e, nullptr, nullptr, nullptr, x0, x, u, nullptr, false, true, S, v,
                                      (char*)ws + L.coef_bytes, ws_bytes - L.coef_bytes, st));
}

lqt_status lqt_solve(const lqt_problem* p, const double* x0, double* S, double* v, double* zeta, double* x,
                     double* u, double* cost, void* ws, size_t ws_bytes, void* stream) {
  t_launches = 0;
  lqt_status s = validate(p);
  if (s != LQT_OK) return s;
  if (!x0 || !S || !v || !x) return LQT_EINVAL;
  const size_t need = lqt_workspace_size(p, LQT_WS_SOLVE);
  if (!ws || ws_bytes < need) return LQT_EWORKSPACE;
  cudaStream_t st = (cudaStream_t)stream;
  const Layout L = make_layout(*p);
  char* base = (char*)ws;
  Coefs cf;
  if (launch_prepare_coefs(*p, L, base, cf, st) != cudaSuccess) return LQT_ECUDA;
  ElemPtrs el = carve_elements(*p, base + L.coef_bytes);
  double* zbuf = (double*)(base + L.coef_bytes + element_bytes(*p));
  double* zout = zeta ? zeta : zbuf;
  char* team_scr = base + L.coef_bytes + element_bytes(*p) + align_up(((size_t)p->T + 1) * 8);
  if (launch_build(*p, L, cf, el, st, (double*)team_scr) != cudaSuccess) return LQT_ECUDA;
  char* scan = team_scr + team_build_scratch_bytes(p->n);
  return from_cuda(run_value_and_traj(*p, L, cf, el, S, v, zout, x0, x, u, cost, true, true, nullptr, nullptr, scan,
                                      ws_bytes - (scan - base), st));
}

lqt_status lqt_solve_mixed(const lqt_problem* p, const double* x0, double* S, double* v, double* zeta, double* x,
                           double* u, double* cost, void* ws, size_t ws_bytes, void* stream) {
  set_mixed_precision(true);
  const lqt_status s = lqt_solve(p, x0, S, v, zeta, x, u, cost, ws, ws_bytes, stream);
  set_mixed_precision(false);
  return s;
}

lqt_status lqt_solve_sequential(const lqt_problem* p, const double* x0, double* S, double* v, double* zeta,
                                double* x, double* u, double* cost, void* ws, size_t ws_bytes, void* stream) {
  t_launches = 0;
  lqt_status s = validate(p);
  if (s != LQT_OK) return s;
  if (p->n > 8) return LQT_EUNSUPPORTED;
  if (!x0 || !S || !v || !x) return LQT_EINVAL;
  const size_t need = lqt_workspace_size(p, LQT_WS_SEQUENTIAL);
  if (!ws || ws_bytes < need) return LQT_EWORKSPACE;
  cudaStream_t st = (cudaStream_t)stream;
  const Layout L = make_layout(*p);
  Coefs cf;
  if (launch_prepare_coefs(*p, L, (char*)ws, cf, st) != cudaSuccess) return LQT_ECUDA;
  return from_cuda(launch_sequential(*p, L, cf, x0, S, v, zeta, x, u, cost, (char*)ws + L.coef_bytes, st));
}

static lqt_status validate_invariant(const lqt_problem* p) {
  lqt_status s = validate(p);
  if (s != LQT_OK) return s;
  if (p->F.mode != LQT_CONST || p->L.mode != LQT_CONST || p->U.mode != LQT_CONST || p->X.mode != LQT_CONST ||
      (p->H.ptr && p->H.mode != LQT_CONST))
    return LQT_EUNSUPPORTED;
  if (!invariant_supported(p->n, make_layout(*p).M)) return LQT_EUNSUPPORTED;
  return LQT_OK;
}

lqt_status lqt_build_elements_invariant(const lqt_problem* p, const lqt_elements* out, void* ws, size_t ws_bytes,
                                        void* stream) {
  t_launches = 0;
  lqt_status s = validate_invariant(p);
  if (s != LQT_OK) return s;
  if (!out || !out->A || !out->b || !out->C || !out->eta || !out->J) return LQT_EINVAL;
  const size_t need = lqt_workspace_size(p, LQT_WS_INVARIANT);
  if (!ws || ws_bytes < need) return LQT_EWORKSPACE;
  cudaStream_t st = (cudaStream_t)stream;
  const Layout L = make_layout(*p);
  Coefs cf;
  if (launch_prepare_coefs(*p, L, (char*)ws, cf, st) != cudaSuccess) return LQT_ECUDA;
  ElemPtrs el{out->A, out->b, out->C, out->eta, out->J, out->zeta};
  return from_cuda(launch_build_invariant(*p, L, cf, el, (double*)((char*)ws + L.coef_bytes), st));
}

lqt_status lqt_solve_invariant(const lqt_problem* p, const double* x0, double* S, double* v, double* zeta, double* x,
                               double* u, double* cost, void* ws, size_t ws_bytes, void* stream) {
  t_launches = 0;
  lqt_status s = validate_invariant(p);
  if (s != LQT_OK) return s;
  if (!x0 || !S || !v || !x) return LQT_EINVAL;
  const size_t need = lqt_workspace_size(p, LQT_WS_SOLVE_INVARIANT);
  if (!ws || ws_bytes < need) return LQT_EWORKSPACE;
  cudaStream_t st = (cudaStream_t)stream;
  const Layout L = make_layout(*p);
  char* base = (char*)ws;
  Coefs cf;
  if (launch_prepare_coefs(*p, L, base, cf, st) != cudaSuccess) return LQT_ECUDA;
  ElemPtrs el = carve_elements(*p, base + L.coef_bytes);
  char* cur = base + L.coef_bytes + element_bytes(*p);
  double* zbuf = (double*)cur;
  double* zout = zeta ? zeta : zbuf;
  cur += align_up(((size_t)p->T + 1) * 8) + team_build_scratch_bytes(p->n);
  const size_t scan_bytes = scan_workspace_bytes(p->n, p->T, true);
  double* table = (double*)(cur + scan_bytes);
  if (launch_build_invariant(*p, L, cf, el, table, st) != cudaSuccess) return LQT_ECUDA;
  return from_cuda(run_value_and_traj(*p, L, cf, el, S, v, zout, x0, x, u, cost, true, true, nullptr, nullptr, cur,
                                      scan_bytes, st));
}

lqt_status lqt_build_elements_forward(const lqt_problem* p, const lqt_elements* out, void* ws, size_t ws_bytes,
                                      void* stream) {
  t_launches = 0;
  lqt_status s = validate(p);
  if (s != LQT_OK) return s;
  if (!out || !out->A || !out->b || !out->C || !out->eta || !out->J) return LQT_EINVAL;
  const Layout L = make_layout(*p);
  if (!ws || ws_bytes < lqt_workspace_size(p, LQT_WS_BUILD)) return LQT_EWORKSPACE;
  cudaStream_t st = (cudaStream_t)stream;
  Coefs cf;
  if (launch_prepare_coefs(*p, L, (char*)ws, cf, st) != cudaSuccess) return LQT_ECUDA;
  ElemPtrs el{out->A, out->b, out->C, out->eta, out->J, out->zeta};
  return from_cuda(launch_build_forward(*p, L, cf, el, st, (double*)((char*)ws + L.coef_bytes)));
}

lqt_status lqt_trajectory_method2(const lqt_problem* p, const lqt_elements* fwd, const double* S, const double* v,
                                  const double* x0, double* x, double* u, void* ws, size_t ws_bytes, void* stream) {
  t_launches = 0;
  lqt_status s = validate(p);
  if (s != LQT_OK) return s;
  if (!fwd || !fwd->A || !fwd->b || !fwd->C || !fwd->eta || !fwd->J || !S || !v || !x0 || !x) return LQT_EINVAL;
  const size_t need = lqt_workspace_size(p, LQT_WS_METHOD2);
  if (!ws || ws_bytes < need) return LQT_EWORKSPACE;
  cudaStream_t st = (cudaStream_t)stream;
  const Layout L = make_layout(*p);
  Coefs cf;
  if (launch_prepare_coefs(*p, L, (char*)ws, cf, st) != cudaSuccess) return LQT_ECUDA;
  ElemPtrs el{fwd->A, fwd->b, fwd->C, fwd->eta, fwd->J, fwd->zeta};
  return from_cuda(run_method2(*p, cf, el, S, v, nullptr, x0, x, u, nullptr, (char*)ws + L.coef_bytes, st));
}

lqt_status lqt_solve_method2(const lqt_problem* p, const double* x0, double* S, double* v, double* zeta, double* x,
                             double* u, double* cost, void* ws, size_t ws_bytes, void* stream) {
  t_launches = 0;
  lqt_status s = validate(p);
  if (s != LQT_OK) return s;
  if (!x0 || !S || !v || !x) return LQT_EINVAL;
  const size_t need = lqt_workspace_size(p, LQT_WS_SOLVE_METHOD2);
  if (!ws || ws_bytes < need) return LQT_EWORKSPACE;
  cudaStream_t st = (cudaStream_t)stream;
  const Layout L = make_layout(*p);
  char* base = (char*)ws;
  Coefs cf;
  if (launch_prepare_coefs(*p, L, base, cf, st) != cudaSuccess) return LQT_ECUDA;
  char* cur = base + L.coef_bytes;
  ElemPtrs bwd = carve_elements(*p, cur);
  cur += element_bytes(*p);
  ElemPtrs fwd = carve_elements(*p, cur);
  cur += element_bytes(*p);
  double* zbuf = (double*)cur;
  cur += align_up(((size_t)p->T + 1) * 8);
  double* zout = zeta ? zeta : zbuf;
  double* team_scr = (double*)cur;  // both element builds (n = 64), one after the other
  cur += team_build_scratch_bytes(p->n);
  // values: backward-ODE elements and the suffix scan (Sec. IV-B, IV-D, IV-A)
  if (launch_build(*p, L, cf, bwd, st, team_scr) != cudaSuccess) return LQT_ECUDA;
  const size_t scan_bytes = scan_workspace_bytes(p->n, p->T, false);
  if (run_value_and_traj(*p, L, cf, bwd, S, v, zout, nullptr, nullptr, nullptr, nullptr, true, false, nullptr,
                         nullptr, cur, scan_bytes, st) != cudaSuccess)
    return LQT_ECUDA;
  cur += scan_bytes;
  // states: forward-ODE elements, prefix scan, Method 2 (Sec. IV-C, IV-E)
  if (launch_build_forward(*p, L, cf, fwd, st, team_scr) != cudaSuccess) return LQT_ECUDA;
  return from_cuda(run_method2(*p, cf, fwd, S, v, zout, x0, x, u, cost, cur, st));
}

lqt_status lqt_densify(const lqt_problem* p, const double* S, const double* v, const double* zeta, const double* x,
                       double* Sd, double* vd, double* zd, double* xd, double* ud, void* ws, size_t ws_bytes,
                       void* stream) {
  t_launches = 0;
  lqt_status s = validate(p);
  if (s != LQT_OK) return s;
  if (!densify_supported(*p)) return LQT_EUNSUPPORTED;
  if (!S || !v || !zeta || !x || !Sd || !vd || !zd || !xd) return LQT_EINVAL;
  const size_t need = lqt_workspace_size(p, LQT_WS_DENSIFY);
  if (!ws || ws_bytes < need) return LQT_EWORKSPACE;
  cudaStream_t st = (cudaStream_t)stream;
  const Layout L = make_layout(*p);
  Coefs cf;
  if (launch_prepare_coefs(*p, L, (char*)ws, cf, st) != cudaSuccess) return LQT_ECUDA;
  return from_cuda(launch_densify(*p, L, cf, S, v, zeta, x, Sd, vd, zd, xd, ud, st));
}

static lqt_status validate_backward(const lqt_problem* p) {
  lqt_status s = validate(p);
  if (s != LQT_OK) return s;
  if (p->n > 8 || p->K > 8 || p->m > 16) return LQT_EUNSUPPORTED;
  if (p->H.ptr || p->Hf || p->c.ptr) return LQT_EUNSUPPORTED;
  const lqt_coef* blockconst[4] = {&p->F, &p->L, &p->X, &p->U};
  for (const lqt_coef* c : blockconst)
    if (c->mode == LQT_PER_STAGE) return LQT_EUNSUPPORTED;
  return LQT_OK;
}

lqt_status lqt_backward(const lqt_problem* p, const double* x0, const double* S, const double* v, const double* x,
                        const double* gS, const double* gv, const double* gzeta, const double* gx, const double* gu,
                        double g_cost, double* gF, double* gL, double* gX, double* gU, double* gr, double* gXf,
                        double* grf, double* gx0, void* ws, size_t ws_bytes, void* stream) {
  t_launches = 0;
  lqt_status s = validate_backward(p);
  if (s != LQT_OK) return s;
  if (gu) return LQT_EUNSUPPORTED;
  if (!x0 || !S || !v || !x) return LQT_EINVAL;
  const size_t need = lqt_workspace_size(p, LQT_WS_BACKWARD);
  if (!ws || ws_bytes < need) return LQT_EWORKSPACE;
  const Layout L = make_layout(*p);
  return from_cuda(run_backward(*p, L, element_bytes(*p), x0, S, v, x, gS, gv, gzeta, gx, g_cost, gF, gL, gX, gU, gr,
                                gXf, grf, gx0, (char*)ws, (cudaStream_t)stream));
}

// ---------------------------------------------------------------------------
// host-buffer call
// ---------------------------------------------------------------------------

static size_t coef_bytes_of(const lqt_coef& c, const lqt_problem& p, size_t per_sample) {
  if (!c.ptr) return 0;
  return (size_t)sample_count(c.mode, p.T, p.K) * per_sample * sizeof(double);
}

size_t lqt_host_staging_size(const lqt_problem* p) {
  if (validate(p) != LQT_OK) return 0;
  const size_t n = p->n, m = p->m, nr = p->nr, T1 = (size_t)p->T + 1;
  size_t b = align_up(T1 * 8);
  b += align_up(coef_bytes_of(p->F, *p, n * n)) + align_up(coef_bytes_of(p->L, *p, n * m)) +
       align_up(coef_bytes_of(p->c, *p, n)) + align_up(coef_bytes_of(p->H, *p, nr * n)) +
       align_up(coef_bytes_of(p->X, *p, nr * nr)) + align_up(coef_bytes_of(p->U, *p, m * m)) +
       align_up(coef_bytes_of(p->r, *p, nr));
  b += align_up(nr * n * 8) + align_up(nr * nr * 8) + align_up(nr * 8) + align_up(n * 8);
  // outputs: S, v, zeta, x, u, cost
  b += align_up(T1 * n * n * 8) + align_up(T1 * n * 8) + align_up(T1 * 8) + align_up(T1 * n * 8) +
       align_up(T1 * m * 8) + 256;
  return b;
}

// Sub-intervals j0 .. j0+cnt-1 of d as a problem of its own: the time points
// and every sampled coefficient start at sub-interval j0's first sample.
static lqt_problem window_problem(const lqt_problem& d, int64_t j0, int64_t cnt) {
  lqt_problem w = d;
  w.T = cnt;
  w.t = d.t + j0;
  const size_t n = d.n, m = d.m, nr = d.nr;
  lqt_coef* cs[7] = {&w.F, &w.L, &w.c, &w.H, &w.X, &w.U, &w.r};
  const size_t per[7] = {n * n, n * m, n, nr * n, nr * nr, m * m, nr};
  for (int i = 0; i < 7; ++i)
    if (cs[i]->ptr) cs[i]->ptr += sample_index(cs[i]->mode, j0, 0, d.K) * per[i];
  return w;
}

// Sub-intervals per overlapped chunk of lqt_solve_host.
static int64_t host_chunk(int64_t T) {
  const int64_t c = (T + 15) / 16;
  return c < (1 << 15) ? (1 << 15) : c;
}

lqt_status lqt_solve_host(const lqt_problem* hp, const double* x0, double* S, double* v, double* zeta, double* x,
                          double* u, double* cost, void* ws, size_t ws_bytes, void* stream) {
  lqt_status s = validate(hp);
  if (s != LQT_OK) return s;
  if (!x0 || !S || !v || !x) return LQT_EINVAL;
  const size_t solve_ws = lqt_workspace_size(hp, LQT_WS_SOLVE);
  const size_t staging = lqt_host_staging_size(hp);
  if (!ws || ws_bytes < solve_ws + staging) return LQT_EWORKSPACE;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t n = hp->n, m = hp->m, nr = hp->nr, T1 = (size_t)hp->T + 1;
  // Chunked path: for n <= 8 and long horizons the sampled coefficients are
  // copied in chunks on a second stream while the derived coefficients and
  // elements of the chunks already copied are built (a chunk's build also
  // waits for the next chunk's copy, which holds its last sample).
  const int64_t chunk = host_chunk(hp->T);
  const bool chunked = hp->n <= 8 && hp->T >= 2 * chunk;
  cudaStream_t cs = st;
  cudaEvent_t evs[20] = {};
  int n_ev = 0;
  cudaError_t e = cudaSuccess;
  if (chunked) {
    e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&evs[n_ev++], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(evs[0], st);  // the workspace is free once st's earlier work is done
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, evs[0], 0);
    if (e != cudaSuccess) {
      if (cs != st) cudaStreamDestroy(cs);
      if (evs[0]) cudaEventDestroy(evs[0]);
      return LQT_ECUDA;
    }
  }
  char* cur = (char*)ws + align_up(solve_ws);
  struct Deferred {
    const lqt_coef* src;
    double* dst;
    size_t per;
  } deferred[7];
  int n_def = 0;
  auto stage = [&](const void* src, size_t bytes) -> const double* {
    if (!src || bytes == 0) return nullptr;
    char* dst = cur;
    cur += align_up(bytes);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, cs);
    return (const double*)dst;
  };
  auto stage_coef = [&](const lqt_coef& c, size_t per) -> const double* {
    if (!c.ptr) return nullptr;
    if (!chunked || c.mode == LQT_CONST) return stage(c.ptr, coef_bytes_of(c, *hp, per));
    double* dst = (double*)cur;
    cur += align_up(coef_bytes_of(c, *hp, per));
    deferred[n_def++] = Deferred{&c, dst, per};
    return dst;
  };
  lqt_problem d = *hp;
  d.t = stage(hp->t, T1 * 8);
  d.F.ptr = stage_coef(hp->F, n * n);
  d.L.ptr = stage_coef(hp->L, n * m);
  d.c.ptr = stage_coef(hp->c, n);
  d.H.ptr = stage_coef(hp->H, nr * n);
  d.X.ptr = stage_coef(hp->X, nr * nr);
  d.U.ptr = stage_coef(hp->U, m * m);
  d.r.ptr = stage_coef(hp->r, nr);
  d.Hf = stage(hp->Hf, nr * n * 8);
  d.Xf = stage(hp->Xf, nr * nr * 8);
  d.rf = stage(hp->rf, nr * 8);
  const double* dx0 = stage(x0, n * 8);
  auto carve = [&](size_t bytes) {
    double* p = (double*)cur;
    cur += align_up(bytes);
    return p;
  };
  double* dS = carve(T1 * n * n * 8);
  double* dv = carve(T1 * n * 8);
  double* dz = carve(T1 * 8);
  double* dxo = carve(T1 * n * 8);
  double* du = carve(T1 * m * 8);
  double* dc = carve(8);
  if (e == cudaSuccess && chunked) {
    t_launches = 0;
    const Layout L = make_layout(d);
    char* base = (char*)ws;
    double* Lt = (double*)(base + L.off_Lt);
    double* Q = (double*)(base + L.off_Q);
    double* qr = (double*)(base + L.off_qr);
    double* Ku = (double*)(base + L.off_Ku);
    const bool ku_const = d.L.mode == LQT_CONST && d.U.mode == LQT_CONST;
    const ElemPtrs el = carve_elements(d, base + L.coef_bytes);
    const int64_t P = (d.T + chunk - 1) / chunk;
    for (int64_t c = 0; c < P && e == cudaSuccess; ++c) {
      const int64_t j0 = c * chunk, j1 = j0 + chunk < d.T ? j0 + chunk : d.T;
      for (int k = 0; k < n_def && e == cudaSuccess; ++k) {
        const Deferred& df = deferred[k];
        const int64_t s0 = sample_index(df.src->mode, j0, 0, d.K);
        const int64_t s1 = c == P - 1 ? sample_count(df.src->mode, d.T, d.K) : sample_index(df.src->mode, j1, 0, d.K);
        e = cudaMemcpyAsync(df.dst + s0 * df.per, df.src->ptr + s0 * df.per, (size_t)(s1 - s0) * df.per * 8,
                            cudaMemcpyHostToDevice, cs);
      }
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&evs[n_ev], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventRecord(evs[n_ev++], cs);
    }
    for (int64_t c = 0; c < P && e == cudaSuccess; ++c) {
      const int64_t j0 = c * chunk, cnt = (j0 + chunk < d.T ? j0 + chunk : d.T) - j0;
      e = cudaStreamWaitEvent(st, evs[1 + (c + 1 < P ? c + 1 : P - 1)], 0);
      if (e != cudaSuccess) break;
      const lqt_problem pw = window_problem(d, j0, cnt);
      const Layout Lw = make_layout(pw);
      Coefs cfw;
      e = launch_prepare_into(pw, Lw, Lt + sample_index(L.mode_Lt, j0, 0, d.K) * n * L.M,
                              Q + sample_index(L.mode_Q, j0, 0, d.K) * n * n,
                              qr + sample_index(L.mode_qr, j0, 0, d.K) * (n + 1), ku_const ? Ku : Ku + j0 * m * n, cfw,
                              st);
      const ElemPtrs elw{el.A + j0 * n * n, el.b + j0 * n, el.C + j0 * n * n, el.eta + j0 * n, el.J + j0 * n * n,
                         el.zeta + j0};
      if (e == cudaSuccess) e = launch_build_range(pw, Lw, cfw, elw, st);
    }
    if (e == cudaSuccess) e = launch_terminal_element(d, el, st);
    if (e == cudaSuccess) {
      const Coefs cf = coefs_view(d, L, Lt, Q, qr, Ku);
      char* team_scr = base + L.coef_bytes + element_bytes(d) + align_up(((size_t)d.T + 1) * 8);
      char* scan = team_scr + team_build_scratch_bytes(d.n);
      e = run_value_and_traj(d, L, cf, el, dS, dv, dz, dx0, dxo, u ? du : nullptr, dc, true, true, nullptr, nullptr,
                             scan, solve_ws - (scan - base), st);
    }
  } else if (e == cudaSuccess) {
    s = lqt_solve(&d, dx0, dS, dv, dz, dxo, u ? du : nullptr, dc, ws, solve_ws, stream);
  }
  if (s == LQT_OK && e == cudaSuccess) {
    e = cudaMemcpyAsync(S, dS, T1 * n * n * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(v, dv, T1 * n * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && zeta) e = cudaMemcpyAsync(zeta, dz, T1 * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(x, dxo, T1 * n * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && u) e = cudaMemcpyAsync(u, du, T1 * m * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && cost) e = cudaMemcpyAsync(cost, dc, 8, cudaMemcpyDeviceToHost, st);
  }
  const cudaError_t sync = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = sync;
  if (chunked) {
    cudaStreamSynchronize(cs);
    for (int k = 0; k < n_ev; ++k) cudaEventDestroy(evs[k]);
    cudaStreamDestroy(cs);
  }
  if (s != LQT_OK) return s;
  return from_cuda(e);
}

// ---------------------------------------------------------------------------
// status
// ---------------------------------------------------------------------------

lqt_status lqt_get_status(void* stream, int32_t timeout_ms) {
  cudaStream_t st = (cudaStream_t)stream;
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    const cudaError_t q = cudaStreamQuery(st);
    if (q == cudaSuccess) break;
    if (q != cudaErrorNotReady) return LQT_ECUDA;
    if (timeout_ms >= 0) {
      const auto ms =
          std::chrono::duration_cast<std::chrono::milliseconds>(std::chrono::steady_clock::now() - t0).count();
      if (ms > timeout_ms) return LQT_ETIMEOUT;
    }
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
  unsigned word = 0;
  if (cudaMemcpyFromSymbol(&word, g_status_word, sizeof(word)) != cudaSuccess) return LQT_ECUDA;
  const unsigned zero = 0;
  if (cudaMemcpyToSymbol(g_status_word, &zero, sizeof(zero)) != cudaSuccess) return LQT_ECUDA;
  if (word & kStatusNonFinite) return LQT_ENONFINITE;
  if (word & kStatusSingular) return LQT_ESINGULAR;
  if (word & kStatusNonUniform) return LQT_EINVAL;
  if (word & kStatusTimeout) return LQT_ETIMEOUT;
  return LQT_OK;
}

const char* lqt_strerror(lqt_status s) {
  switch (s) {
    case LQT_OK: return "ok";
    case LQT_EINVAL: return "invalid argument";
    case LQT_EWORKSPACE: return "workspace missing or too small";
    case LQT_ENONFINITE: return "non-finite value produced on the device";
    case LQT_ESINGULAR: return "singular matrix met on the device";
    case LQT_ETIMEOUT: return "timed out waiting for the stream";
    case LQT_ECUDA: return "CUDA runtime error";
    case LQT_EUNSUPPORTED: return "dimension not supported by this build";
    default: return "unknown status";
  }
}

// ---------------------------------------------------------------------------
// grid method (Sec. VI-B, App. E)
// ---------------------------------------------------------------------------

static lqt_status validate_grid(const lqt_grid_problem* p) {
  if (!p) return LQT_EINVAL;
  if (p->G < 3 || p->G > 16384 || p->substeps < 1 || p->T < 1 || p->T > INT32_MAX) return LQT_EINVAL;
  if (!(p->dx > 0.0) || !(p->tau > 0.0) || !(p->rho > 0.0)) return LQT_EINVAL;
  if (p->interp != 0 && p->interp != 1) return LQT_EINVAL;
  const double vals[] = {p->x_min, p->dx, p->d0, p->d1, p->d2, p->q, p->rho, p->qf, p->tau};
  for (double v : vals)
    if (!std::isfinite(v)) return LQT_EINVAL;
  return LQT_OK;
}

static bool overlaps(const void* a, size_t na, const void* b, size_t nb) {
  const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
  return x < y + nb && y < x + na;
}

size_t lqt_grid_workspace_size(const lqt_grid_problem* p, int32_t which) {
  if (validate_grid(p) != LQT_OK || (which != 0 && which != 1)) return 0;
  return grid_workspace_bytes(*p, which);
}

lqt_status lqt_grid_block(const lqt_grid_problem* p, double* Vblock, void* ws, size_t ws_bytes, void* stream) {
  t_launches = 0;
  lqt_status s = validate_grid(p);
  if (s != LQT_OK) return s;
  if (!Vblock || !aligned8(Vblock)) return LQT_EINVAL;
  const size_t need = grid_workspace_bytes(*p, 0);
  if (!ws || ws_bytes < need || !aligned8(ws)) return LQT_EWORKSPACE;
  if (overlaps(Vblock, (size_t)p->G * p->G * 8, ws, need)) return LQT_EINVAL;
  return from_cuda(run_grid_block(*p, Vblock, (char*)ws, (cudaStream_t)stream));
}

lqt_status lqt_grid_combine(const lqt_grid_problem* p, const double* A, const double* B, double* out, void* stream) {
  t_launches = 0;
  lqt_status s = validate_grid(p);
  if (s != LQT_OK) return s;
  if (!A || !B || !out || !aligned8(A) || !aligned8(B) || !aligned8(out)) return LQT_EINVAL;
  const size_t bytes = (size_t)p->G * p->G * 8;
  if (overlaps(out, bytes, A, bytes) || overlaps(out, bytes, B, bytes)) return LQT_EINVAL;
  return from_cuda(run_grid_combine(*p, A, B, out, (cudaStream_t)stream));
}

lqt_status lqt_grid_values(const lqt_grid_problem* p, const double* Vblock, double* V, void* ws, size_t ws_bytes,
                           void* stream) {
  t_launches = 0;
  lqt_status s = validate_grid(p);
  if (s != LQT_OK) return s;
  if (!Vblock || !V || !aligned8(Vblock) || !aligned8(V)) return LQT_EINVAL;
  const size_t need = grid_workspace_bytes(*p, 1);
  if (!ws || ws_bytes < need || !aligned8(ws)) return LQT_EWORKSPACE;
  const size_t vb = ((size_t)p->T + 1) * p->G * 8, gb = (size_t)p->G * p->G * 8;
  if (overlaps(V, vb, Vblock, gb) || overlaps(V, vb, ws, need)) return LQT_EINVAL;
  return from_cuda(run_grid_values(*p, Vblock, V, (char*)ws, (cudaStream_t)stream));
}

int32_t lqt_last_launch_count(void) { return t_launches; }

}  // extern "C"
