/*
 * lqt.h - C ABI of the GB300 (sm_103a) temporally parallel continuous-time LQT
 * solver.
 *
 * Method: Sarkka & Garcia-Fernandez, "Temporal Parallelisation of the HJB
 * Equation and Continuous-Time Linear Quadratic Control" (arXiv 2212.11744).
 * The problem (Sec. II-B, eq. LQT_Control_problem) is
 *
 *     dx/dt = F(t) x + L(t) u + c(t)
 *     cost  = 1/2 (Hf x(tf) - rf)' Xf (Hf x(tf) - rf)
 *           + int 1/2 (r - H x)' X (r - H x) + 1/2 u' U u dt
 *
 * on [t_0, t_T] split into T sub-intervals t_0 < t_1 < ... < t_T.  The solver
 *   (a) integrates every sub-interval's conditional value function
 *       (A, b, C, eta, J, zeta) with K classical RK4 steps of the backward
 *       conditional HJB ODEs (Sec. IV-B, Theorem Backward_HJB_LQT, boundary
 *       eq. abcej_boundary), element T being the terminal cost (Sec. IV-D,
 *       eq. LQT_final_initialisation);
 *   (b) scans the elements from the right with the combination rule of
 *       Sec. IV-A (eq. lqt_comb), giving the value function
 *       V(x, t_k) = zeta_k + 1/2 x' S_k x - v_k' x at every t_k (eq. eJ_vS);
 *   (c) scans the one-sub-interval affine maps x_{k+1} = Psi_k x_k + alpha_k
 *       (Sec. IV-E, Method 1 combination eqs. Psi_comb/alpha_comb, with the
 *       maps from the one-sub-interval form of Method 2) for the optimal
 *       states, and evaluates u_k = U^-1 L' (v_k - S_k x_k) (eq.
 *       LQT_optimal_control).
 *
 * Conventions for every entry point
 *  - All array pointers are DEVICE pointers unless stated otherwise; the caller
 *    owns every buffer.  The library allocates no device memory: scratch space
 *    is caller-provided and sized by lqt_workspace_size().
 *  - Calls are asynchronous on `stream` (a cudaStream_t passed as void*; NULL is
 *    the legacy default stream) and never synchronise, except lqt_get_status()
 *    and lqt_solve_host().
 *  - Matrices are row-major and dense; symmetric outputs are written in full.
 *    Arrays indexed by boundary run over k = 0..T (T+1 entries).
 *  - FP64 throughout.
 *  - Errors: invalid arguments are rejected on the host before any launch and
 *    returned directly.  Numerical trouble found on the device (a non-finite
 *    value in an output; a singular system) is recorded in a per-device status
 *    word read and cleared by lqt_get_status().  A system W x = r of a
 *    combination (W = I + C J, App. B: eigenvalues >= 1 for PSD C, J) or of a
 *    control law counts as singular when an LU pivot's magnitude is at most
 *    2^-40 (about 9.1e-13) times the largest magnitude of its row in the
 *    original W: its condition number is then beyond ~1e12 and FP64 no longer
 *    carries the digits of a 1e-9 result.  A non-positive Cholesky pivot of
 *    U counts too.
 *  - Supported state dimensions n: 1, 2, 3, 4, 8 (one thread per element),
 *    16 and 64 (a warp / a CTA per element).  Other n return
 *    LQT_EUNSUPPORTED.  m <= 16, nr <= 64.
 */
#ifndef LQT_H
#define LQT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LQT_OK = 0,
  LQT_EINVAL = 1,       /* bad dimension, NULL pointer, bad sampling mode       */
  LQT_EWORKSPACE = 2,   /* workspace NULL or smaller than lqt_workspace_size()   */
  LQT_ENONFINITE = 3,   /* device found a NaN/Inf in an output                   */
  LQT_ESINGULAR = 4,    /* device found a (numerically) singular system: see
                           "Errors" above                                          */
  LQT_ETIMEOUT = 5,     /* lqt_get_status() deadline passed before the stream     */
  LQT_ECUDA = 6,        /* a CUDA runtime call failed                             */
  LQT_EUNSUPPORTED = 7  /* dimension not compiled in                              */
} lqt_status;

/* How a time-varying coefficient is sampled.  For sub-interval j with
 * h_j = (t_{j+1} - t_j)/K the RK4 stages of the element ODE need the
 * coefficients at the half-step times t_j + p h_j / 2, p = 0..2K. */
typedef enum {
  LQT_CONST = 0,        /* 1 sample                                              */
  LQT_PER_INTERVAL = 1, /* T samples; sample j holds on all of sub-interval j     */
  LQT_PER_STAGE = 2     /* 2KT+1 samples; sample 2Kj+p is at t_j + p h_j / 2      */
} lqt_sampling;

/* One coefficient: `ptr` points at its samples, each sample a row-major matrix
 * or vector of the coefficient's shape, samples back to back. */
typedef struct {
  const double *ptr;
  int32_t mode; /* lqt_sampling */
} lqt_coef;

/* The problem of Sec. II-B.  Shapes per sample:
 *   F n x n, L n x m, c n (ptr NULL = zero), H nr x n (ptr NULL = identity,
 *   then nr must equal n), X nr x nr symmetric PSD, U m x m symmetric PD,
 *   r nr (ptr NULL = zero); Hf nr x n (NULL = identity), Xf nr x nr, rf nr
 *   (NULL = zero).  t: T+1 strictly increasing block boundaries. */
typedef struct {
  int32_t n, m, nr;
  int64_t T;
  int32_t K; /* RK4 steps per sub-interval, >= 1 */
  const double *t;
  lqt_coef F, L, c, H, X, U, r;
  const double *Hf, *Xf, *rf;
} lqt_problem;

/* Conditional value function elements of Sec. IV-A (eq. LQT_V_form2), T+1 of
 * them (index T = terminal element): A[T+1][n][n], b[T+1][n], C[T+1][n][n],
 * eta[T+1][n], J[T+1][n][n], zeta[T+1].  Device pointers. */
typedef struct {
  double *A, *b, *C, *eta, *J, *zeta;
} lqt_elements;

/* Which call a workspace is for. */
enum {
  LQT_WS_BUILD = 0,
  LQT_WS_VALUE = 1,
  LQT_WS_TRAJ = 2,
  LQT_WS_SOLVE = 3,
  LQT_WS_SEQUENTIAL = 4,
  LQT_WS_BACKWARD = 5,
  LQT_WS_DENSIFY = 6,
  LQT_WS_METHOD2 = 7,
  LQT_WS_SOLVE_METHOD2 = 8,
  LQT_WS_INVARIANT = 9,
  LQT_WS_SOLVE_INVARIANT = 10
};

/* Bytes of device workspace the call `which` needs for problem p (host call,
 * reads only the scalar fields and sampling modes of p).  0 if p is invalid. */
size_t lqt_workspace_size(const lqt_problem *p, int32_t which);

/* Stage (a): every element a_j, j = 0..T-1, by K RK4 steps of the backward
 * conditional HJB ODEs of Sec. IV-B (Theorem Backward_HJB_LQT) from the
 * boundary A=I, b=C=eta=J=0, zeta=0 at s = t_{j+1} down to s = t_j, and the
 * terminal element a_T of Sec. IV-D (A=b=C=0, J=Hf'XfHf, eta=Hf'Xf rf,
 * zeta = 1/2 rf'Xf rf).  zeta obeys d zeta/ds = -1/2 r'Xr + 1/2 eta'B eta +
 * eta'c (B = L U^-1 L'), the state-free part of the same HJB.
 * out: caller-owned device arrays (see lqt_elements). */
lqt_status lqt_build_elements(const lqt_problem *p, const lqt_elements *out, void *ws, size_t ws_bytes,
                              void *stream);

/* Stage (b): the reverse all-prefix-sums sbar_k = a_k (x) ... (x) a_T of the
 * T+1 elements (Sec. III-D, Theorem parallel_HJB, eq. parallel_V_HJB) with the
 * combination of Sec. IV-A, as a chunked reduce / scan / value-form
 * down-sweep.  Writes S_k = J(sbar_k) [T+1][n][n], v_k = eta(sbar_k) [T+1][n]
 * and zeta_k [T+1] (eq. eJ_vS).  zeta may be NULL. */
lqt_status lqt_scan_value(const lqt_problem *p, const lqt_elements *el, double *S, double *v, double *zeta,
                          void *ws, size_t ws_bytes, void *stream);

/* Stage (c): optimal states and controls at the boundaries.  For each k the
 * one-sub-interval map of Method 2 (Sec. IV-E, eq. Opt_trajectory_method2 with
 * t_0 replaced by t_k): Psi_k = (I + C_k S_{k+1})^-1 A_k,
 * alpha_k = (I + C_k S_{k+1})^-1 (b_k + C_k v_{k+1}); the maps are composed
 * with the associative rule of Method 1 (eqs. Psi_comb, alpha_comb) in a
 * prefix scan applied to x0, giving x[T+1][n]; then u_k = U^-1 L' (v_k - S_k
 * x_k) (eq. LQT_optimal_control) with the coefficients at t_k, u[T+1][m].
 * x0: device [n].  u may be NULL. */
lqt_status lqt_scan_trajectory(const lqt_problem *p, const lqt_elements *el, const double *S, const double *v,
                               const double *x0, double *x, double *u, void *ws, size_t ws_bytes, void *stream);

/* Stages (a)+(b)+(c) in one call, with the elements and the maps kept in the
 * workspace.  cost (device, 1 double, may be NULL) receives the optimal cost
 * V(x0, t_0) = zeta_0 + 1/2 x0'S_0 x0 - v_0'x0 (eq. V_quadratic_LQT).  zeta, u
 * may be NULL.  Graph-capturable (no allocation, no synchronisation). */
lqt_status lqt_solve(const lqt_problem *p, const double *x0, double *S, double *v, double *zeta, double *x,
                     double *u, double *cost, void *ws, size_t ws_bytes, void *stream);

/* Mixed-precision variant of lqt_solve (same arguments, same workspace size):
 * the element build (RK4 of the conditional HJB ODEs) and the LU solves of
 * I + C J inside every combination stay FP64, while the matrix products of the
 * combinations in both scans (forming I + C J, and every product after the
 * solve) run in FP32 with FP32 accumulation: on the CUDA cores for n <= 16,
 * and for n = 64 on the tensor core (tcgen05.mma kind::tf32 with each FP32
 * operand split into three TF32 pieces, so that the products keep FP32
 * accuracy).  Results are FP64 arrays; their error against the FP64 path is a
 * property of the problem (reported by the benchmark and tested against a
 * 1e-4 relative target). */
lqt_status lqt_solve_mixed(const lqt_problem *p, const double *x0, double *S, double *v, double *zeta, double *x,
                           double *u, double *cost, void *ws, size_t ws_bytes, void *stream);

/* The sequential method of Sec. VI-A as ONE GPU thread (the comparison
 * baseline): K RK4 steps per sub-interval of the Riccati ODEs for S, v, zeta
 * (Sec. II-B, eq. LQT_differential_S_v) backward from t_T, then K RK4 steps
 * per sub-interval of the closed-loop ODE (eq. optimal_trajectory_ODE_LQT)
 * forward from x0, with S, v at the step midpoints from the cubic Hermite
 * interpolant of the backward solution.  Same outputs as lqt_solve. */
lqt_status lqt_solve_sequential(const lqt_problem *p, const double *x0, double *S, double *v, double *zeta,
                                double *x, double *u, double *cost, void *ws, size_t ws_bytes, void *stream);

/* Time-invariant specialisation of the element build (row a1 for problems
 * with F, L, U, X constant and H constant or NULL; c and r may vary; n <= 8,
 * or n = 16 with 5 <= m <= 8).
 * With such coefficients and sub-intervals of one length h K, every
 * sub-interval's RK4 of Theorem Backward_HJB_LQT (Sec. IV-B) gives the same
 * A, C, J and passes through the same A, J at every RK4 stage (the paper's
 * observation in Sec. VI-B that a time-invariant model has one conditional
 * value function per block): one thread integrates A, C, J once and records the
 * stage matrices; one thread per sub-interval then integrates only b, eta,
 * zeta.  The elements equal lqt_build_elements' up to rounding.  The grid must
 * be uniform: a sub-interval whose length differs from the first one's by
 * more than 1e-12 relative plus the rounding of its end points
 * (8 DBL_EPSILON (|t_j| + |t_j+1| + |t_0| + |t_1|)) sets the status word
 * (lqt_get_status gives LQT_EINVAL).  Coefficients not constant, or other n, m: LQT_EUNSUPPORTED.
 * lqt_build_elements_invariant: as lqt_build_elements (T+1 elements incl. the
 * terminal one); workspace lqt_workspace_size(p, LQT_WS_INVARIANT).
 * lqt_solve_invariant: as lqt_solve with this build; workspace
 * lqt_workspace_size(p, LQT_WS_SOLVE_INVARIANT).  Asynchronous, allocation-free. */
lqt_status lqt_build_elements_invariant(const lqt_problem *p, const lqt_elements *out, void *ws, size_t ws_bytes,
                                        void *stream);
lqt_status lqt_solve_invariant(const lqt_problem *p, const double *x0, double *S, double *v, double *zeta, double *x,
                               double *u, double *cost, void *ws, size_t ws_bytes, void *stream);

/* Method 2 of the optimal-trajectory recovery (Sec. IV-E, eq.
 * Opt_trajectory_method2) with elements from the forward conditional HJB ODEs
 * (Sec. IV-C, Theorem Forward_HJB_LQT).  Supported: every n of lqt_solve
 * (n <= 8 one thread per element; n = 16 one warp, n = 64 one 256-thread CTA
 * per element and per combination).  All three are asynchronous and
 * allocation-free.
 *
 * lqt_build_elements_forward: the T elements a_j = V(., t_j; ., t_{j+1}),
 * j = 0..T-1 (no terminal element), each by K classical RK4 steps of the
 * forward conditional ODEs in tau from A = I, b = C = eta = J = 0, zeta = 0 at
 * tau = t_j (eq. abcej_boundary) to t_{j+1}, stage samples at half-steps 2i,
 * 2i+1, 2i+2 of step i.  zeta (not given in the paper) follows
 * dzeta/dtau = r'Xr/2 - b'H'Xr + b'H'XHb/2, the state-free part of the forward
 * conditional HJB at x = 0, z = b.  Output layout as lqt_build_elements, T
 * entries; workspace lqt_workspace_size(p, LQT_WS_BUILD).
 *
 * lqt_trajectory_method2: from those T elements and the values S, v (device,
 * [T+1], e.g. from lqt_solve), the prefixes V(., t_0; ., t_k) =
 * a_0 (x) ... (x) a_{k-1} by a parallel prefix scan with the combination of
 * Sec. IV-A (eq. lqt_comb), and then
 *   x_k = (I + C_k S_k)^-1 (A_k x0 + b_k + C_k v_k),  k = 0..T,
 * with (A_k, b_k, C_k) the prefix's parameters, and u_k by eq.
 * LQT_optimal_control.  x [T+1][n], u [T+1][m] (u may be NULL).  Workspace
 * lqt_workspace_size(p, LQT_WS_METHOD2).
 *
 * lqt_solve_method2: the whole path of the paper's Method 2 variant: values by
 * the backward-ODE elements and the suffix scan (as lqt_solve), states by the
 * forward-ODE elements, the prefix scan and the formula above; outputs and
 * cost as lqt_solve.  Workspace lqt_workspace_size(p, LQT_WS_SOLVE_METHOD2). */
lqt_status lqt_build_elements_forward(const lqt_problem *p, const lqt_elements *out, void *ws, size_t ws_bytes,
                                      void *stream);
lqt_status lqt_trajectory_method2(const lqt_problem *p, const lqt_elements *fwd, const double *S, const double *v,
                                  const double *x0, double *x, double *u, void *ws, size_t ws_bytes, void *stream);
lqt_status lqt_solve_method2(const lqt_problem *p, const double *x0, double *S, double *v, double *zeta, double *x,
                             double *u, double *cost, void *ws, size_t ws_bytes, void *stream);

/* Within-block densification: the optimal solution at every RK4 sub-step
 * t_j + i h_j (h_j = (t_{j+1} - t_j)/K, i = 0..K-1) of every sub-interval and at
 * t_T, from the solution at the sub-interval boundaries (Sec. IV-E: the optimal
 * trajectory inside a sub-interval; Sec. VI-A: the K-step fine grid).
 * Inputs (device): S [T+1][n][n], v [T+1][n], zeta [T+1], x [T+1][n], e.g. the
 * outputs of lqt_solve.  Per sub-interval j, independently: K classical RK4
 * steps of the Riccati ODEs (Sec. II-B, eq. LQT_differential_S_v, plus the zeta
 * equation) backward from (S, v, zeta) at t_{j+1} with the element build's
 * half-step samples, then RK4 of the closed-loop ODE (eq.
 * optimal_trajectory_ODE_LQT) forward from x_j with S, v at step midpoints from
 * the cubic Hermite interpolant of the backward values; controls by eq.
 * LQT_optimal_control with the L, U sample at each sub-step.  At the
 * boundaries (i = 0 and t_T) the outputs are the inputs themselves.
 * Outputs (device, fine index g = j K + i, last g = T K): Sd [TK+1][n][n],
 * vd [TK+1][n], zd [TK+1], xd [TK+1][n], ud [TK+1][m] (ud may be NULL).
 * Workspace: lqt_workspace_size(p, LQT_WS_DENSIFY) (derived coefficients).
 * Supported: n <= 8, K <= 16 (otherwise LQT_EUNSUPPORTED).  Asynchronous,
 * allocation-free. */
lqt_status lqt_densify(const lqt_problem *p, const double *S, const double *v, const double *zeta, const double *x,
                       double *Sd, double *vd, double *zd, double *xd, double *ud, void *ws, size_t ws_bytes,
                       void *stream);

/* Reverse mode of lqt_solve: gradients of a scalar loss with respect to the
 * coefficients, given the forward outputs S, v, x of lqt_solve (device) and the
 * loss's gradients with respect to them: gS [T+1][n][n], gv [T+1][n],
 * gzeta [T+1], gx [T+1][n] (each may be NULL = zero) and g_cost (host scalar,
 * the weight of the optimal cost V(x0,t0)).  gu must be NULL (controls are not
 * differentiated).
 * Outputs (device, each may be NULL): gF, gL, gX, gU, gr in the layout and
 * sampling mode of F, L, X, U, r (one gradient per sample); gXf [n][n],
 * grf [n]; gx0 [n].
 * The elements and the optimal-state maps are recomputed from the problem and
 * S, v; the RK4 stage inputs that the discrete adjoint needs are recomputed
 * in segments of 2^15 sub-intervals just before that segment's reverse sweep,
 * each from its sub-interval's fixed initial condition (A = I, the rest 0), so
 * the workspace holds at most one segment's stage inputs, not T's.  Steps:
 * state adjoint (a reverse linear
 * recurrence run as a forward affine scan), map adjoint, value adjoint (a
 * forward congruence scan Sigma_{k+1} = P_k Sigma_k P_k^T + D_{k+1} with the
 * homogeneous optimal-state maps P_k), element adjoint from the saddle point of
 * the dual form (Sec. IV-A, eq. LQT_V_form2), and the discrete adjoint of the K
 * RK4 steps of Theorem Backward_HJB_LQT (Sec. IV-B).
 * Supported: n <= 8, K <= 8, H = Hf = c = NULL, F, L, X, U constant or per
 * sub-interval (r any mode); otherwise LQT_EUNSUPPORTED. */
lqt_status lqt_backward(const lqt_problem *p, const double *x0, const double *S, const double *v, const double *x,
                        const double *gS, const double *gv, const double *gzeta, const double *gx, const double *gu,
                        double g_cost, double *gF, double *gL, double *gX, double *gU, double *gr, double *gXf,
                        double *grf, double *gx0, void *ws, size_t ws_bytes, void *stream);

/* Batches: many independent problems of ONE state dimension n solved by one
 * call (problems of several dimensions: one call per dimension, e.g. captured
 * together in one CUDA graph).  All problems share n, m, nr = n, K and the
 * sampling mode of r; F, L, X, U (and c, if given) are constant per problem;
 * H = Hf = NULL.  Each problem keeps its own T, time grid and data.
 * The problems are laid end to end: problem b's boundaries are
 * [off_b, off_b + T_b] of the concatenated outputs, off_b = sum_{b'<b}
 * (T_b' + 1): S [total][n][n], v [total][n], zeta [total], x [total][n],
 * u [total][m] (may be NULL), cost [count] (may be NULL), total =
 * lqt_batch_boundaries().  Internally one value scan and one state scan run
 * over the whole concatenation: a terminal element (A = b = C = 0, Sec. IV-D)
 * separates the problems' values exactly; the only leak, additive in zeta, is
 * removed afterwards, and the state map at each problem's end is replaced by
 * a jump to the next problem's x0. */
typedef struct {
  int32_t count;                 /* number of problems B >= 1 */
  const lqt_problem *problems;   /* HOST array of B descriptors (their data pointers are device pointers) */
  const double *const *x0;       /* HOST array of B device pointers, each [n] */
} lqt_batch;

/* Tunables of the batched solve, chosen by the caller's autotuner.
 * chunk: sub-intervals per thread (per team for n >= 16) in the first scan
 * level, a power of two in [2, 32]; 0 = built-in choice; anything else gives
 * LQT_EINVAL.  lqt_batch_workspace_size() covers every allowed value.
 * flags: LQT_TUNE_INVARIANT_BUILD selects the time-invariant element build
 * (see lqt_build_elements_invariant): every problem of a batch already has
 * constant F, L, U, X; each must also have sub-intervals of one length (else
 * the status word reports LQT_EINVAL); n <= 8, or n = 16 with 5 <= m <= 8
 * (else LQT_EUNSUPPORTED).  Other bits: LQT_EINVAL. */
enum { LQT_TUNE_INVARIANT_BUILD = 1 };
typedef struct {
  int32_t chunk;
  int32_t flags;
} lqt_tuning;

size_t lqt_batch_workspace_size(const lqt_batch *b);
int64_t lqt_batch_boundaries(const lqt_batch *b);

/* Writes the batch's device-side tables (per-problem descriptors, offsets)
 * into the workspace and synchronises the stream.  Call once per batch and
 * workspace, before lqt_solve_batched (and before any stream capture). */
lqt_status lqt_batch_plan(const lqt_batch *b, void *ws, size_t ws_bytes, void *stream);

/* Solves the planned batch: launches only (no copies, no synchronisation), so
 * it can be captured in a CUDA graph. */
lqt_status lqt_solve_batched(const lqt_batch *b, const lqt_tuning *tune, double *S, double *v, double *zeta,
                             double *x, double *u, double *cost, void *ws, size_t ws_bytes, void *stream);

/* End-to-end convenience call on HOST buffers: the problem's pointers (t, the
 * coefficients, Hf, Xf, rf) and x0 point at host memory, and so do the
 * outputs.  Copies the inputs to the caller's device workspace (its size from
 * lqt_workspace_size(p, LQT_WS_SOLVE) + lqt_host_staging_size(p)), runs
 * lqt_solve on `stream`, copies the outputs back and synchronises the stream.
 * For n <= 8 and T >= 2^16 the sampled coefficients are copied in up to 16
 * chunks on a stream of the call's own, each chunk's derived coefficients and
 * elements built on `stream` as soon as it (and the next chunk, which holds its
 * last sample) has arrived; the results are lqt_solve's, bit for bit.  Host
 * buffers should be pinned for full copy speed (pageable ones work, with
 * copies that complete before they return). */
size_t lqt_host_staging_size(const lqt_problem *p);
lqt_status lqt_solve_host(const lqt_problem *p, const double *x0, double *S, double *v, double *zeta, double *x,
                          double *u, double *cost, void *ws, size_t ws_bytes, void *stream);

/* Allocation-free value scan.  The paper has no counterpart: this is a
 * deployment variant of lqt_scan_value for callers that may not allocate
 * device memory while they run (a control loop whose memory budget is fixed at
 * start-up, a plugin inside an application that owns the device allocator) and
 * so cannot hand in a workspace.  It computes exactly what lqt_scan_value
 * computes, with the scan's scratch in a fixed array inside the library of
 * LQT_STATIC_SCRATCH_BYTES bytes, held on every device that loads the library
 * until the process exits.
 *  - Problems whose scan needs more scratch than that (see
 *    lqt_workspace_size(p, LQT_WS_VALUE)) return LQT_EWORKSPACE before any
 *    launch.  The largest T admitted, by state dimension: n = 1: 7 454 719;
 *    n = 2: 2 795 391; n = 3: 44 607; n = 4: 26 877; n = 8: 7 429;
 *    n = 16: 1 951; n = 64: none (every n = 64 problem is rejected).
 *  - The first call on a device looks up the array's device address (with that
 *    device current) and caches it: make that first call before any stream
 *    capture.
 *  - All calls share the one array: calls that overlap on the GPU (several
 *    streams or host threads at once) race and give wrong results.  Nothing
 *    needs clearing between calls (every scratch byte read is written earlier
 *    in the same call).
 *  - Calls no allocator (no cudaMalloc/cudaFree, no library routine that
 *    allocates).
 * Arguments as for lqt_scan_value. */
#define LQT_STATIC_SCRATCH_BYTES (16u << 20)
lqt_status lqt_scan_value_noalloc(const lqt_problem *p, const lqt_elements *el, double *S, double *v, double *zeta,
                                  void *stream);

/* ------------------------------------------------------------------------
 * The general method on a state grid (Sec. VI-B, App. E)
 *
 * The scalar nonlinear problem of Sec. VI-B, generalised to a quadratic drift:
 *     dx/dt = d0 + d1 x + d2 x^2 + u,   cost  qf x(tf)^2/2 + int q x^2/2 + rho u^2/2 dt
 * (the paper's falling body: d0 = 1, d1 = 0, d2 = -1/10, q = rho = 1, qf = 4,
 * blocks of length 1/10 split into 10 steps).  Functions of the state are held
 * at the G grid points x_i = x_min + i dx; a conditional value function
 * V(x_i, s; x_j, s') is a G x G row-major array (row: start point, column: end
 * point).  Its combination (Theorem HJB-comb) is the minimisation over the
 * grid of the intermediate state,
 *     (A (x) B)(i, j) = min_k A(i, k) + B(k, j),
 * the lowest k winning ties, refined (interp = 1) by App. E's quadratic
 * interpolation: with a, b the summed curvature and slope of the quadratics
 * through (k-1, k, k+1) of A(i, .) and B(., j), the minimum is lowered by
 * b^2 / (4a) when a > 0 and k is not at an end of the grid.
 *
 * The block's conditional value function is built from the one-step function
 * of an explicit Euler step dt = tau / substeps (from x_i to x_j with control
 * u = (x_j - x_i)/dt - drift(x_i), cost dt (q x_i^2 + rho u^2)/2), combined
 * with itself `substeps` times left to right.  This replaces the paper's
 * direct-shooting solve of the block problem.
 *
 * Every floating-point operation is IEEE round-to-nearest double in the order
 * the formulas above state, without multiply-add contraction.
 * ---------------------------------------------------------------------- */
typedef struct {
  int32_t G;         /* grid points, 3 <= G <= 16384                            */
  double x_min, dx;  /* x_i = x_min + i dx, dx > 0                               */
  double d0, d1, d2; /* drift d0 + d1 x + d2 x^2                                 */
  double q, rho, qf; /* running state weight, control weight (> 0), terminal     */
  double tau;        /* block length (> 0)                                       */
  int32_t substeps;  /* Euler steps per block (>= 1)                             */
  int64_t T;         /* blocks, 1 <= T < 2^31                                    */
  int32_t interp;    /* 1: App. E refinement of every minimisation; 0: plain     */
} lqt_grid_problem;

/* Workspace bytes: which = 0 for lqt_grid_block (2 G^2 doubles), 1 for
 * lqt_grid_values (3 G^2 ceil(log2(T+1)) + 1 + (T+1) G doubles: the powers,
 * their App. E curvatures and slopes, one value buffer).  0 when p is invalid
 * or `which` unknown. */
size_t lqt_grid_workspace_size(const lqt_grid_problem *p, int32_t which);

/* The block's conditional value function Vblock (G x G, device) as described
 * above.  Workspace: lqt_grid_workspace_size(p, 0).  Non-finite outputs are
 * recorded in the status word. */
lqt_status lqt_grid_block(const lqt_grid_problem *p, double *Vblock, void *ws, size_t ws_bytes, void *stream);

/* out = A (x) B, all G x G device arrays; out must not overlap A or B.  No
 * workspace. */
lqt_status lqt_grid_combine(const lqt_grid_problem *p, const double *A, const double *B, double *out, void *stream);

/* The value functions V(., t_k) = V[k][0..G-1], k = 0..T (device,
 * (T+1) x G), of the time-invariant problem whose every block has the
 * conditional value function Vblock (G x G, device; Sec. VI-B: one block
 * function serves every block).  V[T] is the terminal cost.  Evaluation order
 * (Theorem parallel_HJB, grouped for a logarithmic span): the powers
 * P_0 = Vblock, P_{l+1} = P_l (x) P_l; then V[k] = P_{l_r} (x) (... (P_{l_1} (x) phi))
 * over the set bits l_1 < ... < l_r of T - k.  Without the refinement this
 * equals the sequential fold V[k] = Vblock (x) V[k+1] exactly (the grid
 * minimum is associative); with it the two differ by the interpolation error.
 * Workspace: lqt_grid_workspace_size(p, 1).  V must not overlap Vblock or the
 * workspace. */
lqt_status lqt_grid_values(const lqt_grid_problem *p, const double *Vblock, double *V, void *ws, size_t ws_bytes,
                           void *stream);

/* Waits for `stream` (polling, at most timeout_ms; < 0 waits forever), then
 * reads and clears the current device's status word.  Returns LQT_OK,
 * LQT_ENONFINITE, LQT_ESINGULAR, LQT_ETIMEOUT or LQT_ECUDA. */
lqt_status lqt_get_status(void *stream, int32_t timeout_ms);

/* Throughput probe of the FMA pipes, a measurement aid with no counterpart in
 * the paper: the roofline denominator of this library's FP64-bound kernels
 * (Sec. IV-A and IV-B give their work; the chip's FP64 rate bounds it), taken
 * on the device they run on.  Launches `blocks` CTAs of `threads` threads
 * (a multiple of 32, <= 1024); every thread whose lane index is below
 * `active_lanes` (1..32) runs 8 independent chains x <- x a + b for `iters`
 * rounds; precision 0 = FP64 (DFMA), 1 = FP32 (FFMA).  Work:
 * 2 * 8 * iters * blocks * threads * active_lanes / 32 flop (FMA = 2); the
 * caller times the launch on `stream`.  out: device scratch of
 * blocks * threads doubles, caller-owned (written, meaningless).  Invalid
 * sizes: LQT_EINVAL before any launch. */
lqt_status lqt_probe_fma_rate(int32_t precision, int32_t blocks, int32_t threads, int32_t iters,
                              int32_t active_lanes, double *out, void *stream);

/* Human-readable name of a status code (static string). */
const char *lqt_strerror(lqt_status s);

/* Number of kernel launches the last call on this host thread made (for
 * launch accounting). */
int32_t lqt_last_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* LQT_H */
