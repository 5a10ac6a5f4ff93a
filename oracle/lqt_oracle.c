/*
 * Oracle for the temporally parallel continuous-time LQT method of
 * Sarkka & Garcia-Fernandez, "Temporal Parallelisation of the HJB Equation and
 * Continuous-Time Linear Quadratic Control" (arXiv 2212.11744).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, sequential FP64 CPU
 * restatement of what the GPU path computes.  Only the tests, the smoke check
 * and the CPU-baseline leg of the benchmark may load it; the product path never
 * does.  It shares no code, header or constant with the CUDA sources.
 *
 * Two solvers live here:
 *
 *  O1  "same discretisation" solver: every sub-interval's conditional value
 *      function (A, b, C, eta, J, zeta) is integrated with classical RK4 from the
 *      backward conditional HJB ODEs (Sec. IV-B, Theorem "Backward_HJB_LQT",
 *      boundary eq. abcej_boundary), the terminal element is eq.
 *      LQT_final_initialisation (Sec. IV-D), the elements are folded right to
 *      left with the LQT combination rule (Sec. IV-A, eq. lqt_comb), which gives
 *      S = J and v = eta at every block boundary (eq. eJ_vS), and the optimal
 *      states follow from the one-block form of Method 2 (Sec. IV-E).
 *
 *  O2  the sequential method of Sec. VI-A: RK4 of the Riccati ODEs for S, v
 *      (Sec. II-B, eq. LQT_differential_S_v) on the fine grid, backward from
 *      t_f, then a forward RK4 of the closed-loop ODE (eq.
 *      optimal_trajectory_ODE_LQT) with the control law eq. LQT_optimal_control.
 *
 * and, further down, the within-block densification (Sec. IV-E, Sec. VI-A),
 * Method 2 with forward-ODE elements (Sec. IV-C, Theorem Forward_HJB_LQT;
 * Sec. IV-E) and the grid method for the nonlinear scalar example (Sec. VI-B,
 * App. E), each with its own header comment.
 *
 * Readings where the paper is silent (each is listed in the design notes):
 *  - zeta (the state-free part of V, eq. V_quadratic_LQT) is carried along:
 *    element ODE d zeta/ds = -1/2 r'Xr + 1/2 eta'B eta + eta'c, terminal
 *    1/2 rf'Xf rf, combination term derived from the minimisation in
 *    Definition "Assoc_operator_HJB" (see lqt_combine below).
 *  - Coefficients are supplied as samples on the half-step grid of each block
 *    (PER_STAGE), once per block (PER_INTERVAL) or once (CONST).
 *  - O2 needs S, v at RK4 midpoints of the forward pass; it takes them from a
 *    cubic Hermite interpolant of the backward solution (values and the Riccati
 *    right-hand side at the two ends of the step), which is fourth order.
 *  - C and J are symmetric by the paper's statement; after every right-hand
 *    side and every combination they are replaced by (X + X')/2.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

enum { ORC_CONST = 0, ORC_PER_INTERVAL = 1, ORC_PER_STAGE = 2 };

/* Problem description.  Every matrix is row-major.  A coefficient pointer with
 * mode CONST holds one sample, PER_INTERVAL holds T samples (sample j is used on
 * the whole of block j), PER_STAGE holds 2*K*T+1 samples at the times
 * t_j + p*h_j/2, p = 0..2K, block ends shared (global index 2*K*j + p). */
typedef struct {
  int n, m, nr;
  long T;
  int K;
  const double *t; /* [T+1] block boundaries */
  const double *F; int F_mode; /* n x n                     */
  const double *L; int L_mode; /* n x m                     */
  const double *c; int c_mode; /* n, NULL = zero            */
  const double *H; int H_mode; /* nr x n, NULL = identity   */
  const double *X; int X_mode; /* nr x nr                   */
  const double *U; int U_mode; /* m x m                     */
  const double *r; int r_mode; /* nr, NULL = zero           */
  const double *Hf;            /* nr x n, NULL = identity   */
  const double *Xf;            /* nr x nr                   */
  const double *rf;            /* nr, NULL = zero           */
} orc_problem;

/* ------------------------------------------------------------------------ */
/* small dense linear algebra                                               */
/* ------------------------------------------------------------------------ */

/* out[p x q] = a[p x k] * b[k x q] */
static void mm(int p, int k, int q, const double *a, const double *b, double *out) {
  for (int i = 0; i < p; ++i)
    for (int j = 0; j < q; ++j) {
      double s = 0.0;
      for (int l = 0; l < k; ++l) s += a[i * k + l] * b[l * q + j];
      out[i * q + j] = s;
    }
}
/* out[p x q] = a[k x p]^T * b[k x q] */
static void mtm(int p, int k, int q, const double *a, const double *b, double *out) {
  for (int i = 0; i < p; ++i)
    for (int j = 0; j < q; ++j) {
      double s = 0.0;
      for (int l = 0; l < k; ++l) s += a[l * p + i] * b[l * q + j];
      out[i * q + j] = s;
    }
}
/* out[p x q] = a[p x k] * b[q x k]^T */
static void mmt(int p, int k, int q, const double *a, const double *b, double *out) {
  for (int i = 0; i < p; ++i)
    for (int j = 0; j < q; ++j) {
      double s = 0.0;
      for (int l = 0; l < k; ++l) s += a[i * k + l] * b[j * k + l];
      out[i * q + j] = s;
    }
}
static void transpose(int p, int q, const double *a, double *out) {
  for (int i = 0; i < p; ++i)
    for (int j = 0; j < q; ++j) out[j * p + i] = a[i * q + j];
}
static void symmetrise(int n, double *a) {
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j) {
      double s = 0.5 * (a[i * n + j] + a[j * n + i]);
      a[i * n + j] = s;
      a[j * n + i] = s;
    }
}
static void eye(int n, double *a) {
  memset(a, 0, sizeof(double) * n * n);
  for (int i = 0; i < n; ++i) a[i * n + i] = 1.0;
}

/* Solve W * Xs = Bs for Xs (W n x n, Bs n x q) by Gaussian elimination with
 * partial pivoting.  W and Bs are overwritten; the solution is left in Bs.
 * Returns 0, or 1 if a pivot is exactly zero. */
static int solve(int n, int q, double *W, double *Bs) {
  for (int k = 0; k < n; ++k) {
    int piv = k;
    double best = fabs(W[k * n + k]);
    for (int i = k + 1; i < n; ++i)
      if (fabs(W[i * n + k]) > best) { best = fabs(W[i * n + k]); piv = i; }
    if (best == 0.0) return 1;
    if (piv != k) {
      for (int j = 0; j < n; ++j) { double s = W[k * n + j]; W[k * n + j] = W[piv * n + j]; W[piv * n + j] = s; }
      for (int j = 0; j < q; ++j) { double s = Bs[k * q + j]; Bs[k * q + j] = Bs[piv * q + j]; Bs[piv * q + j] = s; }
    }
    for (int i = k + 1; i < n; ++i) {
      double f = W[i * n + k] / W[k * n + k];
      if (f == 0.0) continue;
      for (int j = k; j < n; ++j) W[i * n + j] -= f * W[k * n + j];
      for (int j = 0; j < q; ++j) Bs[i * q + j] -= f * Bs[k * q + j];
    }
  }
  for (int k = n - 1; k >= 0; --k)
    for (int j = 0; j < q; ++j) {
      double s = Bs[k * q + j];
      for (int l = k + 1; l < n; ++l) s -= W[k * n + l] * Bs[l * q + j];
      Bs[k * q + j] = s / W[k * n + k];
    }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* coefficients                                                             */
/* ------------------------------------------------------------------------ */

/* Sample of a coefficient for block j at half-step p (0..2K). */
static const double *sample(const double *base, int mode, size_t size, long j, int p, int K) {
  if (mode == ORC_CONST) return base;
  if (mode == ORC_PER_INTERVAL) return base + (size_t)j * size;
  return base + ((size_t)(2 * K) * (size_t)j + (size_t)p) * size;
}

/* Coefficients evaluated at one time point (one sample of each). */
typedef struct {
  double *F, *L, *c, *H, *X, *U, *r; /* copies, with identity / zero filled in */
  double *B;   /* L U^{-1} L^T                         n x n  */
  double *Q;   /* H^T X H                              n x n  */
  double *q;   /* H^T X r                              n      */
  double rho;  /* r^T X r                                     */
  double *G;   /* U^{-1} L^T, the feedback map          m x n  */
} coefs;

static double *take(double **cur, size_t count) { double *p = *cur; *cur += count; return p; }

static void coefs_alloc(coefs *cf, int n, int m, int nr, double **cur) {
  cf->F = take(cur, (size_t)n * n);
  cf->L = take(cur, (size_t)n * m);
  cf->c = take(cur, (size_t)n);
  cf->H = take(cur, (size_t)nr * n);
  cf->X = take(cur, (size_t)nr * nr);
  cf->U = take(cur, (size_t)m * m);
  cf->r = take(cur, (size_t)nr);
  cf->B = take(cur, (size_t)n * n);
  cf->Q = take(cur, (size_t)n * n);
  cf->q = take(cur, (size_t)n);
  cf->G = take(cur, (size_t)m * n);
}
static size_t coefs_size(int n, int m, int nr) {
  return (size_t)n * n + (size_t)n * m + n + (size_t)nr * n + (size_t)nr * nr + (size_t)m * m + nr +
         2 * (size_t)n * n + n + (size_t)m * n;
}

/* Evaluate all coefficients at block j, half-step p. */
static int coefs_eval(const orc_problem *P, long j, int p, coefs *cf) {
  int n = P->n, m = P->m, nr = P->nr, K = P->K;
  memcpy(cf->F, sample(P->F, P->F_mode, (size_t)n * n, j, p, K), sizeof(double) * n * n);
  memcpy(cf->L, sample(P->L, P->L_mode, (size_t)n * m, j, p, K), sizeof(double) * n * m);
  if (P->c) memcpy(cf->c, sample(P->c, P->c_mode, n, j, p, K), sizeof(double) * n);
  else memset(cf->c, 0, sizeof(double) * n);
  if (P->H) memcpy(cf->H, sample(P->H, P->H_mode, (size_t)nr * n, j, p, K), sizeof(double) * nr * n);
  else eye(n, cf->H);
  memcpy(cf->X, sample(P->X, P->X_mode, (size_t)nr * nr, j, p, K), sizeof(double) * nr * nr);
  memcpy(cf->U, sample(P->U, P->U_mode, (size_t)m * m, j, p, K), sizeof(double) * m * m);
  if (P->r) memcpy(cf->r, sample(P->r, P->r_mode, nr, j, p, K), sizeof(double) * nr);
  else memset(cf->r, 0, sizeof(double) * nr);

  /* G = U^{-1} L^T  (m x n), B = L G (n x n) */
  double *W = (double *)malloc(sizeof(double) * (m * m + (size_t)nr * n + nr + (size_t)nr * nr));
  memcpy(W, cf->U, sizeof(double) * m * m);
  transpose(n, m, cf->L, cf->G);
  if (solve(m, n, W, cf->G)) { free(W); return 1; }
  mm(n, m, n, cf->L, cf->G, cf->B);
  symmetrise(n, cf->B);
  /* Q = H^T X H, q = H^T X r, rho = r^T X r */
  double *XH = W;                 /* nr x n */
  double *Xr = W + (size_t)nr * n; /* nr */
  mm(nr, nr, n, cf->X, cf->H, XH);
  mtm(n, nr, n, cf->H, XH, cf->Q);
  symmetrise(n, cf->Q);
  mm(nr, nr, 1, cf->X, cf->r, Xr);
  mtm(n, nr, 1, cf->H, Xr, cf->q);
  double rho = 0.0;
  for (int i = 0; i < nr; ++i) rho += cf->r[i] * Xr[i];
  cf->rho = rho;
  free(W);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* elements: (A, b, C, eta, J, zeta), stored contiguously                   */
/* ------------------------------------------------------------------------ */

static size_t elem_size(int n) { return (size_t)3 * n * n + 2 * (size_t)n + 1; }
typedef struct { double *A, *b, *C, *eta, *J, *zeta; } elem_view;
static elem_view view(int n, double *e) {
  elem_view v;
  v.A = e;
  v.b = v.A + n * n;
  v.C = v.b + n;
  v.eta = v.C + n * n;
  v.J = v.eta + n;
  v.zeta = v.J + n * n;
  return v;
}

/* Right-hand side of the backward conditional HJB ODEs in s (Sec. IV-B,
 * Theorem "Backward_HJB_LQT"), plus the zeta equation:
 *   dA/ds    =  A B J - A F
 *   db/ds    = -A B eta - A c
 *   dC/ds    = -A B A^T
 *   deta/ds  = -H^T X r - F^T eta + J c + J B eta
 *   dJ/ds    = -H^T X H - J F - F^T J + J B J
 *   dzeta/ds = -1/2 r^T X r + 1/2 eta^T B eta + eta^T c
 * with B = L U^{-1} L^T.  tmp needs 4 n^2 doubles. */
static void element_rhs(int n, const coefs *cf, const double *y, double *dy, double *tmp) {
  elem_view s = view(n, (double *)y), d = view(n, dy);
  double *BJ = tmp, *AB = tmp + n * n, *M1 = tmp + 2 * n * n, *M2 = tmp + 3 * n * n;
  /* dA = A (B J) - A F */
  mm(n, n, n, cf->B, s.J, BJ);
  mm(n, n, n, s.A, BJ, M1);
  mm(n, n, n, s.A, cf->F, M2);
  for (int i = 0; i < n * n; ++i) d.A[i] = M1[i] - M2[i];
  /* db = -A (B eta) - A c */
  double *Beta = M1; /* n */
  mm(n, n, 1, cf->B, s.eta, Beta);
  for (int i = 0; i < n; ++i) {
    double acc = 0.0;
    for (int k = 0; k < n; ++k) acc += s.A[i * n + k] * (Beta[k] + cf->c[k]);
    d.b[i] = -acc;
  }
  /* dC = -A B A^T */
  mm(n, n, n, s.A, cf->B, AB);
  mmt(n, n, n, AB, s.A, M2);
  for (int i = 0; i < n * n; ++i) d.C[i] = -M2[i];
  symmetrise(n, d.C);
  /* deta = -q - F^T eta + J c + J B eta */
  for (int i = 0; i < n; ++i) {
    double acc = -cf->q[i];
    for (int k = 0; k < n; ++k) acc -= cf->F[k * n + i] * s.eta[k];
    for (int k = 0; k < n; ++k) acc += s.J[i * n + k] * cf->c[k];
    for (int k = 0; k < n; ++k) acc += s.J[i * n + k] * Beta[k];
    d.eta[i] = acc;
  }
  /* dJ = -Q - J F - F^T J + J B J */
  double *JF = M2;
  mm(n, n, n, s.J, cf->F, JF);
  double *JBJ = AB;
  mm(n, n, n, s.J, BJ, JBJ);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      d.J[i * n + j] = -cf->Q[i * n + j] - JF[i * n + j] - JF[j * n + i] + JBJ[i * n + j];
  symmetrise(n, d.J);
  /* dzeta */
  double z = -0.5 * cf->rho;
  for (int i = 0; i < n; ++i) z += 0.5 * s.eta[i] * Beta[i] + s.eta[i] * cf->c[i];
  *d.zeta = z;
}

/* Element a_j = V(., t_j; ., t_{j+1}) by K classical RK4 steps of the backward
 * conditional ODEs, from the boundary A=I, b=C=eta=J=0, zeta=0 at s=t_{j+1}
 * (eq. abcej_boundary) down to s=t_j.  Step i runs from t_j+(i+1)h to t_j+ih and
 * uses the samples at half-steps p = 2i+2, 2i+1, 2i. */
static int build_block(const orc_problem *P, long j, double *e) {
  int n = P->n, K = P->K;
  size_t es = elem_size(n);
  double h = (P->t[j + 1] - P->t[j]) / K;
  double *buf = (double *)malloc(sizeof(double) * (5 * es + 4 * (size_t)n * n + coefs_size(n, P->m, P->nr)));
  double *y = buf, *yt = y + es, *k = yt + es, *acc = k + es, *tmp = acc + es;
  double *cur = tmp + 4 * (size_t)n * n + es;
  coefs cf;
  coefs_alloc(&cf, n, P->m, P->nr, &cur);
  memset(y, 0, sizeof(double) * es);
  eye(n, view(n, y).A);
  int bad = 0;
  for (int i = K - 1; i >= 0; --i) {
    /* k1 at s = t_j + (i+1) h */
    bad |= coefs_eval(P, j, 2 * i + 2, &cf);
    element_rhs(n, &cf, y, k, tmp);
    for (size_t q = 0; q < es; ++q) { acc[q] = k[q]; yt[q] = y[q] - 0.5 * h * k[q]; }
    /* k2, k3 at s - h/2 */
    bad |= coefs_eval(P, j, 2 * i + 1, &cf);
    element_rhs(n, &cf, yt, k, tmp);
    for (size_t q = 0; q < es; ++q) { acc[q] += 2.0 * k[q]; yt[q] = y[q] - 0.5 * h * k[q]; }
    element_rhs(n, &cf, yt, k, tmp);
    for (size_t q = 0; q < es; ++q) { acc[q] += 2.0 * k[q]; yt[q] = y[q] - h * k[q]; }
    /* k4 at s - h */
    bad |= coefs_eval(P, j, 2 * i, &cf);
    element_rhs(n, &cf, yt, k, tmp);
    for (size_t q = 0; q < es; ++q) { acc[q] += k[q]; y[q] = y[q] - (h / 6.0) * acc[q]; }
  }
  memcpy(e, y, sizeof(double) * es);
  free(buf);
  return bad;
}

/* Terminal element a_T = V(., t_f) (Sec. IV-D, eq. LQT_final_initialisation):
 * A = b = C = 0, J = Hf^T Xf Hf, eta = Hf^T Xf rf, zeta = 1/2 rf^T Xf rf. */
static void terminal_element(const orc_problem *P, double *e) {
  int n = P->n, nr = P->nr;
  size_t es = elem_size(n);
  memset(e, 0, sizeof(double) * es);
  elem_view v = view(n, e);
  double *Hf = (double *)malloc(sizeof(double) * ((size_t)nr * n * 2 + 2 * (size_t)nr));
  double *XH = Hf + (size_t)nr * n, *rf = XH + (size_t)nr * n, *Xr = rf + nr;
  if (P->Hf) memcpy(Hf, P->Hf, sizeof(double) * nr * n);
  else eye(n, Hf);
  if (P->rf) memcpy(rf, P->rf, sizeof(double) * nr);
  else memset(rf, 0, sizeof(double) * nr);
  mm(nr, nr, n, P->Xf, Hf, XH);
  mtm(n, nr, n, Hf, XH, v.J);
  symmetrise(n, v.J);
  mm(nr, nr, 1, P->Xf, rf, Xr);
  mtm(n, nr, 1, Hf, Xr, v.eta);
  double z = 0.0;
  for (int i = 0; i < nr; ++i) z += rf[i] * Xr[i];
  *v.zeta = 0.5 * z;
  free(Hf);
}

/* LQT combination e = e1 (x) e2 (Sec. IV-A, eq. lqt_comb), written out as in
 * the lemma with M = (I + C1 J2)^{-1} and (I + J2 C1)^{-1} = M^T:
 *   A   = A2 M A1
 *   b   = A2 M (b1 + C1 eta2) + b2
 *   C   = A2 M C1 A2^T + C2
 *   eta = A1^T M^T (eta2 - J2 b1) + eta1
 *   J   = A1^T M^T J2 A1 + J1
 * and the state-free term: with z0 = M (b1 + C1 eta2) (the minimiser at
 * x = 0 of Definition "Assoc_operator_HJB") and lambda0 = J2 z0 - eta2,
 *   zeta = zeta1 + zeta2 + 1/2 lambda0^T C1 lambda0 + 1/2 z0^T J2 z0 - z0^T eta2.
 * Returns nonzero if I + C1 J2 is singular. */
int orc_combine(int n, const double *e1, const double *e2, double *out) {
  size_t nn = (size_t)n * n;
  elem_view a = view(n, (double *)e1), c = view(n, (double *)e2);
  double *buf = (double *)malloc(sizeof(double) * (10 * nn + 6 * (size_t)n + elem_size(n)));
  double *W = buf, *MA1 = W + nn, *MC1 = MA1 + nn, *Mt = MC1 + nn, *T1 = Mt + nn, *T2 = T1 + nn;
  double *Minv = T2 + nn, *Wc = Minv + nn, *MtJ2A1 = Wc + nn, *J2A1 = MtJ2A1 + nn;
  double *z0 = J2A1 + nn, *rhs = z0 + n, *lam = rhs + n, *w = lam + n, *tv = w + n, *tv2 = tv + n;
  double *res = tv2 + n;
  elem_view o = view(n, res);
  /* M = (I + C1 J2)^{-1} as an explicit inverse (solve against the identity) */
  mm(n, n, n, a.C, c.J, W);
  for (int i = 0; i < n; ++i) W[i * n + i] += 1.0;
  memcpy(Wc, W, sizeof(double) * nn);
  eye(n, Minv);
  if (solve(n, n, Wc, Minv)) { free(buf); return 1; }
  transpose(n, n, Minv, Mt);
  /* A = A2 M A1 */
  mm(n, n, n, Minv, a.A, MA1);
  mm(n, n, n, c.A, MA1, o.A);
  /* b = A2 M (b1 + C1 eta2) + b2 */
  mm(n, n, 1, a.C, c.eta, tv);
  for (int i = 0; i < n; ++i) rhs[i] = a.b[i] + tv[i];
  mm(n, n, 1, Minv, rhs, z0);
  mm(n, n, 1, c.A, z0, tv);
  for (int i = 0; i < n; ++i) o.b[i] = tv[i] + c.b[i];
  /* C = A2 M C1 A2^T + C2 */
  mm(n, n, n, Minv, a.C, MC1);
  mm(n, n, n, c.A, MC1, T1);
  mmt(n, n, n, T1, c.A, T2);
  for (size_t i = 0; i < nn; ++i) o.C[i] = T2[i] + c.C[i];
  symmetrise(n, o.C);
  /* eta = A1^T M^T (eta2 - J2 b1) + eta1 */
  mm(n, n, 1, c.J, a.b, tv);
  for (int i = 0; i < n; ++i) w[i] = c.eta[i] - tv[i];
  mm(n, n, 1, Mt, w, tv);
  mtm(n, n, 1, a.A, tv, tv2);
  for (int i = 0; i < n; ++i) o.eta[i] = tv2[i] + a.eta[i];
  /* J = A1^T M^T J2 A1 + J1 */
  mm(n, n, n, c.J, a.A, J2A1);
  mm(n, n, n, Mt, J2A1, MtJ2A1);
  mtm(n, n, n, a.A, MtJ2A1, T1);
  for (size_t i = 0; i < nn; ++i) o.J[i] = T1[i] + a.J[i];
  symmetrise(n, o.J);
  /* zeta */
  mm(n, n, 1, c.J, z0, tv);
  for (int i = 0; i < n; ++i) lam[i] = tv[i] - c.eta[i];
  mm(n, n, 1, a.C, lam, tv2);
  double z = *a.zeta + *c.zeta;
  for (int i = 0; i < n; ++i) z += 0.5 * lam[i] * tv2[i] + 0.5 * z0[i] * tv[i] - z0[i] * c.eta[i];
  *o.zeta = z;
  memcpy(out, res, sizeof(double) * elem_size(n));
  free(buf);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* O1                                                                       */
/* ------------------------------------------------------------------------ */

/* Elements j in [j0, j1) with 0 <= j0 <= j1 <= T+1; j = T is the terminal
 * element.  Output: elems[(j - j0) * (3n^2+2n+1)], packed as A,b,C,eta,J,zeta.
 * Returns nonzero if some U sample was singular. */
int orc_build_elements(const orc_problem *P, long j0, long j1, double *elems) {
  size_t es = elem_size(P->n);
  int bad = 0;
  for (long j = j0; j < j1; ++j) {
    double *e = elems + (size_t)(j - j0) * es;
    if (j == P->T) terminal_element(P, e);
    else bad |= build_block(P, j, e);
  }
  return bad;
}

/* Reverse all-prefix-sums of the T+1 elements by the sequential loop of
 * Sec. II-C run right to left: sbar_T = a_T, sbar_k = a_k (x) sbar_{k+1}
 * (Theorem "parallel_HJB", eq. parallel_V_HJB).  The suffix at k is V(., t_k),
 * whose J, eta, zeta are S_k, v_k, zeta_k (eq. eJ_vS).  Writes S[(T+1) n n],
 * v[(T+1) n], zeta[T+1]. */
int orc_suffix_values(int n, long T, const double *elems, double *S, double *v, double *zeta) {
  size_t es = elem_size(n);
  double *s = (double *)malloc(sizeof(double) * 2 * es), *nxt = s + es;
  memcpy(s, elems + (size_t)T * es, sizeof(double) * es);
  int bad = 0;
  for (long k = T;; --k) {
    elem_view sv = view(n, s);
    memcpy(S + (size_t)k * n * n, sv.J, sizeof(double) * n * n);
    memcpy(v + (size_t)k * n, sv.eta, sizeof(double) * n);
    zeta[k] = *sv.zeta;
    if (k == 0) break;
    bad |= orc_combine(n, elems + (size_t)(k - 1) * es, s, nxt);
    memcpy(s, nxt, sizeof(double) * es);
  }
  free(s);
  return bad;
}

/* Control at the block boundary t_i (eq. LQT_optimal_control):
 * u = U^{-1} L^T (v - S x), with the coefficient sample at t_i (for
 * PER_INTERVAL: block i's sample, block T-1's at t_T). */
static int control_at(const orc_problem *P, long i, const double *S, const double *v, const double *x,
                      double *u, double *scratch, coefs *cf) {
  int n = P->n, m = P->m;
  long j = i < P->T ? i : P->T - 1;
  int p = i < P->T ? 0 : 2 * P->K;
  int bad = coefs_eval(P, j, p, cf);
  double *Sx = scratch;
  mm(n, n, 1, S, x, Sx);
  for (int k = 0; k < n; ++k) Sx[k] = v[k] - Sx[k];
  mm(m, n, 1, cf->G, Sx, u);
  return bad;
}

/* Optimal states by the one-block form of Method 2 (Sec. IV-E, with t_0 taken
 * as t_j): x_{j+1} = (I + C_j S_{j+1})^{-1} (A_j x_j + b_j + C_j v_{j+1}),
 * then u_i at every boundary.  x[(T+1) n], u[(T+1) m]. */
int orc_trajectory(const orc_problem *P, const double *elems, const double *S, const double *v,
                   const double *x0, double *x, double *u) {
  int n = P->n;
  long T = P->T;
  size_t es = elem_size(n), nn = (size_t)n * n;
  double *W = (double *)malloc(sizeof(double) * (2 * nn + 4 * (size_t)n + coefs_size(n, P->m, P->nr)));
  double *rhs = W + nn, *tv = rhs + n, *cur = tv + 2 * (size_t)n + nn;
  coefs cf;
  coefs_alloc(&cf, n, P->m, P->nr, &cur);
  int bad = 0;
  memcpy(x, x0, sizeof(double) * n);
  for (long j = 0; j < T; ++j) {
    elem_view e = view(n, (double *)(elems + (size_t)j * es));
    const double *S1 = S + (size_t)(j + 1) * nn, *v1 = v + (size_t)(j + 1) * n;
    mm(n, n, n, e.C, S1, W);
    for (int i = 0; i < n; ++i) W[i * n + i] += 1.0;
    mm(n, n, 1, e.A, x + (size_t)j * n, rhs);
    mm(n, n, 1, e.C, v1, tv);
    for (int i = 0; i < n; ++i) rhs[i] += e.b[i] + tv[i];
    bad |= solve(n, 1, W, rhs);
    memcpy(x + (size_t)(j + 1) * n, rhs, sizeof(double) * n);
  }
  for (long i = 0; i <= T; ++i)
    bad |= control_at(P, i, S + (size_t)i * nn, v + (size_t)i * n, x + (size_t)i * n, u + (size_t)i * P->m, tv,
                      &cf);
  free(W);
  return bad;
}

/* Full O1 solve.  elems (optional, may be NULL) receives the T+1 elements.
 * cost = V(x0, t0) = zeta_0 + 1/2 x0^T S_0 x0 - v_0^T x0 (eq. V_quadratic_LQT). */
int orc_solve(const orc_problem *P, const double *x0, double *S, double *v, double *zeta, double *x, double *u,
              double *cost, double *elems_out) {
  int n = P->n;
  size_t es = elem_size(n);
  double *elems = elems_out ? elems_out : (double *)malloc(sizeof(double) * es * (size_t)(P->T + 1));
  int bad = orc_build_elements(P, 0, P->T + 1, elems);
  bad |= orc_suffix_values(n, P->T, elems, S, v, zeta);
  bad |= orc_trajectory(P, elems, S, v, x0, x, u);
  double c = zeta[0];
  for (int i = 0; i < n; ++i) {
    double sx = 0.0;
    for (int k = 0; k < n; ++k) sx += S[i * n + k] * x0[k];
    c += 0.5 * x0[i] * sx - v[i] * x0[i];
  }
  *cost = c;
  if (!elems_out) free(elems);
  return bad;
}

/* ------------------------------------------------------------------------ */
/* O2: sequential Riccati sweep + forward rollout (Sec. VI-A)                */
/* ------------------------------------------------------------------------ */

/* Riccati right-hand side in t (eq. LQT_differential_S_v) plus zeta:
 *   dS/dt    = -F^T S - S F - H^T X H + S B S
 *   dv/dt    = -H^T X r + S c - F^T v + S B v
 *   dzeta/dt = -1/2 r^T X r + 1/2 v^T B v + v^T c
 * y = (S[n n], v[n], zeta).  tmp needs 3 n^2 doubles. */
static void riccati_rhs(int n, const coefs *cf, const double *y, double *dy, double *tmp) {
  const double *S = y, *v = y + n * n;
  double *dS = dy, *dv = dy + n * n;
  double *SF = tmp, *BS = tmp + n * n, *SBS = tmp + 2 * n * n;
  mm(n, n, n, S, cf->F, SF);
  mm(n, n, n, cf->B, S, BS);
  mm(n, n, n, S, BS, SBS);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      dS[i * n + j] = -SF[j * n + i] - SF[i * n + j] - cf->Q[i * n + j] + SBS[i * n + j];
  symmetrise(n, dS);
  double z = -0.5 * cf->rho;
  for (int i = 0; i < n; ++i) {
    double acc = -cf->q[i];
    for (int k = 0; k < n; ++k) acc += S[i * n + k] * cf->c[k];
    for (int k = 0; k < n; ++k) acc -= cf->F[k * n + i] * v[k];
    double Bv = 0.0;
    for (int k = 0; k < n; ++k) Bv += cf->B[i * n + k] * v[k];
    double SBv = 0.0;
    for (int k = 0; k < n; ++k) {
      double Bvk = 0.0;
      for (int l = 0; l < n; ++l) Bvk += cf->B[k * n + l] * v[l];
      SBv += S[i * n + k] * Bvk;
    }
    dv[i] = acc + SBv;
    z += 0.5 * v[i] * Bv + v[i] * cf->c[i];
  }
  dy[n * n + n] = z;
}

/* Closed-loop right-hand side dx/dt = F x + L u + c with
 * u = -U^{-1} L^T (S x - v)  (eqs. LQT_optimal_control and
 * optimal_trajectory_ODE_LQT). */
static void closed_loop_rhs(int n, int m, const coefs *cf, const double *S, const double *v, const double *x,
                            double *dx, double *tmp) {
  double *e = tmp, *u = tmp + n;
  for (int i = 0; i < n; ++i) {
    double acc = -v[i];
    for (int k = 0; k < n; ++k) acc += S[i * n + k] * x[k];
    e[i] = acc;
  }
  for (int i = 0; i < m; ++i) {
    double acc = 0.0;
    for (int k = 0; k < n; ++k) acc += cf->G[i * n + k] * e[k];
    u[i] = -acc;
  }
  for (int i = 0; i < n; ++i) {
    double acc = cf->c[i];
    for (int k = 0; k < n; ++k) acc += cf->F[i * n + k] * x[k];
    for (int k = 0; k < m; ++k) acc += cf->L[i * m + k] * u[k];
    dx[i] = acc;
  }
}

/* O2.  Fine grid: K steps of h_j = (t_{j+1}-t_j)/K per block.  Backward: RK4 of
 * the Riccati ODEs from S(t_f) = Hf^T Xf Hf, v(t_f) = Hf^T Xf rf,
 * zeta(t_f) = 1/2 rf^T Xf rf.  Forward: RK4 of the closed-loop ODE from x0,
 * with S, v at the step midpoints from the cubic Hermite interpolant
 * y(t+h/2) = (y0 + y1)/2 + h (y0' - y1')/8 of the backward solution, where the
 * end slopes y0', y1' are the Riccati right-hand side evaluated with the current
 * block's coefficients (one-sided at block ends).
 * Outputs at block boundaries: S, v, zeta, x, u (same shapes as orc_solve). */
int orc_sequential(const orc_problem *P, const double *x0, double *S, double *v, double *zeta, double *x, double *u,
                   double *cost) {
  int n = P->n, m = P->m, K = P->K;
  long T = P->T;
  size_t ys = (size_t)n * n + n + 1, nn = (size_t)n * n;
  size_t npts = (size_t)K * T + 1;
  double *grid = (double *)malloc(sizeof(double) * npts * ys); /* backward solution at every fine point */
  double *buf = (double *)malloc(sizeof(double) * (8 * ys + 3 * nn + 8 * (size_t)n + (size_t)m +
                                                   coefs_size(n, m, P->nr)));
  double *y = buf, *yt = y + ys, *k = yt + ys, *acc = k + ys, *ym = acc + ys, *d0 = ym + ys, *d1 = d0 + ys;
  double *tmp = d1 + ys + ys;
  double *xv = tmp + 3 * nn, *xt = xv + n, *kx = xt + n, *ax = kx + n, *t2 = ax + n;
  double *cur = t2 + 4 * (size_t)n + m;
  coefs cf;
  coefs_alloc(&cf, n, m, P->nr, &cur);
  int bad = 0;

  /* terminal values, reusing the terminal element */
  {
    double *e = (double *)malloc(sizeof(double) * elem_size(n));
    terminal_element(P, e);
    elem_view tv = view(n, e);
    memcpy(y, tv.J, sizeof(double) * nn);
    memcpy(y + nn, tv.eta, sizeof(double) * n);
    y[nn + n] = *tv.zeta;
    free(e);
  }
  memcpy(grid + (npts - 1) * ys, y, sizeof(double) * ys);
  for (long j = T - 1; j >= 0; --j) {
    double h = (P->t[j + 1] - P->t[j]) / K;
    for (int i = K - 1; i >= 0; --i) {
      bad |= coefs_eval(P, j, 2 * i + 2, &cf);
      riccati_rhs(n, &cf, y, k, tmp);
      for (size_t q = 0; q < ys; ++q) { acc[q] = k[q]; yt[q] = y[q] - 0.5 * h * k[q]; }
      bad |= coefs_eval(P, j, 2 * i + 1, &cf);
      riccati_rhs(n, &cf, yt, k, tmp);
      for (size_t q = 0; q < ys; ++q) { acc[q] += 2.0 * k[q]; yt[q] = y[q] - 0.5 * h * k[q]; }
      riccati_rhs(n, &cf, yt, k, tmp);
      for (size_t q = 0; q < ys; ++q) { acc[q] += 2.0 * k[q]; yt[q] = y[q] - h * k[q]; }
      bad |= coefs_eval(P, j, 2 * i, &cf);
      riccati_rhs(n, &cf, yt, k, tmp);
      for (size_t q = 0; q < ys; ++q) { acc[q] += k[q]; y[q] = y[q] - (h / 6.0) * acc[q]; }
      memcpy(grid + ((size_t)j * K + i) * ys, y, sizeof(double) * ys);
    }
  }

  for (long j = 0; j <= T; ++j) {
    const double *g = grid + (size_t)j * K * ys;
    memcpy(S + (size_t)j * nn, g, sizeof(double) * nn);
    memcpy(v + (size_t)j * n, g + nn, sizeof(double) * n);
    zeta[j] = g[nn + n];
  }

  /* forward closed-loop rollout */
  memcpy(xv, x0, sizeof(double) * n);
  memcpy(x, x0, sizeof(double) * n);
  for (long j = 0; j < T; ++j) {
    double h = (P->t[j + 1] - P->t[j]) / K;
    bad |= coefs_eval(P, j, 0, &cf);
    riccati_rhs(n, &cf, grid + (size_t)j * K * ys, d0, tmp);
    for (int i = 0; i < K; ++i) {
      size_t g0 = (size_t)j * K + i;
      const double *y0 = grid + g0 * ys, *y1 = grid + (g0 + 1) * ys;
      bad |= coefs_eval(P, j, 2 * i + 2, &cf);
      riccati_rhs(n, &cf, y1, d1, tmp);
      for (size_t q = 0; q < ys; ++q) ym[q] = 0.5 * (y0[q] + y1[q]) + h * (d0[q] - d1[q]) / 8.0;
      bad |= coefs_eval(P, j, 2 * i, &cf);
      closed_loop_rhs(n, m, &cf, y0, y0 + nn, xv, kx, t2);
      for (int q = 0; q < n; ++q) { ax[q] = kx[q]; xt[q] = xv[q] + 0.5 * h * kx[q]; }
      bad |= coefs_eval(P, j, 2 * i + 1, &cf);
      closed_loop_rhs(n, m, &cf, ym, ym + nn, xt, kx, t2);
      for (int q = 0; q < n; ++q) { ax[q] += 2.0 * kx[q]; xt[q] = xv[q] + 0.5 * h * kx[q]; }
      closed_loop_rhs(n, m, &cf, ym, ym + nn, xt, kx, t2);
      for (int q = 0; q < n; ++q) { ax[q] += 2.0 * kx[q]; xt[q] = xv[q] + h * kx[q]; }
      bad |= coefs_eval(P, j, 2 * i + 2, &cf);
      closed_loop_rhs(n, m, &cf, y1, y1 + nn, xt, kx, t2);
      for (int q = 0; q < n; ++q) { ax[q] += kx[q]; xv[q] = xv[q] + (h / 6.0) * ax[q]; }
      memcpy(d0, d1, sizeof(double) * ys);
    }
    memcpy(x + (size_t)(j + 1) * n, xv, sizeof(double) * n);
  }
  for (long i = 0; i <= T; ++i)
    bad |= control_at(P, i, S + (size_t)i * nn, v + (size_t)i * n, x + (size_t)i * n, u + (size_t)i * m, t2, &cf);
  double c = zeta[0];
  for (int i = 0; i < n; ++i) {
    double sx = 0.0;
    for (int q = 0; q < n; ++q) sx += S[i * n + q] * x0[q];
    c += 0.5 * x0[i] * sx - v[i] * x0[i];
  }
  *cost = c;
  free(buf);
  free(grid);
  return bad;
}

/* ------------------------------------------------------------------------ */
/* Method 2: forward-HJB elements, prefix fold, optimal states                 */
/* ------------------------------------------------------------------------ */

/* Right-hand side of the forward conditional HJB ODEs in tau (Sec. IV-C,
 * Theorem "Forward_HJB_LQT"), with Q = H^T X H, q = H^T X r, B = L U^{-1} L^T:
 *   dA/dtau    = -C Q A + F A
 *   db/dtau    =  C q + F b - C Q b + c
 *   dC/dtau    = -C Q C + B + F C + C F^T
 *   deta/dtau  =  A^T q - A^T Q b
 *   dJ/dtau    =  A^T Q A
 *   dzeta/dtau =  1/2 r^T X r - b^T q + 1/2 b^T Q b
 * The zeta equation is the state-free part of the forward conditional HJB
 * (eq. forward_conditional_HJB) at x = 0, z = b, where the multiplier vanishes:
 * the running cost of the target state b.  tmp needs 4 n^2 doubles. */
static void forward_rhs(int n, const coefs *cf, const double *y, double *dy, double *tmp) {
  elem_view s = view(n, (double *)y), d = view(n, dy);
  double *QA = tmp, *CQ = tmp + n * n, *M1 = tmp + 2 * n * n, *M2 = tmp + 3 * n * n;
  mm(n, n, n, cf->Q, s.A, QA);
  mm(n, n, n, s.C, cf->Q, CQ);
  /* dA = -C (Q A) + F A */
  mm(n, n, n, s.C, QA, M1);
  mm(n, n, n, cf->F, s.A, M2);
  for (int i = 0; i < n * n; ++i) d.A[i] = M2[i] - M1[i];
  /* db = C q + F b - C Q b + c */
  for (int i = 0; i < n; ++i) {
    double acc = cf->c[i];
    for (int k = 0; k < n; ++k) acc += s.C[i * n + k] * cf->q[k] + cf->F[i * n + k] * s.b[k];
    for (int k = 0; k < n; ++k) acc -= CQ[i * n + k] * s.b[k];
    d.b[i] = acc;
  }
  /* dC = -C Q C + B + F C + C F^T */
  mm(n, n, n, CQ, s.C, M1);
  mm(n, n, n, cf->F, s.C, M2);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      d.C[i * n + j] = -M1[i * n + j] + cf->B[i * n + j] + M2[i * n + j] + M2[j * n + i];
  symmetrise(n, d.C);
  /* deta = A^T (q - Q b);  dJ = A^T Q A */
  double *w = M1; /* n */
  for (int i = 0; i < n; ++i) {
    double acc = cf->q[i];
    for (int k = 0; k < n; ++k) acc -= cf->Q[i * n + k] * s.b[k];
    w[i] = acc;
  }
  mtm(n, n, 1, s.A, w, d.eta);
  mtm(n, n, n, s.A, QA, d.J);
  symmetrise(n, d.J);
  /* dzeta */
  double z = 0.5 * cf->rho;
  for (int i = 0; i < n; ++i) {
    double Qb = 0.0;
    for (int k = 0; k < n; ++k) Qb += cf->Q[i * n + k] * s.b[k];
    z += -s.b[i] * cf->q[i] + 0.5 * s.b[i] * Qb;
  }
  *d.zeta = z;
}

/* Element a_j = V(., t_j; ., t_{j+1}) by K classical RK4 steps of the forward
 * conditional ODEs in tau, from A = I and the rest 0 at tau = t_j (eq.
 * abcej_boundary) up to tau = t_{j+1}; step i uses the samples at half-steps
 * p = 2i, 2i+1, 2i+2. */
static int build_block_forward(const orc_problem *P, long j, double *e) {
  int n = P->n, K = P->K;
  size_t es = elem_size(n);
  double h = (P->t[j + 1] - P->t[j]) / K;
  double *buf = (double *)malloc(sizeof(double) * (5 * es + 4 * (size_t)n * n + coefs_size(n, P->m, P->nr)));
  double *y = buf, *yt = y + es, *k = yt + es, *acc = k + es, *tmp = acc + es;
  double *cur = tmp + 4 * (size_t)n * n + es;
  coefs cf;
  coefs_alloc(&cf, n, P->m, P->nr, &cur);
  memset(y, 0, sizeof(double) * es);
  eye(n, view(n, y).A);
  int bad = 0;
  for (int i = 0; i < K; ++i) {
    bad |= coefs_eval(P, j, 2 * i, &cf);
    forward_rhs(n, &cf, y, k, tmp);
    for (size_t q = 0; q < es; ++q) { acc[q] = k[q]; yt[q] = y[q] + 0.5 * h * k[q]; }
    bad |= coefs_eval(P, j, 2 * i + 1, &cf);
    forward_rhs(n, &cf, yt, k, tmp);
    for (size_t q = 0; q < es; ++q) { acc[q] += 2.0 * k[q]; yt[q] = y[q] + 0.5 * h * k[q]; }
    forward_rhs(n, &cf, yt, k, tmp);
    for (size_t q = 0; q < es; ++q) { acc[q] += 2.0 * k[q]; yt[q] = y[q] + h * k[q]; }
    bad |= coefs_eval(P, j, 2 * i + 2, &cf);
    forward_rhs(n, &cf, yt, k, tmp);
    for (size_t q = 0; q < es; ++q) { acc[q] += k[q]; y[q] = y[q] + (h / 6.0) * acc[q]; }
  }
  memcpy(e, y, sizeof(double) * es);
  free(buf);
  return bad;
}

/* Forward-ODE elements j in [j0, j1), 0 <= j0 <= j1 <= T (no terminal element). */
int orc_build_elements_forward(const orc_problem *P, long j0, long j1, double *elems) {
  size_t es = elem_size(P->n);
  int bad = 0;
  for (long j = j0; j < j1; ++j) bad |= build_block_forward(P, j, elems + (size_t)(j - j0) * es);
  return bad;
}

/* Prefixes of T elements by the sequential left-to-right fold (Theorem
 * "parallel_HJB", eq. parallel_cond_B_HJB): p_0 = identity element,
 * p_{k+1} = p_k (x) a_k = V(., t_0; ., t_{k+1}).  Writes the T+1 prefixes. */
int orc_prefix(int n, long T, const double *elems, double *prefixes) {
  size_t es = elem_size(n);
  memset(prefixes, 0, sizeof(double) * es);
  eye(n, view(n, prefixes).A);
  int bad = 0;
  for (long k = 0; k < T; ++k)
    bad |= orc_combine(n, prefixes + (size_t)k * es, elems + (size_t)k * es, prefixes + (size_t)(k + 1) * es);
  return bad;
}

/* Method 2 (Sec. IV-E, eq. Opt_trajectory_method2 in the LQT form):
 *   x_k = (I + C(t_0,t_k) S_k)^{-1} (A(t_0,t_k) x0 + b(t_0,t_k) + C(t_0,t_k) v_k)
 * with (A, b, C)(t_0, t_k) from the prefixes of the forward-ODE elements, then
 * the controls of eq. LQT_optimal_control.  x[(T+1) n], u[(T+1) m]. */
int orc_trajectory_method2(const orc_problem *P, const double *S, const double *v, const double *x0, double *x,
                           double *u) {
  int n = P->n;
  long T = P->T;
  size_t es = elem_size(n), nn = (size_t)n * n;
  double *el = (double *)malloc(sizeof(double) * es * (size_t)(2 * T + 1));
  double *pre = el + es * (size_t)T;
  int bad = orc_build_elements_forward(P, 0, T, el);
  bad |= orc_prefix(n, T, el, pre);
  double *W = (double *)malloc(sizeof(double) * (nn + 4 * (size_t)n + coefs_size(n, P->m, P->nr)));
  double *rhs = W + nn, *tv = rhs + n, *cur = tv + 3 * (size_t)n;
  coefs cf;
  coefs_alloc(&cf, n, P->m, P->nr, &cur);
  for (long k = 0; k <= T; ++k) {
    elem_view pk = view(n, pre + (size_t)k * es);
    const double *Sk = S + (size_t)k * nn, *vk = v + (size_t)k * n;
    mm(n, n, n, pk.C, Sk, W);
    for (int i = 0; i < n; ++i) W[i * n + i] += 1.0;
    mm(n, n, 1, pk.A, x0, rhs);
    mm(n, n, 1, pk.C, vk, tv);
    for (int i = 0; i < n; ++i) rhs[i] += pk.b[i] + tv[i];
    bad |= solve(n, 1, W, rhs);
    memcpy(x + (size_t)k * n, rhs, sizeof(double) * n);
    bad |= control_at(P, k, Sk, vk, x + (size_t)k * n, u + (size_t)k * P->m, tv, &cf);
  }
  free(W);
  free(el);
  return bad;
}

/* ------------------------------------------------------------------------ */
/* Densification: values, states and controls at every RK4 sub-step          */
/* ------------------------------------------------------------------------ */

/* Within-block densification (Sec. IV-E: the optimal trajectory inside a
 * sub-interval; Sec. VI-A: the fine grid of K steps per sub-interval).
 * Input: the solution at the block boundaries (S, v, zeta at t_0..t_T, x at
 * t_0..t_T).  For every block j independently:
 *   backward: K RK4 steps of the Riccati ODEs (eq. LQT_differential_S_v plus
 *     the zeta equation) from (S, v, zeta)_{j+1} at t_{j+1} down to t_j, with
 *     the same half-step samples as the element build, giving y_i at
 *     t_j + i h, i = K..0;
 *   forward: K RK4 steps of the closed-loop ODE (eq.
 *     optimal_trajectory_ODE_LQT) from x_j at t_j, with S, v at step midpoints
 *     from the cubic Hermite interpolant of the y_i (slopes = the Riccati
 *     right-hand side at each y_i with the block's sample there), as in O2.
 * Output at fine index g = j K + i (i = 0..K-1) and g = T K: at block
 * boundaries (i = 0, and g = T K) the given boundary solution; inside a block
 * y_i and the forward RK4 state.  Controls by eq. LQT_optimal_control with the
 * sample at each point (block j's sample 2i; block T-1's last sample at t_T).
 * Sd [TK+1][n][n], vd [TK+1][n], zd [TK+1], xd [TK+1][n], ud [TK+1][m]. */
int orc_densify(const orc_problem *P, const double *S, const double *v, const double *zeta, const double *x,
                double *Sd, double *vd, double *zd, double *xd, double *ud) {
  int n = P->n, m = P->m, K = P->K;
  long T = P->T;
  size_t ys = (size_t)n * n + n + 1, nn = (size_t)n * n;
  double *buf = (double *)malloc(sizeof(double) * (2 * (size_t)(K + 1) * ys + 6 * ys + 3 * nn + 8 * (size_t)n +
                                                   (size_t)m + coefs_size(n, m, P->nr)));
  double *Y = buf;                        /* y_i, i = 0..K */
  double *D = Y + (size_t)(K + 1) * ys;   /* slopes d_i, i = 0..K */
  double *yt = D + (size_t)(K + 1) * ys, *k = yt + ys, *acc = k + ys, *ym = acc + ys;
  double *tmp = ym + ys + 2 * ys;
  double *xv = tmp + 3 * nn, *xt = xv + n, *kx = xt + n, *ax = kx + n, *t2 = ax + n;
  double *cur = t2 + 4 * (size_t)n + m;
  coefs cf;
  coefs_alloc(&cf, n, m, P->nr, &cur);
  int bad = 0;
  for (long j = 0; j < T; ++j) {
    double h = (P->t[j + 1] - P->t[j]) / K;
    double *yK = Y + (size_t)K * ys;
    memcpy(yK, S + (size_t)(j + 1) * nn, sizeof(double) * nn);
    memcpy(yK + nn, v + (size_t)(j + 1) * n, sizeof(double) * n);
    yK[nn + n] = zeta[j + 1];
    for (int i = K - 1; i >= 0; --i) {
      const double *y = Y + (size_t)(i + 1) * ys;
      double *yn = Y + (size_t)i * ys;
      bad |= coefs_eval(P, j, 2 * i + 2, &cf);
      riccati_rhs(n, &cf, y, k, tmp);
      memcpy(D + (size_t)(i + 1) * ys, k, sizeof(double) * ys);
      for (size_t q = 0; q < ys; ++q) { acc[q] = k[q]; yt[q] = y[q] - 0.5 * h * k[q]; }
      bad |= coefs_eval(P, j, 2 * i + 1, &cf);
      riccati_rhs(n, &cf, yt, k, tmp);
      for (size_t q = 0; q < ys; ++q) { acc[q] += 2.0 * k[q]; yt[q] = y[q] - 0.5 * h * k[q]; }
      riccati_rhs(n, &cf, yt, k, tmp);
      for (size_t q = 0; q < ys; ++q) { acc[q] += 2.0 * k[q]; yt[q] = y[q] - h * k[q]; }
      bad |= coefs_eval(P, j, 2 * i, &cf);
      riccati_rhs(n, &cf, yt, k, tmp);
      for (size_t q = 0; q < ys; ++q) { acc[q] += k[q]; yn[q] = y[q] - (h / 6.0) * acc[q]; }
    }
    bad |= coefs_eval(P, j, 0, &cf);
    riccati_rhs(n, &cf, Y, D, tmp);
    /* forward */
    memcpy(xv, x + (size_t)j * n, sizeof(double) * n);
    for (int i = 0; i < K; ++i) {
      size_t g = (size_t)j * K + i;
      if (i == 0) {
        memcpy(Sd + g * nn, S + (size_t)j * nn, sizeof(double) * nn);
        memcpy(vd + g * n, v + (size_t)j * n, sizeof(double) * n);
        zd[g] = zeta[j];
        memcpy(xd + g * n, x + (size_t)j * n, sizeof(double) * n);
      } else {
        const double *y = Y + (size_t)i * ys;
        memcpy(Sd + g * nn, y, sizeof(double) * nn);
        memcpy(vd + g * n, y + nn, sizeof(double) * n);
        zd[g] = y[nn + n];
        memcpy(xd + g * n, xv, sizeof(double) * n);
      }
      bad |= coefs_eval(P, j, 2 * i, &cf);
      mm(n, n, 1, Sd + g * nn, xd + g * n, t2);
      for (int q = 0; q < n; ++q) t2[q] = vd[g * n + q] - t2[q];
      mm(m, n, 1, cf.G, t2, ud + g * m);
      if (i == K - 1) break; /* the state at t_{j+1} is the boundary solution */
      const double *y0 = Y + (size_t)i * ys, *y1 = Y + (size_t)(i + 1) * ys;
      const double *d0 = D + (size_t)i * ys, *d1 = D + (size_t)(i + 1) * ys;
      for (size_t q = 0; q < ys; ++q) ym[q] = 0.5 * (y0[q] + y1[q]) + h * (d0[q] - d1[q]) / 8.0;
      closed_loop_rhs(n, m, &cf, y0, y0 + nn, xv, kx, t2);
      for (int q = 0; q < n; ++q) { ax[q] = kx[q]; xt[q] = xv[q] + 0.5 * h * kx[q]; }
      bad |= coefs_eval(P, j, 2 * i + 1, &cf);
      closed_loop_rhs(n, m, &cf, ym, ym + nn, xt, kx, t2);
      for (int q = 0; q < n; ++q) { ax[q] += 2.0 * kx[q]; xt[q] = xv[q] + 0.5 * h * kx[q]; }
      closed_loop_rhs(n, m, &cf, ym, ym + nn, xt, kx, t2);
      for (int q = 0; q < n; ++q) { ax[q] += 2.0 * kx[q]; xt[q] = xv[q] + h * kx[q]; }
      bad |= coefs_eval(P, j, 2 * i + 2, &cf);
      closed_loop_rhs(n, m, &cf, y1, y1 + nn, xt, kx, t2);
      for (int q = 0; q < n; ++q) { ax[q] += kx[q]; xv[q] = xv[q] + (h / 6.0) * ax[q]; }
    }
  }
  size_t g = (size_t)T * K;
  memcpy(Sd + g * nn, S + (size_t)T * nn, sizeof(double) * nn);
  memcpy(vd + g * n, v + (size_t)T * n, sizeof(double) * n);
  zd[g] = zeta[T];
  memcpy(xd + g * n, x + (size_t)T * n, sizeof(double) * n);
  bad |= control_at(P, T, S + (size_t)T * nn, v + (size_t)T * n, x + (size_t)T * n, ud + g * m, t2, &cf);
  free(buf);
  return bad;
}

/* ------------------------------------------------------------------------ */
/* Nonlinear scalar problem on a state grid (Sec. VI-B, App. E)              */
/* ------------------------------------------------------------------------ */

/* Scalar control-affine problem dx/dt = d0 + d1 x + d2 x^2 + u, running cost
 * q x^2 / 2 + rho u^2 / 2, terminal cost qf x^2 / 2 (Sec. VI-B: d0 = 1, d1 = 0,
 * d2 = -1/10, q = rho = 1, qf = 4), on the grid x_i = x_min + i dx,
 * i = 0..G-1; blocks of length tau split into `substeps` steps of
 * dt = tau / substeps, T blocks. */
typedef struct {
  int G;
  double x_min, dx;
  double d0, d1, d2, q, rho, qf;
  double tau;
  int substeps;
  long T;
  int interp; /* 1: every grid minimisation refined by App. E's quadratic interpolation */
} orc_grid_problem;

/* App. E: min over the grid of g_j + f_j, refined by the quadratic
 * interpolants of g and f through the discrete minimiser i and its two
 * neighbours (lowest index on ties; no refinement at the grid ends or when the
 * summed curvature a_g + a_f is not positive). */
static double grid_min(int G, double dx, const double *g, long gs, const double *f, long fs, int interp) {
  int bi = 0;
  double best = g[0] + f[0];
  for (int j = 1; j < G; ++j) {
    double v = g[j * gs] + f[j * fs];
    if (v < best) { best = v; bi = j; }
  }
  if (!interp || bi == 0 || bi == G - 1) return best;
  double gm = g[(bi - 1) * gs], g0 = g[bi * gs], gp = g[(bi + 1) * gs];
  double fm = f[(bi - 1) * fs], f0 = f[bi * fs], fp = f[(bi + 1) * fs];
  double ag = (gp + gm - 2.0 * g0) / (2.0 * dx * dx), bg = (gp - gm) / (2.0 * dx);
  double af = (fp + fm - 2.0 * f0) / (2.0 * dx * dx), bf = (fp - fm) / (2.0 * dx);
  double a = ag + af, b = bg + bf;
  if (!(a > 0.0)) return best;
  return best - b * b / (4.0 * a);
}

/* out(i, j) = min_k A(i, k) + B(k, j) (Theorem "HJB-comb" on the grid: the
 * combination of conditional value functions V(x_i; x_k) and V(x_k; x_j)),
 * G x G row-major. */
int orc_grid_combine(const orc_grid_problem *P, const double *A, const double *B, double *out) {
  int G = P->G;
  for (int i = 0; i < G; ++i)
    for (int j = 0; j < G; ++j) out[(size_t)i * G + j] = grid_min(G, P->dx, A + (size_t)i * G, 1, B + j, G, P->interp);
  return 0;
}

/* out(i) = min_k M(i, k) + w(k): a conditional value function combined with a
 * value function (the last step of the fold, Theorem "parallel_HJB"). */
int orc_grid_apply(const orc_grid_problem *P, const double *M, const double *w, double *out) {
  int G = P->G;
  for (int i = 0; i < G; ++i) out[i] = grid_min(G, P->dx, M + (size_t)i * G, 1, w, 1, P->interp);
  return 0;
}

/* One step's conditional value function: from x_i to x_j in dt with the
 * explicit Euler step x_j = x_i + dt (drift(x_i) + u), so
 * u = (x_j - x_i)/dt - drift(x_i), cost dt (q x_i^2 + rho u^2)/2. */
static void grid_one_step(const orc_grid_problem *P, double *C) {
  int G = P->G;
  double dt = P->tau / P->substeps;
  for (int i = 0; i < G; ++i) {
    double xi = P->x_min + i * P->dx;
    double drift = P->d0 + P->d1 * xi + P->d2 * xi * xi;
    for (int j = 0; j < G; ++j) {
      double xj = P->x_min + j * P->dx;
      double u = (xj - xi) / dt - drift;
      C[(size_t)i * G + j] = dt * 0.5 * (P->q * xi * xi + P->rho * u * u);
    }
  }
}

/* The block's conditional value function V(x_i, t; x_j, t + tau): the one-step
 * function combined with itself substeps times, left to right
 * (M_1 = C, M_{m+1} = M_m (x) C).  Out: G x G. */
int orc_grid_block(const orc_grid_problem *P, double *out) {
  size_t GG = (size_t)P->G * P->G;
  double *C = (double *)malloc(sizeof(double) * 2 * GG), *tmp = C + GG;
  grid_one_step(P, C);
  memcpy(out, C, sizeof(double) * GG);
  for (int m = 1; m < P->substeps; ++m) {
    orc_grid_combine(P, out, C, tmp);
    memcpy(out, tmp, sizeof(double) * GG);
  }
  free(C);
  return 0;
}

/* Terminal value phi(x_i) = qf x_i^2 / 2. */
static void grid_terminal(const orc_grid_problem *P, double *phi) {
  for (int i = 0; i < P->G; ++i) {
    double x = P->x_min + i * P->dx;
    phi[i] = 0.5 * P->qf * x * x;
  }
}

/* Values V(., t_k), k = 0..T, by the sequential right-to-left fold
 * V_T = phi, V_k = Vblock (x) V_{k+1} (Theorem "parallel_HJB" with one
 * conditional value function for every block: the model is time-invariant,
 * Sec. VI-B).  Out: [T+1][G]. */
int orc_grid_values_sequential(const orc_grid_problem *P, const double *Vblock, double *V) {
  int G = P->G;
  long T = P->T;
  grid_terminal(P, V + (size_t)T * G);
  for (long k = T - 1; k >= 0; --k) orc_grid_apply(P, Vblock, V + (size_t)(k + 1) * G, V + (size_t)k * G);
  return 0;
}

/* The same values in the order of the doubling scan: the powers
 * P_0 = Vblock, P_{l+1} = P_l (x) P_l, and for every k, with T - k =
 * sum of 2^{l_1} < 2^{l_2} < ..., V_k = P_{l_r} (x) (... (P_{l_1} (x) phi)).
 * Without the interpolation this is the sequential fold exactly (the grid
 * minimum is associative); with it, the two differ by the interpolation
 * error.  Out: [T+1][G]. */
int orc_grid_values(const orc_grid_problem *P, const double *Vblock, double *V) {
  int G = P->G;
  long T = P->T;
  size_t GG = (size_t)G * G;
  int L = 0;
  while ((1L << L) <= T) ++L;
  double *pw = (double *)malloc(sizeof(double) * ((size_t)L * GG + 2 * (size_t)G));
  double *w = pw + (size_t)L * GG, *w2 = w + G;
  memcpy(pw, Vblock, sizeof(double) * GG);
  for (int l = 1; l < L; ++l) orc_grid_combine(P, pw + (size_t)(l - 1) * GG, pw + (size_t)(l - 1) * GG, pw + (size_t)l * GG);
  grid_terminal(P, V + (size_t)T * G);
  for (long k = 0; k < T; ++k) {
    long e = T - k;
    memcpy(w, V + (size_t)T * G, sizeof(double) * G);
    for (int l = 0; l < L; ++l)
      if (e & (1L << l)) {
        orc_grid_apply(P, pw + (size_t)l * GG, w, w2);
        memcpy(w, w2, sizeof(double) * G);
      }
    memcpy(V + (size_t)k * G, w, sizeof(double) * G);
  }
  free(pw);
  return 0;
}

/* Size in doubles of one packed element, for callers. */
long orc_element_size(int n) { return (long)elem_size(n); }
