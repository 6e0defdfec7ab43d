/*
 * swe_oracle.c -- plain, slow FP64 CPU oracle for the quadrature-free
 * discontinuous Galerkin scheme for the 2D shallow water equations of
 * Faghih-Naini et al., "p-adaptive discontinuous Galerkin method for the
 * shallow water equations on heterogeneous computing architectures" (2023).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py may load this file's library.  It
 * shares no code, header, table or constant generator with the CUDA library.
 *
 * What is followed, passage by passage:
 *   Sect. 2, Eqs. (1)-(5)  : conservative SWE, flux A(c,u), source r(c,u),
 *                            H = h_b + xi; bottom friction (linear and
 *                            quadratic law) and Coriolis as parameters, zero
 *                            by default; the body force F is zero.
 *   Sect. 2, Eqs. (8)-(9)  : semi-discrete weak form, orthonormal basis so the
 *                            mass matrix is the identity.
 *   Sect. 2, LF flux       : A_hat = 1/2((A(c)+A(c+)).n + lambda (c - c+)).
 *   Sect. 2, Eq. (10)      : lambda from edge-midpoint values.
 *   Sect. 2, Eqs. (11)-(12): modal expansion, K(p) = 1,3,6,10 (15 for p=4).
 *   Sect. 2 (end)          : SSP Runge-Kutta time stepping.
 *   Sect. 3, Eq. (13)      : element integrals as sums over coefficient
 *                            products times integrals of basis products
 *                            ("quadrature-free"); base/correction split.
 *   Sect. 3 (end)          : truncated auxiliary system uH = q with K(p,i,j).
 *
 * Readings where the paper is silent or garbled:
 *   - basis: orthonormal Dubiner polynomials on the reference triangle,
 *     ordered by total degree, then by the Jacobi index;
 *   - K(p,i,j) = K(max(deg i, deg j));
 *   - lambda uses element means only (Sect. 3): u_bar = u_1/sqrt|Omega|,
 *     H_bar(x_E) = xi_1/sqrt|Omega| + h_b(x_E);
 *   - land boundary: mirror ghost state; open sea: xi+ = xi_hat(t), q+ = q;
 *   - h_b is the continuous P1 interpolant of vertex depths;
 *   - SSP-RK2 is Heun's method, SSP-RK3 the Shu-Osher scheme;
 *   - dt = cfl * min_e d_e / ((|u_bar| + sqrt(g H_bar)) (2p+1)), d_e the
 *     inscribed diameter.
 *
 * Every reference-element integral is computed exactly from monomial
 * integrals (int_T x^a y^b = a! b! / (a+b+2)!; int_0^1 s^m = 1/(m+1)).
 *
 * Threads: built with -fopenmp, the loops over elements (and the elementwise
 * RK update) run in parallel.  Every element's arithmetic is the same
 * sequence of operations either way and the only reductions are a minimum
 * and integer counts, so a threaded build gives bitwise the results of the
 * serial one (the mass and energy sums stay serial).
 */
#define _USE_MATH_DEFINES
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define KMAX 15   /* K(4) */
#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif
#define PD 16     /* polynomial coefficient grid: degrees 0..15 */
#ifdef _OPENMP
#include <omp.h>
void or_set_threads(int n) { if (n > 0) omp_set_num_threads(n); }
int or_max_threads(void) { return omp_get_max_threads(); }
#else
void or_set_threads(int n) { (void)n; }
int or_max_threads(void) { return 1; }
#endif

/* ------------------------------------------------------------------ */
/* Double-double numbers (error-free transformations; Dekker, Knuth):   */
/* the monomial expansions of degree-12 products cancel by ~1e9, so    */
/* every exact integral is accumulated in ~106-bit precision and only  */
/* rounded to FP64 at the end.                                         */
/* ------------------------------------------------------------------ */
typedef struct { double hi, lo; } dd;

static dd dd_d(double a) { dd r = {a, 0.0}; return r; }
static dd quick_two_sum(double a, double b) { dd r; r.hi = a + b; r.lo = b - (r.hi - a); return r; }
static dd two_sum(double a, double b) {
  dd r; r.hi = a + b;
  double bb = r.hi - a;
  r.lo = (a - (r.hi - bb)) + (b - bb);
  return r;
}
static dd dd_add(dd a, dd b) {
  dd s = two_sum(a.hi, b.hi), t = two_sum(a.lo, b.lo);
  s.lo += t.hi; s = quick_two_sum(s.hi, s.lo);
  s.lo += t.lo; return quick_two_sum(s.hi, s.lo);
}
static dd dd_neg(dd a) { dd r = {-a.hi, -a.lo}; return r; }
static dd dd_mul(dd a, dd b) {
  double p = a.hi * b.hi;
  double e = fma(a.hi, b.hi, -p);
  e += a.hi * b.lo + a.lo * b.hi;
  return quick_two_sum(p, e);
}
static dd dd_div(dd a, dd b) {
  double q1 = a.hi / b.hi;
  dd r = dd_add(a, dd_neg(dd_mul(dd_d(q1), b)));
  double q2 = r.hi / b.hi;
  r = dd_add(r, dd_neg(dd_mul(dd_d(q2), b)));
  double q3 = r.hi / b.hi;
  dd q = quick_two_sum(q1, q2);
  return dd_add(q, dd_d(q3));
}
static dd dd_sqrt_d(double x) {
  double s = sqrt(x);
  double res = fma(-s, s, x);  /* exact residual x - s^2 */
  return quick_two_sum(s, res / (2.0 * s));
}
static dd dd_ratio(double a, double b) { return dd_div(dd_d(a), dd_d(b)); }
static int dd_is_zero(dd a) { return a.hi == 0.0 && a.lo == 0.0; }

/* ------------------------------------------------------------------ */
/* Polynomials in (x, y) on the reference triangle: c[a][b] x^a y^b.  */
/* ------------------------------------------------------------------ */
typedef struct { dd c[PD][PD]; } poly2;
typedef struct { dd c[4 * PD]; } poly1; /* in s */

static void p2_zero(poly2* p) { memset(p, 0, sizeof *p); }

static void p2_mul(const poly2* a, const poly2* b, poly2* out) {
  static poly2 r;
  p2_zero(&r);
  for (int i = 0; i < PD; ++i) for (int j = 0; i + j < PD; ++j) {
    if (dd_is_zero(a->c[i][j])) continue;
    for (int k = 0; i + k < PD; ++k) for (int l = 0; i + k + j + l < PD; ++l)
      if (!dd_is_zero(b->c[k][l])) r.c[i + k][j + l] = dd_add(r.c[i + k][j + l], dd_mul(a->c[i][j], b->c[k][l]));
  }
  *out = r;
}

static void p2_axpy(dd alpha, const poly2* x, poly2* y) {
  for (int i = 0; i < PD; ++i) for (int j = 0; j < PD; ++j)
    if (!dd_is_zero(x->c[i][j])) y->c[i][j] = dd_add(y->c[i][j], dd_mul(alpha, x->c[i][j]));
}

static void p2_dx(const poly2* a, poly2* out) {
  static poly2 r;
  p2_zero(&r);
  for (int i = 1; i < PD; ++i) for (int j = 0; j < PD; ++j) r.c[i - 1][j] = dd_mul(dd_d((double)i), a->c[i][j]);
  *out = r;
}

static void p2_dy(const poly2* a, poly2* out) {
  static poly2 r;
  p2_zero(&r);
  for (int i = 0; i < PD; ++i) for (int j = 1; j < PD; ++j) r.c[i][j - 1] = dd_mul(dd_d((double)j), a->c[i][j]);
  *out = r;
}

static double fact(int n) { double f = 1.0; for (int i = 2; i <= n; ++i) f *= i; return f; } /* exact to 18! */

/* int over {x>=0, y>=0, x+y<=1} of x^a y^b = a! b! / (a+b+2)! */
static dd p2_int_tri(const poly2* a) {
  dd s = dd_d(0.0);
  for (int i = 0; i < PD; ++i) for (int j = 0; i + j < PD; ++j)
    if (!dd_is_zero(a->c[i][j])) s = dd_add(s, dd_mul(a->c[i][j], dd_ratio(fact(i) * fact(j), fact(i + j + 2))));
  return s;
}

/* restriction to the straight line (x0 + dx s, y0 + dy s); the line
 * coefficients are small integers, so the powers are exact */
static void p2_on_line(const poly2* a, double x0, double dxs, double y0, double dys, poly1* out) {
  static double px[PD][PD], py[PD][PD];
  memset(px, 0, sizeof px); memset(py, 0, sizeof py);
  px[0][0] = 1.0; py[0][0] = 1.0;
  for (int k = 1; k < PD; ++k)
    for (int m = 0; m < PD; ++m) {
      px[k][m] = x0 * px[k - 1][m] + (m > 0 ? dxs * px[k - 1][m - 1] : 0.0);
      py[k][m] = y0 * py[k - 1][m] + (m > 0 ? dys * py[k - 1][m - 1] : 0.0);
    }
  memset(out, 0, sizeof *out);
  for (int i = 0; i < PD; ++i) for (int j = 0; i + j < PD; ++j) {
    if (dd_is_zero(a->c[i][j])) continue;
    for (int m = 0; m < PD; ++m) for (int n = 0; n < PD; ++n)
      if (px[i][m] != 0.0 && py[j][n] != 0.0)
        out->c[m + n] = dd_add(out->c[m + n], dd_mul(a->c[i][j], dd_d(px[i][m] * py[j][n])));
  }
}

static void p1_mul(const poly1* a, const poly1* b, poly1* out) {
  static poly1 r;
  memset(&r, 0, sizeof r);
  for (int i = 0; i < 4 * PD; ++i) {
    if (dd_is_zero(a->c[i])) continue;
    for (int j = 0; i + j < 4 * PD; ++j)
      if (!dd_is_zero(b->c[j])) r.c[i + j] = dd_add(r.c[i + j], dd_mul(a->c[i], b->c[j]));
  }
  *out = r;
}

static dd p1_int01(const poly1* a) {
  dd s = dd_d(0.0);
  for (int i = 0; i < 4 * PD; ++i)
    if (!dd_is_zero(a->c[i])) s = dd_add(s, dd_div(a->c[i], dd_d((double)(i + 1))));
  return s;
}

/* ------------------------------------------------------------------ */
/* Orthonormal Dubiner basis (Sect. 2: hierarchical, orthonormal).     */
/* With r = 2x-1, s = 2y-1, eta1 = 2(1+r)/(1-s)-1, eta2 = s:           */
/*   phi_{a,b} = N_{ab} P_a(eta1) ((1-eta2)/2)^a P_b^{(2a+1,0)}(eta2), */
/*   N_{ab}^2 = 2 (2a+1)(a+b+1)  (normalised on the reference triangle) */
/* Q_a := P_a(eta1)((1-eta2)/2)^a is a polynomial in (x,y):            */
/*   Q_0 = 1, Q_1 = 2x+y-1,                                            */
/*   (a+1) Q_{a+1} = (2a+1)(2x+y-1) Q_a - a (1-y)^2 Q_{a-1}.            */
/* Modes are ordered by total degree a+b, then by b.                   */
/* ------------------------------------------------------------------ */
static poly2 g_phi[KMAX], g_dphi[2][KMAX];
static int g_deg[KMAX];
static int g_ready = 0;

static const int KP[5] = {1, 3, 6, 10, 15};

static void build_basis(void) {
  static poly2 Q[5], J[5], lin, omy2, sv, q1, q2, ph;
  p2_zero(&Q[0]); Q[0].c[0][0] = dd_d(1.0);
  p2_zero(&lin); lin.c[1][0] = dd_d(2.0); lin.c[0][1] = dd_d(1.0); lin.c[0][0] = dd_d(-1.0);
  p2_zero(&omy2); omy2.c[0][0] = dd_d(1.0); omy2.c[0][1] = dd_d(-2.0); omy2.c[0][2] = dd_d(1.0); /* (1-y)^2 */
  p2_zero(&sv); sv.c[0][0] = dd_d(-1.0); sv.c[0][1] = dd_d(2.0);                                  /* s = 2y-1 */
  Q[1] = lin;
  for (int a = 1; a < 4; ++a) {
    p2_mul(&lin, &Q[a], &q1);
    p2_mul(&omy2, &Q[a - 1], &q2);
    p2_zero(&Q[a + 1]);
    p2_axpy(dd_ratio(2.0 * a + 1.0, a + 1.0), &q1, &Q[a + 1]);
    p2_axpy(dd_ratio(-(double)a, a + 1.0), &q2, &Q[a + 1]);
  }
  int idx = 0;
  for (int d = 0; d <= 4; ++d) {
    for (int b = 0; b <= d; ++b) {
      int a = d - b;
      /* Jacobi P_b^{(al,0)}(s), s = 2y-1, as a polynomial in y */
      double al = 2.0 * a + 1.0;
      p2_zero(&J[0]); J[0].c[0][0] = dd_d(1.0);
      /* P_1^{(al,0)}(s) = ((al+2) s + al)/2 = (al+2) y - 1 */
      p2_zero(&J[1]); J[1].c[0][0] = dd_d(-1.0); J[1].c[0][1] = dd_d(al + 2.0);
      for (int n = 1; n < b; ++n) {
        /* three-term recurrence of P_n^{(al,be)} with be = 0:
         * a1 P_{n+1} = (a2 + a3 s) P_n - a4 P_{n-1} */
        double a1 = 2.0 * (n + 1) * (n + al + 1) * (2 * n + al);
        double a2 = (2 * n + al + 1) * (al * al);
        double a3 = (2 * n + al) * (2 * n + al + 1) * (2 * n + al + 2);
        double a4 = 2.0 * (n + al) * n * (2 * n + al + 2);
        p2_mul(&sv, &J[n], &q1);
        p2_zero(&J[n + 1]);
        p2_axpy(dd_ratio(a2, a1), &J[n], &J[n + 1]);
        p2_axpy(dd_ratio(a3, a1), &q1, &J[n + 1]);
        p2_axpy(dd_ratio(-a4, a1), &J[n - 1], &J[n + 1]);
      }
      p2_mul(&Q[a], &J[b], &ph);
      p2_zero(&g_phi[idx]);
      p2_axpy(dd_sqrt_d(2.0 * (2.0 * a + 1.0) * (a + b + 1.0)), &ph, &g_phi[idx]);
      g_deg[idx] = d;
      ++idx;
    }
  }
  for (int i = 0; i < KMAX; ++i) { p2_dx(&g_phi[i], &g_dphi[0][i]); p2_dy(&g_phi[i], &g_dphi[1][i]); }
}

/* ------------------------------------------------------------------ */
/* Reference tensors (Eq. 13 and its triple-product analogues).        */
/* ------------------------------------------------------------------ */
static double D_[2][KMAX][KMAX];           /* D_k[q][i] = int phi_i d_k phi_q        */
static double G_[2][KMAX][KMAX][KMAX];     /* G_k[q][i][j] = int phi_i phi_j d_k phi_q */
static double T_[KMAX][KMAX][KMAX];        /* T[n][i][j] = int phi_n phi_i phi_j      */
static double S2_[3][KMAX][KMAX];          /* int_0^1 phi_q phi_i (gamma_k(s)) ds     */
static double S3_[3][KMAX][KMAX][KMAX];    /* int_0^1 phi_q phi_i phi_j (gamma_k(s))  */
static double X2_[3][3][KMAX][KMAX];       /* int phi_q(gamma_k(s)) phi_i(gamma_k'(1-s)) */
static double X3_[3][3][KMAX][KMAX][KMAX]; /* ... phi_i phi_j (gamma_k'(1-s))         */
static double L_[3][KMAX];                 /* int lambda_v phi_i (P1 hat functions)   */
static double M_[KMAX][KMAX];              /* int phi_i phi_j (identity; for pins)    */

/* Local edge k is opposite vertex k: gamma_0(s)=(1-s,s), gamma_1(s)=(0,1-s),
 * gamma_2(s)=(s,0); all run counter-clockwise. */
static const double GX0[3] = {1.0, 0.0, 0.0}, GDX[3] = {-1.0, 0.0, 1.0};
static const double GY0[3] = {0.0, 1.0, 0.0}, GDY[3] = {1.0, -1.0, 0.0};

static void build_tensors(void) {
  static poly2 pp, t, t2;
  static poly1 fw[3][KMAX], bw[3][KMAX], t1, t3, tx, tx3;
  for (int i = 0; i < KMAX; ++i) for (int j = 0; j < KMAX; ++j) {
    p2_mul(&g_phi[i], &g_phi[j], &pp);
    M_[i][j] = p2_int_tri(&pp).hi;
    for (int k = 0; k < 2; ++k) {
      p2_mul(&g_phi[i], &g_dphi[k][j], &t);
      D_[k][j][i] = p2_int_tri(&t).hi;
    }
    for (int n = 0; n < KMAX; ++n) {
      p2_mul(&pp, &g_phi[n], &t);
      T_[n][i][j] = p2_int_tri(&t).hi;
      for (int k = 0; k < 2; ++k) {
        p2_mul(&pp, &g_dphi[k][n], &t2);
        G_[k][n][i][j] = p2_int_tri(&t2).hi;
      }
    }
  }
  for (int k = 0; k < 3; ++k) for (int i = 0; i < KMAX; ++i) {
    p2_on_line(&g_phi[i], GX0[k], GDX[k], GY0[k], GDY[k], &fw[k][i]);
    /* reversed traversal: gamma_k(1-s) = gamma_k(1) - s * dgamma */
    p2_on_line(&g_phi[i], GX0[k] + GDX[k], -GDX[k], GY0[k] + GDY[k], -GDY[k], &bw[k][i]);
  }
  for (int k = 0; k < 3; ++k) for (int q = 0; q < KMAX; ++q) for (int i = 0; i < KMAX; ++i) {
    p1_mul(&fw[k][q], &fw[k][i], &t1);
    S2_[k][q][i] = p1_int01(&t1).hi;
    for (int j = 0; j < KMAX; ++j) { p1_mul(&t1, &fw[k][j], &t3); S3_[k][q][i][j] = p1_int01(&t3).hi; }
    for (int kk = 0; kk < 3; ++kk) {
      p1_mul(&fw[k][q], &bw[kk][i], &tx);
      X2_[k][kk][q][i] = p1_int01(&tx).hi;
      for (int j = 0; j < KMAX; ++j) {
        p1_mul(&tx, &bw[kk][j], &tx3);
        X3_[k][kk][q][i][j] = p1_int01(&tx3).hi;
      }
    }
  }
  /* barycentric hat functions lambda_0 = 1-x-y, lambda_1 = x, lambda_2 = y */
  static poly2 lam[3];
  for (int v = 0; v < 3; ++v) p2_zero(&lam[v]);
  lam[0].c[0][0] = dd_d(1.0); lam[0].c[1][0] = dd_d(-1.0); lam[0].c[0][1] = dd_d(-1.0);
  lam[1].c[1][0] = dd_d(1.0); lam[2].c[0][1] = dd_d(1.0);
  for (int v = 0; v < 3; ++v) for (int i = 0; i < KMAX; ++i) {
    p2_mul(&lam[v], &g_phi[i], &t); L_[v][i] = p2_int_tri(&t).hi;
  }
}

static void ensure_ready(void) {
  if (g_ready) return;
  build_basis();
  build_tensors();
  g_ready = 1;
}

/* K(p,i,j) of the truncated auxiliary system (Sect. 3), read as
 * K(max(deg phi_i, deg phi_j)). */
static int Ktr(int i, int j) { int d = g_deg[i] > g_deg[j] ? g_deg[i] : g_deg[j]; return KP[d]; }

/* ------------------------------------------------------------------ */
/* Exports for the pins.                                               */
/* ------------------------------------------------------------------ */
void or_basis_monomials(double* out /* [15][PD][PD] */) {
  ensure_ready();
  for (int i = 0; i < KMAX; ++i)
    for (int a = 0; a < PD; ++a)
      for (int b = 0; b < PD; ++b) out[((size_t)i * PD + a) * PD + b] = g_phi[i].c[a][b].hi;
}
int or_poly_grid(void) { return PD; }
void or_degrees(int* out) { ensure_ready(); for (int i = 0; i < KMAX; ++i) out[i] = g_deg[i]; }
void or_tensor_D(double* o) { ensure_ready(); memcpy(o, D_, sizeof D_); }
void or_tensor_G(double* o) { ensure_ready(); memcpy(o, G_, sizeof G_); }
void or_tensor_T(double* o) { ensure_ready(); memcpy(o, T_, sizeof T_); }
void or_tensor_S2(double* o) { ensure_ready(); memcpy(o, S2_, sizeof S2_); }
void or_tensor_S3(double* o) { ensure_ready(); memcpy(o, S3_, sizeof S3_); }
void or_tensor_X2(double* o) { ensure_ready(); memcpy(o, X2_, sizeof X2_); }
void or_tensor_X3(double* o) { ensure_ready(); memcpy(o, X3_, sizeof X3_); }
void or_tensor_M(double* o) { ensure_ready(); memcpy(o, M_, sizeof M_); }
void or_tensor_L(double* o) { ensure_ready(); memcpy(o, L_, sizeof L_); }
int or_Ktr(int i, int j) { ensure_ready(); return Ktr(i, j); }

/* ------------------------------------------------------------------ */
/* Mesh, geometry and bathymetry.                                      */
/* ------------------------------------------------------------------ */
typedef struct {
  int64_t nv, ne;
  double* vx; double* vy; double* hv;  /* vertices and vertex depths */
  int32_t* tri;                        /* [ne][3], counter-clockwise  */
  int8_t* p;                           /* orders 0..4                 */
  double* area; double* s;             /* |Omega_e|, sqrt|det J|      */
  double* Jinv;                        /* [ne][2][2]: Jinv[k][d] = d xhat_k / d x_d */
  double* hb;                          /* [ne][3] modal P1 bathymetry  */
  double* dhb;                         /* [ne][2] grad h_b            */
  double* diam;                        /* inscribed diameter 4|Omega|/perimeter */
  double* elen; double* enx; double* eny; double* ehb; /* [ne][3]: |E|, n, h_b(x_E) */
  int64_t* nb; int8_t* nbk; int8_t* bc; /* [ne][3]: neighbour, its local edge, 0/1/2 */
} or_mesh;

typedef struct {
  double g, cfl, h_min;
  int rk_order;
  double tide_amp, tide_period, tide_phase;
  /* source terms of Eq. (5): bottom friction tau_bf = fric_lin H + fric_quad |u|
   * (the linear and the quadratic law of the paper's setups) and Coriolis f_c */
  double fric_lin, fric_quad, f_c;
} or_params;

#define C_(c, f, i, e, ne) (c)[((int64_t)(f) * KMAX + (i)) * (ne) + (e)]

typedef struct { int64_t a, b, e; int k; } edge_key;

static int cmp_key(const void* x, const void* y) {
  const edge_key* p = (const edge_key*)x; const edge_key* q = (const edge_key*)y;
  if (p->a != q->a) return p->a < q->a ? -1 : 1;
  if (p->b != q->b) return p->b < q->b ? -1 : 1;
  if (p->e != q->e) return p->e < q->e ? -1 : 1;
  return p->k - q->k;
}

void or_mesh_free(or_mesh* m) {
  if (!m) return;
  free(m->vx); free(m->vy); free(m->hv); free(m->tri); free(m->p); free(m->area); free(m->s);
  free(m->Jinv); free(m->hb); free(m->dhb); free(m->diam); free(m->elen); free(m->enx); free(m->eny);
  free(m->ehb); free(m->nb); free(m->nbk); free(m->bc);
  free(m);
}

/* Build the mesh.  bc_tag[e][k] for the edge opposite vertex k of the
 * triangle as given: 0 = interior (or land if unmatched), 1 = land, 2 = open
 * sea; NULL means every unmatched edge is land.  Returns NULL on a degenerate
 * triangle or an edge shared by more than two triangles (*err = -2). */
or_mesh* or_mesh_new(int64_t nv, const double* xy, const double* hv, int64_t ne, const int32_t* tri,
                     const int8_t* bc_tag, const int8_t* p, int* err) {
  ensure_ready();
  *err = 0;
  or_mesh* m = (or_mesh*)calloc(1, sizeof(or_mesh));
  m->nv = nv; m->ne = ne;
  m->vx = malloc(sizeof(double) * nv); m->vy = malloc(sizeof(double) * nv); m->hv = malloc(sizeof(double) * nv);
  for (int64_t v = 0; v < nv; ++v) { m->vx[v] = xy[2 * v]; m->vy[v] = xy[2 * v + 1]; m->hv[v] = hv ? hv[v] : 0.0; }
  m->tri = malloc(sizeof(int32_t) * 3 * ne); m->p = malloc(ne);
  m->area = malloc(sizeof(double) * ne); m->s = malloc(sizeof(double) * ne);
  m->Jinv = malloc(sizeof(double) * 4 * ne); m->hb = malloc(sizeof(double) * 3 * ne);
  m->dhb = malloc(sizeof(double) * 2 * ne); m->diam = malloc(sizeof(double) * ne);
  m->elen = malloc(sizeof(double) * 3 * ne); m->enx = malloc(sizeof(double) * 3 * ne);
  m->eny = malloc(sizeof(double) * 3 * ne); m->ehb = malloc(sizeof(double) * 3 * ne);
  m->nb = malloc(sizeof(int64_t) * 3 * ne); m->nbk = malloc(3 * ne); m->bc = malloc(3 * ne);
  int8_t* tag = malloc(3 * ne);
  for (int64_t e = 0; e < ne; ++e) {
    int32_t v0 = tri[3 * e], v1 = tri[3 * e + 1], v2 = tri[3 * e + 2];
    int8_t t0 = bc_tag ? bc_tag[3 * e] : 0, t1 = bc_tag ? bc_tag[3 * e + 1] : 0, t2 = bc_tag ? bc_tag[3 * e + 2] : 0;
    double cr = (xy[2 * v1] - xy[2 * v0]) * (xy[2 * v2 + 1] - xy[2 * v0 + 1]) -
                (xy[2 * v2] - xy[2 * v0]) * (xy[2 * v1 + 1] - xy[2 * v0 + 1]);
    if (!(cr != 0.0) || v0 < 0 || v1 < 0 || v2 < 0 || v0 >= nv || v1 >= nv || v2 >= nv) { *err = -2; break; }
    if (cr < 0) { int32_t tv = v1; v1 = v2; v2 = tv; int8_t tt = t1; t1 = t2; t2 = tt; } /* edge k stays opposite vertex k */
    m->tri[3 * e] = v0; m->tri[3 * e + 1] = v1; m->tri[3 * e + 2] = v2;
    tag[3 * e] = t0; tag[3 * e + 1] = t1; tag[3 * e + 2] = t2;
    m->p[e] = p ? p[e] : 1;
    if (m->p[e] < 0 || m->p[e] > 4) { *err = -1; break; }
  }
  if (*err) { free(tag); or_mesh_free(m); return NULL; }
  /* geometry */
  for (int64_t e = 0; e < ne; ++e) {
    int32_t v[3] = {m->tri[3 * e], m->tri[3 * e + 1], m->tri[3 * e + 2]};
    double x0 = m->vx[v[0]], y0 = m->vy[v[0]];
    double J00 = m->vx[v[1]] - x0, J01 = m->vx[v[2]] - x0; /* dx/dxhat, dx/dyhat */
    double J10 = m->vy[v[1]] - y0, J11 = m->vy[v[2]] - y0; /* dy/dxhat, dy/dyhat */
    double det = J00 * J11 - J01 * J10;
    m->area[e] = 0.5 * det;
    m->s[e] = sqrt(det);
    double* Ji = m->Jinv + 4 * e;
    Ji[0] = J11 / det;  Ji[1] = -J01 / det;  /* d xhat / dx, d xhat / dy */
    Ji[2] = -J10 / det; Ji[3] = J00 / det;   /* d yhat / dx, d yhat / dy */
    /* h_b: continuous P1 interpolant; modal coefficients hb_i = int h_b phi_i
     * = s_e * sum_v h_v int_T lambda_v phihat_i. */
    for (int i = 0; i < 3; ++i) {
      double acc = 0.0;
      for (int w = 0; w < 3; ++w) acc += m->hv[v[w]] * L_[w][i];
      m->hb[3 * e + i] = m->s[e] * acc;
    }
    double dh1 = m->hv[v[1]] - m->hv[v[0]], dh2 = m->hv[v[2]] - m->hv[v[0]];
    m->dhb[2 * e] = dh1 * Ji[0] + dh2 * Ji[2];
    m->dhb[2 * e + 1] = dh1 * Ji[1] + dh2 * Ji[3];
    double per = 0.0;
    for (int k = 0; k < 3; ++k) {
      int32_t a = v[(k + 1) % 3], b = v[(k + 2) % 3];
      double dx = m->vx[b] - m->vx[a], dy = m->vy[b] - m->vy[a];
      double L = sqrt(dx * dx + dy * dy);
      m->elen[3 * e + k] = L;
      m->enx[3 * e + k] = dy / L;
      m->eny[3 * e + k] = -dx / L;
      m->ehb[3 * e + k] = 0.5 * (m->hv[a] + m->hv[b]);
      per += L;
    }
    m->diam[e] = 4.0 * m->area[e] / per;
  }
  /* neighbours: match each edge by its sorted vertex pair */
  edge_key* keys = malloc(sizeof(edge_key) * 3 * ne);
  for (int64_t e = 0; e < ne; ++e) for (int k = 0; k < 3; ++k) {
    int64_t a = m->tri[3 * e + (k + 1) % 3], b = m->tri[3 * e + (k + 2) % 3];
    keys[3 * e + k].a = a < b ? a : b; keys[3 * e + k].b = a < b ? b : a;
    keys[3 * e + k].e = e; keys[3 * e + k].k = k;
    m->nb[3 * e + k] = -1; m->nbk[3 * e + k] = -1;
  }
  qsort(keys, 3 * ne, sizeof(edge_key), cmp_key);
  for (int64_t r = 0; r < 3 * ne;) {
    int64_t s = r;
    while (s < 3 * ne && keys[s].a == keys[r].a && keys[s].b == keys[r].b) ++s;
    if (s - r > 2) { *err = -2; break; }
    if (s - r == 2) {
      edge_key A = keys[r], B = keys[r + 1];
      m->nb[3 * A.e + A.k] = B.e; m->nbk[3 * A.e + A.k] = (int8_t)B.k;
      m->nb[3 * B.e + B.k] = A.e; m->nbk[3 * B.e + B.k] = (int8_t)A.k;
    }
    r = s;
  }
  free(keys);
  for (int64_t e = 0; e < ne && !*err; ++e) for (int k = 0; k < 3; ++k) {
    if (m->nb[3 * e + k] >= 0) m->bc[3 * e + k] = 0;
    else m->bc[3 * e + k] = tag[3 * e + k] == 2 ? 2 : 1;
  }
  free(tag);
  if (*err) { or_mesh_free(m); return NULL; }
  return m;
}

void or_set_orders(or_mesh* m, const int8_t* p) { for (int64_t e = 0; e < m->ne; ++e) m->p[e] = p[e]; }

/* geometry exports for tests */
void or_mesh_geometry(const or_mesh* m, double* area, double* s, double* hb, double* dhb) {
  for (int64_t e = 0; e < m->ne; ++e) {
    if (area) area[e] = m->area[e];
    if (s) s[e] = m->s[e];
    for (int i = 0; i < 3; ++i) if (hb) hb[3 * e + i] = m->hb[3 * e + i];
    for (int i = 0; i < 2; ++i) if (dhb) dhb[2 * e + i] = m->dhb[2 * e + i];
  }
}
void or_mesh_neighbours(const or_mesh* m, int64_t* nb, int8_t* nbk, int8_t* bc, int32_t* tri) {
  for (int64_t i = 0; i < 3 * m->ne; ++i) { nb[i] = m->nb[i]; nbk[i] = m->nbk[i]; bc[i] = m->bc[i]; tri[i] = m->tri[i]; }
}

/* Modal coefficients of the continuous P1 interpolant of vertex values
 * (used for h_b and for P1 initial states): out[i][e], i < 3. */
void or_p1_modes(const or_mesh* m, const double* vals, double* out) {
  for (int64_t e = 0; e < m->ne; ++e)
    for (int i = 0; i < 3; ++i) {
      double acc = 0.0;
      for (int w = 0; w < 3; ++w) acc += vals[m->tri[3 * e + w]] * L_[w][i];
      out[(int64_t)i * m->ne + e] = m->s[e] * acc;
    }
}

/* ------------------------------------------------------------------ */
/* L2 projection onto the element basis with a collapsed Gauss rule.   */
/* ------------------------------------------------------------------ */
static void gauss_legendre(int n, double* x, double* w) {
  for (int i = 0; i < n; ++i) {
    double z = cos(M_PI * (i + 0.75) / (n + 0.5)), pp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) { double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k; p0 = p1; p1 = p2; }
      if (n == 1) { p1 = z; p0 = 1.0; }
      pp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / pp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= n; ++k) { double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k; p0 = p1; p1 = p2; }
    pp = n * (z * p1 - p0) / (z * z - 1.0);
    x[i] = z; w[i] = 2.0 / ((1.0 - z * z) * pp * pp);
  }
}

static double p2_eval(const poly2* a, double x, double y) {
  double s = 0.0, xp = 1.0;
  for (int i = 0; i < PD; ++i) {
    double yp = 1.0;
    for (int j = 0; i + j < PD; ++j) { s += (a->c[i][j].hi + a->c[i][j].lo) * xp * yp; yp *= y; }
    xp *= x;
  }
  return s;
}

/* reference points of an n x n collapsed rule: xh[n*n], yh[n*n], w[n*n] */
void or_tri_rule(int n, double* xh, double* yh, double* w) {
  double gx[64], gw[64];
  gauss_legendre(n, gx, gw);
  for (int i = 0; i < n; ++i) for (int j = 0; j < n; ++j) {
    double a = gx[i], b = gx[j];
    xh[i * n + j] = 0.25 * (1.0 + a) * (1.0 - b);
    yh[i * n + j] = 0.5 * (1.0 + b);
    w[i * n + j] = gw[i] * gw[j] * (1.0 - b) / 8.0;
  }
}

/* Physical points of the rule on every element: xy[e][n*n][2]. */
void or_proj_points(const or_mesh* m, int n, double* xy) {
  int nq = n * n;
  double xh[4096], yh[4096], w[4096];
  or_tri_rule(n, xh, yh, w);
  #pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < m->ne; ++e) {
    int32_t v0 = m->tri[3 * e], v1 = m->tri[3 * e + 1], v2 = m->tri[3 * e + 2];
    for (int q = 0; q < nq; ++q) {
      xy[(e * nq + q) * 2] = m->vx[v0] + (m->vx[v1] - m->vx[v0]) * xh[q] + (m->vx[v2] - m->vx[v0]) * yh[q];
      xy[(e * nq + q) * 2 + 1] = m->vy[v0] + (m->vy[v1] - m->vy[v0]) * xh[q] + (m->vy[v2] - m->vy[v0]) * yh[q];
    }
  }
}

/* c_i = int_Omega_e f phi_{e,i} for i < K(p_e): vals[e][n*n] -> out[i][e]
 * (out has 15 rows; rows >= K(p_e) are set to zero). */
void or_project(const or_mesh* m, int n, const double* vals, double* out) {
  int nq = n * n;
  double xh[4096], yh[4096], w[4096];
  or_tri_rule(n, xh, yh, w);
  #pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < m->ne; ++e) {
    int K = KP[m->p[e]];
    for (int i = 0; i < KMAX; ++i) {
      double acc = 0.0;
      if (i < K)
        for (int q = 0; q < nq; ++q) acc += w[q] * vals[e * nq + q] * p2_eval(&g_phi[i], xh[q], yh[q]);
      /* int_Omega f phi_i = int_T f phihat_i / s * s^2 */
      out[(int64_t)i * m->ne + e] = acc * m->s[e];
    }
  }
}

/* ------------------------------------------------------------------ */
/* Auxiliary system uH = q (Sect. 3, truncated with K(p,i,j)).          */
/* ------------------------------------------------------------------ */
static int lu_solve(int K, double A[KMAX][KMAX], double* b1, double* b2) {
  /* Doolittle LU without pivoting (the matrix is symmetric positive definite
   * for positive depth), then forward and back substitution for two
   * right-hand sides. */
  for (int k = 0; k < K; ++k) {
    if (A[k][k] == 0.0) return -4;
    for (int i = k + 1; i < K; ++i) {
      double l = A[i][k] / A[k][k];
      A[i][k] = l;
      for (int j = k + 1; j < K; ++j) A[i][j] -= l * A[k][j];
    }
  }
  double* bs[2] = {b1, b2};
  for (int r = 0; r < 2; ++r) {
    double* b = bs[r];
    for (int i = 0; i < K; ++i) for (int j = 0; j < i; ++j) b[i] -= A[i][j] * b[j];
    for (int i = K - 1; i >= 0; --i) {
      for (int j = i + 1; j < K; ++j) b[i] -= A[i][j] * b[j];
      b[i] /= A[i][i];
    }
  }
  return 0;
}

/* u[l][i][e] (l = 0: u, 1: v).  Returns -3 when an element mean of H is
 * <= h_min. */
int or_usolve(const or_mesh* m, const or_params* P, const double* c, double* u) {
  int64_t ne = m->ne;
  int bad_depth = 0, bad_solve = 0;
#pragma omp parallel for schedule(dynamic, 256) reduction(| : bad_depth, bad_solve)
  for (int64_t e = 0; e < ne; ++e) {
    int K = KP[m->p[e]];
    double H[KMAX], A[KMAX][KMAX], bu[KMAX], bv[KMAX];
    for (int n = 0; n < KMAX; ++n) H[n] = (n < K ? C_(c, 0, n, e, ne) : 0.0) + (n < 3 ? m->hb[3 * e + n] : 0.0);
    if (!(H[0] / sqrt(m->area[e]) > P->h_min)) bad_depth = 1;
    for (int i = 0; i < K; ++i) for (int j = 0; j < K; ++j) {
      double acc = 0.0;
      int nt = Ktr(i, j);
      for (int n = 0; n < nt; ++n) acc += H[n] * T_[n][i][j];
      A[i][j] = acc / m->s[e];
    }
    for (int i = 0; i < K; ++i) { bu[i] = C_(c, 1, i, e, ne); bv[i] = C_(c, 2, i, e, ne); }
    if (lu_solve(K, A, bu, bv)) bad_solve = 1;
    for (int i = 0; i < KMAX; ++i) {
      u[((int64_t)0 * KMAX + i) * ne + e] = i < K ? bu[i] : 0.0;
      u[((int64_t)1 * KMAX + i) * ne + e] = i < K ? bv[i] : 0.0;
    }
  }
  return bad_depth ? -3 : bad_solve ? -4 : 0;
}

/* ------------------------------------------------------------------ */
/* Semi-discrete right-hand side (Eq. 8 with the LF flux).             */
/* part: 0 = whole scheme, 1 = base (every index <= 3), 2 = correction */
/* ------------------------------------------------------------------ */
static int use_term(int part, int is_base) { return part == 0 || (part == 1 && is_base) || (part == 2 && !is_base); }

static double tide(const or_params* P, double t) {
  if (P->tide_period <= 0.0) return P->tide_amp;
  return P->tide_amp * sin(2.0 * M_PI * t / P->tide_period + P->tide_phase);
}

int or_rhs(const or_mesh* m, const or_params* P, const double* c, double t, double* rhs, int part, double* u_out) {
  ensure_ready();
  int64_t ne = m->ne;
  double g = P->g;
  double* u = u_out ? u_out : malloc(sizeof(double) * 2 * KMAX * ne);
  int status = or_usolve(m, P, c, u);
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t e = 0; e < ne; ++e) {
    int K = KP[m->p[e]];
    double se = m->s[e];
    const double* Ji = m->Jinv + 4 * e;
    double xi[KMAX], U[KMAX], V[KMAX], uu[KMAX], vv[KMAX], hb[KMAX];
    for (int i = 0; i < KMAX; ++i) {
      xi[i] = C_(c, 0, i, e, ne) * (i < K); U[i] = C_(c, 1, i, e, ne) * (i < K); V[i] = C_(c, 2, i, e, ne) * (i < K);
      uu[i] = u[(int64_t)i * ne + e]; vv[i] = u[((int64_t)KMAX + i) * ne + e];
      hb[i] = i < 3 ? m->hb[3 * e + i] : 0.0;
    }
    /* fields vanish beyond K; h_b keeps its three P1 modes even when K = 1 */
    int Kx = K < 3 ? 3 : K;
    /* bottom friction coefficient from the element means (Sect. 3): H and |u|
     * of the piecewise constant part; mode 0 of a field is its mean times
     * sqrt|Omega_e| */
    double rA = 1.0 / sqrt(m->area[e]);
    double Hm = (xi[0] + hb[0]) * rA, um = uu[0] * rA, vm = vv[0] * rA;
    double tau = P->fric_lin * Hm + P->fric_quad * sqrt(um * um + vm * vm);
    double r[3][KMAX];
    memset(r, 0, sizeof r);
    /* volume terms (A, grad phi_q) and source (r, phi_q) */
    for (int q = 0; q < K; ++q) {
      for (int i = 0; i < Kx; ++i) {
        double Dx = Ji[0] * D_[0][q][i] + Ji[2] * D_[1][q][i];
        double Dy = Ji[1] * D_[0][q][i] + Ji[3] * D_[1][q][i];
        if (use_term(part, q < 3 && i < 3)) r[0][q] += U[i] * Dx + V[i] * Dy;
        for (int j = 0; j < Kx; ++j) {
          if (!use_term(part, q < 3 && i < 3 && j < 3)) continue;
          double Gx = (Ji[0] * G_[0][q][i][j] + Ji[2] * G_[1][q][i][j]) / se;
          double Gy = (Ji[1] * G_[0][q][i][j] + Ji[3] * G_[1][q][i][j]) / se;
          double pres = g * (0.5 * xi[i] * xi[j] + xi[i] * hb[j]);
          r[1][q] += (U[i] * uu[j] + pres) * Gx + U[i] * vv[j] * Gy;
          r[2][q] += V[i] * uu[j] * Gx + (V[i] * vv[j] + pres) * Gy;
        }
      }
      if (use_term(part, q < 3)) {
        /* (r, phi_q) of Eq. (5); tau_bf and f_c are constant on the element, so
         * with the orthonormal basis (tau u, phi_q) = tau u_q */
        r[1][q] += g * m->dhb[2 * e] * xi[q] - tau * uu[q] + P->f_c * V[q];
        r[2][q] += g * m->dhb[2 * e + 1] * xi[q] - tau * vv[q] - P->f_c * U[q];
      }
    }
    /* edge terms -<A_hat, phi_q> */
    for (int k = 0; k < 3; ++k) {
      double L = m->elen[3 * e + k], nx = m->enx[3 * e + k], ny = m->eny[3 * e + k];
      int bc = m->bc[3 * e + k];
      double xo[KMAX], Uo[KMAX], Vo[KMAX], uo[KMAX], vo[KMAX], ho[KMAX];
      int Ko;
      double lin_x, tri_x, areao;
      const double(*X2)[KMAX]; const double(*X3)[KMAX][KMAX];
      double xihat = 0.0;
      if (bc == 0) {
        int64_t n = m->nb[3 * e + k]; int kk = m->nbk[3 * e + k];
        Ko = KP[m->p[n]];
        for (int i = 0; i < KMAX; ++i) {
          xo[i] = C_(c, 0, i, n, ne) * (i < Ko); Uo[i] = C_(c, 1, i, n, ne) * (i < Ko); Vo[i] = C_(c, 2, i, n, ne) * (i < Ko);
          uo[i] = u[(int64_t)i * ne + n]; vo[i] = u[((int64_t)KMAX + i) * ne + n];
          ho[i] = i < 3 ? m->hb[3 * n + i] : 0.0;
        }
        lin_x = L / (se * m->s[n]); tri_x = L / (se * m->s[n] * m->s[n]);
        X2 = X2_[k][kk]; X3 = X3_[k][kk]; areao = m->area[n];
      } else {
        Ko = K;
        for (int i = 0; i < KMAX; ++i) {
          ho[i] = hb[i];
          if (bc == 1) { /* land: mirror the normal component */
            double qn = nx * U[i] + ny * V[i], un = nx * uu[i] + ny * vv[i];
            xo[i] = xi[i]; Uo[i] = U[i] - 2.0 * nx * qn; Vo[i] = V[i] - 2.0 * ny * qn;
            uo[i] = uu[i] - 2.0 * nx * un; vo[i] = vv[i] - 2.0 * ny * un;
          } else { /* open sea: xi+ = xi_hat(t) as a constant, q+ = q */
            xo[i] = 0.0; Uo[i] = U[i]; Vo[i] = V[i]; uo[i] = uu[i]; vo[i] = vv[i];
          }
        }
        if (bc == 2) { xihat = tide(P, t); xo[0] = xihat * sqrt(m->area[e]); }
        lin_x = L / (se * se); tri_x = L / (se * se * se);
        X2 = S2_[k]; X3 = S3_[k]; areao = m->area[e];
      }
      int Kox = Ko < 3 ? 3 : Ko;
      double lin_o = L / (se * se), tri_o = L / (se * se * se);
      /* lambda (Eq. 10) from the element means (Sect. 3) */
      double ra = 1.0 / sqrt(m->area[e]), rb = 1.0 / sqrt(areao);
      double un_a = (uu[0] * nx + vv[0] * ny) * ra, un_b = (uo[0] * nx + vo[0] * ny) * rb;
      double Ha = xi[0] * ra + m->ehb[3 * e + k], Hb = xo[0] * rb + m->ehb[3 * e + k];
      double lam = fmax(fabs(un_a), fabs(un_b)) + fmax(sqrt(g * Ha), sqrt(g * Hb));
      for (int q = 0; q < K; ++q) {
        double F[3] = {0.0, 0.0, 0.0};
        for (int i = 0; i < KMAX; ++i) {
          /* own side, linear parts: A_xi.n and lambda c */
          if (i < Kx && use_term(part, q < 3 && i < 3)) {
            double w = S2_[k][q][i] * lin_o;
            F[0] += (U[i] * nx + V[i] * ny) * w + lam * xi[i] * w;
            F[1] += lam * U[i] * w;
            F[2] += lam * V[i] * w;
          }
          if (i < Kox && use_term(part, q < 3 && i < 3)) {
            double w = X2[q][i] * lin_x;
            F[0] += (Uo[i] * nx + Vo[i] * ny) * w - lam * xo[i] * w;
            F[1] -= lam * Uo[i] * w;
            F[2] -= lam * Vo[i] * w;
          }
          for (int j = 0; j < KMAX; ++j) {
            if (i < Kx && j < Kx && use_term(part, q < 3 && i < 3 && j < 3)) {
              double w = S3_[k][q][i][j] * tri_o;
              double unj = uu[j] * nx + vv[j] * ny;
              double pres = g * (0.5 * xi[i] * xi[j] + xi[i] * hb[j]);
              F[1] += (U[i] * unj + pres * nx) * w;
              F[2] += (V[i] * unj + pres * ny) * w;
            }
            if (i < Kox && j < Kox && use_term(part, q < 3 && i < 3 && j < 3)) {
              double w = X3[q][i][j] * tri_x;
              double unj = uo[j] * nx + vo[j] * ny;
              double pres = g * (0.5 * xo[i] * xo[j] + xo[i] * ho[j]);
              F[1] += (Uo[i] * unj + pres * nx) * w;
              F[2] += (Vo[i] * unj + pres * ny) * w;
            }
          }
        }
        for (int f = 0; f < 3; ++f) r[f][q] -= 0.5 * F[f];
      }
    }
    for (int f = 0; f < 3; ++f)
      for (int q = 0; q < KMAX; ++q) C_(rhs, f, q, e, ne) = q < K ? r[f][q] : 0.0;
  }
  if (!u_out) free(u);
  for (int64_t i = 0; i < 3 * KMAX * ne && status == 0; ++i) if (!isfinite(rhs[i])) status = -4;
  return status;
}

/* ------------------------------------------------------------------ */
/* Time step and SSP Runge-Kutta (Sect. 2).                            */
/* ------------------------------------------------------------------ */
double or_dt(const or_mesh* m, const or_params* P, const double* c, const double* u) {
  double best = INFINITY;
  int64_t ne = m->ne;
#pragma omp parallel for schedule(static) reduction(min : best)
  for (int64_t e = 0; e < ne; ++e) {
    double ra = 1.0 / sqrt(m->area[e]);
    double ub = u[e] * ra, vb = u[(int64_t)KMAX * ne + e] * ra;
    double Hb = (C_(c, 0, 0, e, ne) + m->hb[3 * e]) * ra;
    double sp = sqrt(ub * ub + vb * vb) + sqrt(P->g * Hb);
    double d = m->diam[e] / (sp * (2.0 * m->p[e] + 1.0));
    if (d < best) best = d;
  }
  return P->cfl * best;
}

/* One SSP-RK step in place; dt <= 0 takes the CFL step.  *dt_used and *t
 * are updated. */
int or_step(const or_mesh* m, const or_params* P, double* c, double* t, double dt, double* dt_used) {
  int64_t n = 3 * KMAX * m->ne;
  double* c0 = malloc(sizeof(double) * n);
  double* cs = malloc(sizeof(double) * n);
  double* r = malloc(sizeof(double) * n);
  double* u = malloc(sizeof(double) * 2 * KMAX * m->ne);
  memcpy(c0, c, sizeof(double) * n);
  memcpy(cs, c, sizeof(double) * n);
  int status = 0;
  if (dt <= 0.0) {
    status = or_usolve(m, P, c, u);
    dt = or_dt(m, P, c, u);
  }
  int ns = P->rk_order == 3 ? 3 : 2;
  /* stage s: c^(s+1) = a_s c^n + b_s (c^(s) + dt L(c^(s), t + tau_s dt)) */
  double a2[2] = {0.0, 0.5}, b2[2] = {1.0, 0.5}, tau2[2] = {0.0, 1.0};
  double a3[3] = {0.0, 0.75, 1.0 / 3.0}, b3[3] = {1.0, 0.25, 2.0 / 3.0}, tau3[3] = {0.0, 1.0, 0.5};
  for (int s = 0; s < ns && status == 0; ++s) {
    double a = ns == 3 ? a3[s] : a2[s], b = ns == 3 ? b3[s] : b2[s], tau = ns == 3 ? tau3[s] : tau2[s];
    status = or_rhs(m, P, cs, *t + tau * dt, r, 0, u);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) cs[i] = a * c0[i] + b * (cs[i] + dt * r[i]);
  }
  if (status == 0) { memcpy(c, cs, sizeof(double) * n); *t += dt; }
  if (dt_used) *dt_used = dt;
  free(c0); free(cs); free(r); free(u);
  return status;
}

int or_run(const or_mesh* m, const or_params* P, double* c, double* t, int64_t nsteps, double dt) {
  for (int64_t s = 0; s < nsteps; ++s) {
    int st = or_step(m, P, c, t, dt, NULL);
    if (st) return st;
  }
  return 0;
}

/* Mass = int xi = sum_e sqrt|Omega_e| xi_e1. */
double or_mass(const or_mesh* m, const double* c) {
  double s = 0.0;
  for (int64_t e = 0; e < m->ne; ++e) s += sqrt(m->area[e]) * c[e];
  return s;
}

/* Energy = 1/2 g int xi^2 + 1/2 int q.u (orthonormal basis: sums of squares). */
double or_energy(const or_mesh* m, const or_params* P, const double* c, int* status) {
  int64_t ne = m->ne;
  double* u = malloc(sizeof(double) * 2 * KMAX * ne);
  *status = or_usolve(m, P, c, u);
  double s = 0.0;
  for (int64_t e = 0; e < ne; ++e) {
    int K = KP[m->p[e]];
    for (int i = 0; i < K; ++i) {
      double x = C_(c, 0, i, e, ne);
      s += 0.5 * P->g * x * x + 0.5 * (C_(c, 1, i, e, ne) * u[(int64_t)i * ne + e] +
                                       C_(c, 2, i, e, ne) * u[((int64_t)KMAX + i) * ne + e]);
    }
  }
  free(u);
  return s;
}

/* ------------------------------------------------------------------ */
/* p-adaptivity (Sect. 2, end; Sect. 3: with a hierarchical basis an   */
/* order change adds or removes terms).  The paper's JRL indicator is  */
/* defined elsewhere; the reading used here is a modal-decay indicator: */
/*   s_e = sum_{deg i = p_e} xi_i^2 / sum_{deg i >= 1} xi_i^2           */
/* p_e + 1 if s_e > theta_up and p_e < p_max, p_e - 1 if s_e <         */
/* theta_down and p_e > p_min (s_e = 0 for p_e = 0 or a flat element).  */
/* ------------------------------------------------------------------ */
int64_t or_indicator(const or_mesh* m, const double* c, double theta_up, double theta_down, int p_min, int p_max,
                     int8_t* p_out, double* s_out) {
  ensure_ready();
  int64_t ne = m->ne, changed = 0;
#pragma omp parallel for schedule(static) reduction(+ : changed)
  for (int64_t e = 0; e < ne; ++e) {
    int p = m->p[e], K = KP[p];
    double num = 0.0, den = 0.0;
    for (int i = 1; i < K; ++i) {
      double x = C_(c, 0, i, e, ne);
      den += x * x;
      if (g_deg[i] == p) num += x * x;
    }
    double s = (p > 0 && den > 0.0) ? num / den : 0.0;
    int q = p;
    if (s > theta_up && p < p_max) q = p + 1;
    else if (s < theta_down && p > p_min) q = p - 1;
    p_out[e] = (int8_t)q;
    if (s_out) s_out[e] = s;
    changed += q != p;
  }
  return changed;
}
