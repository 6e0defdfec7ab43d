// Reference-element tables of libswedg, generated on the host by numerical
// quadrature (independent of any symbolic expansion):
//   - the orthonormal Dubiner basis on T = {x, y >= 0, x + y <= 1}, evaluated
//     from its collapsed-coordinate recurrences (value and gradient);
//   - Gauss-Legendre rules on [0,1] and collapsed (Duffy) rules on T;
//   - the volume tensors D, G and the auxiliary-system tensor T of Eq. (13)
//     and Sect. 3, integrated with a 14 x 14 collapsed rule (exact for the
//     degree <= 12 integrands);
//   - edge trace tables B_k[i][g] = phihat_i(gamma_k(s_g)), which apply the
//     edge tensors of the quadrature-free scheme in factored form.
#include "tables.h"

#include <cmath>
#include <cstring>

namespace swedg {

// Dubiner basis (Sect. 2: hierarchical and orthonormal on the element).  In
// collapsed coordinates eta1 = (2x + y - 1)/(1 - y), eta2 = 2y - 1 the mode
// (a, b) is  N_ab P_a(eta1) (1-y)^a P_b^(2a+1,0)(eta2),  N_ab^2 = 2(2a+1)(a+b+1).
// R_a = P_a(eta1) (1-y)^a is evaluated without the singular division through
// (a+1) R_{a+1} = (2a+1) l R_a - a m^2 R_{a-1},  l = 2x + y - 1, m = 1 - y.
// Modes are ordered by total degree a + b, then by b.
void dubiner(double x, double y, double* v, double* vx, double* vy) {
  const double l = 2.0 * x + y - 1.0, m = 1.0 - y;
  double R[5], Rx[5], Ry[5];
  R[0] = 1.0; Rx[0] = 0.0; Ry[0] = 0.0;
  R[1] = l;   Rx[1] = 2.0; Ry[1] = 1.0;
  for (int a = 1; a < 4; ++a) {
    const double c1 = (2.0 * a + 1.0) / (a + 1.0), c2 = (double)a / (a + 1.0);
    R[a + 1] = c1 * l * R[a] - c2 * m * m * R[a - 1];
    Rx[a + 1] = c1 * (2.0 * R[a] + l * Rx[a]) - c2 * m * m * Rx[a - 1];
    Ry[a + 1] = c1 * (R[a] + l * Ry[a]) - c2 * (m * m * Ry[a - 1] - 2.0 * m * R[a - 1]);
  }
  const double t = 2.0 * y - 1.0;
  int idx = 0;
  for (int d = 0; d <= 4; ++d) {
    for (int b = 0; b <= d; ++b) {
      const int a = d - b;
      const double al = 2.0 * a + 1.0;
      // Jacobi P_n^(al,0)(t) and its t-derivative by the three-term recurrence
      double P0 = 1.0, dP0 = 0.0;
      double P1 = 0.5 * ((al + 2.0) * t + al), dP1 = 0.5 * (al + 2.0);
      double P = P0, dP = dP0;
      if (b >= 1) { P = P1; dP = dP1; }
      for (int n = 1; n < b; ++n) {
        const double s = 2.0 * n + al;
        const double A1 = 2.0 * (n + 1) * (n + al + 1) * s;
        const double A2 = (s + 1) * al * al;
        const double A3 = s * (s + 1) * (s + 2);
        const double A4 = 2.0 * (n + al) * n * (s + 2);
        const double P2 = ((A2 + A3 * t) * P1 - A4 * P0) / A1;
        const double dP2 = (A3 * P1 + (A2 + A3 * t) * dP1 - A4 * dP0) / A1;
        P0 = P1; dP0 = dP1; P1 = P2; dP1 = dP2;
        P = P2; dP = dP2;
      }
      const double N = std::sqrt(2.0 * (2.0 * a + 1.0) * (a + b + 1.0));
      v[idx] = N * R[a] * P;
      if (vx) vx[idx] = N * Rx[a] * P;
      if (vy) vy[idx] = N * (Ry[a] * P + R[a] * 2.0 * dP);
      ++idx;
    }
  }
}

// Gauss-Legendre nodes and weights on [0,1], by Newton's method on P_n.
void gauss01(int n, double* s, double* w) {
  for (int i = 0; i < n; ++i) {
    double z = -std::cos(M_PI * (i + 0.75) / (n + 0.5));  // ascending
    double dp = 1.0;
    for (int it = 0; it < 60; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 1; k < n; ++k) {
        const double p2 = ((2.0 * k + 1.0) * z * p1 - k * p0) / (k + 1.0);
        p0 = p1; p1 = p2;
      }
      const double pn = n == 0 ? 1.0 : p1, pm = n == 1 ? 1.0 : p0;
      dp = n * (pm - z * pn) / (1.0 - z * z);
      const double step = pn / dp;
      z -= step;
      if (std::fabs(step) < 1e-17) break;
    }
    double p0 = 1.0, p1 = z;
    for (int k = 1; k < n; ++k) {
      const double p2 = ((2.0 * k + 1.0) * z * p1 - k * p0) / (k + 1.0);
      p0 = p1; p1 = p2;
    }
    dp = n * (p0 - z * p1) / (1.0 - z * z);
    s[i] = 0.5 * (1.0 + z);
    w[i] = 1.0 / ((1.0 - z * z) * dp * dp);  // = 2/((1-z^2) P'^2) / 2
  }
}

void edge_point(int k, double s, double* x, double* y) {
  // gamma_0(s) = (1-s, s), gamma_1(s) = (0, 1-s), gamma_2(s) = (s, 0)
  if (k == 0) { *x = 1.0 - s; *y = s; }
  else if (k == 1) { *x = 0.0; *y = 1.0 - s; }
  else { *x = s; *y = 0.0; }
}

void build_tables(RefTables* R) {
  std::memset(R, 0, sizeof(*R));
  const int n = 14;
  double s[32], w[32];
  gauss01(n, s, w);
  for (int a = 0; a < n; ++a) {
    for (int b = 0; b < n; ++b) {
      // Duffy map of the unit square onto T: x = u (1 - v), y = v, dx dy = (1 - v) du dv
      const double u = s[a], v = s[b];
      const double x = u * (1.0 - v), y = v, wt = w[a] * w[b] * (1.0 - v);
      double ph[KMAX], px[KMAX], py[KMAX];
      dubiner(x, y, ph, px, py);
      const double* dk[2] = {px, py};
      for (int i = 0; i < KMAX; ++i) {
        for (int q = 0; q < KMAX; ++q) {
          R->M[q][i] += wt * ph[q] * ph[i];
          for (int k = 0; k < 2; ++k) R->D[k][q][i] += wt * ph[i] * dk[k][q];
        }
        for (int j = 0; j < KMAX; ++j) {
          const double pij = wt * ph[i] * ph[j];
          for (int q = 0; q < KMAX; ++q) {
            R->T[q][i][j] += pij * ph[q];
            R->G[0][q][i][j] += pij * px[q];
            R->G[1][q][i][j] += pij * py[q];
          }
        }
      }
    }
  }
  // gradients of the degree-1 modes (constant)
  double ph[KMAX], px[KMAX], py[KMAX];
  dubiner(0.25, 0.25, ph, px, py);
  for (int q = 0; q < 3; ++q) { R->grad1[q][0] = px[q]; R->grad1[q][1] = py[q]; }
  R->phi0 = ph[0];
  // barycentric hat functions against the basis: Lv[v][i] = int lambda_v phihat_i
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b) {
      const double u = s[a], v = s[b];
      const double x = u * (1.0 - v), y = v, wt = w[a] * w[b] * (1.0 - v);
      dubiner(x, y, ph, nullptr, nullptr);
      const double lam[3] = {1.0 - x - y, x, y};
      for (int vv = 0; vv < 3; ++vv)
        for (int i = 0; i < 3; ++i) R->Lv[vv][i] += wt * lam[vv] * ph[i];
    }
  // edge trace tables for every rule size used
  for (int np = 1; np <= 8; ++np) {
    gauss01(np, R->es[np], R->ew[np]);
    for (int k = 0; k < 3; ++k)
      for (int g = 0; g < np; ++g) {
        double x, y;
        edge_point(k, R->es[np][g], &x, &y);
        dubiner(x, y, ph, nullptr, nullptr);
        for (int i = 0; i < KMAX; ++i) R->EB[np][k][i][g] = ph[i];
      }
  }
  for (int k = 0; k < 3; ++k)
    for (int a = 0; a < 2; ++a) {
      double x, y;
      edge_point(k, (double)a, &x, &y);
      dubiner(x, y, ph, nullptr, nullptr);
      for (int i = 0; i < 3; ++i) R->EV[k][a][i] = ph[i];
    }
}

const RefTables& tables() {
  static RefTables* R = nullptr;
  if (!R) {
    RefTables* t = new RefTables;
    build_tables(t);
    R = t;
  }
  return *R;
}

}  // namespace swedg
