// Reference-element tables of libswedg (host side).
#pragma once
#include "common.h"

namespace swedg {

struct RefTables {
  double D[2][KMAX][KMAX];          // D_k[q][i] = int phi_i d_k phi_q
  double G[2][KMAX][KMAX][KMAX];    // G_k[q][i][j] = int phi_i phi_j d_k phi_q
  double T[KMAX][KMAX][KMAX];       // T[n][i][j] = int phi_n phi_i phi_j
  double M[KMAX][KMAX];             // int phi_q phi_i (identity up to rounding)
  double grad1[3][2];               // grad phihat_q for q < 3 (constant)
  double phi0;                      // phihat_1 = sqrt 2
  double Lv[3][3];                  // int lambda_v phihat_i, i < 3
  double es[9][8], ew[9][8];        // Gauss-Legendre rules on [0,1], 1..8 points
  double EB[9][3][KMAX][8];         // EB[n][k][i][g] = phihat_i(gamma_k(s_g)) with the n-point rule
  double EV[3][2][3];               // EV[k][a][i] = phihat_i(gamma_k(a)), a = 0, 1: degree-1 modes at the edge ends
};

void dubiner(double x, double y, double* v, double* vx, double* vy);
void gauss01(int n, double* s, double* w);
const RefTables& tables();

}  // namespace swedg
