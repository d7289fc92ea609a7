/*
 * Legendre-Gauss-Lobatto nodes, weights and the 1D differentiation matrix
 * (Sec. 3.1, Eqs. expansion, expansionDerivs and basisDerivatives).
 * Test infrastructure only (see oracle.h).
 *
 *   nodes   xi_0 = -1, xi_N = +1 and the N-1 roots of P_N'(x)
 *   weights w_i = 2 / (N (N+1) P_N(xi_i)^2)
 *   D_ij    = L_j'(xi_i), the derivative of the j-th Lagrange polynomial
 *             at node i, from barycentric weights; D_ii = -sum_{j!=i} D_ij.
 */
#include <math.h>
#include "oracle.h"

/* Legendre polynomial P_N(x) and its derivative by the three-term recurrence. */
static void legendre(int N, double x, double *P, double *dP) {
  double p0 = 1.0, p1 = x, d0 = 0.0, d1 = 1.0;
  if (N == 0) { *P = 1.0; *dP = 0.0; return; }
  for (int k = 2; k <= N; ++k) {
    double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
    double d2 = d0 + (2.0 * k - 1.0) * p1;   /* P_k' = P_{k-2}' + (2k-1) P_{k-1} */
    p0 = p1; p1 = p2; d0 = d1; d1 = d2;
  }
  *P = p1; *dP = d1;
}

void orc_lgl(int N, double *xi, double *w, double *D) {
  int Nq = N + 1;
  /* Interior nodes: Newton on q(x) = P_N'(x), started from the
   * Chebyshev-Gauss-Lobatto points -cos(pi i / N). */
  for (int i = 0; i < Nq; ++i) {
    double x = -cos(M_PI * i / N);
    if (i > 0 && i < N) {
      for (int it = 0; it < 100; ++it) {
        /* P_N'' from the Legendre ODE: (1-x^2) P'' = 2x P' - N(N+1) P */
        double P, dP;
        legendre(N, x, &P, &dP);
        double ddP = (2.0 * x * dP - N * (N + 1.0) * P) / (1.0 - x * x);
        double dx = dP / ddP;
        x -= dx;
        if (fabs(dx) < 1e-16) break;
      }
    }
    xi[i] = x;
  }
  xi[0] = -1.0; xi[N] = 1.0;
  /* symmetrise: xi_{N-i} = -xi_i exactly */
  for (int i = 0; i < Nq / 2; ++i) {
    double a = 0.5 * (xi[N - i] - xi[i]);
    xi[i] = -a; xi[N - i] = a;
  }
  if (Nq % 2 == 1) xi[N / 2] = 0.0;
  for (int i = 0; i < Nq; ++i) {
    double P, dP;
    legendre(N, xi[i], &P, &dP);
    w[i] = 2.0 / (N * (N + 1.0) * P * P);
  }
  /* barycentric weights lambda_j = 1 / prod_{k != j} (xi_j - xi_k) */
  double lam[ORC_MAXQ];
  for (int j = 0; j < Nq; ++j) {
    double prod = 1.0;
    for (int k = 0; k < Nq; ++k)
      if (k != j) prod *= (xi[j] - xi[k]);
    lam[j] = 1.0 / prod;
  }
  for (int i = 0; i < Nq; ++i) {
    double diag = 0.0;
    for (int j = 0; j < Nq; ++j) {
      if (j == i) continue;
      double dij = (lam[j] / lam[i]) / (xi[i] - xi[j]);
      D[i * Nq + j] = dij;
      diag -= dij;
    }
    D[i * Nq + i] = diag;
  }
}
