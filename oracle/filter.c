/*
 * Exponential modal filter (Eq. exponential_filter): in every element and
 * along every direction, the nodal values are expanded in Legendre modes
 * P_k (k = 0..N), mode k is multiplied by sigma(k/N) = exp(-alpha (k/N)^s),
 * and the values are evaluated back at the LGL nodes.  Reading: eta = k/N
 * (no cut-off mode), and the filter acts on the momentum components (the
 * velocity field of the mountain-wave cases, whose balanced background is
 * zero), selected by a bit mask over the six variables.
 * Test infrastructure only (see oracle.h).
 */
#include <math.h>
#include <string.h>
#include "oracle.h"
#include "oracle_internal.h"

/* Legendre P_0..P_N at x by the three-term recurrence
 * (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1}. */
static void legendre_all(int N, double x, double *P) {
  P[0] = 1.0;
  if (N >= 1) P[1] = x;
  for (int k = 1; k < N; ++k) P[k + 1] = ((2.0 * k + 1.0) * x * P[k] - k * P[k - 1]) / (k + 1.0);
}

/* inverse of an n x n matrix by Gauss-Jordan elimination with partial pivoting */
static int invert(int n, const double *A, double *Ainv) {
  double M[ORC_MAXQ][2 * ORC_MAXQ];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < 2 * n; ++j) M[i][j] = j < n ? A[i * n + j] : (j - n == i ? 1.0 : 0.0);
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (fabs(M[r][c]) > fabs(M[piv][c])) piv = r;
    if (M[piv][c] == 0.0) return -1;
    if (piv != c)
      for (int j = 0; j < 2 * n; ++j) {
        double t = M[c][j];
        M[c][j] = M[piv][j];
        M[piv][j] = t;
      }
    double d = M[c][c];
    for (int j = 0; j < 2 * n; ++j) M[c][j] /= d;
    for (int r = 0; r < n; ++r)
      if (r != c) {
        double f = M[r][c];
        for (int j = 0; j < 2 * n; ++j) M[r][j] -= f * M[c][j];
      }
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) Ainv[i * n + j] = M[i][j + n];
  return 0;
}

void orc_filter_matrix(int N, const double *xi, int order, double alpha, double *F) {
  const int Nq = N + 1;
  double V[ORC_MAXQ * ORC_MAXQ], Vi[ORC_MAXQ * ORC_MAXQ], P[ORC_MAXQ];
  for (int i = 0; i < Nq; ++i) {
    legendre_all(N, xi[i], P);
    for (int k = 0; k < Nq; ++k) V[i * Nq + k] = P[k]; /* V_ik = P_k(xi_i) */
  }
  invert(Nq, V, Vi);
  for (int i = 0; i < Nq; ++i)
    for (int j = 0; j < Nq; ++j) {
      double acc = 0.0;
      for (int k = 0; k < Nq; ++k) acc += V[i * Nq + k] * exp(-alpha * pow((double)k / N, order)) * Vi[k * Nq + j];
      F[i * Nq + j] = acc;
    }
}

void orc_filter(orc_solver *s, double *Q, int order, double alpha, int mask) {
  const int N = s->N, Nq = s->Nq, Np = s->Np;
  double F[ORC_MAXQ * ORC_MAXQ];
  orc_filter_matrix(N, s->xi, order, alpha, F);
  double a[ORC_MAXQ * ORC_MAXQ * ORC_MAXQ], b[ORC_MAXQ * ORC_MAXQ * ORC_MAXQ];
  for (int e = 0; e < s->E; ++e)
    for (int v = 0; v < 6; ++v) {
      if (!(mask & (1 << v))) continue;
      double *q = Q + ((size_t)e * 6 + v) * Np;
      memcpy(a, q, (size_t)Np * sizeof(double));
      /* along x (index i), then y (j), then z (k); node n = i + Nq (j + Nq k) */
      for (int dir = 0; dir < 3; ++dir) {
        for (int k = 0; k < Nq; ++k)
          for (int j = 0; j < Nq; ++j)
            for (int i = 0; i < Nq; ++i) {
              double acc = 0.0;
              for (int m = 0; m < Nq; ++m) {
                int idx = dir == 0 ? m + Nq * (j + Nq * k) : (dir == 1 ? i + Nq * (m + Nq * k) : i + Nq * (j + Nq * m));
                int row = dir == 0 ? i : (dir == 1 ? j : k);
                acc += F[row * Nq + m] * a[idx];
              }
              b[i + Nq * (j + Nq * k)] = acc;
            }
        memcpy(a, b, (size_t)Np * sizeof(double));
      }
      memcpy(q, a, (size_t)Np * sizeof(double));
    }
}
