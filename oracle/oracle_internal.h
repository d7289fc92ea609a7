/*
 * Private layout of the oracle solver, shared by the oracle's own source
 * files only.  Test infrastructure only (see oracle.h).
 */
#ifndef CMLES_ORACLE_INTERNAL_H
#define CMLES_ORACLE_INTERNAL_H
#include "oracle.h"

struct orc_solver {
  orc_mesh m;
  orc_params p;
  int N, Nq, Np, E;
  double xi[ORC_MAXQ], w[ORC_MAXQ], D[ORC_MAXQ * ORC_MAXQ];
  double *x, *y, *z, *J, *Ja; /* Ja[e][n][r][c] = J * d xi_r / d x_c */
  double *Delta;              /* [E] */
  double *Dm;                 /* [E][3], L_m / N from the element's extent along axis m */
  int *EToE;                  /* [E][6], -1 = wall */
  double *rho_r, *p_r, *tau;  /* [E][Np] */
  double *qt_r;               /* [E][Np] reference total water of the HEVI linearisation (0 unless set) */
  /* work arrays of the last RHS */
  double *G, *gradG, *nut, *Dt, *F2, *aux, *Ftot;
  /* learned closure (FP64 copy) */
  int has_mlp;
  double mlp_W1[64 * 13], mlp_b1[64], mlp_W2[64 * 64], mlp_b2[64], mlp_W3[2 * 64], mlp_b3[2];
  double mlp_in[13], mlp_out[2];
};

#endif
