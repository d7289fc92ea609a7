/*
 * HEVI time stepping of Sec. 3.2 (horizontally explicit, vertically
 * implicit): the CPU oracle's vertical linear operator.  Test
 * infrastructure only: the CUDA path never links or calls it.
 *
 * Sec. 3.2 names "a variant of the HEVI schemes of Bao et al. (2015)" with
 * a 1-D IMEX additive Runge-Kutta method but prints neither the implicit
 * operator nor the tableau.  Reading: the implicit part is the vertical
 * acoustic-gravity operator linearised about the hydrostatic reference
 * state (rho_r(z), p_r(z)) and the rest state, discretised like the full
 * operator (strong-form nodal DG along z on the LGL nodes, Sec. 3.1) with a
 * Rusanov flux at the reference sound speed; it acts on the deviations
 *   y = (rho - rho_r, rho w, rho e - rho e_r)
 * with the linear equation of state of dry air at rest,
 *   p = R_d T_0 rho + (R_d / c_vd) (rho e - rho Phi),   Phi = g z,
 * (Eq. eos with the internal energy of Eq. internal_energies), so that
 *   d rho'/dt  = -d(rho w)/dz
 *   d(rho w)/dt = -d p'/dz - g rho',    p' = (R_d T_0 - kappa Phi) rho' + kappa (rho e)'
 *   d(rho e)'/dt = -d(h_r rho w)/dz,    h_r = (rho e_r + p_r) / rho_r,
 * kappa = R_d / c_vd, rho e_r = (p_r - R_d T_0 rho_r) / kappa + rho_r Phi.
 * The face flux of the full operator applies Rusanov dissipation at the
 * sound speed to every component on vertical faces; for the horizontal
 * momentum and rho q_t the linear operator keeps that dissipation,
 * -(1/2) c_r [q] lifted on the z-faces, and nothing else.  Flat meshes only.
 */
#include <math.h>
#include <string.h>

#include "oracle_internal.h"

/* the reference quantities of the linear operator at node q */
static void lin_ref(const orc_solver *s, size_t q, double *phi, double *rhoe_r, double *h_r, double *c_r) {
  const orc_params *P = &s->p;
  const double kappa = P->Rd / P->cvd;
  const double rr = s->rho_r[q], pr = s->p_r[q];
  *phi = P->g * s->z[q];
  *rhoe_r = (pr - P->Rd * P->T0 * rr) / kappa + rr * (*phi);
  *h_r = (*rhoe_r + pr) / rr;
  *c_r = sqrt((P->cvd + P->Rd) / P->cvd * pr / rr);
}

/* The state the operator is linearised about: (rho_r, 0, 0, 0, rho e_r, 0). */
void orc_vlin_reference(orc_solver *s, double *Qref) {
  const int Np = s->Np;
  for (int e = 0; e < s->E; ++e)
    for (int n = 0; n < Np; ++n) {
      const size_t q = (size_t)e * Np + n;
      double phi, rer, hr, cr;
      lin_ref(s, q, &phi, &rer, &hr, &cr);
      for (int v = 0; v < 6; ++v) Qref[((size_t)e * 6 + v) * Np + n] = 0.0;
      Qref[((size_t)e * 6 + 0) * Np + n] = s->rho_r[q];
      Qref[((size_t)e * 6 + 4) * Np + n] = rer;
    }
}

/* vertical flux of the deviations y = (rho', m, E') at a node */
static void vflux(const orc_params *P, double phi, double hr, const double y[3], double F[3]) {
  const double kappa = P->Rd / P->cvd;
  F[0] = y[1];
  F[1] = (P->Rd * P->T0 - kappa * phi) * y[0] + kappa * y[2];
  F[2] = hr * y[1];
}

/* out = L (Q - Qref): components 0, 3, 4 (rho, rho w, rho e); the others 0. */
void orc_vlin_apply(orc_solver *s, const double *Q, double *out) {
  const int Nq = s->Nq, Np = s->Np, N = s->N;
  const orc_params *P = &s->p;
  const double hz = s->m.Lz / s->m.nez;
  const double jz = 2.0 / hz, lift = 2.0 / (hz * s->w[0]);
  const int comp[3] = {0, 3, 4};
  memset(out, 0, (size_t)s->E * 6 * Np * sizeof(double));
  for (int e = 0; e < s->E; ++e) {
    /* deviations and fluxes of the element's nodes */
    double y[ORC_MAXQ * ORC_MAXQ * ORC_MAXQ][3], F[ORC_MAXQ * ORC_MAXQ * ORC_MAXQ][3];
    for (int n = 0; n < Np; ++n) {
      const size_t q = (size_t)e * Np + n;
      double phi, rer, hr, cr;
      lin_ref(s, q, &phi, &rer, &hr, &cr);
      y[n][0] = Q[((size_t)e * 6 + 0) * Np + n] - s->rho_r[q];
      y[n][1] = Q[((size_t)e * 6 + 3) * Np + n];
      y[n][2] = Q[((size_t)e * 6 + 4) * Np + n] - rer;
      vflux(P, phi, hr, y[n], F[n]);
    }
    for (int n = 0; n < Np; ++n) {
      const int i = n % Nq, j = (n / Nq) % Nq, k = n / (Nq * Nq);
      double r[3] = {0.0, 0.0, 0.0};
      /* volume: -d F / dz along the element's vertical line */
      for (int m = 0; m < Nq; ++m) {
        const int nm = i + Nq * (j + Nq * m);
        for (int c = 0; c < 3; ++c) r[c] -= jz * s->D[k * Nq + m] * F[nm][c];
      }
      r[1] -= P->g * y[n][0];
      /* faces: bottom (k = 0, n_z = -1, face 4) and top (k = N, n_z = +1, face 5) */
      for (int side = 0; side < 2; ++side) {
        if ((side == 0 && k != 0) || (side == 1 && k != N)) continue;
        const double nz = side == 0 ? -1.0 : 1.0;
        const int nb = s->EToE[e * 6 + (side == 0 ? 4 : 5)];
        const size_t q = (size_t)e * Np + n;
        double phi, rer, hr, cr;
        lin_ref(s, q, &phi, &rer, &hr, &cr);
        double yp[3], Fp[3];
        if (nb >= 0) {
          const int np = i + Nq * (j + Nq * (side == 0 ? N : 0));
          const size_t qp = (size_t)nb * Np + np;
          double phip, rerp, hrp, crp;
          lin_ref(s, qp, &phip, &rerp, &hrp, &crp);
          yp[0] = Q[((size_t)nb * 6 + 0) * Np + np] - s->rho_r[qp];
          yp[1] = Q[((size_t)nb * 6 + 3) * Np + np];
          yp[2] = Q[((size_t)nb * 6 + 4) * Np + np] - rerp;
        } else {
          /* reflecting wall: the normal momentum mirrored */
          yp[0] = y[n][0];
          yp[1] = -y[n][1];
          yp[2] = y[n][2];
        }
        /* the shared face node has the face's height, hence the same reference */
        vflux(P, phi, hr, yp, Fp);
        for (int c = 0; c < 3; ++c) {
          const double Fstar = 0.5 * nz * (F[n][c] + Fp[c]) + 0.5 * cr * (y[n][c] - yp[c]);
          r[c] += lift * (nz * F[n][c] - Fstar);
        }
      }
      for (int c = 0; c < 3; ++c) out[((size_t)e * 6 + comp[c]) * Np + n] = r[c];
      /* horizontal momentum and rho q_t: the vertical faces' dissipation */
      for (int side = 0; side < 2; ++side) {
        if ((side == 0 && k != 0) || (side == 1 && k != N)) continue;
        const int nb = s->EToE[e * 6 + (side == 0 ? 4 : 5)];
        const size_t q = (size_t)e * Np + n;
        double phi, rer, hr, cr;
        lin_ref(s, q, &phi, &rer, &hr, &cr);
        const int np = i + Nq * (j + Nq * (side == 0 ? N : 0));
        const int vs[3] = {1, 2, 5};
        for (int c = 0; c < 3; ++c) {
          const double qm = Q[((size_t)e * 6 + vs[c]) * Np + n];
          double qp;
          if (nb >= 0)
            qp = Q[((size_t)nb * 6 + vs[c]) * Np + np];
          else
            qp = qm;  /* a wall mirrors only the normal momentum */
          out[((size_t)e * 6 + vs[c]) * Np + n] += lift * (-0.5 * cr * (qm - qp));
        }
      }
    }
  }
}
