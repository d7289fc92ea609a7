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
 * with the equation of state of unsaturated air at rest and fixed total
 * water q_r(z) (Eqs. eos and internal_energies with q_l = 0), linear in
 * (rho, rho e):
 *   p = R_m T_0 rho + kappa_m (rho e - rho Phi - rho q_r I_v0),   Phi = g z,
 * kappa_m = R_m / c_vm, R_m and c_vm the mixture constants at q_r, so that
 *   d rho'/dt  = -d(rho w)/dz
 *   d(rho w)/dt = -d p'/dz - g rho',    p' = a rho' + kappa_m (rho e)',
 *   d(rho e)'/dt = -d(h_r rho w)/dz,    h_r = (rho e_r + p_r) / rho_r,
 * a = R_m T_0 - kappa_m (Phi + q_r I_v0), rho e_r = rho_r (c_vm (T_r - T_0) +
 * q_r I_v0 + Phi), T_r = p_r / (rho_r R_m), c_r^2 = (1 + kappa_m) p_r / rho_r.
 * The linearisation point is the reference (rho_r, p_r) with the reference
 * total water q_r (zero unless set): linearising a moist state about a dry
 * energy would leave a deviation (rho e)' as large as the latent part of
 * rho e, whose cancellation between the explicit and implicit parts costs
 * digits in rho'.
 * The face flux of the full operator applies Rusanov dissipation at the
 * sound speed to every component on vertical faces; for the horizontal
 * momentum and rho q_t the linear operator keeps that dissipation,
 * -(1/2) c_r [q] lifted on the z-faces, and nothing else.  Flat meshes only.
 */
#include <math.h>
#include <string.h>

#include "oracle_internal.h"

/* the reference quantities of the linear operator at node q: Phi, rho e_r,
 * h_r, c_r, kappa_m and a */
typedef struct {
  double phi, rhoe_r, h_r, c_r, kappa, a;
} lin_coef;
static lin_coef lin_ref(const orc_solver *s, size_t q) {
  const orc_params *P = &s->p;
  const double rr = s->rho_r[q], pr = s->p_r[q], qr = s->qt_r[q];
  const double Rm = (1.0 - qr) * P->Rd + qr * P->Rv, cvm = (1.0 - qr) * P->cvd + qr * P->cvv;
  const double Iv0 = P->Lv0 - P->Rv * P->T0;
  lin_coef c;
  c.phi = P->g * s->z[q];
  c.kappa = Rm / cvm;
  const double Tr = pr / (rr * Rm);
  c.rhoe_r = rr * (cvm * (Tr - P->T0) + qr * Iv0 + c.phi);
  c.h_r = (c.rhoe_r + pr) / rr;
  c.c_r = sqrt((1.0 + c.kappa) * pr / rr);
  c.a = Rm * P->T0 - c.kappa * (c.phi + qr * Iv0);
  return c;
}

/* The state the operator is linearised about: (rho_r, 0, 0, 0, rho e_r, 0). */
void orc_vlin_reference(orc_solver *s, double *Qref) {
  const int Np = s->Np;
  for (int e = 0; e < s->E; ++e)
    for (int n = 0; n < Np; ++n) {
      const size_t q = (size_t)e * Np + n;
      const lin_coef c = lin_ref(s, q);
      for (int v = 0; v < 6; ++v) Qref[((size_t)e * 6 + v) * Np + n] = 0.0;
      Qref[((size_t)e * 6 + 0) * Np + n] = s->rho_r[q];
      Qref[((size_t)e * 6 + 4) * Np + n] = c.rhoe_r;
    }
}

/* vertical flux of the deviations y = (rho', m, E') at a node */
static void vflux(const lin_coef *c, const double y[3], double F[3]) {
  F[0] = y[1];
  F[1] = c->a * y[0] + c->kappa * y[2];
  F[2] = c->h_r * y[1];
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
      const lin_coef c = lin_ref(s, q);
      y[n][0] = Q[((size_t)e * 6 + 0) * Np + n] - s->rho_r[q];
      y[n][1] = Q[((size_t)e * 6 + 3) * Np + n];
      y[n][2] = Q[((size_t)e * 6 + 4) * Np + n] - c.rhoe_r;
      vflux(&c, y[n], F[n]);
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
        const lin_coef c = lin_ref(s, q);
        const double cr = c.c_r;
        double yp[3], Fp[3];
        if (nb >= 0) {
          const int np = i + Nq * (j + Nq * (side == 0 ? N : 0));
          const size_t qp = (size_t)nb * Np + np;
          const lin_coef cp = lin_ref(s, qp);
          yp[0] = Q[((size_t)nb * 6 + 0) * Np + np] - s->rho_r[qp];
          yp[1] = Q[((size_t)nb * 6 + 3) * Np + np];
          yp[2] = Q[((size_t)nb * 6 + 4) * Np + np] - cp.rhoe_r;
        } else {
          /* reflecting wall: the normal momentum mirrored */
          yp[0] = y[n][0];
          yp[1] = -y[n][1];
          yp[2] = y[n][2];
        }
        /* the shared face node has the face's height, hence the same reference */
        vflux(&c, yp, Fp);
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
        const double cr = lin_ref(s, (size_t)e * Np + n).c_r;
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
