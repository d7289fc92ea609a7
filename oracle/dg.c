/*
 * The oracle's nodal DG right-hand side (Sec. 3.1, Eq. matrixProblem) on
 * hexahedral LGL elements, with the BR1 auxiliary gradient for the second-order
 * terms, the SGS closure (Sec. 4), wall boundary conditions (App. A.3), the
 * Rayleigh sponge (App. A.2) and the sources of Eq. momentum.
 * Test infrastructure only (see oracle.h).
 *
 * Layout: state Q[e][v][n], v = (rho, rho u, rho v, rho w, rho e_tot, rho q_t),
 * node n = i + Nq (j + Nq k) with i along xi (x), j along eta (y), k along
 * zeta (z); element e = ex + nex (ey + ney ez).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

#include "oracle_internal.h"

static int nidx(int Nq, int i, int j, int k) { return i + Nq * (j + Nq * k); }

/* node index of face node (t1, t2) on the face normal to direction d at end a */
static int face_node(int Nq, int d, int a, int t1, int t2) {
  if (d == 0) return nidx(Nq, a, t1, t2);
  if (d == 1) return nidx(Nq, t1, a, t2);
  return nidx(Nq, t1, t2, a);
}

/* the line index of node n along direction r, and the node obtained by
 * replacing that index with m */
static void node_ijk(int Nq, int n, int ijk[3]) {
  ijk[0] = n % Nq;
  ijk[1] = (n / Nq) % Nq;
  ijk[2] = n / (Nq * Nq);
}
static int replace_idx(int Nq, const int ijk[3], int r, int m) {
  int t[3] = {ijk[0], ijk[1], ijk[2]};
  t[r] = m;
  return nidx(Nq, t[0], t[1], t[2]);
}

/* derivative along xi_b of component a of a nodal vector field V[n][3] */
static double dvec(const orc_solver *s, const double *V, const int ijk[3], int a, int b) {
  double acc = 0.0;
  for (int q = 0; q < s->Nq; ++q) acc += s->D[ijk[b] * s->Nq + q] * V[replace_idx(s->Nq, ijk, b, q) * 3 + a];
  return acc;
}

/* ------------------------------------------------------------------ mesh */

static double surface_height(const orc_mesh *m, double x) {
  if (!m->warp) return 0.0;
  double s = (x - m->hill_xc) / m->hill_a;
  return m->hill_h * exp(-s * s);
}

orc_solver *orc_create(const orc_mesh *m, const orc_params *p) {
  orc_solver *s = (orc_solver *)calloc(1, sizeof(orc_solver));
  s->m = *m;
  s->p = *p;
  int N = m->N, Nq = N + 1, Np = Nq * Nq * Nq;
  int E = m->nex * m->ney * m->nez;
  s->N = N; s->Nq = Nq; s->Np = Np; s->E = E;
  orc_lgl(N, s->xi, s->w, s->D);
  size_t nn = (size_t)E * Np;
  s->x = (double *)malloc(nn * sizeof(double));
  s->y = (double *)malloc(nn * sizeof(double));
  s->z = (double *)malloc(nn * sizeof(double));
  s->J = (double *)malloc(nn * sizeof(double));
  s->Ja = (double *)malloc(nn * 9 * sizeof(double));
  s->Delta = (double *)malloc((size_t)E * sizeof(double));
  s->Dm = (double *)malloc((size_t)E * 3 * sizeof(double));
  s->EToE = (int *)malloc((size_t)E * 6 * sizeof(int));
  s->rho_r = (double *)calloc(nn, sizeof(double));
  s->qt_r = (double *)calloc(nn, sizeof(double));
  s->p_r = (double *)calloc(nn, sizeof(double));
  s->tau = (double *)calloc(nn, sizeof(double));
  s->G = (double *)malloc(nn * 6 * sizeof(double));
  s->gradG = (double *)malloc(nn * 18 * sizeof(double));
  s->nut = (double *)malloc(nn * sizeof(double));
  s->Dt = (double *)malloc(nn * sizeof(double));
  s->F2 = (double *)malloc(nn * 15 * sizeof(double));
  s->aux = (double *)malloc(nn * 4 * sizeof(double));
  s->Ftot = (double *)malloc(nn * 18 * sizeof(double));

  double hx = m->Lx / m->nex, hy = m->Ly / m->ney, hz = m->Lz / m->nez;
  /* Node coordinates: affine map of the reference cube onto each element;
   * with warping, z' = z + z_s(x) (1 - (z - z0)/Lz), i.e. linear damping of the
   * terrain to a flat top (Sec. 4.3, stacked and warped elements). */
  for (int ez = 0; ez < m->nez; ++ez)
    for (int ey = 0; ey < m->ney; ++ey)
      for (int ex = 0; ex < m->nex; ++ex) {
        int e = ex + m->nex * (ey + m->ney * ez);
        for (int k = 0; k < Nq; ++k)
          for (int j = 0; j < Nq; ++j)
            for (int i = 0; i < Nq; ++i) {
              int n = nidx(Nq, i, j, k);
              double X = m->x0 + (ex + 0.5 * (s->xi[i] + 1.0)) * hx;
              double Y = m->y0 + (ey + 0.5 * (s->xi[j] + 1.0)) * hy;
              double Z = m->z0 + (ez + 0.5 * (s->xi[k] + 1.0)) * hz;
              if (m->warp) Z = Z + surface_height(m, X) * (1.0 - (Z - m->z0) / m->Lz);
              s->x[(size_t)e * Np + n] = X;
              s->y[(size_t)e * Np + n] = Y;
              s->z[(size_t)e * Np + n] = Z;
            }
        /* neighbours; -1 marks a wall */
        int nb[6];
        nb[0] = ex > 0 ? e - 1 : (m->periodic_x ? e + (m->nex - 1) : -1);
        nb[1] = ex < m->nex - 1 ? e + 1 : (m->periodic_x ? e - (m->nex - 1) : -1);
        nb[2] = ey > 0 ? e - m->nex : (m->periodic_y ? e + m->nex * (m->ney - 1) : -1);
        nb[3] = ey < m->ney - 1 ? e + m->nex : (m->periodic_y ? e - m->nex * (m->ney - 1) : -1);
        int sl = m->nex * m->ney;
        nb[4] = ez > 0 ? e - sl : (m->periodic_z ? e + sl * (m->nez - 1) : -1);
        nb[5] = ez < m->nez - 1 ? e + sl : (m->periodic_z ? e - sl * (m->nez - 1) : -1);
        for (int f = 0; f < 6; ++f) s->EToE[e * 6 + f] = nb[f];
      }

  /* Metric terms (Eq. mapping).  dX_c/dxi_r by the LGL derivative matrix;
   * J = det(dX/dxi); J grad(xi_r) in the conservative curl form of Kopriva
   * (2006) (reading: the paper does not state how metrics are evaluated):
   *   (J a^r)_c = -[ curl_xi ( X_l grad_xi X_m ) ]_r,  (c, m, l) cyclic. */
  /* The curl form is invariant under translation of the coordinates (the
   * derivative operators along different directions commute), so the metric
   * terms are evaluated from element-local coordinates X - X(node 0), which
   * keeps their rounding independent of the element's distance from the
   * origin. */
  double *V = (double *)malloc((size_t)Np * 3 * sizeof(double));
  double *XL = (double *)malloc((size_t)Np * 3 * sizeof(double));
  for (int e = 0; e < E; ++e) {
    for (int c = 0; c < 3; ++c) {
      const double *Xa = (c == 0 ? s->x : (c == 1 ? s->y : s->z)) + (size_t)e * Np;
      for (int n = 0; n < Np; ++n) XL[c * Np + n] = Xa[n] - Xa[0];
    }
    const double *X[3] = {XL, XL + Np, XL + 2 * Np};
    double vol = 0.0;
    for (int n = 0; n < Np; ++n) {
      int ijk[3];
      node_ijk(Nq, n, ijk);
      double dX[3][3]; /* dX[c][r] = d X_c / d xi_r */
      for (int c = 0; c < 3; ++c)
        for (int r = 0; r < 3; ++r) {
          double acc = 0.0;
          for (int q = 0; q < Nq; ++q) acc += s->D[ijk[r] * Nq + q] * X[c][replace_idx(Nq, ijk, r, q)];
          dX[c][r] = acc;
        }
      double det = dX[0][0] * (dX[1][1] * dX[2][2] - dX[1][2] * dX[2][1]) -
                   dX[0][1] * (dX[1][0] * dX[2][2] - dX[1][2] * dX[2][0]) +
                   dX[0][2] * (dX[1][0] * dX[2][1] - dX[1][1] * dX[2][0]);
      s->J[(size_t)e * Np + n] = det;
      vol += s->w[ijk[0]] * s->w[ijk[1]] * s->w[ijk[2]] * det;
    }
    s->Delta[e] = cbrt(vol) / N;
    for (int c = 0; c < 3; ++c) {
      const double *Xa = (c == 0 ? s->x : (c == 1 ? s->y : s->z)) + (size_t)e * Np;
      double lo = Xa[0], hi = Xa[0];
      for (int n = 1; n < Np; ++n) {
        if (Xa[n] < lo) lo = Xa[n];
        if (Xa[n] > hi) hi = Xa[n];
      }
      s->Dm[e * 3 + c] = (hi - lo) / N;
    }
    for (int c = 0; c < 3; ++c) {
      int mm = (c + 1) % 3, ll = (c + 2) % 3;
      /* V_r = X_l * d X_m / d xi_r at every node */
      for (int n = 0; n < Np; ++n) {
        int ijk[3];
        node_ijk(Nq, n, ijk);
        for (int r = 0; r < 3; ++r) {
          double acc = 0.0;
          for (int q = 0; q < Nq; ++q) acc += s->D[ijk[r] * Nq + q] * X[mm][replace_idx(Nq, ijk, r, q)];
          V[n * 3 + r] = X[ll][n] * acc;
        }
      }
      for (int n = 0; n < Np; ++n) {
        int ijk[3];
        node_ijk(Nq, n, ijk);
        double curl0 = dvec(s, V, ijk, 2, 1) - dvec(s, V, ijk, 1, 2);
        double curl1 = dvec(s, V, ijk, 0, 2) - dvec(s, V, ijk, 2, 0);
        double curl2 = dvec(s, V, ijk, 1, 0) - dvec(s, V, ijk, 0, 1);
        double *ja = s->Ja + ((size_t)e * Np + n) * 9;
        ja[0 * 3 + c] = -curl0;
        ja[1 * 3 + c] = -curl1;
        ja[2 * 3 + c] = -curl2;
      }
    }
  }
  free(V);
  free(XL);

  /* Rayleigh sponge coefficient (Eq. sponge).  Reading of the garbled
   * profile: tau_s = alpha sin^gamma( pi/2 (z - z_s)/(z_top - z_s) ) above z_s;
   * the optional lateral layers use the same shape in x, and the largest of
   * the top and lateral values is taken. */
  double ztop = m->z0 + m->Lz;
  for (size_t q = 0; q < nn; ++q) {
    double t = 0.0;
    if (p->sponge_alpha > 0.0) {
      double zz = s->z[q];
      if (zz > p->sponge_zs) {
        double a = 0.5 * M_PI * (zz - p->sponge_zs) / (ztop - p->sponge_zs);
        t = p->sponge_alpha * pow(sin(a), p->sponge_gamma);
      }
      if (p->lateral_sponge_frac > 0.0) {
        double width = p->lateral_sponge_frac * m->Lx;
        double xl = m->x0 + width, xr = m->x0 + m->Lx - width;
        double xx = s->x[q], tl = 0.0;
        if (xx < xl) tl = p->sponge_alpha * pow(sin(0.5 * M_PI * (xl - xx) / width), p->sponge_gamma);
        if (xx > xr) tl = p->sponge_alpha * pow(sin(0.5 * M_PI * (xx - xr) / width), p->sponge_gamma);
        if (tl > t) t = tl;
      }
    }
    s->tau[q] = t;
  }
  return s;
}

void orc_destroy(orc_solver *s) {
  if (!s) return;
  free(s->x); free(s->y); free(s->z); free(s->J); free(s->Ja); free(s->Delta); free(s->Dm); free(s->EToE);
  free(s->rho_r); free(s->p_r); free(s->tau); free(s->qt_r);
  free(s->G); free(s->gradG); free(s->nut); free(s->Dt); free(s->F2); free(s->aux); free(s->Ftot);
  free(s);
}

int64_t orc_num_nodes(const orc_solver *s) { return (int64_t)s->E * s->Np; }
int orc_num_elements(const orc_solver *s) { return s->E; }

void orc_geometry(const orc_solver *s, double *x, double *y, double *z, double *J, double *wJ) {
  size_t nn = (size_t)s->E * s->Np;
  for (size_t q = 0; q < nn; ++q) {
    int n = (int)(q % s->Np), ijk[3];
    node_ijk(s->Nq, n, ijk);
    if (x) x[q] = s->x[q];
    if (y) y[q] = s->y[q];
    if (z) z[q] = s->z[q];
    if (J) J[q] = s->J[q];
    if (wJ) wJ[q] = s->w[ijk[0]] * s->w[ijk[1]] * s->w[ijk[2]] * s->J[q];
  }
}

void orc_set_reference(orc_solver *s, const double *rho_r, const double *p_r) {
  size_t nn = (size_t)s->E * s->Np;
  memcpy(s->rho_r, rho_r, nn * sizeof(double));
  memcpy(s->p_r, p_r, nn * sizeof(double));
}

void orc_set_reference_qt(orc_solver *s, const double *qt_r) {
  memcpy(s->qt_r, qt_r, (size_t)s->E * s->Np * sizeof(double));
}

void orc_set_mlp(orc_solver *s, const double *W1, const double *b1, const double *W2, const double *b2,
                 const double *W3, const double *b3, const double *in_scale, const double *out_scale) {
  memcpy(s->mlp_W1, W1, sizeof(s->mlp_W1));
  memcpy(s->mlp_b1, b1, sizeof(s->mlp_b1));
  memcpy(s->mlp_W2, W2, sizeof(s->mlp_W2));
  memcpy(s->mlp_b2, b2, sizeof(s->mlp_b2));
  memcpy(s->mlp_W3, W3, sizeof(s->mlp_W3));
  memcpy(s->mlp_b3, b3, sizeof(s->mlp_b3));
  memcpy(s->mlp_in, in_scale, sizeof(s->mlp_in));
  memcpy(s->mlp_out, out_scale, sizeof(s->mlp_out));
  s->has_mlp = 1;
}

/* outward unit normal and surface Jacobian J_s = |J grad xi_d| at a face node */
static void face_normal(const orc_solver *s, int e, int n, int d, int side, double nrm[3], double *Js) {
  const double *ja = s->Ja + ((size_t)e * s->Np + n) * 9 + d * 3;
  double mag = sqrt(ja[0] * ja[0] + ja[1] * ja[1] + ja[2] * ja[2]);
  double sg = side ? 1.0 : -1.0;
  for (int c = 0; c < 3; ++c) nrm[c] = sg * ja[c] / mag;
  *Js = mag;
}

/* Reflecting wall state (Eq. bc-velocity-impenetrable):
 * u+ = u- - 2 (n.u-) n, scalars copied (homogeneous Neumann reading of
 * Eq. bc-general_tracer). */
static void wall_ghost(const double Ym[6], const double nrm[3], int noslip, double Yp[6]) {
  /* u+ = 2 u_bc - u- (Eq. bc-velocity-impenetrable): u_bc = u- - (n.u-) n
   * reflects the normal component; no-slip, u_bc = 0, reverses all three */
  double mn = Ym[1] * nrm[0] + Ym[2] * nrm[1] + Ym[3] * nrm[2];
  Yp[0] = Ym[0];
  for (int c = 0; c < 3; ++c) Yp[1 + c] = noslip ? -Ym[1 + c] : Ym[1 + c] - 2.0 * mn * nrm[c];
  Yp[4] = Ym[4];
  Yp[5] = Ym[5];
}

/* ------------------------------------------------------------------ RHS */

int orc_rhs(orc_solver *s, const double *Q, double *RHS, int form) {
  const orc_params *P = &s->p;
  const int N = s->N, Nq = s->Nq, Np = s->Np, E = s->E;
  int fails = 0;

  /* 1. pointwise thermodynamics: G = (u, v, w, h_tot, q_t, theta_v) and
   *    aux = (p - p_r, c, T, q_l) at every node. */
#pragma omp parallel for reduction(+ : fails) schedule(static)
  for (int e = 0; e < E; ++e)
    for (int n = 0; n < Np; ++n) {
      size_t q = (size_t)e * Np + n;
      double Y[6];
      for (int v = 0; v < 6; ++v) Y[v] = Q[((size_t)e * 6 + v) * Np + n];
      orc_thermo_state st;
      if (orc_thermo(P, Y, s->z[q], &st) != 0) fails++;
      double *G = s->G + (size_t)e * 6 * Np;
      G[0 * Np + n] = st.u[0];
      G[1 * Np + n] = st.u[1];
      G[2 * Np + n] = st.u[2];
      G[3 * Np + n] = st.htot;
      G[4 * Np + n] = st.qt;
      G[5 * Np + n] = st.thetav;
      double *A = s->aux + (size_t)e * 4 * Np;
      A[0 * Np + n] = st.p - s->p_r[q];
      A[1 * Np + n] = st.c;
      A[2 * Np + n] = st.T;
      A[3 * Np + n] = st.ql;
    }

  /* 2. BR1 auxiliary gradient (Sec. 3.1, strong form):
   *    grad G_i = (1/J_i) sum_r (J a^r)_i sum_m D_{i_r m} G_m
   *             + (w_s J_s)/(w_i J_i) n (G* - G-),  G* = (G- + G+)/2. */
#pragma omp parallel for schedule(static)
  for (int e = 0; e < E; ++e) {
    const double *G = s->G + (size_t)e * 6 * Np;
    double *gG = s->gradG + (size_t)e * 18 * Np;
    for (int n = 0; n < Np; ++n) {
      int ijk[3];
      node_ijk(Nq, n, ijk);
      size_t q = (size_t)e * Np + n;
      const double *ja = s->Ja + q * 9;
      for (int v = 0; v < 6; ++v) {
        double dxi[3];
        for (int r = 0; r < 3; ++r) {
          double acc = 0.0;
          for (int m = 0; m < Nq; ++m) acc += s->D[ijk[r] * Nq + m] * G[v * Np + replace_idx(Nq, ijk, r, m)];
          dxi[r] = acc;
        }
        for (int c = 0; c < 3; ++c) {
          double acc = 0.0;
          for (int r = 0; r < 3; ++r) acc += ja[r * 3 + c] * dxi[r];
          gG[(v * 3 + c) * Np + n] = acc / s->J[q];
        }
      }
    }
    for (int f = 0; f < 6; ++f) {
      int d = f / 2, side = f % 2, a = side ? N : 0;
      int nb = s->EToE[e * 6 + f];
      for (int t2 = 0; t2 < Nq; ++t2)
        for (int t1 = 0; t1 < Nq; ++t1) {
          int n = face_node(Nq, d, a, t1, t2);
          double nrm[3], Js;
          face_normal(s, e, n, d, side, nrm, &Js);
          double Gm[6], Gp[6];
          for (int v = 0; v < 6; ++v) Gm[v] = G[v * Np + n];
          if (nb >= 0) {
            int np = face_node(Nq, d, N - a, t1, t2);
            for (int v = 0; v < 6; ++v) Gp[v] = s->G[((size_t)nb * 6 + v) * Np + np];
          } else {
            /* the wall ghost of the velocity as in the flux pass (reflected
             * normal component, or reversed at a no-slip wall); scalars
             * copied */
            double un = Gm[0] * nrm[0] + Gm[1] * nrm[1] + Gm[2] * nrm[2];
            const int ns = (P->noslip >> f) & 1;
            for (int c = 0; c < 3; ++c) Gp[c] = ns ? -Gm[c] : Gm[c] - 2.0 * un * nrm[c];
            for (int v = 3; v < 6; ++v) Gp[v] = Gm[v];
          }
          double lift = Js / (s->w[a] * s->J[(size_t)e * Np + n]);
          for (int v = 0; v < 6; ++v) {
            double jump = 0.5 * (Gm[v] + Gp[v]) - Gm[v];
            for (int c = 0; c < 3; ++c) gG[(v * 3 + c) * Np + n] += lift * nrm[c] * jump;
          }
        }
    }
  }

  /* 3. closure and diffusive fluxes F2 (Sec. 4):
   *    d_qt = -D_t grad q_t (Eq. diff_moisture_flux), rho tau = -2 rho nu_t S
   *    (Eq. stress_tensor), rho (J + D) = -rho D_t grad h_tot
   *    (Eq. diff_energy_flux), D_t = nu_t / Pr_t (Eq. Diffusivity).
   *    Row i of F2 (flux in direction i): [rho d_i, rho tau_i. + d_i rho u_.,
   *    rho (J+D)_i + (rho tau u)_i]; the mass equation carries rho d_qt too. */
#pragma omp parallel for schedule(static)
  for (int e = 0; e < E; ++e)
    for (int n = 0; n < Np; ++n) {
      size_t q = (size_t)e * Np + n;
      const double *gG = s->gradG + (size_t)e * 18 * Np;
      double gu[9];
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) gu[3 * i + j] = gG[(i * 3 + j) * Np + n];
      double gh[3], gq[3], gth[3];
      for (int c = 0; c < 3; ++c) {
        gh[c] = gG[(3 * 3 + c) * Np + n];
        gq[c] = gG[(4 * 3 + c) * Np + n];
        gth[c] = gG[(5 * 3 + c) * Np + n];
      }
      double thv = s->G[((size_t)e * 6 + 5) * Np + n];
      double nut = 0.0, Dt = 0.0;
      if (P->closure == ORC_CLOSURE_SL) {
        nut = orc_smagorinsky(P, gu, gth[2], thv, s->Delta[e]);
        Dt = nut / P->Prt;
      } else if (P->closure == ORC_CLOSURE_VREMAN) {
        nut = orc_vreman(P, gu, gth[2], thv, s->Dm + (size_t)e * 3);
        Dt = nut / P->Prt;
      } else if (P->closure == ORC_CLOSURE_MLP && s->has_mlp) {
        double xin[13], yout[2];
        for (int k = 0; k < 9; ++k) xin[k] = gu[k] * s->mlp_in[k];
        for (int k = 0; k < 3; ++k) xin[9 + k] = gth[k] * s->mlp_in[9 + k];
        xin[12] = s->Delta[e] * s->mlp_in[12];
        orc_mlp_forward_bf16(1, xin, s->mlp_W1, s->mlp_b1, s->mlp_W2, s->mlp_b2, s->mlp_W3, s->mlp_b3, yout);
        nut = (yout[0] > 0.0 ? yout[0] : 0.0) * s->mlp_out[0];
        Dt = (yout[1] > 0.0 ? yout[1] : 0.0) * s->mlp_out[1];
      }
      s->nut[q] = nut;
      s->Dt[q] = Dt;
      double rho = Q[((size_t)e * 6 + 0) * Np + n];
      double rhou[3] = {Q[((size_t)e * 6 + 1) * Np + n], Q[((size_t)e * 6 + 2) * Np + n],
                        Q[((size_t)e * 6 + 3) * Np + n]};
      double u[3] = {s->G[((size_t)e * 6 + 0) * Np + n], s->G[((size_t)e * 6 + 1) * Np + n],
                     s->G[((size_t)e * 6 + 2) * Np + n]};
      double *F2 = s->F2 + (size_t)e * 15 * Np;
      for (int i = 0; i < 3; ++i) {
        double di = -Dt * gq[i];
        double rtau[3];
        for (int j = 0; j < 3; ++j) rtau[j] = -2.0 * rho * nut * 0.5 * (gu[3 * i + j] + gu[3 * j + i]);
        F2[(i * 5 + 0) * Np + n] = rho * di;
        for (int j = 0; j < 3; ++j) F2[(i * 5 + 1 + j) * Np + n] = rtau[j] + di * rhou[j];
        F2[(i * 5 + 4) * Np + n] = -rho * Dt * gh[i] + (rtau[0] * u[0] + rtau[1] * u[1] + rtau[2] * u[2]);
      }
    }

  /* 4. total flux F = F1 + F2 at every node, Ftot[e][v][c][n]. */
#pragma omp parallel for schedule(static)
  for (int e = 0; e < E; ++e)
    for (int n = 0; n < Np; ++n) {
      size_t q = (size_t)e * Np + n;
      double Y[6];
      for (int v = 0; v < 6; ++v) Y[v] = Q[((size_t)e * 6 + v) * Np + n];
      double pp = s->aux[((size_t)e * 4 + 0) * Np + n] + s->p_r[q];
      double pprime = s->aux[((size_t)e * 4 + 0) * Np + n];
      const double *F2 = s->F2 + (size_t)e * 15 * Np;
      double *Ft = s->Ftot + (size_t)e * 18 * Np;
      double u[3] = {Y[1] / Y[0], Y[2] / Y[0], Y[3] / Y[0]};
      for (int c = 0; c < 3; ++c) {
        double f[6];
        f[0] = Y[1 + c];
        for (int j = 0; j < 3; ++j) f[1 + j] = Y[1 + j] * u[c] + (j == c ? pprime : 0.0);
        f[4] = (Y[4] + pp) * u[c];
        f[5] = Y[5] * u[c];
        f[0] += F2[(c * 5 + 0) * Np + n];
        for (int j = 0; j < 3; ++j) f[1 + j] += F2[(c * 5 + 1 + j) * Np + n];
        f[4] += F2[(c * 5 + 4) * Np + n];
        f[5] += F2[(c * 5 + 0) * Np + n];
        for (int v = 0; v < 6; ++v) Ft[(v * 3 + c) * Np + n] = f[v];
      }
    }

  /* 5. volume term of Eq. matrixProblem and the surface lift, then sources. */
  double ztop = s->m.z0 + s->m.Lz;
  (void)ztop;
#pragma omp parallel for schedule(static)
  for (int e = 0; e < E; ++e) {
    const double *Ft = s->Ftot + (size_t)e * 18 * Np;
    double *R = RHS + (size_t)e * 6 * Np;
    for (int n = 0; n < Np; ++n) {
      int ijk[3];
      node_ijk(Nq, n, ijk);
      size_t q = (size_t)e * Np + n;
      for (int v = 0; v < 6; ++v) {
        double div = 0.0;
        for (int r = 0; r < 3; ++r) {
          double acc = 0.0;
          for (int m = 0; m < Nq; ++m) {
            int nm = replace_idx(Nq, ijk, r, m);
            const double *ja = s->Ja + ((size_t)e * Np + nm) * 9 + r * 3;
            double fhat = ja[0] * Ft[(v * 3 + 0) * Np + nm] + ja[1] * Ft[(v * 3 + 1) * Np + nm] +
                          ja[2] * Ft[(v * 3 + 2) * Np + nm];
            if (form == 0)
              acc += s->D[ijk[r] * Nq + m] * fhat;
            else /* weak form: (1/(w_i J_i)) sum_m w_m D_{m i} fhat_m along the line */
              acc -= s->w[m] / s->w[ijk[r]] * s->D[m * Nq + ijk[r]] * fhat;
          }
          div += acc;
        }
        R[v * Np + n] = -div / s->J[q];
      }
    }
    /* surface terms */
    for (int f = 0; f < 6; ++f) {
      int d = f / 2, side = f % 2, a = side ? N : 0;
      int nb = s->EToE[e * 6 + f];
      for (int t2 = 0; t2 < Nq; ++t2)
        for (int t1 = 0; t1 < Nq; ++t1) {
          int n = face_node(Nq, d, a, t1, t2);
          size_t q = (size_t)e * Np + n;
          double nrm[3], Js;
          face_normal(s, e, n, d, side, nrm, &Js);
          double Ym[6], Yp[6], Fm[6], F1s[6], F2s[6];
          for (int v = 0; v < 6; ++v) Ym[v] = Q[((size_t)e * 6 + v) * Np + n];
          for (int v = 0; v < 6; ++v)
            Fm[v] = nrm[0] * Ft[(v * 3 + 0) * Np + n] + nrm[1] * Ft[(v * 3 + 1) * Np + n] +
                    nrm[2] * Ft[(v * 3 + 2) * Np + n];
          const double *F2m = s->F2 + (size_t)e * 15 * Np;
          double f2m[5];
          for (int k = 0; k < 5; ++k)
            f2m[k] = nrm[0] * F2m[(0 * 5 + k) * Np + n] + nrm[1] * F2m[(1 * 5 + k) * Np + n] +
                     nrm[2] * F2m[(2 * 5 + k) * Np + n];
          double f2s[5];
          if (nb >= 0) {
            int np = face_node(Nq, d, N - a, t1, t2);
            for (int v = 0; v < 6; ++v) Yp[v] = Q[((size_t)nb * 6 + v) * Np + np];
            const double *F2p = s->F2 + (size_t)nb * 15 * Np;
            for (int k = 0; k < 5; ++k) {
              double f2p = nrm[0] * F2p[(0 * 5 + k) * Np + np] + nrm[1] * F2p[(1 * 5 + k) * Np + np] +
                           nrm[2] * F2p[(2 * 5 + k) * Np + np];
              f2s[k] = 0.5 * (f2m[k] + f2p);  /* central flux for F2 (BR1) */
            }
          } else {
            wall_ghost(Ym, nrm, (P->noslip >> f) & 1, Yp);
            /* Wall-normal diffusive fluxes are specified directly (App. A.3):
             * zero at free-slip, insulated, impermeable walls; at the bottom
             * with prescribed surface fluxes, the upward energy flux is
             * SHF + LHF and the upward water (and mass) flux LHF / L_v0. */
            for (int k = 0; k < 5; ++k) f2s[k] = 0.0;
            if (d == 2 && side == 0 && P->surface_flux) {
              double E_w = P->lhf / P->Lv0;
              /* outward normal points down: n.F = -(upward flux) */
              f2s[0] = -E_w * (-nrm[2]);
              f2s[4] = -(P->shf + P->lhf) * (-nrm[2]);
            }
            if (d == 2 && side == 0 && P->drag_cd > 0.0) {
              /* Aerodynamic drag law (Eq. drag_law): with n the inward
               * normal, n.(rho tau) = -rho C_d |u_p| u_p, u_p the
               * wall-parallel velocity at the interior point, read as the
               * node of the first interior layer (k = 1) above this face
               * node, and rho the density at the wall node.  The outward
               * normal is -n, so n_out.(rho tau) = +rho C_d |u_p| u_p.  The
               * energy flux is unchanged (its kinetic part is neglected). */
              int ni = face_node(Nq, 2, 1, t1, t2);
              double ui[3], un = 0.0, up2 = 0.0;
              for (int c = 0; c < 3; ++c) {
                ui[c] = Q[((size_t)e * 6 + 1 + c) * Np + ni] / Q[((size_t)e * 6 + 0) * Np + ni];
                un += ui[c] * nrm[c];
              }
              for (int c = 0; c < 3; ++c) {
                ui[c] -= un * nrm[c];
                up2 += ui[c] * ui[c];
              }
              double drag = Ym[0] * P->drag_cd * sqrt(up2);
              for (int c = 0; c < 3; ++c) f2s[1 + c] = drag * ui[c];
            }
          }
          if (P->flux == ORC_FLUX_HLLC)
            orc_hllc(P, Ym, Yp, s->z[q], s->p_r[q], nrm, F1s);
          else if (P->flux == ORC_FLUX_ROE)
            orc_roe(P, Ym, Yp, s->z[q], s->p_r[q], nrm, F1s);
          else
            orc_rusanov(P, Ym, Yp, s->z[q], s->p_r[q], nrm, F1s);
          F2s[0] = f2s[0];
          F2s[1] = f2s[1];
          F2s[2] = f2s[2];
          F2s[3] = f2s[3];
          F2s[4] = f2s[4];
          F2s[5] = f2s[0];
          double lift = Js / (s->w[a] * s->J[q]);
          for (int v = 0; v < 6; ++v) {
            double fstar = F1s[v] + F2s[v];
            if (form == 0)
              R[v * Np + n] += lift * (Fm[v] - fstar);
            else
              R[v * Np + n] -= lift * fstar;
          }
        }
    }
    /* sources (Eq. momentum, Eq. sponge): -(rho - rho_r) g k,
     * -tau_s (rho u - rho u_relax), -2 Omega x rho u. */
    for (int n = 0; n < Np; ++n) {
      size_t q = (size_t)e * Np + n;
      double rho = Q[((size_t)e * 6 + 0) * Np + n];
      double m[3] = {Q[((size_t)e * 6 + 1) * Np + n], Q[((size_t)e * 6 + 2) * Np + n],
                     Q[((size_t)e * 6 + 3) * Np + n]};
      double S[3] = {0.0, 0.0, 0.0};
      S[2] -= (rho - s->rho_r[q]) * P->g;
      for (int c = 0; c < 3; ++c) S[c] -= s->tau[q] * (m[c] - rho * P->u_relax[c]);
      S[0] -= 2.0 * (P->Omega[1] * m[2] - P->Omega[2] * m[1]);
      S[1] -= 2.0 * (P->Omega[2] * m[0] - P->Omega[0] * m[2]);
      S[2] -= 2.0 * (P->Omega[0] * m[1] - P->Omega[1] * m[0]);
      for (int c = 0; c < 3; ++c) R[(1 + c) * Np + n] += S[c];
    }
  }
  return fails;
}

void orc_intermediates(const orc_solver *s, double *G, double *gradG, double *nut, double *F2, double *aux) {
  size_t nn = (size_t)s->E * s->Np;
  if (G) memcpy(G, s->G, nn * 6 * sizeof(double));
  if (gradG) memcpy(gradG, s->gradG, nn * 18 * sizeof(double));
  if (nut) memcpy(nut, s->nut, nn * sizeof(double));
  if (F2) memcpy(F2, s->F2, nn * 15 * sizeof(double));
  if (aux) memcpy(aux, s->aux, nn * 4 * sizeof(double));
}

/* ------------------------------------------------------------------ LSRK */

/* Five-stage fourth-order 2N-storage coefficients of Carpenter & Kennedy
 * (1994), cited in Sec. 3.2:  dQ <- A_s dQ + dt RHS(Q);  Q <- Q + B_s dQ. */
void orc_lsrk54_coefficients(double A[5], double B[5], double c[5]) {
  A[0] = 0.0;
  A[1] = -567301805773.0 / 1357537059087.0;
  A[2] = -2404267990393.0 / 2016746695238.0;
  A[3] = -3550918686646.0 / 2091501179385.0;
  A[4] = -1275806237668.0 / 842570457699.0;
  B[0] = 1432997174477.0 / 9575080441755.0;
  B[1] = 5161836677717.0 / 13612068292357.0;
  B[2] = 1720146321549.0 / 2090206949498.0;
  B[3] = 3134564353537.0 / 4481467310338.0;
  B[4] = 2277821191437.0 / 14882151754819.0;
  c[0] = 0.0;
  c[1] = 1432997174477.0 / 9575080441755.0;
  c[2] = 2526269341429.0 / 6820363962896.0;
  c[3] = 2006345519317.0 / 3224310063776.0;
  c[4] = 2802321613138.0 / 2924317926251.0;
}

/* Fourteen-stage fourth-order 2N-storage coefficients of Niegemann, Diehl &
 * Busch (2012), the integrator Sec. 3.2 names for the isotropic benchmarks
 * (a large real-axis stability interval, about [-18.5, 0]). */
void orc_lsrk144_coefficients(double A[14], double B[14], double c[14]) {
  static const double a[14] = {0.0,
                               -0.7188012108672410,
                               -0.7785331173421570,
                               -0.0053282796654044,
                               -0.8552979934029281,
                               -3.9564138245774565,
                               -1.5780575380587385,
                               -2.0837094552574054,
                               -0.7483334182761610,
                               -0.7032861106563359,
                               0.0013917096117681,
                               -0.0932075369637460,
                               -0.9514200470875948,
                               -7.1151571693922548};
  static const double b[14] = {0.0367762454319673, 0.3136296607553959, 0.1531848691869027, 0.0030097086818182,
                               0.3326293790646110, 0.2440251405350864, 0.3718879239592277, 0.6204126221582444,
                               0.1524043173028741, 0.0760894927419266, 0.0077604214040978, 0.0024647284755382,
                               0.0780348340049386, 5.5059777270269628};
  static const double cc[14] = {0.0, 0.0367762454319673, 0.1249685262725025, 0.2446177702277698,
                                0.2476149531070420, 0.2969311120382472, 0.3978149645802642, 0.5270854589440328,
                                0.6981269994175695, 0.8190890835352128, 0.8527059887098624, 0.8604711817462826,
                                0.8627060376969976, 0.8734213127600976};
  for (int k = 0; k < 14; ++k) {
    A[k] = a[k];
    B[k] = b[k];
    c[k] = cc[k];
  }
}

/* nsteps steps of a 2N-storage scheme with S stages (Sec. 3.2):
 * per stage dQ <- A_s dQ + dt RHS(Q), Q <- Q + B_s dQ. */
static int lsrk_2n(orc_solver *s, double *Q, int nsteps, double dt, const double *A, const double *B, int S) {
  size_t n6 = (size_t)s->E * s->Np * 6;
  double *dQ = (double *)calloc(n6, sizeof(double));
  double *R = (double *)malloc(n6 * sizeof(double));
  int fails = 0;
  for (int st = 0; st < nsteps; ++st)
    for (int k = 0; k < S; ++k) {
      fails += orc_rhs(s, Q, R, 0);
      for (size_t q = 0; q < n6; ++q) {
        dQ[q] = A[k] * dQ[q] + dt * R[q];
        Q[q] = Q[q] + B[k] * dQ[q];
      }
    }
  free(dQ);
  free(R);
  return fails;
}

int orc_lsrk54(orc_solver *s, double *Q, int nsteps, double dt) {
  double A[5], B[5], c[5];
  orc_lsrk54_coefficients(A, B, c);
  return lsrk_2n(s, Q, nsteps, dt, A, B, 5);
}

int orc_lsrk144(orc_solver *s, double *Q, int nsteps, double dt) {
  double A[14], B[14], c[14];
  orc_lsrk144_coefficients(A, B, c);
  return lsrk_2n(s, Q, nsteps, dt, A, B, 14);
}

/* ------------------------------------------------------------ diagnostics */

/* Domain integrals by LGL quadrature (the integrals of Sec. 6). */
int orc_budgets(const orc_solver *s, const double *Q, double out[6]) {
  const int Np = s->Np, Nq = s->Nq;
  for (int v = 0; v < 6; ++v) out[v] = 0.0;
  int bad = 0;
  for (int e = 0; e < s->E; ++e)
    for (int n = 0; n < Np; ++n) {
      int ijk[3];
      node_ijk(Nq, n, ijk);
      double wJ = s->w[ijk[0]] * s->w[ijk[1]] * s->w[ijk[2]] * s->J[(size_t)e * Np + n];
      for (int v = 0; v < 6; ++v) {
        double val = Q[((size_t)e * 6 + v) * Np + n];
        if (!isfinite(val)) bad = 1;
        out[v] += wJ * val;
      }
    }
  return bad;
}

/* Favre (density-weighted) horizontal means per node level (App. C):
 * phi_bar = <rho phi>/<rho>, variances and vertical eddy fluxes
 * <rho w' phi'>/<rho>, with <.> the horizontal quadrature mean at a level. */
void orc_favre_profiles(const orc_solver *s, const double *Q, double *out) {
  const int Np = s->Np, Nq = s->Nq, nl = s->m.nez * Nq;
  const orc_params *P = &s->p;
  double cpd = P->cvd + P->Rd;
  double *acc = (double *)calloc((size_t)nl * 8, sizeof(double));
  /* pass 1: <1>, <rho>, <rho theta>, <rho qt>, <rho ql>, <rho u>, <rho v>, <rho w>, and theta_l */
  double *tl = (double *)calloc((size_t)nl, sizeof(double));
  for (int e = 0; e < s->E; ++e) {
    int ez = e / (s->m.nex * s->m.ney);
    for (int n = 0; n < Np; ++n) {
      int ijk[3];
      node_ijk(Nq, n, ijk);
      int lev = ez * Nq + ijk[2];
      double wh = s->w[ijk[0]] * s->w[ijk[1]];
      double Y[6];
      for (int v = 0; v < 6; ++v) Y[v] = Q[((size_t)e * 6 + v) * Np + n];
      orc_thermo_state st;
      orc_thermo(P, Y, s->z[(size_t)e * Np + n], &st);
      double thl = st.theta * (1.0 - P->Lv0 * st.ql / (cpd * st.T));
      double *a = acc + (size_t)lev * 8;
      a[0] += wh;
      a[1] += wh * st.rho;
      a[2] += wh * st.rho * st.theta;
      a[3] += wh * st.rho * st.qt;
      a[4] += wh * st.rho * st.ql;
      a[5] += wh * st.rho * st.u[0];
      a[6] += wh * st.rho * st.u[1];
      a[7] += wh * st.rho * st.u[2];
      tl[lev] += wh * st.rho * thl;
    }
  }
  double *acc2 = (double *)calloc((size_t)nl * 3, sizeof(double));
  for (int e = 0; e < s->E; ++e) {
    int ez = e / (s->m.nex * s->m.ney);
    for (int n = 0; n < Np; ++n) {
      int ijk[3];
      node_ijk(Nq, n, ijk);
      int lev = ez * Nq + ijk[2];
      double wh = s->w[ijk[0]] * s->w[ijk[1]];
      double Y[6];
      for (int v = 0; v < 6; ++v) Y[v] = Q[((size_t)e * 6 + v) * Np + n];
      orc_thermo_state st;
      orc_thermo(P, Y, s->z[(size_t)e * Np + n], &st);
      double *a = acc + (size_t)lev * 8;
      double wbar = a[7] / a[1], thbar = a[2] / a[1], qbar = a[3] / a[1];
      double wp = st.u[2] - wbar;
      acc2[lev * 3 + 0] += wh * st.rho * wp * wp;
      acc2[lev * 3 + 1] += wh * st.rho * wp * (st.theta - thbar);
      acc2[lev * 3 + 2] += wh * st.rho * wp * (st.qt - qbar);
    }
  }
  for (int l = 0; l < nl; ++l) {
    double *a = acc + (size_t)l * 8, *o = out + (size_t)l * 11;
    o[0] = a[1] / a[0];
    o[1] = a[2] / a[1];
    o[2] = a[3] / a[1];
    o[3] = a[4] / a[1];
    o[4] = a[5] / a[1];
    o[5] = a[6] / a[1];
    o[6] = a[7] / a[1];
    o[7] = acc2[l * 3 + 0] / a[1];
    o[8] = acc2[l * 3 + 1] / a[1];
    o[9] = acc2[l * 3 + 2] / a[1];
    o[10] = tl[l] / a[1];
  }
  free(acc);
  free(acc2);
  free(tl);
}
