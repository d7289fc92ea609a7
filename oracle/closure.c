/*
 * The oracle of the learned closure's training samples.  Test
 * infrastructure only (see oracle.h).
 *
 * The paper has no learned closure.  Its extension of Sec. 4 is trained on
 * fine-resolution runs of the plain method, filtered onto a coarser mesh.  The
 * definitions below are readings, stated where they are used:
 *
 *  1. Primitive fields at every fine node: the velocity u_i and the virtual
 *     potential temperature theta_v of the node's thermodynamic state (Sec. 2,
 *     orc_thermo).
 *  2. Fine-node derivatives d_j f: the element-local LGL derivative,
 *     (2 / h_j) sum_m D_{a m} f_m along each line (Eq. basisDerivatives on a
 *     box element; no face term).
 *  3. The filter: a top-hat of width Delta_c = H_d / N in each direction
 *     (H_d the coarse element length, so Delta_c is the coarse node
 *     spacing), centred on a coarse node x_c.  The filtered value <f> is the
 *     average of f over every fine node (every element's own copy, so a node
 *     on a shared face counts once per element) whose distance to x_c is at
 *     most Delta_c / 2 in each direction, weighted by its LGL quadrature
 *     weight w_a w_b w_c.  A distance within 1e-9 of Delta_c / 2 (relative)
 *     counts as inside.  Periodic directions measure the distance to the
 *     nearest periodic image; across a wall the box is cut off.
 *  4. From the filtered moments:
 *       tau_ij   = <u_i u_j> - <u_i><u_j>          (subgrid stress)
 *       tau_th,j = <u_j theta_v> - <u_j><theta_v>  (subgrid theta_v flux)
 *       S_ij     = (<d_j u_i> + <d_i u_j>) / 2,   g_j = <d_j theta_v>
 *     and the least-squares eddy viscosity and diffusivity
 *       nu*    = max(0, -tau:S / (2 S:S))         (0 when S:S = 0)
 *       kappa* = max(0, -tau_th.g / |g|^2)        (0 when |g| = 0),
 *     the minimisers of |tau + 2 nu S|^2 and |tau_th + kappa g|^2.
 *  5. The network inputs: X[3i + j] = <d_j u_i>, X[9 + j] = g_j and
 *     X[12] = Delta = (H_x H_y H_z)^(1/3) / N, the filter width of a coarse
 *     element (the Delta of Sec. 4.1 on the coarse mesh).
 *
 * The coarse mesh has nex/factor x ney/factor x nez/factor elements of the
 * same order N over the same box; samples are ordered coarse element-major,
 * node-minor, like a state.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"
#include "oracle_internal.h"

void orc_closure_primitives(const orc_solver *s, const double *Q, double *prim) {
  const int Np = s->Np;
#pragma omp parallel for schedule(static)
  for (int e = 0; e < s->E; ++e)
    for (int n = 0; n < Np; ++n) {
      double Y[6];
      for (int v = 0; v < 6; ++v) Y[v] = Q[((size_t)e * 6 + v) * Np + n];
      orc_thermo_state th;
      orc_thermo(&s->p, Y, s->z[(size_t)e * Np + n], &th);
      double *o = prim + (size_t)e * 4 * Np + n;
      o[0] = th.u[0];
      o[Np] = th.u[1];
      o[2 * Np] = th.u[2];
      o[3 * Np] = th.thetav;
    }
}

/* One direction of the filter box: the fine (element, node) pairs along that
 * axis whose position lies within the half-width b of xc, with their 1-D
 * weights.  Returns how many were found (at most cap). */
static int box_1d(const orc_solver *s, int d, double xc, double b, int *elem, int *node, double *wt, int cap) {
  const int nel = d == 0 ? s->m.nex : (d == 1 ? s->m.ney : s->m.nez);
  const double L = d == 0 ? s->m.Lx : (d == 1 ? s->m.Ly : s->m.Lz);
  const double x0 = d == 0 ? s->m.x0 : (d == 1 ? s->m.y0 : s->m.z0);
  const int periodic = d == 0 ? s->m.periodic_x : (d == 1 ? s->m.periodic_y : s->m.periodic_z);
  const double h = L / nel;
  int cnt = 0;
  for (int f = 0; f < nel; ++f)
    for (int a = 0; a < s->Nq; ++a) {
      const double x = x0 + (f + 0.5 * (s->xi[a] + 1.0)) * h;
      double dist = x - xc;
      if (periodic) dist -= L * floor(dist / L + 0.5); /* nearest periodic image */
      if (fabs(dist) <= b * (1.0 + 1e-9) && cnt < cap) {
        elem[cnt] = f;
        node[cnt] = a;
        wt[cnt] = s->w[a];
        ++cnt;
      }
    }
  return cnt;
}

long long orc_closure_samples(const orc_solver *s, const double *prim, int factor, double *X, double *T,
                              double *thv_bar) {
  const int N = s->N, Nq = s->Nq, Np = s->Np;
  const orc_mesh *m = &s->m;
  if (factor < 1 || m->nex % factor || m->ney % factor || m->nez % factor || m->warp) return -1;
  const int cn[3] = {m->nex / factor, m->ney / factor, m->nez / factor};
  const double h[3] = {m->Lx / m->nex, m->Ly / m->ney, m->Lz / m->nez};
  const double H[3] = {factor * h[0], factor * h[1], factor * h[2]};
  const double org[3] = {m->x0, m->y0, m->z0};
  const double Delta_c = cbrt(H[0] * H[1] * H[2]) / N;
  const long long nce = (long long)cn[0] * cn[1] * cn[2];

  /* step 2: element-local derivatives of the four primitive fields at every
   * fine node, dprim[e][f][j][n] = d_j f */
  double *dprim = (double *)malloc((size_t)s->E * 12 * Np * sizeof(double));
#pragma omp parallel for schedule(static)
  for (int e = 0; e < s->E; ++e)
    for (int n = 0; n < Np; ++n) {
      const int ijk[3] = {n % Nq, (n / Nq) % Nq, n / (Nq * Nq)};
      for (int f = 0; f < 4; ++f)
        for (int j = 0; j < 3; ++j) {
          double acc = 0.0;
          for (int q = 0; q < Nq; ++q) {
            int t[3] = {ijk[0], ijk[1], ijk[2]};
            t[j] = q;
            acc += s->D[ijk[j] * Nq + q] * prim[((size_t)e * 4 + f) * Np + t[0] + Nq * (t[1] + Nq * t[2])];
          }
          dprim[(((size_t)e * 4 + f) * 3 + j) * Np + n] = 2.0 / h[j] * acc;
        }
    }

  const int cap = 4 * Nq * (m->nex + m->ney + m->nez);
#pragma omp parallel
  {
    int *el[3], *nd[3];
    double *wt[3];
    for (int d = 0; d < 3; ++d) {
      el[d] = (int *)malloc(cap * sizeof(int));
      nd[d] = (int *)malloc(cap * sizeof(int));
      wt[d] = (double *)malloc(cap * sizeof(double));
    }
#pragma omp for schedule(dynamic, 4)
    for (long long ce = 0; ce < nce; ++ce) {
      const int cidx[3] = {(int)(ce % cn[0]), (int)((ce / cn[0]) % cn[1]), (int)(ce / ((long long)cn[0] * cn[1]))};
      for (int n = 0; n < Np; ++n) {
        const int nidx[3] = {n % Nq, (n / Nq) % Nq, n / (Nq * Nq)};
        /* step 3: the box around the coarse node, one axis at a time */
        int cnt[3];
        for (int d = 0; d < 3; ++d) {
          const double xc = org[d] + (cidx[d] + 0.5 * (s->xi[nidx[d]] + 1.0)) * H[d];
          cnt[d] = box_1d(s, d, xc, 0.5 * H[d] / N, el[d], nd[d], wt[d], cap);
        }
        double W = 0.0, mu[3] = {0, 0, 0}, muu[3][3] = {{0}}, mth = 0.0, muth[3] = {0, 0, 0};
        double mdu[3][3] = {{0}}, mdth[3] = {0, 0, 0};
        for (int c = 0; c < cnt[2]; ++c)
          for (int b = 0; b < cnt[1]; ++b)
            for (int a = 0; a < cnt[0]; ++a) {
              const long long fe = el[0][a] + (long long)m->nex * (el[1][b] + (long long)m->ney * el[2][c]);
              const int fn = nd[0][a] + Nq * (nd[1][b] + Nq * nd[2][c]);
              const double w = wt[0][a] * wt[1][b] * wt[2][c];
              double u[3], th, du[3][3], dth[3];
              for (int i = 0; i < 3; ++i) u[i] = prim[((size_t)fe * 4 + i) * Np + fn];
              th = prim[((size_t)fe * 4 + 3) * Np + fn];
              for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) du[i][j] = dprim[(((size_t)fe * 4 + i) * 3 + j) * Np + fn];
              for (int j = 0; j < 3; ++j) dth[j] = dprim[(((size_t)fe * 4 + 3) * 3 + j) * Np + fn];
              W += w;
              mth += w * th;
              for (int i = 0; i < 3; ++i) {
                mu[i] += w * u[i];
                muth[i] += w * u[i] * th;
                mdth[i] += w * dth[i];
                for (int j = 0; j < 3; ++j) {
                  muu[i][j] += w * u[i] * u[j];
                  mdu[i][j] += w * du[i][j];
                }
              }
            }
        /* step 4: filtered moments, subgrid fluxes and the least-squares targets */
        double ub[3], thb = mth / W, tau[3][3], tth[3], S[3][3], g[3], gu[3][3];
        for (int i = 0; i < 3; ++i) ub[i] = mu[i] / W;
        for (int i = 0; i < 3; ++i) {
          tth[i] = muth[i] / W - ub[i] * thb;
          g[i] = mdth[i] / W;
          for (int j = 0; j < 3; ++j) {
            tau[i][j] = muu[i][j] / W - ub[i] * ub[j];
            gu[i][j] = mdu[i][j] / W;
          }
        }
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) S[i][j] = 0.5 * (gu[i][j] + gu[j][i]);
        double tS = 0.0, SS = 0.0, tg = 0.0, gg = 0.0;
        for (int i = 0; i < 3; ++i) {
          tg += tth[i] * g[i];
          gg += g[i] * g[i];
          for (int j = 0; j < 3; ++j) {
            tS += tau[i][j] * S[i][j];
            SS += S[i][j] * S[i][j];
          }
        }
        const double nu = SS > 0.0 ? fmax(0.0, -tS / (2.0 * SS)) : 0.0;
        const double ka = gg > 0.0 ? fmax(0.0, -tg / gg) : 0.0;
        /* step 5: the sample */
        const long long q = ce * Np + n;
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) X[q * 13 + 3 * i + j] = gu[i][j];
        for (int j = 0; j < 3; ++j) X[q * 13 + 9 + j] = g[j];
        X[q * 13 + 12] = Delta_c;
        T[q * 2] = nu;
        T[q * 2 + 1] = ka;
        if (thv_bar) thv_bar[q] = thb;
      }
    }
    for (int d = 0; d < 3; ++d) {
      free(el[d]);
      free(nd[d]);
      free(wt[d]);
    }
  }
  free(dprim);
  return nce * Np;
}
