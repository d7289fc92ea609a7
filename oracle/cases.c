/*
 * Initial states of the synthetic cases, evaluated at the oracle's own node
 * coordinates.  These are inputs for the tests, not part of the method: the
 * background states follow the hydrostatic profiles the paper prints
 * (Eq. pressureDistrib for neutral air, Eqs. pressure_hs_brunt and
 * density_hs_brunt for constant Brunt-Vaisala frequency), perturbations follow
 * the case descriptions, and seeded noise comes from a counter-based
 * SplitMix64 stream.  Test infrastructure only (see oracle.h).
 */
#include <math.h>
#include <stdlib.h>
#include "oracle.h"
#include "oracle_internal.h"

/* SplitMix64 (Steele, Lea & Flood 2014): the generator's state advances by the
 * golden-ratio increment; output number `counter` is the mix of
 * seed + (counter + 1) * 0x9E3779B97F4A7C15. */
double orc_uniform(uint64_t seed, uint64_t counter) {
  uint64_t z = seed + (counter + 1ULL) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  z = z ^ (z >> 31);
  return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

/* ---- background profiles ---- */

typedef struct {
  const orc_params *P;
  const orc_case *c;
} prof_ctx;

/* moist-layer potential temperature and total water (case 2): theta_l constant
 * in the mixed layer then a constant lapse; q_t linear in the mixed layer,
 * then linear to q_top at the lid. */
static double prof_theta(const prof_ctx *x, double z, double Lz) {
  const orc_case *c = x->c;
  if (c->id == 2) return z <= c->z_ml ? c->theta0 : c->theta0 + c->dthdz_above * (z - c->z_ml);
  if (c->id == 5 || c->id == 3) return c->theta0 * exp(c->NBV * c->NBV * z / x->P->g);
  (void)Lz;
  return c->theta0;
}
static double prof_qt(const prof_ctx *x, double z, double Lz) {
  const orc_case *c = x->c;
  if (!c->moist) return 0.0;
  if (c->id == 2) {
    if (z <= c->z_ml) return c->qt_sfc + (c->qt_ml - c->qt_sfc) * z / c->z_ml;
    return c->qt_ml + (c->qt_top - c->qt_ml) * (z - c->z_ml) / (Lz - c->z_ml);
  }
  if (c->id == 5) return c->qt_sfc * exp(-z / c->qt_H);
  return 0.0;
}

/* dp/dz = -g p / (R_m T),  T = theta (p/p0)^{R_d/c_pd}, q_l = 0 (reading). */
static double dpdz(const prof_ctx *x, double z, double p, double Lz) {
  const orc_params *P = x->P;
  double cpd = P->cvd + P->Rd;
  double th = prof_theta(x, z, Lz), qt = prof_qt(x, z, Lz);
  double T = th * pow(p / P->p0, P->Rd / cpd);
  double Rm = P->Rd * (1.0 - qt) + P->Rv * qt;
  return -P->g * p / (Rm * T);
}
static double rk4(const prof_ctx *x, double z, double p, double h, double Lz) {
  double k1 = dpdz(x, z, p, Lz);
  double k2 = dpdz(x, z + 0.5 * h, p + 0.5 * h * k1, Lz);
  double k3 = dpdz(x, z + 0.5 * h, p + 0.5 * h * k2, Lz);
  double k4 = dpdz(x, z + h, p + h * k3, Lz);
  return p + h / 6.0 * (k1 + 2.0 * k2 + 2.0 * k3 + k4);
}

/* Hydrostatic pressure by classical RK4 on the fixed grid z_m = m h0,
 * h0 = 0.5 m, from p(0) = p0, and a last partial step to z. */
typedef struct {
  double h0;
  int M;
  double *pm;
} hydro_table;
static void hydro_build(hydro_table *t, const prof_ctx *x, double zmax, double Lz) {
  t->h0 = 0.5;
  t->M = (int)ceil(zmax / t->h0) + 2;
  t->pm = (double *)malloc((size_t)(t->M + 1) * sizeof(double));
  t->pm[0] = x->P->p0;
  for (int m = 0; m < t->M; ++m) t->pm[m + 1] = rk4(x, m * t->h0, t->pm[m], t->h0, Lz);
}
static double hydro_p(const hydro_table *t, const prof_ctx *x, double z, double Lz) {
  int m = (int)floor(z / t->h0);
  if (m < 0) m = 0;
  if (m > t->M) m = t->M;
  double zm = m * t->h0;
  if (z == zm) return t->pm[m];
  return rk4(x, zm, t->pm[m], z - zm, Lz);
}

/* background pressure at height z for each case */
static double background_p(const prof_ctx *x, const hydro_table *t, double z, double Lz) {
  const orc_params *P = x->P;
  const orc_case *c = x->c;
  double cpd = P->cvd + P->Rd;
  if (c->id == 1 || c->id == 11) /* Eq. pressureDistrib */
    return P->p0 * pow(1.0 - P->g / (cpd * c->theta0) * z, cpd / P->Rd);
  if ((c->id == 3 || c->id == 5) && !c->moist) { /* Eq. pressure_hs_brunt */
    double N2 = c->NBV * c->NBV;
    double pi = 1.0 + P->g * P->g / (cpd * c->theta0 * N2) * (exp(-z * N2 / P->g) - 1.0);
    return P->p0 * pow(pi, cpd / P->Rd);
  }
  return hydro_p(t, x, z, Lz);
}

/* conserved state from theta, q_t (q_l = 0), pressure and velocity:
 * T = theta (p/p0)^{R_d/c_pd}, rho = p/(R_m T),
 * rho e = rho (I(T, q_t, 0) + |u|^2/2 + g z). */
static void state_from(const orc_params *P, double theta, double qt, double p, const double u[3], double z,
                       double Y[6]) {
  double cpd = P->cvd + P->Rd;
  double T = theta * pow(p / P->p0, P->Rd / cpd);
  double Rm = P->Rd * (1.0 - qt) + P->Rv * qt;
  double rho = p / (Rm * T);
  double I = orc_internal_energy(P, T, qt, 0.0);
  double ke = 0.5 * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
  Y[0] = rho;
  Y[1] = rho * u[0];
  Y[2] = rho * u[1];
  Y[3] = rho * u[2];
  Y[4] = rho * (I + ke + P->g * z);
  Y[5] = rho * qt;
}

static void vortex_state(const orc_solver *s, const orc_case *c, double t, size_t q, double Y[6]) {
  const orc_params *P = &s->p;
  double cpd = P->cvd + P->Rd, gam = cpd / P->cvd;
  double Lx = s->m.Lx, Ly = s->m.Ly;
  double cx = c->xc + c->vortex_U * t;
  double dx = s->x[q] - cx, dy = s->y[q] - c->yc;
  dx -= Lx * floor(dx / Lx + 0.5);
  dy -= Ly * floor(dy / Ly + 0.5);
  double R = c->vortex_R, bU = c->vortex_beta * c->vortex_U;
  double f = exp(0.5 * (1.0 - (dx * dx + dy * dy) / (R * R)));
  double u[3] = {c->vortex_U - bU * dy / R * f, bU * dx / R * f, 0.0};
  double T = c->vortex_T - bU * bU / (2.0 * cpd) * f * f;
  double rho = c->vortex_rho * pow(T / c->vortex_T, 1.0 / (gam - 1.0));
  double I = orc_internal_energy(P, T, 0.0, 0.0);
  double ke = 0.5 * (u[0] * u[0] + u[1] * u[1]);
  Y[0] = rho;
  Y[1] = rho * u[0];
  Y[2] = rho * u[1];
  Y[3] = 0.0;
  Y[4] = rho * (I + ke + P->g * s->z[q]);
  Y[5] = 0.0;
}

void orc_vortex_exact(orc_solver *s, const orc_case *c, double t, double *Q) {
  const int Np = s->Np;
  for (int e = 0; e < s->E; ++e)
    for (int n = 0; n < Np; ++n) {
      double Y[6];
      vortex_state(s, c, t, (size_t)e * Np + n, Y);
      for (int v = 0; v < 6; ++v) Q[((size_t)e * 6 + v) * Np + n] = Y[v];
    }
}

void orc_init_case(orc_solver *s, const orc_case *c, double *Q, double *rho_r, double *p_r) {
  const orc_params *P = &s->p;
  const int Np = s->Np;
  const double Lz = s->m.Lz;
  prof_ctx x = {P, c};
  hydro_table t = {0};
  int need_table = (c->id == 2) || ((c->id == 3 || c->id == 5) && c->moist);
  if (need_table) {
    double zmax = 0.0;
    for (size_t q = 0; q < (size_t)s->E * Np; ++q)
      if (s->z[q] > zmax) zmax = s->z[q];
    hydro_build(&t, &x, zmax, Lz);
  }
  for (int e = 0; e < s->E; ++e)
    for (int n = 0; n < Np; ++n) {
      size_t q = (size_t)e * Np + n;
      uint64_t gid = (uint64_t)q;
      double Y[6];
      if (c->id == 10) {
        vortex_state(s, c, 0.0, q, Y);
        rho_r[q] = c->vortex_rho;
        p_r[q] = c->vortex_rho * P->Rd * c->vortex_T;
      } else {
        double z = s->z[q];
        double pb = background_p(&x, &t, z, Lz);
        double th0 = prof_theta(&x, z, Lz), qt0 = prof_qt(&x, z, Lz);
        double zero[3] = {0.0, 0.0, 0.0};
        double Yr[6];
        state_from(P, th0, qt0, pb, zero, z, Yr);
        rho_r[q] = Yr[0];
        p_r[q] = pb;
        double th = th0, qt = qt0;
        double u[3] = {c->u0[0], c->u0[1], c->u0[2]};
        if (c->id == 1) { /* cosine-squared bubble, Eq. tracer_perturbation shape */
          double dx = s->x[q] - c->xc, dy = s->y[q] - c->yc, dz = z - c->zc;
          double r = sqrt(dx * dx + dy * dy + dz * dz);
          if (r <= c->r0) {
            double cs = cos(M_PI * r / (2.0 * c->r0));
            th += c->dtheta * cs * cs;
          }
        }
        if (c->id == 11) { /* Eq. densityCurrentEqn, r read as an ellipse radius */
          double ax = (s->x[q] - c->xc) / c->r0, az = (z - c->zc) / (0.5 * c->r0);
          double r = sqrt(ax * ax + az * az);
          if (r <= 1.0) th += 0.5 * c->dtheta * (1.0 + cos(M_PI * r));
        }
        if (c->modes) { /* random-phase velocity modes (throughput box, training runs) */
          for (int k = 0; k < c->nmodes; ++k) {
            const double *md = c->modes + (size_t)k * 7;
            double ph = md[0] * s->x[q] + md[1] * s->y[q] + md[2] * z + md[6];
            double cs = cos(ph);
            u[0] += md[3] * cs;
            u[1] += md[4] * cs;
            u[2] += md[5] * cs;
          }
        }
        if (z <= c->noise_zmax) {
          th += c->noise_theta * (2.0 * orc_uniform(c->seed, 4 * gid + 0) - 1.0);
          if (c->moist) qt += c->noise_qt * (2.0 * orc_uniform(c->seed, 4 * gid + 1) - 1.0);
        }
        state_from(P, th, qt, pb, u, z, Y);
      }
      for (int v = 0; v < 6; ++v) Q[((size_t)e * 6 + v) * Np + n] = Y[v];
    }
  free(t.pm);
  orc_set_reference(s, rho_r, p_r);
}
