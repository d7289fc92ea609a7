/*
 * Pointwise physics of the oracle: thermodynamics and saturation adjustment
 * (Sec. 2), the inviscid flux and the Rusanov numerical flux (Sec. 3.1,
 * Eq. nonviscFlux) and the Smagorinsky-Lilly closure with the Richardson
 * correction (Sec. 4, Eqs. smago and richardson).
 * Test infrastructure only (see oracle.h).
 */
#include <math.h>
#include "oracle.h"

/* Saturation vapour pressure over liquid from the Clausius-Clapeyron relation
 * integrated with constant heat capacities (Sec. 2.7 cites Romps 2008 for
 * this closed form; values of p_tr, T_tr are a reading):
 *   p_v*(T) = p_tr (T/T_tr)^{(c_pv - c_pl)/R_v}
 *             exp[ (L_v0 - (c_pv - c_pl) T_0)/R_v (1/T_tr - 1/T) ],
 * with c_pv = c_vv + R_v and c_pl = c_vl. */
double orc_pvsat(const orc_params *p, double T) {
  double cpv = p->cvv + p->Rv;
  double cpl = p->cvl;
  double dcp = cpv - cpl;
  return p->ptr * pow(T / p->Ttr, dcp / p->Rv) *
         exp((p->Lv0 - dcp * p->T0) / p->Rv * (1.0 / p->Ttr - 1.0 / T));
}

/* Saturation specific humidity q_sat = p_v* / (rho R_v T) (ideal-gas vapour). */
double orc_qsat(const orc_params *p, double T, double rho) {
  return orc_pvsat(p, T) / (rho * p->Rv * T);
}

/* I(T, q) = (1-q_t) I_d + q_v I_v + q_l I_l  (Eqs. total_internal_energy,
 * internal_energies; q_i = 0), I_v0 = L_v0 - R_v T_0. */
double orc_internal_energy(const orc_params *p, double T, double qt, double ql) {
  double qv = qt - ql;
  double Iv0 = p->Lv0 - p->Rv * p->T0;
  double Id = p->cvd * (T - p->T0);
  double Iv = p->cvv * (T - p->T0) + Iv0;
  double Il = p->cvl * (T - p->T0);
  return (1.0 - qt) * Id + qv * Iv + ql * Il;
}

/* Saturation adjustment (Eq. sat_adjustment): find T with I*(T; rho, q_t) = I.
 * Unsaturated: q_v = q_t, closed form T = T_0 + (I - q_t I_v0)/c_vm.
 * Saturated: Newton on f(T) = I*(T) - I with q_v = q_sat(T, rho),
 * q_l = q_t - q_v, and the analytic derivative
 *   f'(T) = c_vm + dq_sat/dT [ (c_vv - c_vl)(T - T_0) + I_v0 ],
 *   dq_sat/dT = q_sat ( L(T)/(R_v T^2) - 1/T ),  L(T) = L_v0 + (c_pv - c_pl)(T - T_0).
 * Reading: liquid only (all cases are warm); stop when |dT| <= 1e-10 K, cap 50. */
int orc_saturation_adjustment(const orc_params *p, double rho, double qt, double I, double *T, double *ql) {
  double Iv0 = p->Lv0 - p->Rv * p->T0;
  double cvm_u = (1.0 - qt) * p->cvd + qt * p->cvv;
  double Tu = p->T0 + (I - qt * Iv0) / cvm_u;
  if (!p->moist || qt <= orc_qsat(p, Tu, rho)) {
    *T = Tu;
    *ql = 0.0;
    return 0;
  }
  double cpv = p->cvv + p->Rv;
  double dcp = cpv - p->cvl;
  double Tn = Tu;
  for (int it = 1; it <= 50; ++it) {
    double qs = orc_qsat(p, Tn, rho);
    double qv = qs;
    double qln = qt - qv;
    double cvm = (1.0 - qt) * p->cvd + qv * p->cvv + qln * p->cvl;
    double f = cvm * (Tn - p->T0) + qv * Iv0 - I;
    double L = p->Lv0 + dcp * (Tn - p->T0);
    double dqs = qs * (L / (p->Rv * Tn * Tn) - 1.0 / Tn);
    double fp = cvm + dqs * ((p->cvv - p->cvl) * (Tn - p->T0) + Iv0);
    double dT = f / fp;
    Tn -= dT;
    if (fabs(dT) <= 1e-10) {
      double qsf = orc_qsat(p, Tn, rho);
      *T = Tn;
      *ql = qt - qsf;
      if (*ql < 0.0) *ql = 0.0;
      return it;
    }
  }
  *T = Tn;
  *ql = qt - orc_qsat(p, Tn, rho);
  return -1;
}

/* Diagnostic state of one node (Sec. 2): u = rho u / rho, q_t, e_tot,
 * I = e_tot - |u|^2/2 - g z (Eq. total_energy_def with Phi = g z),
 * saturation adjustment, R_m (Eq. R_m), p = rho R_m T (Eq. eos),
 * c_vm, c_pm = c_vm + R_m, sound speed c = sqrt(c_pm/c_vm R_m T),
 * total enthalpy h_tot = e_tot + R_m T, potential temperature with the dry
 * Exner function (p/p0)^{R_d/c_pd} and theta_v = theta R_m / R_d. */
int orc_thermo(const orc_params *p, const double Y[6], double z, orc_thermo_state *s) {
  s->rho = Y[0];
  for (int d = 0; d < 3; ++d) s->u[d] = Y[1 + d] / Y[0];
  s->etot = Y[4] / Y[0];
  s->qt = Y[5] / Y[0];
  double ke = 0.5 * (s->u[0] * s->u[0] + s->u[1] * s->u[1] + s->u[2] * s->u[2]);
  s->I = s->etot - ke - p->g * z;
  int it = orc_saturation_adjustment(p, s->rho, s->qt, s->I, &s->T, &s->ql);
  s->newton = it;
  s->qv = s->qt - s->ql;
  s->Rm = p->Rd * (1.0 - s->qt) + p->Rv * s->qv;
  s->cvm = (1.0 - s->qt) * p->cvd + s->qv * p->cvv + s->ql * p->cvl;
  s->cpm = s->cvm + s->Rm;
  s->p = s->rho * s->Rm * s->T;
  s->c = sqrt(s->cpm / s->cvm * s->Rm * s->T);
  s->htot = s->etot + s->Rm * s->T;
  double cpd = p->cvd + p->Rd;
  double exner = pow(s->p / p->p0, p->Rd / cpd);
  s->theta = s->T / exner;
  s->thetav = s->theta * s->Rm / p->Rd;
  return it < 0 ? -1 : 0;
}

/* n . F1(Y): F1 = [rho u, rho u (x) u + (p - p_r) I_3, (rho e + p) u, rho q_t u]
 * (Eqs. mass, moisture, momentum and energy_balance, advective parts). */
void orc_flux1_normal(const orc_params *p, const double Y[6], double z, double pr, const double n[3], double out[6]) {
  orc_thermo_state s;
  orc_thermo(p, Y, z, &s);
  double un = s.u[0] * n[0] + s.u[1] * n[1] + s.u[2] * n[2];
  out[0] = Y[0] * un;
  for (int j = 0; j < 3; ++j) out[1 + j] = Y[1 + j] * un + (s.p - pr) * n[j];
  out[4] = (Y[4] + s.p) * un;
  out[5] = Y[5] * un;
}

/* Rusanov flux, Eq. nonviscFlux with the standard reading of its garbled
 * dissipation term:  n.F* = 1/2 n.(F(Y-) + F(Y+)) + lambda/2 (Y- - Y+),
 * lambda = max over both sides of |u.n| + c. */
void orc_rusanov(const orc_params *p, const double Ym[6], const double Yp[6], double z, double pr,
                 const double n[3], double out[6]) {
  double fm[6], fp[6];
  orc_flux1_normal(p, Ym, z, pr, n, fm);
  orc_flux1_normal(p, Yp, z, pr, n, fp);
  orc_thermo_state sm, sp;
  orc_thermo(p, Ym, z, &sm);
  orc_thermo(p, Yp, z, &sp);
  double lm = fabs(sm.u[0] * n[0] + sm.u[1] * n[1] + sm.u[2] * n[2]) + sm.c;
  double lp = fabs(sp.u[0] * n[0] + sp.u[1] * n[1] + sp.u[2] * n[2]) + sp.c;
  double lam = lm > lp ? lm : lp;
  for (int v = 0; v < 6; ++v) out[v] = 0.5 * (fm[v] + fp[v]) + 0.5 * lam * (Ym[v] - Yp[v]);
}

/* HLLC flux (Toro, Spruce & Speares 1994), in the frame of the face normal n
 * (u = u.n): with the Davis estimates S_L = min(u_L - c_L, u_R - c_R),
 * S_R = max(u_L + c_L, u_R + c_R) (reading: the paper names the flux, not its
 * wave speeds), the contact speed
 *   S* = [p_R - p_L + rho_L u_L (S_L - u_L) - rho_R u_R (S_R - u_R)]
 *        / [rho_L (S_L - u_L) - rho_R (S_R - u_R)],
 * and for side K the star state
 *   U*_K = rho_K (S_K - u_K)/(S_K - S*) [1, S* n + u_t,K,
 *          E_K/rho_K + (S* - u_K)(S* + p_K/(rho_K (S_K - u_K))), q_t,K],
 * the flux is F_L for S_L >= 0, F_L + S_L (U*_L - U_L) for S_L < 0 <= S*,
 * F_R + S_R (U*_R - U_R) for S* < 0 < S_R and F_R for S_R <= 0.  E = rho e_tot
 * (with rho g z, carried by the energy flux (E + p) u) and p the full
 * pressure; F1's momentum flux holds p - p_r, a shift common to both sides
 * that leaves the jump conditions unchanged.  Y- is the left state. */
void orc_hllc(const orc_params *p, const double Ym[6], const double Yp[6], double z, double pr, const double n[3],
              double out[6]) {
  orc_thermo_state sL, sR;
  orc_thermo(p, Ym, z, &sL);
  orc_thermo(p, Yp, z, &sR);
  double uL = sL.u[0] * n[0] + sL.u[1] * n[1] + sL.u[2] * n[2];
  double uR = sR.u[0] * n[0] + sR.u[1] * n[1] + sR.u[2] * n[2];
  double SL = fmin(uL - sL.c, uR - sR.c), SR = fmax(uL + sL.c, uR + sR.c);
  double Ss = (sR.p - sL.p + sL.rho * uL * (SL - uL) - sR.rho * uR * (SR - uR)) /
              (sL.rho * (SL - uL) - sR.rho * (SR - uR));
  double fL[6], fR[6];
  orc_flux1_normal(p, Ym, z, pr, n, fL);
  orc_flux1_normal(p, Yp, z, pr, n, fR);
  if (SL >= 0.0) {
    for (int v = 0; v < 6; ++v) out[v] = fL[v];
    return;
  }
  if (SR <= 0.0) {
    for (int v = 0; v < 6; ++v) out[v] = fR[v];
    return;
  }
  const int left = Ss >= 0.0;
  const orc_thermo_state *s = left ? &sL : &sR;
  const double *Y = left ? Ym : Yp, *f = left ? fL : fR;
  double S = left ? SL : SR, u = left ? uL : uR;
  double chi = (S - u) / (S - Ss);
  double Us[6];
  Us[0] = s->rho * chi;
  for (int c = 0; c < 3; ++c) {
    double ut = s->u[c] - u * n[c];
    Us[1 + c] = s->rho * chi * (Ss * n[c] + ut);
  }
  Us[4] = s->rho * chi * (Y[4] / s->rho + (Ss - u) * (Ss + s->p / (s->rho * (S - u))));
  Us[5] = s->rho * chi * (Y[5] / s->rho);
  for (int v = 0; v < 6; ++v) out[v] = f[v] + S * (Us[v] - Y[v]);
}

/* Roe flux (Roe 1981), n.F* = (n.F(Y-) + n.F(Y+))/2 - |A| (Y+ - Y-)/2 with A
 * the flux Jacobian along n at Roe's averaged state: rho^ = sqrt(rho- rho+)
 * and sqrt(rho)-weighted u, total specific enthalpy H = (rho e_tot + p)/rho
 * and q_t.  Reading (the paper names the flux only): the averaged state uses
 * the frozen moist equation of state (q_l = 0),
 *   p = (R_m/c_vm) (E - rho |u|^2/2 - rho Phi - rho q I_v0) + rho R_m T_0,
 * whose derivatives at fixed other conserved variables are, with
 * G = R_m/c_vm,
 *   dp/dE = G, dp/d(rho u) = -G u,
 *   dp/d(rho q) = (R_v - R_d - G (c_vv - c_vd)) (T - T_0) - G I_v0 + (R_v - R_d) T_0,
 *   dp/drho = (R_d - G c_vd) (T - T_0) + G (|u|^2/2 - Phi) + R_d T_0,
 * T from H, and c^2 = dp/drho + u.dp/d(rho u) + H dp/dE + q dp/d(rho q).
 * The acoustic strengths alpha_-+ = (dp -+ rho^ c du_n)/(2 c^2) (dp and
 * du_n the jumps linearised at the averaged state) with eigenvectors
 * r_-+ = (1, u -+ c n, H -+ u_n c, q), and every other wave travels at u_n:
 *   |A| dY = |u_n - c| a_- r_- + |u_n + c| a_+ r_+ + |u_n| (dY - a_- r_- - a_+ r_+).
 * For dry air this is Roe's exact linearisation.  No entropy fix. */
void orc_roe(const orc_params *p, const double Ym[6], const double Yp[6], double z, double pr, const double n[3],
             double out[6]) {
  orc_thermo_state sL, sR;
  orc_thermo(p, Ym, z, &sL);
  orc_thermo(p, Yp, z, &sR);
  double fL[6], fR[6];
  orc_flux1_normal(p, Ym, z, pr, n, fL);
  orc_flux1_normal(p, Yp, z, pr, n, fR);
  double wL = sqrt(sL.rho), wR = sqrt(sR.rho), iw = 1.0 / (wL + wR);
  double rh = wL * wR;
  double u[3];
  for (int c = 0; c < 3; ++c) u[c] = (wL * sL.u[c] + wR * sR.u[c]) * iw;
  double HL = (Ym[4] + sL.p) / sL.rho, HR = (Yp[4] + sR.p) / sR.rho;
  double H = (wL * HL + wR * HR) * iw;
  double q = (wL * Ym[5] / sL.rho + wR * Yp[5] / sR.rho) * iw;
  double Phi = p->g * z, uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  double Iv0 = p->Lv0 - p->Rv * p->T0;
  double Rm = p->Rd + q * (p->Rv - p->Rd), cvm = p->cvd + q * (p->cvv - p->cvd), G = Rm / cvm;
  /* H = |u|^2/2 + Phi + c_vm (T - T_0) + q I_v0 + R_m T */
  double T = (H - 0.5 * uu - Phi - q * Iv0 + cvm * p->T0) / (cvm + Rm);
  double p_rho = (p->Rd - G * p->cvd) * (T - p->T0) + G * (0.5 * uu - Phi) + p->Rd * p->T0;
  double p_w = ((p->Rv - p->Rd) - G * (p->cvv - p->cvd)) * (T - p->T0) - G * Iv0 + (p->Rv - p->Rd) * p->T0;
  double c2 = p_rho - G * uu + G * H + q * p_w, c = sqrt(c2);
  double dY[6];
  for (int v = 0; v < 6; ++v) dY[v] = Yp[v] - Ym[v];
  double dp = p_rho * dY[0] - G * (u[0] * dY[1] + u[1] * dY[2] + u[2] * dY[3]) + G * dY[4] + p_w * dY[5];
  double un = u[0] * n[0] + u[1] * n[1] + u[2] * n[2];
  double dun = (n[0] * dY[1] + n[1] * dY[2] + n[2] * dY[3] - un * dY[0]) / rh;
  double am = (dp - rh * c * dun) / (2.0 * c2), ap = (dp + rh * c * dun) / (2.0 * c2);
  double rm[6] = {1.0, u[0] - c * n[0], u[1] - c * n[1], u[2] - c * n[2], H - un * c, q};
  double rp[6] = {1.0, u[0] + c * n[0], u[1] + c * n[1], u[2] + c * n[2], H + un * c, q};
  for (int v = 0; v < 6; ++v) {
    double D = fabs(un - c) * am * rm[v] + fabs(un + c) * ap * rp[v] + fabs(un) * (dY[v] - am * rm[v] - ap * rp[v]);
    out[v] = 0.5 * (fL[v] + fR[v]) - 0.5 * D;
  }
}

/* Richardson factor f_b (Eq. richardson) for |S|^2 = 2 S:S > 0. */
static double richardson_factor(const orc_params *p, double dthvdz, double thv, double Smag2) {
  double N2 = p->g / thv * dthvdz;
  double Ri = N2 / Smag2;
  if (Ri <= 0.0) return 1.0;
  double a = 1.0 - Ri / p->Prt;
  return a > 0.0 ? pow(a, 0.25) : 0.0;
}

/* Vreman eddy viscosity (Eq. vreman-sgs): beta_ij = sum_m Delta_m^2 u_i,m u_j,m,
 * B_beta = beta11 beta22 + beta11 beta33 + beta22 beta33 - beta13^2 - beta12^2
 * - beta23^2, nu_t = 2.5 C_s^2 sqrt(B_beta / (u_i,j u_i,j)); zero when the
 * gradient vanishes or B_beta <= 0.  Times f_b when the correction is on. */
double orc_vreman(const orc_params *p, const double gu[9], double dthvdz, double thv, const double Dm[3]) {
  /* beta_ij = sum_m Delta_m^2 u_i,m u_j,m */
  double beta[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double acc = 0.0;
      for (int m = 0; m < 3; ++m) acc += Dm[m] * Dm[m] * gu[3 * i + m] * gu[3 * j + m];
      beta[i][j] = acc;
    }
  double B = beta[0][0] * beta[1][1] + beta[0][0] * beta[2][2] + beta[1][1] * beta[2][2] -
             (beta[0][2] * beta[0][2] + beta[0][1] * beta[0][1] + beta[1][2] * beta[1][2]);
  double uu = 0.0;
  for (int k = 0; k < 9; ++k) uu += gu[k] * gu[k];
  if (uu == 0.0 || B <= 0.0) return 0.0;
  double nut = 2.5 * p->Cs * p->Cs * sqrt(B / uu);
  if (p->richardson) {
    double S2 = 0.0;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        double Sij = 0.5 * (gu[3 * i + j] + gu[3 * j + i]);
        S2 += Sij * Sij;
      }
    if (S2 > 0.0) nut *= richardson_factor(p, dthvdz, thv, 2.0 * S2);
  }
  return nut;
}

/* Smagorinsky-Lilly eddy viscosity nu_t = (C_s Delta)^2 |S| f_b with
 * S = sym(grad u) (Eq. strain_rate), |S| = sqrt(2 S_ij S_ij) (Eq. smago) and
 * f_b the Richardson correction (Eq. richardson):
 *   Ri = (g/theta_v d theta_v/dz) / |S|^2,
 *   f_b = 1 for Ri <= 0, max(0, 1 - Ri/Pr_t)^{1/4} otherwise.
 * Reading: nu_t = 0 when |S| = 0. */
double orc_smagorinsky(const orc_params *p, const double gu[9], double dthvdz, double thv, double Delta) {
  double S2 = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double Sij = 0.5 * (gu[3 * i + j] + gu[3 * j + i]);
      S2 += Sij * Sij;
    }
  double Smag2 = 2.0 * S2;
  if (Smag2 == 0.0) return 0.0;
  double Smag = sqrt(Smag2);
  double fb = 1.0;
  if (p->richardson) {
    double N2 = p->g / thv * dthvdz;
    double Ri = N2 / Smag2;
    if (Ri > 0.0) {
      double a = 1.0 - Ri / p->Prt;
      fb = a > 0.0 ? pow(a, 0.25) : 0.0;
    }
  }
  double l = p->Cs * Delta;
  return l * l * Smag * fb;
}
