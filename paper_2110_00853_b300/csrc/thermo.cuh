// FP64 pointwise thermodynamics of the cmles CUDA path (Sec. 2).
#pragma once

#include "common.cuh"

namespace cmles {

struct Th64 {
  double u[3], q, T, ql, p, c, htot, thv;
};

// Saturation vapour pressure over liquid, integrated Clausius-Clapeyron with
// constant heat capacities (Sec. 2.7):
//   p_v* = p_tr (T/T_tr)^a exp(b (1/T_tr - 1/T)), a = (c_pv - c_pl)/R_v,
//   b = (L_v0 - (c_pv - c_pl) T_0)/R_v, evaluated as one exp of a log-sum.
__device__ __forceinline__ double pvsat64(const KParams &P, double T) {
  return P.pv_ptr * exp(P.pv_a * log(T * P.inv_Ttr) + P.pv_b * (P.inv_Ttr - 1.0 / T));
}

// True when rho q_t is certainly below rho_vs(T): below the tangent of the
// nearest tabulated temperature, with a relative margin of 1e-9 that keeps
// the shortcut clear of the exact test's rounding.
__device__ __forceinline__ bool surely_unsaturated64(const KParams &P, double rhoq, double T) {
  if (P.rvs_n <= 0) return false;
  const double x = (T - P.rvs_T0) / P.rvs_dT;
  if (!(x >= 0.0 && x <= P.rvs_n - 1)) return false;
  const int k = (int)(x + 0.5);
  const double lo = P.rvs_tab[2 * k] + P.rvs_tab[2 * k + 1] * (T - (P.rvs_T0 + k * P.rvs_dT));
  return rhoq <= (1.0 - 1e-9) * lo;
}

// Conserved variables -> diagnostic state (Sec. 2): internal energy from
// Eq. total_energy_def with Phi = g z, temperature from Eq. sat_adjustment
// (closed form when unsaturated, Newton with analytic derivative otherwise,
// liquid only), R_m (Eq. R_m), p (Eq. eos), sound speed, h_tot = e_tot + p/rho,
// theta_v = T / (p/p0)^{R_d/c_pd} * R_m / R_d.
// (p/p0)^-kappa at node level lev: the level's (p_r/p0)^-kappa times the
// binomial series of (1 + v)^-kappa, v = p/p_r - 1, to v^11 for |v| <= 1/32
// (omitted terms below 1e-17 relative); exp(-kappa log(p/p0)) otherwise.
__device__ __forceinline__ double exner_inv64(const KParams &P, double p, int lev) {
  const double pr = P.p_r[lev];
  const double v = (p - pr) / pr;
  if (fabs(v) <= 0.03125) {
    double r = P.kpow64[10];
#pragma unroll
    for (int n = 9; n >= 0; --n) r = fma(r, v, P.kpow64[n]);
    return P.exr[lev] * (1.0 + r * v);
  }
  return exp(-P.kappa * log(p * P.inv_p0));
}

// lev: the node level ez (N + 1) + k of the node, whose reference pressure
// and Exner factor the theta_v evaluation uses.
template <bool MOIST>
__device__ __forceinline__ void thermo64(const KParams &P, const double Y[6], double z, int lev, Th64 &s, int &fail) {
  const double rinv = 1.0 / Y[0];
  s.u[0] = Y[1] * rinv;
  s.u[1] = Y[2] * rinv;
  s.u[2] = Y[3] * rinv;
  const double e = Y[4] * rinv;
  const double q = Y[5] * rinv;
  s.q = q;
  const double ke = 0.5 * (s.u[0] * s.u[0] + s.u[1] * s.u[1] + s.u[2] * s.u[2]);
  const double I = e - ke - P.g * z;
  double T = P.T0 + (I - q * P.Iv0) / ((1.0 - q) * P.cvd + q * P.cvv);
  double ql = 0.0;
  if (MOIST) {
    const double rRv = Y[0] * P.Rv;
    if (!surely_unsaturated64(P, Y[5], T) && q > pvsat64(P, T) / (rRv * T)) {
      bool conv = false;
      for (int it = 0; it < P.satadj_max_iter; ++it) {
        const double qs = pvsat64(P, T) / (rRv * T);
        const double qln = q - qs;
        const double cvm = (1.0 - q) * P.cvd + qs * P.cvv + qln * P.cvl;
        const double f = cvm * (T - P.T0) + qs * P.Iv0 - I;
        const double L = P.Lv0 + P.dcp * (T - P.T0);
        const double dqs = qs * (L / (P.Rv * T * T) - 1.0 / T);
        const double fp = cvm + dqs * ((P.cvv - P.cvl) * (T - P.T0) + P.Iv0);
        const double dT = f / fp;
        T -= dT;
        if (fabs(dT) <= 1e-10) {
          conv = true;
          break;
        }
      }
      if (!conv) fail |= 1;
      ql = q - pvsat64(P, T) / (rRv * T);
      if (ql < 0.0) ql = 0.0;
      // condensate below freezing: kept liquid (no ice phase), counted
      if (ql > 0.0 && T < kTfreeze) fail |= 2;
    }
  }
  const double qv = q - ql;
  const double Rm = P.Rd * (1.0 - q) + P.Rv * qv;
  const double cvm = (1.0 - q) * P.cvd + qv * P.cvv + ql * P.cvl;
  s.T = T;
  s.ql = ql;
  s.p = Y[0] * Rm * T;
  s.c = sqrt((cvm + Rm) / cvm * Rm * T);
  s.htot = e + Rm * T;
  // theta_v = T (p/p0)^-kappa R_m / R_d
  s.thv = T * Rm * P.inv_Rd * exner_inv64(P, s.p, lev);
}

}  // namespace cmles
