// FP32 deviation-form thermodynamics shared by the flat and curvilinear
// FP32 kernels (see dg_fp32.cu for the formulation).
#pragma once

#include "common.cuh"

namespace cmles {

constexpr int kNP = np32(4);  // padded nodes per element in the FP32 arrays up to N = 4

struct Th32 {
  float rho, u[3], qp, Tp, pp, c, hp, thvp;
};

// Divisions in the FP32 path use the approximate quotient (2 ulp), far below
// the FP32 rounding of the deviations they combine.
__device__ __forceinline__ float fdiv(float a, float b) { return __fdividef(a, b); }

// p_v*(T) of the integrated Clausius-Clapeyron relation, FP32.
__device__ __forceinline__ float pvsat32(const KF &F, float T) {
  return F.pv_ptr * expf(F.pv_a * logf(T * F.inv_Ttr) + F.pv_b * (F.inv_Ttr - fdiv(1.0f, T)));
}
// saturation vapour density p_v*(T) / (R_v T)
__device__ __forceinline__ float rhovsat32(const KF &F, float T) { return fdiv(pvsat32(F, T) * F.inv_Rv, T); }

// (1 + v)^-kappa - 1: the binomial series to v^6 for |v| <= 1/32 (the
// omitted terms are below 3e-10 of the result there), expm1(-kappa log1p(v))
// otherwise.
__device__ __forceinline__ float pow_kappa_m1(const KF &F, float v) {
  if (fabsf(v) <= 0.03125f) {
    float r = F.kpow[5];
#pragma unroll
    for (int n = 4; n >= 0; --n) r = fmaf(r, v, F.kpow[n]);
    return r * v;
  }
  return expm1f(-F.kappa * log1pf(v));
}

// Thermodynamics of one node from its deviation state s and its level table L.
template <bool MOIST>
__device__ __forceinline__ void thermo32(const KParams &P, const float *__restrict__ L, const float s[6], Th32 &o,
                                         int &fail) {
  const KF &F = P.f;
  const float rho_r = L[L_RHO], rhoq_r = L[L_RHOQ], Tr = L[L_T], TrT0 = L[L_T_T0];
  const float rp = s[0], qp = s[5];
  const float rho = rho_r + rp;
  const float rinv = fdiv(1.0f, rho);
  o.rho = rho;
  o.u[0] = s[1] * rinv;
  o.u[1] = s[2] * rinv;
  o.u[2] = s[3] * rinv;
  const float rhoq = rhoq_r + qp;
  o.qp = (qp - L[L_QM] * rp) * rinv;  // q_t - q_r
  const float rke = 0.5f * (s[1] * o.u[0] + s[2] * o.u[1] + s[3] * o.u[2]);
  const float dRI = s[4] - rke - rp * L[L_GZ];  // rho I - rho_r I_r
  // unsaturated: rho c_vm (T - T_r) = d(rho I) - d(rho q) I_v0 - d(rho c_vm) (T_r - T_0)
  // drqv = rho q_v - rho q_r is carried as a deviation (never formed as the
  // difference of two near-equal FP32 numbers)
  float rhoqv = rhoq, rhoql = 0.0f, drqv = qp;
  float Tp = fdiv(dRI - qp * F.Iv0 - (rp * F.cvd + qp * (F.cvv - F.cvd)) * TrT0,
                  rho * F.cvd + rhoq * (F.cvv - F.cvd));
  if (MOIST) {
    float T = Tr + Tp;
    // Certainly unsaturated without evaluating p_v*: rho_vs(T) is convex in
    // T on [150, 450] K, so its tangent at T_r bounds it from below there,
    // rho_vs(T) >= rho_vs(T_r) (1 + T' d ln rho_vs/dT(T_r)); the factor
    // 1 - 1e-5 keeps the shortcut clear of the exact test's rounding.
    const float iTr = fdiv(1.0f, Tr);
    const float slope = (F.pv_a - 1.0f + F.pv_b * iTr) * iTr;
    const bool dry = P.rvs_ok && T >= 150.0f && T <= 450.0f && Tr >= 150.0f && Tr <= 450.0f &&
                     rhoq <= 0.99999f * L[L_RVS] * (1.0f + slope * Tp);
    if (!dry && rhoq > rhovsat32(F, T)) {
      bool conv = false;
      for (int it = 0; it < P.satadj_max_iter; ++it) {
        T = Tr + Tp;
        const float rqs = rhovsat32(F, T);
        const float rql = rhoq - rqs;
        const float rcvm = (rho - rhoq) * F.cvd + rqs * F.cvv + rql * F.cvl;
        const float drcvm = (rp - qp) * F.cvd + (rqs - rhoq_r) * F.cvv + rql * F.cvl;
        const float rf = rcvm * Tp + drcvm * TrT0 + (rqs - rhoq_r) * F.Iv0 - dRI;
        const float Lh = F.Lv0 + F.dcp * (T - F.T0);
        const float iT = fdiv(1.0f, T);
        const float drqs = rqs * iT * (Lh * F.inv_Rv * iT - 1.0f);
        const float rfp = rcvm + drqs * ((F.cvv - F.cvl) * (T - F.T0) + F.Iv0);
        const float dT = fdiv(rf, rfp);
        Tp -= dT;
        if (fabsf(dT) <= 5e-5f) {
          conv = true;
          break;
        }
      }
      if (!conv) fail |= 1;
      T = Tr + Tp;
      rhoqv = rhovsat32(F, T);
      rhoql = rhoq - rhoqv;
      drqv = rhoqv - rhoq_r;
      if (rhoql < 0.0f) {
        rhoql = 0.0f;
        rhoqv = rhoq;
        drqv = qp;
      } else if (T < (float)kTfreeze) {
        fail |= 2;  // condensate below freezing: kept liquid (no ice phase), counted
      }
    }
  }
  o.Tp = Tp;
  const float rRm = F.Rd * (rho - rhoq) + F.Rv * rhoqv;
  const float drRm = F.Rd * (rp - qp) + F.Rv * drqv;
  const float pp = rRm * Tp + drRm * Tr;  // p - p_r
  o.pp = pp;
  const float rcvm = (rho - rhoq) * F.cvd + rhoqv * F.cvv + rhoql * F.cvl;
  const float pr = L[L_P];
  o.c = sqrtf(fdiv(rcvm + rRm, rcvm) * (pr + pp) * rinv);
  o.hp = (s[4] + pp - L[L_HM] * rp) * rinv;  // h_tot - h_r
  // theta_v / theta_v,r = (T/T_r)(R_m/R_m,r)(p/p_r)^-kappa with
  // (T/T_r)(R_m/R_m,r) = (1 + a)(1 + b)/(1 + c) = 1 + (a + b + ab - c)/(1 + c),
  // a = T'/T_r, b = (rho R_m)'/(rho R_m)_r, c = rho'/rho_r (exact algebra)
  const float ra = fdiv(Tp, Tr), rb = fdiv(drRm, L[L_RHORM]), rc = fdiv(rp, rho_r);
  // theta_v / theta_v,r = (1 + u)(1 + w), w = (p/p_r)^-kappa - 1
  const float u = fdiv(ra + rb + ra * rb - rc, 1.0f + rc);
  const float w = pow_kappa_m1(F, fdiv(pp, pr));
  o.thvp = L[L_THV] * (u + w + u * w);  // theta_v - theta_v,r
}

// Deviation part of n.F1 along d (sign by the caller):
// [rho u_d, rho u_j u_d + (p - p_r) delta_jd, (rho e' + p') u_d, rho q_t u_d].
// The reference part H_r u_d of the energy flux is handled separately.
__device__ __forceinline__ void flux1_dev32(const float s[6], float rho_r, float rhoq_r, float pp, int d,
                                           float f[6]) {
  // the normal momentum by selection, not by a run-time index, so that the
  // state stays in registers when d is not a compile-time constant
  const float sd = d == 0 ? s[1] : (d == 1 ? s[2] : s[3]);
  const float ud = fdiv(sd, rho_r + s[0]);
  f[0] = sd;
  f[1] = s[1] * ud + (d == 0 ? pp : 0.f);
  f[2] = s[2] * ud + (d == 1 ? pp : 0.f);
  f[3] = s[3] * ud + (d == 2 ? pp : 0.f);
  f[4] = (s[4] + pp) * ud;
  f[5] = (rhoq_r + s[5]) * ud;
}

// The thermodynamic fields of a shadow node s that the two passes read
// (planes of TH per element: p', c, h', theta_v'), stored by whoever writes
// the node's state; np: the arrays' padded nodes per element.
__device__ __forceinline__ void thermo_store32(const KParams &P, const float *L, const float s[6], float *TH,
                                               size_t e, int t, int &fail, int np = kNP) {
  Th32 o;
  if (P.moist)
    thermo32<true>(P, L, s, o, fail);
  else
    thermo32<false>(P, L, s, o, fail);
  TH[(e * 4 + 0) * np + t] = o.pp;
  TH[(e * 4 + 1) * np + t] = o.c;
  TH[(e * 4 + 2) * np + t] = o.hp;
  TH[(e * 4 + 3) * np + t] = o.thvp;
}

}  // namespace cmles
