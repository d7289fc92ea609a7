// FP64 ("plain") DG right-hand side kernels for flat hexahedral meshes.
//
// Two kernels per Runge-Kutta stage (Sec. 3.1, Eq. matrixProblem):
//   k_grad64: the BR1 auxiliary gradient of G = (u, v, w, h_tot, q_t,
//             theta_v) with its centred face term, the SGS closure (Sec. 4)
//             and the diffusive flux F2; writes F2.
//   k_rhs64:  total flux F1 + F2, its divergence by the 1D LGL derivative
//             matrix along each axis, the Rusanov/central surface terms with
//             the lift w_s J_s / (w_i J_i), wall boundary states (App. A.3),
//             sources (gravity with reference subtraction, Rayleigh sponge,
//             Coriolis), and the fused LSRK(5,4) stage update.
// The pointwise thermodynamics with saturation adjustment (Sec. 2) runs once
// per node and state, in the kernel that writes the state: the flux pass for
// the state it advances to, k_thermo64 otherwise.  It stores p - p_r, the
// sound speed, h_tot and theta_v (TH, four planes per element), which the
// next gradient pass (own and neighbour face nodes) and flux pass read.
// One element per 128-thread CTA iteration, one node per thread, element and
// neighbour face nodes staged in shared memory; grid-stride over elements.
#include "common.cuh"
#include "launch.h"
#include "thermo.cuh"

namespace cmles {

// Threads per CTA of the FP64 element kernels: one per node, 128 up to
// N = 4 (125 nodes), else the nodes rounded up to whole warps (N = 5: 224,
// N = 6: 352, N = 7: 512).
__host__ __device__ constexpr int block64(int N) {
  return (N + 1) * (N + 1) * (N + 1) <= 128 ? 128 : ((N + 1) * (N + 1) * (N + 1) + 31) / 32 * 32;
}

// The thermodynamic fields of a node's state Y at height z and level lev.
// Not inlined: the flux pass (for the state it advances to) and k_thermo64
// (for a state set from outside) then run the same compiled code, so that a
// state gets bit-identical fields whichever kernel wrote them (a run resumed
// from a saved state continues bit-identically).
__device__ __noinline__ void thermo_store64(const KParams &P, const double Y[6], double z, int lev, double *TH,
                                               size_t e, int t, int Np, int &fail) {
  Th64 s;
  if (P.moist)
    thermo64<true>(P, Y, z, lev, s, fail);
  else
    thermo64<false>(P, Y, z, lev, s, fail);
  TH[(e * 4 + 0) * Np + t] = s.p - P.p_r[lev];
  TH[(e * 4 + 1) * Np + t] = s.c;
  TH[(e * 4 + 2) * Np + t] = s.htot;
  TH[(e * 4 + 3) * Np + t] = s.thv;
}

template <int N>
__global__ void __launch_bounds__(block64(N)) k_grad64(const double *__restrict__ Q, const double *__restrict__ TH,
                                                       double *__restrict__ F2, const KParams P) {
  constexpr int Nq = N + 1, Np = Nq * Nq * Nq, Nf = Nq * Nq;
  static_assert(Np <= block64(N), "one node per thread");
  __shared__ double sD[Nq * Nq];
  __shared__ double sG[6][Np];
  __shared__ double sGf[6][6][Nf];
  __shared__ int sNb[6];
  const int t = threadIdx.x;
  if (t < Nq * Nq) sD[t] = P.D[t];
  const int i = t % Nq, j = (t / Nq) % Nq, k = t / Nf;
  for (int g = blockIdx.x; g < P.E; g += gridDim.x) {
    int ex, ey, ez;
    const int e = element_lin(P, g, ex, ey, ez);
    if (t < 6) sNb[t] = neighbour(P, ex, ey, ez, t);
    double Y[6], G[6];
    if (t < Np) {
#pragma unroll
      for (int v = 0; v < 6; ++v) Y[v] = Q[((size_t)e * 6 + v) * Np + t];
      // h_tot and theta_v come with the state; u and q_t formed exactly as
      // the thermodynamics forms them
      const double rinv = 1.0 / Y[0];
      G[0] = Y[1] * rinv;
      G[1] = Y[2] * rinv;
      G[2] = Y[3] * rinv;
      G[3] = TH[((size_t)e * 4 + 2) * Np + t];
      G[4] = Y[5] * rinv;
      G[5] = TH[((size_t)e * 4 + 3) * Np + t];
#pragma unroll
      for (int v = 0; v < 6; ++v) sG[v][t] = G[v];
    }
    __syncthreads();
    // neighbour face nodes
    for (int task = t; task < 6 * Nf; task += blockDim.x) {
      const int f = task / Nf, fn = task - f * Nf;
      const int nb = sNb[f];
      if (nb < 0) continue;
      const int d = f >> 1, t1 = fn % Nq, t2 = fn / Nq;
      const int a_nb = (f & 1) ? 0 : N;
      const int nn = face_node<Nq>(d, a_nb, t1, t2);
      const double *Yp = Q + (size_t)nb * 6 * Np + nn;
      const double rinv = 1.0 / Yp[0];
      sGf[f][0][fn] = Yp[1 * Np] * rinv;
      sGf[f][1][fn] = Yp[2 * Np] * rinv;
      sGf[f][2][fn] = Yp[3 * Np] * rinv;
      sGf[f][3][fn] = TH[((size_t)nb * 4 + 2) * Np + nn];
      sGf[f][4][fn] = Yp[5 * Np] * rinv;
      sGf[f][5][fn] = TH[((size_t)nb * 4 + 3) * Np + nn];
    }
    __syncthreads();
    if (t < Np) {
      double gr[6][3];
#pragma unroll
      for (int v = 0; v < 6; ++v) {
        double a0 = 0.0, a1 = 0.0, a2 = 0.0;
#pragma unroll
        for (int m = 0; m < Nq; ++m) {
          a0 += sD[i * Nq + m] * sG[v][m + Nq * (j + Nq * k)];
          a1 += sD[j * Nq + m] * sG[v][i + Nq * (m + Nq * k)];
          a2 += sD[k * Nq + m] * sG[v][i + Nq * (j + Nq * m)];
        }
        gr[v][0] = P.jac[0] * a0;
        gr[v][1] = P.jac[1] * a1;
        gr[v][2] = P.jac[2] * a2;
      }
      // BR1 surface term: (w_s J_s)/(w_i J_i) n (G* - G-), G* = (G- + G+)/2;
      // at walls the velocity ghost reflects the normal component and
      // scalars are copied, so only the normal velocity jumps.
      auto lift = [&](int f, int fn) {
        const int d = f >> 1;
        const double L = (f & 1) ? P.lift[d] : -P.lift[d];
        if (sNb[f] >= 0) {
#pragma unroll
          for (int v = 0; v < 6; ++v) gr[v][d] += L * (0.5 * (G[v] + sGf[f][v][fn]) - G[v]);
        } else if ((P.noslip >> f) & 1) {
          // no-slip wall: every velocity component's ghost is -G
#pragma unroll
          for (int c = 0; c < 3; ++c) gr[c][d] += L * (-G[c]);
        } else {
          gr[d][d] += L * (-G[d]);
        }
      };
      if (i == 0) lift(0, j + Nq * k);
      if (i == N) lift(1, j + Nq * k);
      if (j == 0) lift(2, i + Nq * k);
      if (j == N) lift(3, i + Nq * k);
      if (k == 0) lift(4, i + Nq * j);
      if (k == N) lift(5, i + Nq * j);

      // Smagorinsky-Lilly (Eq. smago) or Vreman (Eq. vreman-sgs), times the
      // Richardson correction (Eq. richardson)
      double nut = 0.0, Dt = 0.0;
      if (P.closure == 1 || P.closure == 3) {
        double S2 = 0.0;
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
          for (int b = 0; b < 3; ++b) {
            const double Sab = 0.5 * (gr[a][b] + gr[b][a]);
            S2 += Sab * Sab;
          }
        const double Smag2 = 2.0 * S2;
        if (P.closure == 1)
          nut = Smag2 > 0.0 ? P.CsDelta2 * sqrt(Smag2) : 0.0;
        else
          nut = vreman_nu<double>(gr, P.vr_c, P.vr_d2);
        if (P.richardson && Smag2 > 0.0) {
          const double Ri = P.g * gr[5][2] / (G[5] * Smag2);
          if (Ri > 0.0) {
            const double a = 1.0 - Ri * P.inv_Prt;
            nut *= a > 0.0 ? sqrt(sqrt(a)) : 0.0;
          }
        }
        Dt = nut * P.inv_Prt;
      }
      // F2 rows: [rho d_i, rho tau_ij + d_i rho u_j, -rho D_t dh/dx_i + (rho tau u)_i],
      // d = -D_t grad q_t, rho tau = -2 rho nu_t S (Eqs. diff_moisture_flux,
      // stress_tensor, diff_energy_flux).
      const double rho = Y[0];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const double di = -Dt * gr[4][d];
        double rt[3];
#pragma unroll
        for (int b = 0; b < 3; ++b) rt[b] = -2.0 * rho * nut * (0.5 * (gr[d][b] + gr[b][d]));
        double *o = F2 + ((size_t)e * 15 + d * 5) * Np + t;
        o[0] = rho * di;
        o[1 * Np] = rt[0] + di * Y[1];
        o[2 * Np] = rt[1] + di * Y[2];
        o[3 * Np] = rt[2] + di * Y[3];
        o[4 * Np] = -rho * Dt * gr[3][d] + (rt[0] * G[0] + rt[1] * G[1] + rt[2] * G[2]);
      }
    }
    __syncthreads();
  }
}

// n.F1 in direction d (sign applied by the caller) of Eq. eom_compact:
// [rho u_d, rho u_j u_d + (p - p_r) delta_jd, (rho e + p) u_d, rho q_t u_d].
__device__ __forceinline__ void flux1_dir(const double Y[6], double rinv, double pprime, double pr, int d,
                                          double f[6]) {
  // the normal momentum by selection, not by a run-time index (which would
  // move the state to local memory when d is not a compile-time constant)
  const double yd = d == 0 ? Y[1] : (d == 1 ? Y[2] : Y[3]);
  const double ud = yd * rinv;
  f[0] = yd;
  f[1] = Y[1] * ud + (d == 0 ? pprime : 0.0);
  f[2] = Y[2] * ud + (d == 1 ? pprime : 0.0);
  f[3] = Y[3] * ud + (d == 2 ? pprime : 0.0);
  f[4] = (Y[4] + (pprime + pr)) * ud;
  f[5] = Y[5] * ud;
}

// FL: numerical flux of F1, 0 Rusanov, 1 HLLC, 2 Roe
// The flux pass's shared memory (dynamic: above N = 4 it exceeds the 48 KB of
// static shared memory).
template <int N>
struct Rhs64Smem {
  static constexpr int Nq = N + 1, Np = Nq * Nq * Nq, Nf = Nq * Nq;
  double sD[Nq * Nq];
  double sF[6][3][Np];
  double sY[6][Np];
  double sL[6][6][Nf];
  int sNb[6];
};

template <int N, bool UPDATE, int FL>
__global__ void __launch_bounds__(block64(N)) k_rhs64(const double *__restrict__ Q, const double *__restrict__ F2,
                                                      const double *__restrict__ TH, double *__restrict__ dQ,
                                                      double *__restrict__ Qout, double *__restrict__ THout,
                                                      const StageCoef sc, const KParams P) {
  constexpr int Nq = N + 1, Np = Nq * Nq * Nq, Nf = Nq * Nq;
  extern __shared__ __align__(16) unsigned char smem_rhs64[];
  Rhs64Smem<N> &SM = *reinterpret_cast<Rhs64Smem<N> *>(smem_rhs64);
  auto &sD = SM.sD;
  auto &sF = SM.sF;
  auto &sY = SM.sY;
  auto &sL = SM.sL;
  auto &sNb = SM.sNb;
  const int t = threadIdx.x;
  if (t < Nq * Nq) sD[t] = P.D[t];
  const int i = t % Nq, j = (t / Nq) % Nq, k = t / Nf;
  int fail = 0;
  for (int g = blockIdx.x; g < P.E; g += gridDim.x) {
    int ex, ey, ez;
    const int e = element_lin(P, g, ex, ey, ez);
    if (t < 6) sNb[t] = neighbour(P, ex, ey, ez, t);
    double Y[6];
    if (t < Np) {
      const int lev = ez * Nq + k;
#pragma unroll
      for (int v = 0; v < 6; ++v) {
        Y[v] = Q[((size_t)e * 6 + v) * Np + t];
        sY[v][t] = Y[v];
      }
      const double pp = TH[((size_t)e * 4) * Np + t];
      const double pr = P.p_r[lev];
      const double rinv = 1.0 / Y[0];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        double f[6];
        flux1_dir(Y, rinv, pp, pr, d, f);
        const double *g2 = F2 + ((size_t)e * 15 + d * 5) * Np + t;
        const double c0 = g2[0];
        sF[0][d][t] = f[0] + c0;
        sF[1][d][t] = f[1] + g2[1 * Np];
        sF[2][d][t] = f[2] + g2[2 * Np];
        sF[3][d][t] = f[3] + g2[3 * Np];
        sF[4][d][t] = f[4] + g2[4 * Np];
        sF[5][d][t] = f[5] + c0;
      }
    }
    __syncthreads();
    // surface terms, one task per (face, face node)
    for (int task = t; task < 6 * Nf; task += blockDim.x) {
      const int f = task / Nf, fn = task - f * Nf;
      const int d = f >> 1, t1 = fn % Nq, t2 = fn / Nq;
      const int a = (f & 1) ? N : 0;
      const double sg = (f & 1) ? 1.0 : -1.0;
      const int n = face_node<Nq>(d, a, t1, t2);
      const int lev = ez * Nq + (d == 2 ? a : t2);
      const double pr = P.p_r[lev];
      double Ym[6], Yp[6];
#pragma unroll
      for (int v = 0; v < 6; ++v) Ym[v] = sY[v][n];
      const double cm = TH[((size_t)e * 4 + 1) * Np + n];
      const int nb = sNb[f];
      if (FL == 0 && nb >= 0) {
        // Rusanov across an interior face.  The own node's total normal flux
        // n.(F1 + F2) is sF from the first phase, so the lifted jump
        // n.F_- - F* is 1/2 n.(F_- - F_+) - lambda/2 (Y_- - Y_+) and only
        // the neighbour's F1 is evaluated here.
        const int nn = face_node<Nq>(d, N - a, t1, t2);
#pragma unroll
        for (int v = 0; v < 6; ++v) Yp[v] = Q[((size_t)nb * 6 + v) * Np + nn];
        const double pp = TH[((size_t)nb * 4) * Np + nn];
        const double cp = TH[((size_t)nb * 4 + 1) * Np + nn];
        const double *g2p = F2 + ((size_t)nb * 15 + d * 5) * Np + nn;
        double fp[6];
        const double ip = 1.0 / Yp[0];
        flux1_dir(Yp, ip, pp, pr, d, fp);
        fp[0] += g2p[0];
        fp[1] += g2p[1 * Np];
        fp[2] += g2p[2 * Np];
        fp[3] += g2p[3 * Np];
        fp[4] += g2p[4 * Np];
        fp[5] += g2p[0];
        const double lm = fabs((d == 0 ? Ym[1] : (d == 1 ? Ym[2] : Ym[3])) / Ym[0]) + cm;
        const double lp = fabs((d == 0 ? Yp[1] : (d == 1 ? Yp[2] : Yp[3])) * ip) + cp;
        const double lam = fmax(lm, lp);
#pragma unroll
        for (int v = 0; v < 6; ++v)
          sL[f][v][fn] = P.lift[d] * (0.5 * sg * (sF[v][d][n] - fp[v]) - 0.5 * lam * (Ym[v] - Yp[v]));
        continue;
      }
      const double pm = TH[((size_t)e * 4) * Np + n];
      double pp, cp, f2s[5];
      if (nb >= 0) {
        const int nn = face_node<Nq>(d, N - a, t1, t2);
#pragma unroll
        for (int v = 0; v < 6; ++v) Yp[v] = Q[((size_t)nb * 6 + v) * Np + nn];
        pp = TH[((size_t)nb * 4) * Np + nn];
        cp = TH[((size_t)nb * 4 + 1) * Np + nn];
        const double *g2m = F2 + ((size_t)e * 15 + d * 5) * Np + n;
        const double *g2p = F2 + ((size_t)nb * 15 + d * 5) * Np + nn;
#pragma unroll
        for (int c = 0; c < 5; ++c) f2s[c] = 0.5 * (sg * g2m[c * Np] + sg * g2p[c * Np]);
      } else {
        // reflecting wall state (Eq. bc-velocity-impenetrable), scalars copied
#pragma unroll
        for (int v = 0; v < 6; ++v) Yp[v] = Ym[v];
        // (no-slip: u_bc = 0, every velocity component reversed)
        const bool ns = (P.noslip >> f) & 1;
        Yp[1] = (ns || d == 0) ? -Ym[1] : Ym[1];
        Yp[2] = (ns || d == 1) ? -Ym[2] : Ym[2];
        Yp[3] = (ns || d == 2) ? -Ym[3] : Ym[3];
        pp = pm;
        cp = cm;
        // wall-normal diffusive fluxes specified directly (App. A.3)
#pragma unroll
        for (int c = 0; c < 5; ++c) f2s[c] = 0.0;
        if (f == 4 && P.surface_flux) {
          f2s[0] = -P.E_water;
          f2s[4] = -P.E_energy;
        }
        if (f == 4 && P.drag_cd > 0.0) {
          // drag law (Eq. drag_law) on the flat bottom: outward flux
          // rho C_d |u_p| u_p of the horizontal momentum, u_p from the node
          // of the first interior layer above this face node
          const int ni = face_node<Nq>(2, 1, t1, t2);
          const double ri = 1.0 / sY[0][ni];
          const double ux = sY[1][ni] * ri, uy = sY[2][ni] * ri;
          const double c = Ym[0] * P.drag_cd * sqrt(ux * ux + uy * uy);
          f2s[1] = c * ux;
          f2s[2] = c * uy;
        }
      }
      double fm[6], fp[6], f1s[6];
      const double im = 1.0 / Ym[0], ip = 1.0 / Yp[0];
      flux1_dir(Ym, im, pm, pr, d, fm);
      flux1_dir(Yp, ip, pp, pr, d, fp);
      if (FL == 1) {
        // HLLC: n.F1(Y_K) + S_K (U*_K - U_K)
        const double uM[3] = {Ym[1] * im, Ym[2] * im, Ym[3] * im}, uP[3] = {Yp[1] * ip, Yp[2] * ip, Yp[3] * ip};
        const double nrm[3] = {d == 0 ? sg : 0.0, d == 1 ? sg : 0.0, d == 2 ? sg : 0.0};
        double J[6];
        const int K = hllc_jump<double>(Ym[0], uM, Ym[5] * im, Ym[4] * im, pm + pr, cm, Yp[0], uP, Yp[5] * ip,
                                        Yp[4] * ip, pp + pr, cp, pp - pm, nrm, J);
#pragma unroll
        for (int v = 0; v < 6; ++v) f1s[v] = sg * (K ? fp[v] : fm[v]) + J[v];
      } else if (FL == 2) {
        // Roe: 1/2 n.(F1- + F1+) - 1/2 |A| (Y+ - Y-)
        const double uM[3] = {Ym[1] * im, Ym[2] * im, Ym[3] * im}, uP[3] = {Yp[1] * ip, Yp[2] * ip, Yp[3] * ip};
        const double nrm[3] = {d == 0 ? sg : 0.0, d == 1 ? sg : 0.0, d == 2 ? sg : 0.0};
        double dY[6], D[6];
#pragma unroll
        for (int v = 0; v < 6; ++v) dY[v] = Yp[v] - Ym[v];
        const RoeConst<double> rk = {P.Rd, P.Rv - P.Rd, P.cvd, P.cvv - P.cvd, P.T0, P.Iv0};
        roe_dissipation<double>(Ym[0], uM, Ym[5] * im, (Ym[4] + pm + pr) * im, Yp[0], uP, Yp[5] * ip,
                                (Yp[4] + pp + pr) * ip, dY, P.g * node_z(P, ez, d == 2 ? a : t2), nrm, rk, D);
#pragma unroll
        for (int v = 0; v < 6; ++v) f1s[v] = 0.5 * (sg * fm[v] + sg * fp[v]) - 0.5 * D[v];
      } else {
        // Rusanov (Eq. nonviscFlux): 1/2 n.(F1- + F1+) + lambda/2 (Y- - Y+)
        const double lm = fabs((d == 0 ? Ym[1] : (d == 1 ? Ym[2] : Ym[3])) * im) + cm;
        const double lp = fabs((d == 0 ? Yp[1] : (d == 1 ? Yp[2] : Yp[3])) * ip) + cp;
        const double lam = fmax(lm, lp);
#pragma unroll
        for (int v = 0; v < 6; ++v) f1s[v] = 0.5 * (sg * fm[v] + sg * fp[v]) + 0.5 * lam * (Ym[v] - Yp[v]);
      }
      const int c_of_v[6] = {0, 1, 2, 3, 4, 0};
#pragma unroll
      for (int v = 0; v < 6; ++v) {
        const double fstar = f1s[v] + f2s[c_of_v[v]];
        sL[f][v][fn] = P.lift[d] * (sg * sF[v][d][n] - fstar);
      }
    }
    __syncthreads();
    if (t < Np) {
      const int lev = ez * Nq + k;
      double R[6];
#pragma unroll
      for (int v = 0; v < 6; ++v) {
        double a0 = 0.0, a1 = 0.0, a2 = 0.0;
#pragma unroll
        for (int m = 0; m < Nq; ++m) {
          a0 += sD[i * Nq + m] * sF[v][0][m + Nq * (j + Nq * k)];
          a1 += sD[j * Nq + m] * sF[v][1][i + Nq * (m + Nq * k)];
          a2 += sD[k * Nq + m] * sF[v][2][i + Nq * (j + Nq * m)];
        }
        double r = -(P.jac[0] * a0 + P.jac[1] * a1 + P.jac[2] * a2);
        if (i == 0) r += sL[0][v][j + Nq * k];
        if (i == N) r += sL[1][v][j + Nq * k];
        if (j == 0) r += sL[2][v][i + Nq * k];
        if (j == N) r += sL[3][v][i + Nq * k];
        if (k == 0) r += sL[4][v][i + Nq * j];
        if (k == N) r += sL[5][v][i + Nq * j];
        R[v] = r;
      }
      // sources: -(rho - rho_r) g k, -tau_s (rho u - rho u_relax), -2 Omega x rho u
      double tau = P.tau_lev[lev];
      if (P.tau_col) tau = fmax(tau, P.tau_col[(ex + P.gx0) * Nq + i]);
      double S[3];
      S[0] = -tau * (Y[1] - Y[0] * P.u_relax[0]);
      S[1] = -tau * (Y[2] - Y[0] * P.u_relax[1]);
      S[2] = -(Y[0] - P.rho_r[lev]) * P.g - tau * (Y[3] - Y[0] * P.u_relax[2]);
      S[0] -= 2.0 * (P.Omega[1] * Y[3] - P.Omega[2] * Y[2]);
      S[1] -= 2.0 * (P.Omega[2] * Y[1] - P.Omega[0] * Y[3]);
      S[2] -= 2.0 * (P.Omega[0] * Y[2] - P.Omega[1] * Y[1]);
      R[1] += S[0];
      R[2] += S[1];
      R[3] += S[2];
      double Yn[6];
#pragma unroll
      for (int v = 0; v < 6; ++v) {
        const size_t idx = ((size_t)e * 6 + v) * Np + t;
        if (UPDATE) {
          const double dq = (sc.A != 0.0 ? sc.A * dQ[idx] : 0.0) + sc.dt * R[v];
          dQ[idx] = dq;
          Yn[v] = Y[v] + sc.B * dq;
          Qout[idx] = Yn[v];
        } else {
          dQ[idx] = R[v];
        }
      }
      // the thermodynamics of the new state, for the next stage's two passes
      if (UPDATE) thermo_store64(P, Yn, node_z(P, ez, k), ez * Nq + k, THout, e, t, Np, fail);
    }
    __syncthreads();
  }
  report_thermo_flags(P, fail);
}

// The thermodynamic fields of a given state Q (one thread per node).
__global__ void k_thermo64(const double *__restrict__ Q, double *__restrict__ TH, const KParams P, int Np, int Nq) {
  const long long n = (long long)P.E * Np;
  int fail = 0;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
    const long long g = q / Np;
    const int node = (int)(q - g * Np);
    int ex, ey, ez;
    const long long e = element_lin(P, g, ex, ey, ez);
    const int k = node / (Nq * Nq);
    double Y[6];
#pragma unroll
    for (int v = 0; v < 6; ++v) Y[v] = Q[(e * 6 + v) * Np + node];
    thermo_store64(P, Y, node_z(P, ez, k), ez * Nq + k, TH, (size_t)e, node, Np, fail);
  }
  report_thermo_flags(P, fail);
}

// ------------------------------------------------------------------ launchers


int grid_for(const void *fn, int E, size_t smem, int threads) {
  int dev = 0, nsm = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, threads, smem);
  if (per < 1) per = 1;
  long long g = (long long)nsm * per;
  return (int)(g < E ? g : E);
}

// Persistent grid of a kernel of `threads` threads and dyn_smem bytes of
// dynamic shared memory that allocates tmem_cols Tensor Memory columns per
// CTA: the resident CTAs per SM from its registers and shared memory (the
// occupancy query reports 1 for such kernels), capped so that the resident
// CTAs' allocations fit in the SM's 512 columns.
int grid_for_tc(const void *fn, int E, int tmem_cols, int threads, size_t dyn_smem) {
  int dev = 0, nsm = 0, regs_sm = 0, smem_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaFuncAttributes a;
  if (cudaFuncGetAttributes(&a, fn) != cudaSuccess) {
    cudaGetLastError();
    return nsm < E ? nsm : E;
  }
  const int regs_cta = ((a.numRegs * 32 + 255) / 256 * 256) * (threads / 32);  // 256-register granules per warp
  int per = regs_cta > 0 ? regs_sm / regs_cta : 1;
  if (2048 / threads < per) per = 2048 / threads;
  const int smem_cta = (int)a.sharedSizeBytes + (int)dyn_smem + 1024;  // + the per-CTA reservation
  if (smem_cta > 0 && smem_sm / smem_cta < per) per = smem_sm / smem_cta;
  if (512 / tmem_cols < per) per = 512 / tmem_cols;
  if (per < 1) per = 1;
  const long long g = (long long)nsm * per;
  return (int)(g < E ? g : E);
}

cudaError_t launch_thermo64(const double *Q, double *TH, const KParams &P, int N, cudaStream_t s) {
  const int Nq = N + 1, Np = Nq * Nq * Nq;
  const long long nodes = (long long)P.E * Np;
  int blocks = (int)((nodes + 127) / 128);
  if (blocks > 148 * 16) blocks = 148 * 16;
  k_thermo64<<<blocks, 128, 0, s>>>(Q, TH, P, Np, Nq);
  return cudaGetLastError();
}

template <int N>
static void grad64_instance(const double *Q, const double *TH, double *F2, const KParams &P, cudaStream_t s) {
  static int grid = 0;
  if (!grid) grid = grid_for((const void *)k_grad64<N>, 1 << 30, 0, block64(N));
  k_grad64<N><<<grid < P.E ? grid : P.E, block64(N), 0, s>>>(Q, TH, F2, P);
}

// the FP64 flat-mesh kernels are instantiated for the orders 1 .. 7 (one
// thread per node)
cudaError_t launch_grad64(const double *Q, const double *TH, double *F2, const KParams &P, cudaStream_t s) {
  switch (P.N) {
    case 1: grad64_instance<1>(Q, TH, F2, P, s); break;
    case 2: grad64_instance<2>(Q, TH, F2, P, s); break;
    case 3: grad64_instance<3>(Q, TH, F2, P, s); break;
    case 4: grad64_instance<4>(Q, TH, F2, P, s); break;
    case 5: grad64_instance<5>(Q, TH, F2, P, s); break;
    case 6: grad64_instance<6>(Q, TH, F2, P, s); break;
    case 7: grad64_instance<7>(Q, TH, F2, P, s); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <int N, bool UPDATE, int FL>
static void rhs64_instance(const double *Q, const double *F2, const double *TH, double *dQ, double *Qout,
                           double *THout, const StageCoef &sc, const KParams &P, cudaStream_t s) {
  static int grid = 0;
  constexpr size_t smem = sizeof(Rhs64Smem<N>);
  if (!grid) {
    if (smem > 48 * 1024)
      cudaFuncSetAttribute((const void *)k_rhs64<N, UPDATE, FL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem);
    grid = grid_for((const void *)k_rhs64<N, UPDATE, FL>, 1 << 30, smem, block64(N));
  }
  k_rhs64<N, UPDATE, FL><<<grid < P.E ? grid : P.E, block64(N), smem, s>>>(Q, F2, TH, dQ, Qout, THout, sc, P);
}

template <int N>
static void rhs64_order(const double *Q, const double *F2, const double *TH, double *dQ, double *Qout,
                        double *THout, const StageCoef &sc, bool update, const KParams &P, cudaStream_t s) {
  if (update) {
    if (P.flux == 2)
      rhs64_instance<N, true, 2>(Q, F2, TH, dQ, Qout, THout, sc, P, s);
    else if (P.flux == 1)
      rhs64_instance<N, true, 1>(Q, F2, TH, dQ, Qout, THout, sc, P, s);
    else
      rhs64_instance<N, true, 0>(Q, F2, TH, dQ, Qout, THout, sc, P, s);
  } else {
    if (P.flux == 2)
      rhs64_instance<N, false, 2>(Q, F2, TH, dQ, Qout, THout, sc, P, s);
    else if (P.flux == 1)
      rhs64_instance<N, false, 1>(Q, F2, TH, dQ, Qout, THout, sc, P, s);
    else
      rhs64_instance<N, false, 0>(Q, F2, TH, dQ, Qout, THout, sc, P, s);
  }
}

cudaError_t launch_rhs64(const double *Q, const double *F2, const double *TH, double *dQ, double *Qout,
                         double *THout, const StageCoef &sc, bool update, const KParams &P, cudaStream_t s) {
  switch (P.N) {
    case 1: rhs64_order<1>(Q, F2, TH, dQ, Qout, THout, sc, update, P, s); break;
    case 2: rhs64_order<2>(Q, F2, TH, dQ, Qout, THout, sc, update, P, s); break;
    case 3: rhs64_order<3>(Q, F2, TH, dQ, Qout, THout, sc, update, P, s); break;
    case 4: rhs64_order<4>(Q, F2, TH, dQ, Qout, THout, sc, update, P, s); break;
    case 5: rhs64_order<5>(Q, F2, TH, dQ, Qout, THout, sc, update, P, s); break;
    case 6: rhs64_order<6>(Q, F2, TH, dQ, Qout, THout, sc, update, P, s); break;
    case 7: rhs64_order<7>(Q, F2, TH, dQ, Qout, THout, sc, update, P, s); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace cmles
