// Shared device-side definitions of the cmles CUDA path (sm_103a).
//
// Layout in HBM (element-major, the variable inside the element):
//   Q[e][v][n]      conserved state, v = rho, rho u, rho v, rho w, rho e_tot, rho q_t
//   F2[e][d][c][n]  diffusive flux in direction d (3) of the 5 distinct components
//                   c = (rho d_qt, momentum row d (3), energy); rho and rho q_t share c = 0
//   aux[e][a][n]    a = 0: p - p_r, a = 1: sound speed c
// with node n = i + Nq (j + Nq k) and element e = ex + nex (ey + ney ez).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace cmles {

constexpr int kMaxQ = 8;

// FP32 copies of the constants used by the FP32 kernels.
struct KF {
  float g, Rd, Rv, cvd, cvv, cvl, T0, Lv0, Iv0, kappa, pv_ptr, pv_Ttr, pv_a, pv_b, dcp;
  float inv_Ttr, inv_Rv;  // 1 / T_tr, 1 / R_v
  float CsDelta2, inv_Prt, Delta;
  float vr_c, vr_d2[3];
  float jac[3], lift[3];
  float inv_w0;  // 1 / w_0, the LGL end weight
  float kpow[6];  // binomial coefficients of (1 + v)^-kappa: kpow[n-1] = C(-kappa, n), n = 1..6
  float u_relax[3], Omega[3];
  float E_water, E_energy;
  float drag_cd;
};

// Per-level FP32 table of the FP32 path (16 floats per node level).
enum {
  L_RHO = 0, L_RHOQ, L_T, L_T_T0, L_GZ, L_P, L_H, L_HM, L_THV, L_DZ_HM, L_DZ_THV, L_RHORM, L_TAU, L_QM, L_DZ_Q,
  L_RVS,  // saturation vapour density p_v*(T_r) / (R_v T_r)
  L_NF = 16
};

// Everything a DG kernel needs, passed by value (kernel parameter space).
struct KParams {
  // thermodynamics (Table t:constants and readings) and derived constants
  double g, p0, Rd, Rv, cvd, cvv, cvl, T0, Lv0;
  double Iv0;        // L_v0 - R_v T_0
  double cpd;        // c_vd + R_d
  double kappa;      // R_d / c_pd (dry Exner exponent)
  double pv_ptr, pv_Ttr, pv_a, pv_b;  // p_v* = p_tr exp(a ln(T/T_tr) + b (1/T_tr - 1/T))
  double dcp;        // c_pv - c_pl
  double inv_Rd, inv_p0, inv_Ttr;
  // (p/p0)^-kappa = (p_r/p0)^-kappa (1 + p'/p_r)^-kappa: exr[level] is the
  // first factor, kpow64[n-1] = C(-kappa, n) (n = 1..11) the series of the second
  const double *exr;
  double kpow64[11];
  // tangents of the saturation vapour density rho_vs(T) = p_v*(T)/(R_v T) at
  // T_k = rvs_T0 + k rvs_dT, k < rvs_n: [k][2] = (rho_vs(T_k), d rho_vs/dT);
  // rho_vs is convex in T on the tabulated range (checked on the host when the
  // table is built; rvs_n = 0 disables the shortcut), so each tangent bounds it
  // from below there
  const double *rvs_tab;
  double rvs_T0, rvs_dT;
  int rvs_n;
  int rvs_ok;        // FP32 path: the tangent test at T_r may be used
  // closure
  double CsDelta2;   // (C_s Delta)^2
  double vr_c;       // 2.5 C_s^2 (Vreman)
  double vr_d2[3];   // Delta_m^2 = (h_m / N)^2 (Vreman)
  double Prt, inv_Prt;
  int richardson, moist, closure;
  int flux;          // numerical flux of F1: 0 Rusanov, 1 HLLC
  // sources
  double Omega[3], u_relax[3];
  int surface_flux;
  double E_water;    // LHF / L_v0 (kg m^-2 s^-1)
  double E_energy;   // SHF + LHF (W m^-2)
  double drag_cd;    // bottom-wall drag coefficient of Eq. drag_law (0: free slip)
  int noslip;        // wall faces (bit f) with the no-slip velocity ghost u+ = -u-
  // mesh (flat, uniform elements); N: the polynomial order
  int N;
  int nex, ney, nez, E;
  int periodic[3];
  double x0, y0, z0, hx, hy, hz;
  double jac[3];     // 2 / h_d: d xi_d / d x_d
  double lift[3];    // 2 / (w_0 h_d): w_s J_s / (w_i J_i) on a face normal to d
  // per node-level tables (level = ez (N+1) + k) and per x-column sponge table
  const double *rho_r, *p_r, *tau_lev, *tau_col;
  int satadj_max_iter;
  int *flags;        // [0] Newton non-convergence count, [1] CTAs whose tensor-core wait gave up
  int tc_stall;      // test hook: 1 the tensor-core kernels also wait on a barrier nothing arrives on;
                    // 2 their first MMA completion wait gives up at once
  int tiled;         // 1: visit elements in 4 x 4 column tiles (nex, ney multiples of 4)
  // one partition of a larger mesh split into (x, y) pencils (cmles_group):
  // the nex x ney x nez elements are the partition's interior, stored with
  // one ghost element on each side in x and y, (nex + 2) x (ney + 2) x nez
  // storage elements.  Ghost elements hold only the face nodes their interior
  // neighbours read, written by the halo exchange.  gx0, gy0: global indices
  // of the first interior element (sponge columns); wall[s] (s = 0 -x, 1 +x,
  // 2 -y, 3 +y): 1 where that side of the partition is a wall of the whole
  // mesh, 0 where a ghost element (a neighbouring partition's, or the
  // partition's own across a periodic boundary) lies.
  int part, gx0, gy0, wall[4];
  // FP32 path tables (see dg_fp32.cu): per level 16 floats, per element layer
  // the 5 x 5 differences of rho e_r + p_r along z, per level FP64 offsets
  const float *lev32, *dH32;
  const double *qref64;
  // FP32 path: sum of the step's stage increments B_s dQ_s so far [E][6][128]
  float *D32;
  const struct MlpPacked *mlp;  // learned-closure weights (closure == 2)
  // curvilinear meshes (dg_curved32.cu): per-node metrics [E][10][128]
  // ((J grad xi_r)_c at 3r + c, J at 9) and per-node tables [E][24][128]
  int curved;
  const float *geo32, *node32;
  // LGL basis
  double D[kMaxQ * kMaxQ], w[kMaxQ], xi[kMaxQ];
  KF f;
};

template <int Nq>
__device__ __forceinline__ int face_node(int d, int a, int t1, int t2) {
  return d == 0 ? a + Nq * (t1 + Nq * t2) : (d == 1 ? t1 + Nq * (a + Nq * t2) : t1 + Nq * (t2 + Nq * a));
}

// Freezing temperature (K).  The saturation adjustment keeps all condensate
// liquid (the ice phase of Sec. 2.7 is not modelled), and a node that
// condenses below it is counted, for information.
constexpr double kTfreeze = 273.15;

// Report a thread's thermodynamic flags (bit 0: the saturation adjustment did
// not converge; bit 1: condensate below freezing) as counts in the device
// flag words 0 and 2.
__device__ __forceinline__ void report_thermo_flags(const KParams &P, int fail) {
  if (fail & 1) atomicAdd(P.flags, 1);
  if (fail & 2) atomicAdd(P.flags + 2, 1);
}

// Padded nodes per element of the FP32 arrays at order N: 128 up to N = 4
// (one node per thread of a 128-thread CTA), above it (N+1)^3 rounded up to
// a whole warp (224, 352, 512), the CTA size of those orders.
__host__ __device__ constexpr int np32(int N) {
  return (N + 1) * (N + 1) * (N + 1) <= 128 ? 128 : ((N + 1) * (N + 1) * (N + 1) + 31) / 32 * 32;
}

// Storage index of the element with (interior) coordinates (ex, ey, ez); on
// a partition, -1 and nex (ney) are its ghost elements in x (y).
__host__ __device__ __forceinline__ int storage_index(const KParams &P, int ex, int ey, int ez) {
  return P.part ? (ex + 1) + (P.nex + 2) * ((ey + 1) + (P.ney + 2) * ez) : ex + P.nex * (ey + P.ney * ez);
}

// Neighbour of element (ex, ey, ez) across face f (0: -x, 1: +x, 2: -y, 3: +y,
// 4: -z, 5: +z) as a storage index; -1 marks a wall.
__device__ __forceinline__ int neighbour(const KParams &P, int ex, int ey, int ez, int f) {
  // selects rather than arrays indexed by the run-time direction
  const int d = f >> 1;
  const int n = d == 0 ? P.nex : (d == 1 ? P.ney : P.nez);
  int v = (d == 0 ? ex : (d == 1 ? ey : ez)) + ((f & 1) ? 1 : -1);
  if (v < 0 || v >= n) {
    if (P.part && d < 2) {
      if (P.wall[f]) return -1;  // otherwise the ghost element at -1 or n
    } else {
      if (!P.periodic[d]) return -1;
      v = v < 0 ? v + n : v - n;
    }
  }
  return storage_index(P, d == 0 ? v : ex, d == 1 ? v : ey, d == 2 ? v : ez);
}

// Element visited at position g of a kernel's traversal (g < P.E, the
// interior elements): its storage index, and its coordinates in (ex, ey, ez).
// With tiling, the traversal walks 4 x 4 columns of elements bottom to top,
// so that the x, y and z neighbours of an element are visited close in time
// and their face data is still in L2 when it is gathered.
__device__ __forceinline__ int element_at(const KParams &P, int g, int &ex, int &ey, int &ez) {
  if (P.tiled) {
    const int per_tile = 16 * P.nez;
    const int t = g / per_tile, r = g - t * per_tile;
    const int tiles_x = P.nex >> 2;
    ez = r >> 4;
    ex = ((t % tiles_x) << 2) + (r & 3);
    ey = ((t / tiles_x) << 2) + ((r >> 2) & 3);
  } else {
    ex = g % P.nex;
    ey = (g / P.nex) % P.ney;
    ez = g / (P.nex * P.ney);
  }
  return storage_index(P, ex, ey, ez);
}

// For the first six lanes of a warp: element g of the traversal, its
// storage index, layer and column to el[0], el[1], el[2] (lane 0), and its
// neighbour across face `lane` to nb[lane].
__device__ __forceinline__ void next_element(const KParams &P, int g, int *el, int *nb) {
  int ex, ey, ez;
  const int e = element_at(P, g, ex, ey, ez);
  const int lane = threadIdx.x & 31;
  nb[lane] = neighbour(P, ex, ey, ez, lane);
  if (lane == 0) {
    el[0] = e;
    el[1] = ez;
    el[2] = ex;
  }
}

// The same in the plain order x fastest (kernels that do not tile).
__device__ __forceinline__ int element_lin(const KParams &P, long long g, int &ex, int &ey, int &ez) {
  ex = (int)(g % P.nex);
  ey = (int)((g / P.nex) % P.ney);
  ez = (int)(g / ((long long)P.nex * P.ney));
  return storage_index(P, ex, ey, ez);
}

__device__ __forceinline__ double node_z(const KParams &P, int ez, int k) {
  return P.z0 + (ez + 0.5 * (P.xi[k] + 1.0)) * P.hz;
}

// LSRK(5,4) stage coefficients (Carpenter & Kennedy 1994, Sec. 3.2).
// last: the final stage of a step, which adds the step's accumulated
// increment to the FP64 state (FP32 path).
// The FP32 kernels use the FP32 copies Af, Bf, dtf (converted once on the
// host: an FP64 operation per thread costs 64 FP32 ones on B300) and
// first (A = 0: no register to read).
struct StageCoef {
  double A, B, dt;
  int last;
  float Af, Bf, dtf;
  int first;
};


// Vreman eddy viscosity (Eq. vreman-sgs) from gr[i][m] = d u_i / d x_m and
// d2[m] = Delta_m^2.  B_beta, the sum of the 2x2 principal minors of
// beta = A A^T with A = grad(u) diag(Delta_m), is evaluated by the
// Cauchy-Binet identity as sum_{i<j} sum_{m<n} Delta_m^2 Delta_n^2
// (u_i,m u_j,n - u_i,n u_j,m)^2: a sum of squares, so rounding cannot turn
// it negative and a nearly rank-one gradient (a shear) loses no digits.
template <typename T>
__device__ __forceinline__ T vreman_nu(const T (&gr)[6][3], T c25, const T (&d2)[3]) {
  T uu = T(0), B = T(0);
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) uu += gr[a][b] * gr[a][b];
  constexpr int lo[3] = {0, 0, 1}, hi[3] = {1, 2, 2};
#pragma unroll
  for (int p = 0; p < 3; ++p) {
    const int m = lo[p], n = hi[p];
    T acc = T(0);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const int i = lo[q], j = hi[q];
      const T det = gr[i][m] * gr[j][n] - gr[i][n] * gr[j][m];
      acc += det * det;
    }
    B += d2[m] * d2[n] * acc;
  }
  return uu > T(0) ? c25 * sqrt(B / uu) : T(0);
}


// HLLC numerical flux (Toro, Spruce & Speares 1994; named in Sec. 3.1) in the
// form n.F* = n.F1(Y_K) + J on a face of unit normal n, with the Davis wave
// speeds S_L = min(u_L - c_L, u_R - c_R), S_R = max(u_L + c_L, u_R + c_R),
// u = u.n.  Returns the side K (0 = left, the own element; 1 = right) whose
// flux is used and writes J = S_K (U*_K - U_K) (zero in the supersonic cases).
// The star-state jump is formed as products of small factors,
//   rho* - rho = rho (S* - u)/(S - S*) =: dr,
//   (rho u)* - rho u = dr u + rho chi (S* - u) n,  chi = (S - u)/(S - S*),
//   E* - E = e dr + rho chi (S* - u)(S* + p / (rho (S - u))),
//   (rho q)* - rho q = q dr,
// so that no large state is differenced.  Per side: density, velocity,
// specific water q, total energy per unit mass e = E/rho (with g z), full
// pressure p and sound speed c; dp = p_R - p_L.
template <typename T>
__device__ __forceinline__ int hllc_jump(T rL, const T (&uL)[3], T qL, T eL, T pL, T cL, T rR, const T (&uR)[3], T qR,
                                         T eR, T pR, T cR, T dp, const T (&n)[3], T J[6]) {
  const T unL = uL[0] * n[0] + uL[1] * n[1] + uL[2] * n[2];
  const T unR = uR[0] * n[0] + uR[1] * n[1] + uR[2] * n[2];
  const T SL = fmin(unL - cL, unR - cR), SR = fmax(unL + cL, unR + cR);
#pragma unroll
  for (int v = 0; v < 6; ++v) J[v] = T(0);
  if (SL >= T(0)) return 0;
  if (SR <= T(0)) return 1;
  const T Ss = (dp + rL * unL * (SL - unL) - rR * unR * (SR - unR)) / (rL * (SL - unL) - rR * (SR - unR));
  const int K = Ss >= T(0) ? 0 : 1;
  const T r = K ? rR : rL, un = K ? unR : unL, S = K ? SR : SL;
  const T q = K ? qR : qL, e = K ? eR : eL, p = K ? pR : pL;
  const T iden = T(1) / (S - Ss);
  const T chi = (S - un) * iden;
  const T dr = r * (Ss - un) * iden;
  const T rcs = r * chi * (Ss - un);
  J[0] = S * dr;
#pragma unroll
  for (int c = 0; c < 3; ++c) J[1 + c] = S * (dr * (K ? uR[c] : uL[c]) + rcs * n[c]);
  J[4] = S * (e * dr + rcs * (Ss + p / (r * (S - un))));
  J[5] = S * q * dr;
  return K;
}


// Roe flux (Roe 1981; named in Sec. 3.1): the dissipation |A| dY of
// n.F* = (n.F(Y-) + n.F(Y+))/2 - |A| dY / 2, A the flux Jacobian along n at
// Roe's averaged state (sqrt(rho)-weighted u, total specific enthalpy H and
// q_t) with the frozen (q_l = 0) moist equation of state,
//   p = G (E - rho |u|^2/2 - rho Phi - rho q I_v0) + rho R_m T_0,  G = R_m/c_vm,
// whose derivatives give c^2 = p_rho + u.p_m + H p_E + q p_w.  Acoustic
// strengths a_-+ = (dp -+ rho^ c du_n)/(2 c^2) on r_-+ = (1, u -+ c n,
// H -+ u_n c, q); every other wave moves at u_n:
//   |A| dY = |u_n - c| a_- r_- + |u_n + c| a_+ r_+ + |u_n| (dY - a_- r_- - a_+ r_+).
template <typename T>
struct RoeConst {
  T Rd, dR, cvd, dc, T0, Iv0;  // R_d, R_v - R_d, c_vd, c_vv - c_vd, T_0, L_v0 - R_v T_0
};
template <typename T>
__device__ __forceinline__ void roe_dissipation(T rL, const T (&uL)[3], T qL, T HL, T rR, const T (&uR)[3], T qR,
                                                T HR, const T (&dY)[6], T Phi, const T (&n)[3],
                                                const RoeConst<T> &k, T D[6]) {
  const T wL = sqrt(rL), wR = sqrt(rR), iw = T(1) / (wL + wR), rh = wL * wR;
  T u[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) u[c] = (wL * uL[c] + wR * uR[c]) * iw;
  const T H = (wL * HL + wR * HR) * iw, q = (wL * qL + wR * qR) * iw;
  const T uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  const T Rm = k.Rd + q * k.dR, cvm = k.cvd + q * k.dc, G = Rm / cvm;
  const T Tt = (H - T(0.5) * uu - Phi - q * k.Iv0 + cvm * k.T0) / (cvm + Rm);
  const T p_rho = (k.Rd - G * k.cvd) * (Tt - k.T0) + G * (T(0.5) * uu - Phi) + k.Rd * k.T0;
  const T p_w = (k.dR - G * k.dc) * (Tt - k.T0) - G * k.Iv0 + k.dR * k.T0;
  const T c2 = p_rho - G * uu + G * H + q * p_w, c = sqrt(c2);
  const T dp = p_rho * dY[0] - G * (u[0] * dY[1] + u[1] * dY[2] + u[2] * dY[3]) + G * dY[4] + p_w * dY[5];
  const T un = u[0] * n[0] + u[1] * n[1] + u[2] * n[2];
  const T dun = (n[0] * dY[1] + n[1] * dY[2] + n[2] * dY[3] - un * dY[0]) / rh;
  const T am = (dp - rh * c * dun) / (T(2) * c2), ap = (dp + rh * c * dun) / (T(2) * c2);
  const T lm = fabs(un - c), lp = fabs(un + c), l0 = fabs(un);
  const T rm[6] = {T(1), u[0] - c * n[0], u[1] - c * n[1], u[2] - c * n[2], H - un * c, q};
  const T rp[6] = {T(1), u[0] + c * n[0], u[1] + c * n[1], u[2] + c * n[2], H + un * c, q};
#pragma unroll
  for (int v = 0; v < 6; ++v) {
    const T wm = am * rm[v], wp = ap * rp[v];
    D[v] = lm * wm + lp * wp + l0 * (dY[v] - wm - wp);
  }
}

}  // namespace cmles
