// C ABI of the cmles library (declared in include/cmles.h): handle set-up on
// the host (LGL basis, mesh tables, reference state, sponge), device buffers,
// and the stage loop that launches the DG kernels.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <string>
#include <utility>
#include <vector>

#include "handle.h"

namespace {

// LSRK(5,4), Carpenter & Kennedy (1994), 2N-storage form:
//   dQ <- A_s dQ + dt RHS(Q),  Q <- Q + B_s dQ.
const double kLsrkA[5] = {0.0, -567301805773.0 / 1357537059087.0, -2404267990393.0 / 2016746695238.0,
                          -3550918686646.0 / 2091501179385.0, -1275806237668.0 / 842570457699.0};
const double kLsrkB[5] = {1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0,
                          1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0,
                          2277821191437.0 / 14882151754819.0};

// LSRK(14,4), Niegemann, Diehl & Busch (2012), the same 2N-storage form.
const double kLsrk14A[14] = {0.0,
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
const double kLsrk14B[14] = {0.0367762454319673, 0.3136296607553959, 0.1531848691869027, 0.0030097086818182,
                             0.3326293790646110, 0.2440251405350864, 0.3718879239592277, 0.6204126221582444,
                             0.1524043173028741, 0.0760894927419266, 0.0077604214040978, 0.0024647284755382,
                             0.0780348340049386, 5.5059777270269628};

// Legendre P_N and P_{N-1} at x by the three-term recurrence.
void legendre_pair(int N, double x, double *PN, double *PNm1) {
  double pm = 1.0, p = x;
  if (N == 0) {
    *PN = 1.0;
    *PNm1 = 0.0;
    return;
  }
  for (int k = 1; k < N; ++k) {
    double pn = ((2.0 * k + 1.0) * x * p - k * pm) / (k + 1.0);
    pm = p;
    p = pn;
  }
  *PN = p;
  *PNm1 = pm;
}

// LGL nodes as the zeros of f(x) = (1 - x^2) P_N'(x) = N (P_{N-1} - x P_N),
// found by Newton with f'(x) = -N (N+1) P_N(x) (Legendre's equation) from the
// Chebyshev-Lobatto points; weights 2 / (N (N+1) P_N^2); derivative matrix in
// the classical closed form D_ij = P_N(x_i) / (P_N(x_j) (x_i - x_j)),
// D_00 = -N(N+1)/4, D_NN = N(N+1)/4, other diagonal entries 0.
void lgl_basis(int N, std::vector<double> &x, std::vector<double> &w, std::vector<double> &D) {
  const int Nq = N + 1;
  x.assign(Nq, 0.0);
  w.assign(Nq, 0.0);
  D.assign(Nq * Nq, 0.0);
  for (int i = 0; i < Nq; ++i) {
    double xi = -cos(M_PI * i / N);
    if (i > 0 && i < N) {
      for (int it = 0; it < 200; ++it) {
        double PN, PNm1;
        legendre_pair(N, xi, &PN, &PNm1);
        const double step = (PNm1 - xi * PN) / ((N + 1.0) * PN);
        xi += step;
        if (fabs(step) < 1e-17) break;
      }
    }
    x[i] = xi;
  }
  x[0] = -1.0;
  x[N] = 1.0;
  for (int i = 0; i < Nq / 2; ++i) {  // exact symmetry about 0
    const double h = 0.5 * (x[N - i] - x[i]);
    x[i] = -h;
    x[N - i] = h;
  }
  if (N % 2 == 0) x[N / 2] = 0.0;
  std::vector<double> PN(Nq);
  for (int i = 0; i < Nq; ++i) {
    double pm;
    legendre_pair(N, x[i], &PN[i], &pm);
    w[i] = 2.0 / (N * (N + 1.0) * PN[i] * PN[i]);
  }
  for (int i = 0; i < Nq; ++i)
    for (int j = 0; j < Nq; ++j) D[i * Nq + j] = i == j ? 0.0 : PN[i] / (PN[j] * (x[i] - x[j]));
  D[0] = -N * (N + 1.0) / 4.0;
  D[N * Nq + N] = N * (N + 1.0) / 4.0;
}

}  // namespace


namespace cmles_host {

cmles_status fail(cmles_handle h, cmles_status st, const std::string &msg) {
  if (h) h->err = msg;
  return st;
}

cmles_status dalloc(cmles_handle h, void **p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(h, CMLES_ERR_OOM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed: " +
                                      cudaGetErrorString(e));
  }
  h->bytes += (long long)bytes;
  return CMLES_OK;
}

// launch bookkeeping: count every kernel; with timing on, bracket by events
LaunchScope::LaunchScope(cmles_handle h_, int kind_, int nkernels) : h(h_), kind(kind_), nk(nkernels) {
  h->launches += nk;
  if (h->timing) {
    cudaEventCreate(&tl.a);
    cudaEventCreate(&tl.b);
    cudaEventRecord(tl.a, h->stream);
  }
}
LaunchScope::~LaunchScope() {
  if (h->timing) {
    cudaEventRecord(tl.b, h->stream);
    tl.kind = kind;
    h->timed.push_back(tl);
  }
}

void fill_kparams(cmles_handle h) {
  const cmles_params &p = h->prm;
  const cmles_mesh &m = h->mesh;
  KParams &K = h->K;
  memset(&K, 0, sizeof(K));
  K.g = p.g;
  K.p0 = p.p0;
  K.Rd = p.Rd;
  K.Rv = p.Rv;
  K.cvd = p.cvd;
  K.cvv = p.cvv;
  K.cvl = p.cvl;
  K.T0 = p.T0;
  K.Lv0 = p.Lv0;
  K.Iv0 = p.Lv0 - p.Rv * p.T0;
  K.cpd = p.cvd + p.Rd;
  K.kappa = p.Rd / K.cpd;
  K.dcp = (p.cvv + p.Rv) - p.cvl;
  K.pv_ptr = p.ptr;
  K.pv_Ttr = p.Ttr;
  K.pv_a = K.dcp / p.Rv;
  K.pv_b = (p.Lv0 - K.dcp * p.T0) / p.Rv;
  K.inv_Rd = 1.0 / p.Rd;
  K.inv_p0 = 1.0 / p.p0;
  K.inv_Ttr = 1.0 / p.Ttr;
  {
    double c = 1.0;
    for (int n = 1; n <= 11; ++n) {
      c *= (-K.kappa - (n - 1)) / n;
      K.kpow64[n - 1] = c;
    }
  }
  K.exr = h->exr;
  K.Prt = p.Prt;
  K.inv_Prt = 1.0 / p.Prt;
  K.richardson = p.richardson;
  K.moist = p.moist;
  K.closure = p.closure;
  K.flux = p.flux;
  for (int c = 0; c < 3; ++c) {
    K.Omega[c] = p.Omega[c];
    K.u_relax[c] = p.u_relax[c];
    K.periodic[c] = m.periodic[c];
  }
  K.surface_flux = p.surface_flux;
  K.E_water = p.lhf / p.Lv0;
  K.E_energy = p.shf + p.lhf;
  K.drag_cd = p.drag_cd;
  K.noslip = p.noslip;
  K.N = h->N;
  K.nex = m.nex;
  K.ney = m.ney;
  K.nez = m.nez;
  K.E = (int)h->E;
  K.x0 = m.x0;
  K.y0 = m.y0;
  K.z0 = m.z0;
  K.hx = m.Lx / m.nex;
  K.hy = m.Ly / m.ney;
  K.hz = m.Lz / m.nez;
  const double hd[3] = {K.hx, K.hy, K.hz};
  for (int d = 0; d < 3; ++d) {
    K.jac[d] = 2.0 / hd[d];
    K.lift[d] = 2.0 / (h->w[0] * hd[d]);
  }
  // Delta = (element volume)^(1/3) / N (Sec. 4.1, geometric mean of L_d / N)
  const double Delta = cbrt(K.hx * K.hy * K.hz) / h->N;
  K.CsDelta2 = (p.Cs * Delta) * (p.Cs * Delta);
  // Vreman: Delta_m = h_m / N per direction
  K.vr_c = 2.5 * p.Cs * p.Cs;
  for (int d = 0; d < 3; ++d) K.vr_d2[d] = (hd[d] / h->N) * (hd[d] / h->N);
  K.satadj_max_iter = p.satadj_max_iter > 0 ? p.satadj_max_iter : 20;
  for (int a = 0; a < h->Nq; ++a) {
    K.w[a] = h->w[a];
    K.xi[a] = h->xi[a];
    for (int b = 0; b < h->Nq; ++b) K.D[a * h->Nq + b] = h->D[a * h->Nq + b];
  }
  KF &F = K.f;
  F.g = (float)p.g;
  F.Rd = (float)p.Rd;
  F.Rv = (float)p.Rv;
  F.cvd = (float)p.cvd;
  F.cvv = (float)p.cvv;
  F.cvl = (float)p.cvl;
  F.T0 = (float)p.T0;
  F.Lv0 = (float)p.Lv0;
  F.Iv0 = (float)K.Iv0;
  F.kappa = (float)K.kappa;
  F.pv_ptr = (float)K.pv_ptr;
  F.pv_Ttr = (float)K.pv_Ttr;
  F.pv_a = (float)K.pv_a;
  F.pv_b = (float)K.pv_b;
  F.inv_Ttr = (float)(1.0 / K.pv_Ttr);
  F.inv_Rv = (float)(1.0 / p.Rv);
  F.dcp = (float)K.dcp;
  F.CsDelta2 = (float)K.CsDelta2;
  F.Delta = (float)Delta;
  F.vr_c = (float)K.vr_c;
  F.inv_w0 = (float)(1.0 / h->w[0]);
  {
    double c = 1.0;
    for (int n = 1; n <= 6; ++n) {
      c *= (-K.kappa - (n - 1)) / n;
      F.kpow[n - 1] = (float)c;
    }
  }
  for (int d = 0; d < 3; ++d) F.vr_d2[d] = (float)K.vr_d2[d];
  K.mlp = h->mlp_dev;
  F.inv_Prt = (float)K.inv_Prt;
  for (int d = 0; d < 3; ++d) {
    F.jac[d] = (float)K.jac[d];
    F.lift[d] = (float)K.lift[d];
    F.u_relax[d] = (float)p.u_relax[d];
    F.Omega[d] = (float)p.Omega[d];
  }
  F.E_water = (float)K.E_water;
  F.E_energy = (float)K.E_energy;
  F.drag_cd = (float)K.drag_cd;
  K.tiled = (m.nex % 4 == 0 && m.ney % 4 == 0) ? 1 : 0;
  K.lev32 = h->lev32;
  K.dH32 = h->dH32;
  K.qref64 = h->qref64;
  K.D32 = h->D32;
  K.rho_r = h->rho_r;
  K.p_r = h->p_r;
  K.tau_lev = h->tau_lev;
  K.tau_col = h->tau_col;
  K.flags = h->flags;
  K.tc_stall = h->tc_stall;
}

double level_z(cmles_handle h, int lev) {
  const int ez = lev / h->Nq, k = lev % h->Nq;
  return h->K.z0 + (ez + 0.5 * (h->xi[k] + 1.0)) * h->K.hz;
}

// One gradient pass and one flux pass on the shadow S32[in]; with update the
// stage's new shadow and its thermodynamic fields go to buffer 1 - in.
cmles_status run_stage_pair32(cmles_handle h, int in, double *Rout, const StageCoef &sc, bool update) {
  const float *Sin = h->S32[in];
  float *Sout = update ? h->S32[1 - in] : nullptr;
  {
    LaunchScope ls(h, 0, 1);
    if (h->curved)
      CK(launch_grad32c(Sin, h->TH32[in], h->F2_32, h->K, h->stream));
    else
      CK(launch_grad32(Sin, h->TH32[in], h->F2_32, h->K, h->stream));
  }
  {
    LaunchScope ls(h, 1, 1);
    float *THout = update ? h->TH32[1 - in] : nullptr;
    if (h->curved)
      CK(launch_rhs32c(Sin, h->F2_32, h->TH32[in], h->dQ32, h->Q[0], Sout, THout, Rout, sc, update, h->K, h->stream));
    else
      CK(launch_rhs32(Sin, h->F2_32, h->TH32[in], h->dQ32, h->Q[0], Sout, THout, Rout, sc, update, h->K, h->stream));
  }
  return CMLES_OK;
}

// the shadow of the FP64 state Q (with its thermodynamic fields) into buffer i
cmles_status write_shadow(cmles_handle h, const double *Q, int i) {
  LaunchScope ls(h, 2, 1);
  if (h->curved)
    CK(launch_shadow32c(Q, h->S32[i], h->TH32[i], h->K, h->N, h->stream));
  else
    CK(launch_shadow32(Q, h->S32[i], h->TH32[i], h->K, h->N, h->stream));
  return CMLES_OK;
}

// the thermodynamic fields of the FP64 state Q into TH
cmles_status write_thermo64(cmles_handle h, const double *Q, double *TH) {
  LaunchScope ls(h, 2, 1);
  CK(launch_thermo64(Q, TH, h->K, h->N, h->stream));
  return CMLES_OK;
}

// FP32: the shadow of the state and its thermodynamic fields; FP64: the
// state's thermodynamic fields (both built when the state has changed).
cmles_status ensure_shadow(cmles_handle h) {
  if (!h->shadow_valid) {
    cmles_status st = h->fp32 ? write_shadow(h, h->Q[0], h->scur) : write_thermo64(h, h->Q[h->cur], h->TH64[h->cur]);
    if (st != CMLES_OK) return st;
    h->shadow_valid = true;
  }
  return CMLES_OK;
}

// One gradient pass and one flux pass of the FP64 path on Qin, whose
// thermodynamic fields are THin; with update the stage's new state and its
// fields go to Qout and THout.
cmles_status run_stage_pair(cmles_handle h, const double *Qin, const double *THin, double *Qout, double *THout,
                            double *dQ, const StageCoef &sc, bool update) {
  {
    LaunchScope ls(h, 0, 1);
    CK(launch_grad64(Qin, THin, h->F2, h->K, h->stream));
  }
  {
    LaunchScope ls(h, 1, 1);
    CK(launch_rhs64(Qin, h->F2, THin, dQ, Qout, THout, sc, update, h->K, h->stream));
  }
  return CMLES_OK;
}


// ---- curvilinear (warped) meshes ----

// Terrain height of the warped mesh: z_s(x) = h exp(-((x - x_c)/a)^2).
double terrain(const cmles_mesh &m, double x) {
  const double s = (x - m.hill_xc) / m.hill_a;
  return m.hill_h * exp(-s * s);
}

// Node coordinates (z' = z + z_s(x)(1 - (z - z0)/Lz)), Jacobian, metric terms
// in the conservative curl form (J a^r)_c = -[curl_xi(X_l grad_xi X_m)]_r with
// (c, m, l) cyclic, and the per-element filter width; uploads the FP32
// metrics [E][10][np32(N)] and the quadrature weights w_n J_n.
cmles_status build_curved(cmles_handle h) {
  const cmles_mesh &m = h->mesh;
  const int Nq = h->Nq, Np = h->Np, np = np32(h->N);
  const long long E = h->E;
  const double hx = m.Lx / m.nex, hy = m.Ly / m.ney, hz = m.Lz / m.nez;
  h->hx_.resize((size_t)E * Np);
  h->hz_.resize((size_t)E * Np);
  h->hJ_.resize((size_t)E * Np);
  h->hJa_.resize((size_t)E * Np * 9);
  h->hdelta_.resize(E);
  h->hvr_.resize((size_t)E * 3);
  std::vector<float> geo((size_t)E * 10 * np, 0.0f);
  std::vector<double> wJ((size_t)E * Np);
  std::vector<double> X(3 * Np), dX(9 * Np), V(3 * Np);
  auto at = [&](int i, int j, int k) { return i + Nq * (j + Nq * k); };
  // derivative along reference direction r of nodal field f at node n
  auto dref = [&](const double *f, int n, int r) {
    int ijk[3] = {n % Nq, (n / Nq) % Nq, n / (Nq * Nq)};
    double acc = 0.0;
    for (int q = 0; q < Nq; ++q) {
      int t[3] = {ijk[0], ijk[1], ijk[2]};
      t[r] = q;
      acc += h->D[ijk[r] * Nq + q] * f[at(t[0], t[1], t[2])];
    }
    return acc;
  };
  for (long long e = 0; e < E; ++e) {
    const int ex = (int)(e % m.nex), ey = (int)((e / m.nex) % m.ney), ez = (int)(e / ((long long)m.nex * m.ney));
    for (int n = 0; n < Np; ++n) {
      const int i = n % Nq, j = (n / Nq) % Nq, k = n / (Nq * Nq);
      const double x = m.x0 + (ex + 0.5 * (h->xi[i] + 1.0)) * hx;
      const double y = m.y0 + (ey + 0.5 * (h->xi[j] + 1.0)) * hy;
      double z = m.z0 + (ez + 0.5 * (h->xi[k] + 1.0)) * hz;
      if (m.warp) z = z + terrain(m, x) * (1.0 - (z - m.z0) / m.Lz);
      X[n] = x;
      X[Np + n] = y;
      X[2 * Np + n] = z;
      h->hx_[e * Np + n] = x;
      h->hz_[e * Np + n] = z;
    }
    // Vreman's directional lengths: the extent of the element's nodes along
    // x, y and z over N (reading for a curved element: its bounding box)
    for (int c = 0; c < 3; ++c) {
      double lo = X[c * Np], hi = X[c * Np];
      for (int n = 1; n < Np; ++n) {
        lo = fmin(lo, X[c * Np + n]);
        hi = fmax(hi, X[c * Np + n]);
      }
      h->hvr_[e * 3 + c] = ((hi - lo) / h->N) * ((hi - lo) / h->N);
    }
    // metrics from element-local coordinates (the curl form is translation
    // invariant; local coordinates keep the rounding independent of position)
    for (int c = 0; c < 3; ++c) {
      const double x0n = X[c * Np];
      for (int n = 0; n < Np; ++n) X[c * Np + n] -= x0n;
    }
    for (int c = 0; c < 3; ++c)
      for (int r = 0; r < 3; ++r)
        for (int n = 0; n < Np; ++n) dX[(c * 3 + r) * Np + n] = dref(&X[c * Np], n, r);
    double vol = 0.0;
    for (int n = 0; n < Np; ++n) {
      const double *a = &dX[n];
      auto d = [&](int c, int r) { return a[(c * 3 + r) * Np]; };
      const double J = d(0, 0) * (d(1, 1) * d(2, 2) - d(1, 2) * d(2, 1)) -
                       d(0, 1) * (d(1, 0) * d(2, 2) - d(1, 2) * d(2, 0)) +
                       d(0, 2) * (d(1, 0) * d(2, 1) - d(1, 1) * d(2, 0));
      h->hJ_[e * Np + n] = J;
      const int i = n % Nq, j = (n / Nq) % Nq, k = n / (Nq * Nq);
      wJ[e * Np + n] = h->w[i] * h->w[j] * h->w[k] * J;
      vol += wJ[e * Np + n];
    }
    h->hdelta_[e] = cbrt(vol) / h->N;
    for (int c = 0; c < 3; ++c) {
      const int mm = (c + 1) % 3, ll = (c + 2) % 3;
      for (int r = 0; r < 3; ++r)
        for (int n = 0; n < Np; ++n) V[r * Np + n] = X[ll * Np + n] * dX[(mm * 3 + r) * Np + n];
      for (int n = 0; n < Np; ++n) {
        const double c0 = dref(&V[2 * Np], n, 1) - dref(&V[1 * Np], n, 2);
        const double c1 = dref(&V[0 * Np], n, 2) - dref(&V[2 * Np], n, 0);
        const double c2 = dref(&V[1 * Np], n, 0) - dref(&V[0 * Np], n, 1);
        double *ja = &h->hJa_[(e * Np + n) * 9];
        ja[0 * 3 + c] = -c0;
        ja[1 * 3 + c] = -c1;
        ja[2 * 3 + c] = -c2;
      }
    }
    for (int n = 0; n < Np; ++n) {
      for (int q = 0; q < 9; ++q) geo[((size_t)e * 10 + q) * np + n] = (float)h->hJa_[(e * Np + n) * 9 + q];
      geo[((size_t)e * 10 + 9) * np + n] = (float)h->hJ_[e * Np + n];
    }
  }
  CK(cudaMemcpy(h->geo32, geo.data(), geo.size() * sizeof(float), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(h->wJn, wJ.data(), wJ.size() * sizeof(double), cudaMemcpyHostToDevice));
  return CMLES_OK;
}

// Per-node FP32 tables and FP64 offsets of a curvilinear mesh from the
// per-node reference (rho_r, p_r, q_r): the level-table fields of the flat
// path per node, the full reference gradients of h_r, q_r, theta_v,r (the
// DG gradient operator applied to the nodal reference values), Delta,
// (C_s Delta)^2 and the sponge coefficient.
// saturation vapour density p_v*(T) / (R_v T) in FP64 (integrated
// Clausius-Clapeyron relation with the constants of the handle)
static double rhovsat64(cmles_handle h, double T) {
  const KParams &K = h->K;
  return K.pv_ptr * exp(K.pv_a * log(T / K.pv_Ttr) + K.pv_b * (1.0 / K.pv_Ttr - 1.0 / T)) / (h->prm.Rv * T);
}

cmles_status curved_reference(cmles_handle h, const double *rho_r, const double *p_r, const double *qt_r) {
  const cmles_params &p = h->prm;
  const cmles_mesh &m = h->mesh;
  const KParams &K = h->K;
  const int Nq = h->Nq, Np = h->Np, NF = kCurvedNF, np = np32(h->N);
  const long long E = h->E;
  std::vector<float> tab((size_t)E * NF * np, 0.0f);
  std::vector<double> qref((size_t)E * 3 * Np);
  std::vector<double> hr(Np), thr(Np), qr(Np);
  const double ztop = m.z0 + m.Lz;
  for (long long e = 0; e < E; ++e) {
    for (int n = 0; n < Np; ++n) {
      const size_t g = (size_t)e * Np + n;
      const double q = qt_r ? qt_r[g] : 0.0, z = h->hz_[g], x = h->hx_[g];
      const double Rm = p.Rd * (1.0 - q) + p.Rv * q;
      const double Tr = p_r[g] / (rho_r[g] * Rm);
      const double I = (1.0 - q) * p.cvd * (Tr - p.T0) + q * (p.cvv * (Tr - p.T0) + K.Iv0);
      const double rhoe = rho_r[g] * (I + p.g * z);
      qref[((size_t)e * 3 + 0) * Np + n] = rho_r[g];
      qref[((size_t)e * 3 + 1) * Np + n] = rhoe;
      qref[((size_t)e * 3 + 2) * Np + n] = rho_r[g] * q;
      hr[n] = (rhoe + p_r[g]) / rho_r[g];
      thr[n] = Tr * pow(p.p0 / p_r[g], K.kappa) * Rm / p.Rd;
      qr[n] = q;
      double tau = 0.0;
      if (p.sponge_alpha > 0.0) {
        if (z > p.sponge_zs) tau = p.sponge_alpha * pow(sin(0.5 * M_PI * (z - p.sponge_zs) / (ztop - p.sponge_zs)),
                                                        p.sponge_gamma);
        if (p.lateral_sponge_frac > 0.0) {
          const double width = p.lateral_sponge_frac * m.Lx, xl = m.x0 + width, xr = m.x0 + m.Lx - width;
          double tl = 0.0;
          if (x < xl) tl = p.sponge_alpha * pow(sin(0.5 * M_PI * (xl - x) / width), p.sponge_gamma);
          if (x > xr) tl = p.sponge_alpha * pow(sin(0.5 * M_PI * (x - xr) / width), p.sponge_gamma);
          tau = fmax(tau, tl);
        }
      }
      float *T = &tab[(size_t)e * NF * np + n];
      T[L_RHO * np] = (float)rho_r[g];
      T[L_RHOQ * np] = (float)(rho_r[g] * q);
      T[L_T * np] = (float)Tr;
      T[L_T_T0 * np] = (float)(Tr - p.T0);
      T[L_GZ * np] = (float)(p.g * z);
      T[L_P * np] = (float)p_r[g];
      T[L_H * np] = (float)(rhoe + p_r[g]);
      T[L_HM * np] = (float)hr[n];
      T[L_THV * np] = (float)thr[n];
      T[L_RHORM * np] = (float)(rho_r[g] * Rm);
      T[L_TAU * np] = (float)tau;
      T[L_QM * np] = (float)q;
      T[L_RVS * np] = (float)rhovsat64(h, Tr);
      const double delta = h->hdelta_[e];
      T[kCurvedDelta * np] = (float)delta;
      T[kCurvedCsd2 * np] = (float)((p.Cs * delta) * (p.Cs * delta));
      for (int c = 0; c < 3; ++c) T[(kCurvedVr + c) * np] = (float)(h->hvr_[e * 3 + c]);
    }
    // reference gradients: (1/J) sum_r (J a^r)_c d/dxi_r
    const double *fields[3] = {hr.data(), qr.data(), thr.data()};
    const int zslot[3] = {L_DZ_HM, L_DZ_Q, L_DZ_THV}, xslot[3] = {L_NF, L_NF + 2, L_NF + 4};
    for (int n = 0; n < Np; ++n) {
      const int ijk[3] = {n % Nq, (n / Nq) % Nq, n / (Nq * Nq)};
      const double *ja = &h->hJa_[((size_t)e * Np + n) * 9];
      const double Jn = h->hJ_[(size_t)e * Np + n];
      for (int fi = 0; fi < 3; ++fi) {
        double dr[3];
        for (int r = 0; r < 3; ++r) {
          double acc = 0.0;
          for (int q = 0; q < Nq; ++q) {
            int t[3] = {ijk[0], ijk[1], ijk[2]};
            t[r] = q;
            acc += h->D[ijk[r] * Nq + q] * fields[fi][t[0] + Nq * (t[1] + Nq * t[2])];
          }
          dr[r] = acc;
        }
        double gc[3];
        for (int c = 0; c < 3; ++c) gc[c] = (ja[0 + c] * dr[0] + ja[3 + c] * dr[1] + ja[6 + c] * dr[2]) / Jn;
        float *T = &tab[(size_t)e * NF * np + n];
        T[xslot[fi] * np] = (float)gc[0];
        T[(xslot[fi] + 1) * np] = (float)gc[1];
        T[zslot[fi] * np] = (float)gc[2];
      }
    }
  }
  CK(cudaMemcpy(h->node32, tab.data(), tab.size() * sizeof(float), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(h->qref64, qref.data(), qref.size() * sizeof(double), cudaMemcpyHostToDevice));
  h->have_ref = true;
  h->shadow_valid = false;
  return CMLES_OK;
}

}  // namespace cmles_host

using namespace cmles_host;

// Order the handle's stream after the latest asynchronous host download, so
// that work that writes a state buffer cannot overwrite one it still reads
// (a wait on the device; the host does not block).
static cmles_status order_after_fetch(cmles_handle h) {
  if (h->fetch_unordered) {
    CK(cudaStreamWaitEvent(h->stream, h->fetch_done_ev, 0));
    h->fetch_unordered = false;
  }
  return CMLES_OK;
}

// Element range [lo, hi) of chunk i of a state of n doubles.
static void fetch_chunk(size_t n, int i, size_t &lo, size_t &hi) {
  lo = n * (size_t)i / kFetchChunks;
  hi = n * (size_t)(i + 1) / kFetchChunks;
}

extern "C" {

void cmles_default_params(cmles_params *p) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  // Table t:constants; g, p0, p_tr, T_tr are readings (not in the table)
  p->g = 9.81;
  p->p0 = 1.0e5;
  p->Rd = 287.0;
  p->Rv = 462.0;
  p->cvd = 717.5;
  p->cvv = 1397.5;
  p->cvl = 4181.0;
  p->cvi = 2100.0;
  p->T0 = 273.16;
  p->Lv0 = 2.5008e6;
  p->Lf0 = 0.3336e6;
  p->ptr = 611.657;
  p->Ttr = 273.16;
  p->closure = CMLES_CLOSURE_SL;
  p->Cs = 0.21;
  p->Prt = 1.0 / 3.0;
  p->richardson = 1;
  p->moist = 0;
  p->sponge_gamma = 2.0;
  p->precision = CMLES_FP64;
  p->dt = 0.02;
  p->satadj_max_iter = 20;
  p->flux = CMLES_FLUX_RUSANOV;
  p->filter_order = 0;
  p->filter_alpha = -log(pow(2.0, -52));
  p->filter_vars = 0xE;
  p->integrator = CMLES_LSRK54;
  p->drag_cd = 0.0;
  p->noslip = 0;
}

// Tangent table of the saturation vapour density rho_vs(T) = p_v*(T)/(R_v T)
// for the certainly-unsaturated shortcut of the thermodynamics: knots every
// 5 K on [150, 450] K.  The shortcut relies on rho_vs being convex there;
// that is checked here by second differences on a 0.1 K grid, and the
// shortcut is disabled (rvs_n = 0, rvs_ok = 0) if it fails.
static constexpr int kRvsN = 61;
static cudaError_t build_rvs_table(cmles_handle h) {
  KParams &K = h->K;
  auto rvs = [&](double T) {
    return K.pv_ptr * exp(K.pv_a * log(T / K.pv_Ttr) + K.pv_b * (1.0 / K.pv_Ttr - 1.0 / T)) / (h->prm.Rv * T);
  };
  bool convex = true;
  const double dT = 0.1;
  for (double T = 150.0 + dT; T < 450.0; T += dT)
    if (!(rvs(T - dT) - 2.0 * rvs(T) + rvs(T + dT) > 0.0)) convex = false;
  std::vector<double> tab(kRvsN * 2);
  for (int k = 0; k < kRvsN; ++k) {
    const double T = 150.0 + 5.0 * k, f = rvs(T);
    tab[2 * k] = f;
    tab[2 * k + 1] = f * (K.pv_a - 1.0 + K.pv_b / T) / T;
  }
  K.rvs_tab = h->rvs_tab;
  K.rvs_T0 = 150.0;
  K.rvs_dT = 5.0;
  K.rvs_n = convex ? kRvsN : 0;
  K.rvs_ok = convex ? 1 : 0;
  return cudaMemcpy(h->rvs_tab, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice);
}

// 1D exponential filter matrix F = V diag(sigma_k) V^-1 with V_ik = P_k(xi_i)
// (Legendre polynomials by their three-term recurrence) and
// sigma_k = exp(-alpha (k/N)^s); V^-1 by LU with partial pivoting.
static void build_expfilter(cmles_handle h) {
  const int N = h->N, Nq = h->Nq;
  std::vector<double> V(Nq * Nq), LU(Nq * Nq), Vinv(Nq * Nq);
  for (int i = 0; i < Nq; ++i) {
    double p0 = 1.0, p1 = h->xi[i];
    V[i * Nq] = p0;
    if (N >= 1) V[i * Nq + 1] = p1;
    for (int k = 2; k <= N; ++k) {
      const double p2 = ((2 * k - 1) * h->xi[i] * p1 - (k - 1) * p0) / k;
      V[i * Nq + k] = p2;
      p0 = p1;
      p1 = p2;
    }
  }
  LU = V;
  std::vector<int> piv(Nq);
  for (int c = 0; c < Nq; ++c) {
    int r = c;
    for (int q = c + 1; q < Nq; ++q)
      if (fabs(LU[q * Nq + c]) > fabs(LU[r * Nq + c])) r = q;
    piv[c] = r;
    if (r != c)
      for (int q = 0; q < Nq; ++q) std::swap(LU[c * Nq + q], LU[r * Nq + q]);
    for (int q = c + 1; q < Nq; ++q) {
      LU[q * Nq + c] /= LU[c * Nq + c];
      for (int m = c + 1; m < Nq; ++m) LU[q * Nq + m] -= LU[q * Nq + c] * LU[c * Nq + m];
    }
  }
  for (int col = 0; col < Nq; ++col) {  // solve V x = e_col
    std::vector<double> x(Nq, 0.0);
    x[col] = 1.0;
    for (int c = 0; c < Nq; ++c) std::swap(x[c], x[piv[c]]);
    for (int q = 0; q < Nq; ++q)
      for (int m = 0; m < q; ++m) x[q] -= LU[q * Nq + m] * x[m];
    for (int q = Nq - 1; q >= 0; --q) {
      for (int m = q + 1; m < Nq; ++m) x[q] -= LU[q * Nq + m] * x[m];
      x[q] /= LU[q * Nq + q];
    }
    for (int q = 0; q < Nq; ++q) Vinv[q * Nq + col] = x[q];
  }
  const double s = h->prm.filter_order, alpha = h->prm.filter_alpha;
  for (int i = 0; i < Nq; ++i)
    for (int j = 0; j < Nq; ++j) {
      double acc = 0.0;
      for (int k = 0; k < Nq; ++k) acc += V[i * Nq + k] * exp(-alpha * pow((double)k / N, s)) * Vinv[k * Nq + j];
      h->expf.F[i * Nq + j] = acc;
    }
  h->expf.mask = h->prm.filter_vars;
}

static cmles_status apply_expfilter(cmles_handle h) {
  LaunchScope ls(h, 2, 1);
  if (h->fp32) {
    CK(launch_expfilter(h->Q[0], h->shadow_valid ? h->S32[h->scur] : nullptr, h->expf, h->N, (int)h->E, h->stream));
    // the filtered shadow's thermodynamic fields
    if (h->shadow_valid) {
      if (h->curved)
        CK(launch_shadow32c(nullptr, h->S32[h->scur], h->TH32[h->scur], h->K, h->N, h->stream));
      else
        CK(launch_shadow32(nullptr, h->S32[h->scur], h->TH32[h->scur], h->K, h->N, h->stream));
    }
  } else {
    CK(launch_expfilter(h->Q[h->cur], nullptr, h->expf, h->N, (int)h->E, h->stream));
    if (h->shadow_valid) CK(launch_thermo64(h->Q[h->cur], h->TH64[h->cur], h->K, h->N, h->stream));
  }
  return CMLES_OK;
}

}  // extern "C"

// cmles_create of a whole mesh (ps null), or of one partition of a mesh
// split into (x, y) pencils: `mesh` is then the partition's interior as a mesh
// of its own extent and origin, and ps gives the whole mesh, the partition's
// place in it and its sides that are walls.
cmles_status cmles_host::create_handle(const cmles_mesh *mesh, const cmles_params *params, const PartSpec *ps,
                                       cmles_handle *out) {
  if (!mesh || !params || !out) return CMLES_ERR_ARG;
  *out = nullptr;
  // the kernels are instantiated for the orders 1 .. 7: flat meshes in both
  // precisions, warped meshes (FP32), HEVI
  if (mesh->N < 1 || mesh->N > 7) return CMLES_ERR_ARG;
  if (mesh->nex < 1 || mesh->ney < 1 || mesh->nez < 1 || !(mesh->Lx > 0) || !(mesh->Ly > 0) || !(mesh->Lz > 0))
    return CMLES_ERR_MESH;
  // warped (curvilinear) meshes run on the FP32 path
  if (mesh->warp && params->precision != CMLES_FP32_ACC64) return CMLES_ERR_ARG;
  if (params->precision != CMLES_FP64 && params->precision != CMLES_FP32_ACC64) return CMLES_ERR_ARG;
  if (params->closure != CMLES_CLOSURE_NONE && params->closure != CMLES_CLOSURE_SL &&
      params->closure != CMLES_CLOSURE_MLP && params->closure != CMLES_CLOSURE_VREMAN)
    return CMLES_ERR_ARG;
  if (params->flux != CMLES_FLUX_RUSANOV && params->flux != CMLES_FLUX_HLLC && params->flux != CMLES_FLUX_ROE)
    return CMLES_ERR_ARG;
  if (params->filter_order < 0 || !(params->filter_alpha >= 0.0) || (params->filter_vars & ~0xE) != 0)
    return CMLES_ERR_ARG;
  if (!(params->drag_cd >= 0.0) || !std::isfinite(params->drag_cd)) return CMLES_ERR_ARG;
  if (params->noslip & ~0x3F) return CMLES_ERR_ARG;
  if (params->integrator != CMLES_LSRK54 && params->integrator != CMLES_LSRK144 &&
      params->integrator != CMLES_ARK2_HEVI)
    return CMLES_ERR_ARG;
  // HEVI: flat meshes with walls at the bottom and top
  if (params->integrator == CMLES_ARK2_HEVI && (mesh->warp || mesh->periodic[2] || mesh->nez < 2))
    return CMLES_ERR_ARG;
  // the learned closure runs on BF16 tensor cores inside the FP32 kernels
  if (params->closure == CMLES_CLOSURE_MLP && params->precision != CMLES_FP32_ACC64) return CMLES_ERR_ARG;
  long long E = (long long)mesh->nex * mesh->ney * mesh->nez;
  const long long Es = ps ? (long long)(mesh->nex + 2) * (mesh->ney + 2) * mesh->nez : E;
  if (Es > 0x7fffffffLL / 8) return CMLES_ERR_MESH;
  cmles_handle h = new cmles_t();
  h->mesh = *mesh;
  h->prm = *params;
  h->N = mesh->N;
  h->Nq = h->N + 1;
  h->Np = h->Nq * h->Nq * h->Nq;
  h->E = E;
  h->nodes = E * h->Np;
  h->Es = Es;
  h->snodes = Es * h->Np;
  h->part = ps != nullptr;
  lgl_basis(h->N, h->xi, h->w, h->D);
  if (params->filter_order > 0) build_expfilter(h);
  const size_t n6 = (size_t)h->snodes * 6;
  const int nlev = mesh->nez * h->Nq;
  cmles_status st = CMLES_OK;
#define ALLOC(ptr, bytes)                                   \
  do {                                                      \
    st = dalloc(h, (void **)&(ptr), (bytes));               \
    if (st != CMLES_OK) {                                   \
      std::string msg = h->err;                             \
      cmles_destroy(h);                                     \
      fprintf(stderr, "cmles_create: %s\n", msg.c_str());   \
      return st;                                            \
    }                                                       \
  } while (0)
  h->fp32 = params->precision == CMLES_FP32_ACC64;
  ALLOC(h->Q[0], n6 * sizeof(double));
  if (!h->fp32) {
    ALLOC(h->Q[1], n6 * sizeof(double));
    ALLOC(h->dQ, n6 * sizeof(double));
    ALLOC(h->F2, (size_t)h->snodes * 15 * sizeof(double));
    ALLOC(h->TH64[0], (size_t)h->snodes * 4 * sizeof(double));
    ALLOC(h->TH64[1], (size_t)h->snodes * 4 * sizeof(double));
  } else {
    const size_t n32 = (size_t)Es * np32(mesh->N);  // padded nodes
    ALLOC(h->S32[0], n32 * 6 * sizeof(float));
    ALLOC(h->S32[1], n32 * 6 * sizeof(float));
    ALLOC(h->dQ32, n32 * 6 * sizeof(float));
    ALLOC(h->D32, n32 * 6 * sizeof(float));
    ALLOC(h->F2_32, n32 * 15 * sizeof(float));
    ALLOC(h->TH32[0], n32 * 4 * sizeof(float));
    ALLOC(h->TH32[1], n32 * 4 * sizeof(float));
  }
  h->curved = mesh->warp != 0;
  ALLOC(h->lev32, (size_t)nlev * L_NF * sizeof(float));
  ALLOC(h->dH32, (size_t)mesh->nez * h->Nq * h->Nq * sizeof(float));
  if (h->curved) {
    ALLOC(h->qref64, (size_t)E * 3 * h->Np * sizeof(double));
    ALLOC(h->geo32, (size_t)E * 10 * np32(mesh->N) * sizeof(float));
    ALLOC(h->node32, (size_t)E * kCurvedNF * np32(mesh->N) * sizeof(float));
    ALLOC(h->wJn, (size_t)E * h->Np * sizeof(double));
  } else {
    ALLOC(h->qref64, (size_t)nlev * 4 * sizeof(double));
  }
  ALLOC(h->mlp_dev, sizeof(MlpPacked));
  ALLOC(h->rho_r, nlev * sizeof(double));
  ALLOC(h->p_r, nlev * sizeof(double));
  ALLOC(h->qt_r, nlev * sizeof(double));
  ALLOC(h->tau_lev, nlev * sizeof(double));
  // lateral sponge: one value per node column of the whole mesh in x
  const cmles_mesh &gm = ps ? ps->global : *mesh;
  ALLOC(h->tau_col, (size_t)gm.nex * h->Nq * sizeof(double));
  ALLOC(h->wq, h->Np * sizeof(double));
  ALLOC(h->flags, 16 * sizeof(int));
  ALLOC(h->rvs_tab, kRvsN * 2 * sizeof(double));
  ALLOC(h->exr, nlev * sizeof(double));
  h->budget_nblocks = budget_blocks(h->nodes);
  ALLOC(h->partials, (size_t)h->budget_nblocks * 7 * sizeof(double));
  ALLOC(h->budget_out, 8 * sizeof(double));
  ALLOC(h->prof, (size_t)nlev * 12 * sizeof(double));
#undef ALLOC
  fill_kparams(h);
  if (ps) {
    h->K.part = 1;
    h->K.gx0 = ps->gx0;
    h->K.gy0 = ps->gy0;
    for (int f = 0; f < 4; ++f) h->K.wall[f] = ps->wall[f];
  }
  // sponge tables (Eq. sponge, reading tau_s = alpha sin^gamma(pi/2 (z - z_s)/(z_top - z_s)))
  std::vector<double> tl(nlev, 0.0), tc((size_t)gm.nex * h->Nq, 0.0);
  const double ztop = mesh->z0 + mesh->Lz;
  for (int l = 0; l < nlev; ++l) {
    const double z = level_z(h, l);
    if (params->sponge_alpha > 0.0 && z > params->sponge_zs)
      tl[l] = params->sponge_alpha * pow(sin(0.5 * M_PI * (z - params->sponge_zs) / (ztop - params->sponge_zs)),
                                         params->sponge_gamma);
  }
  bool lateral = params->sponge_alpha > 0.0 && params->lateral_sponge_frac > 0.0;
  if (lateral) {
    const double width = params->lateral_sponge_frac * gm.Lx;
    const double xl = gm.x0 + width, xr = gm.x0 + gm.Lx - width;
    for (int ex = 0; ex < gm.nex; ++ex)
      for (int i = 0; i < h->Nq; ++i) {
        const double x = gm.x0 + (ex + 0.5 * (h->xi[i] + 1.0)) * h->K.hx;
        double t = 0.0;
        if (x < xl) t = params->sponge_alpha * pow(sin(0.5 * M_PI * (xl - x) / width), params->sponge_gamma);
        if (x > xr) t = params->sponge_alpha * pow(sin(0.5 * M_PI * (x - xr) / width), params->sponge_gamma);
        tc[(size_t)ex * h->Nq + i] = t;
      }
  }
  std::vector<double> wq(h->Np);
  for (int k = 0; k < h->Nq; ++k)
    for (int j = 0; j < h->Nq; ++j)
      for (int i = 0; i < h->Nq; ++i) wq[i + h->Nq * (j + h->Nq * k)] = h->w[i] * h->w[j] * h->w[k];
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = cudaMemcpy(h->tau_lev, tl.data(), nlev * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(h->tau_col, tc.data(), tc.size() * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(h->wq, wq.data(), h->Np * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(h->flags, 0, 16 * sizeof(int));
  if (e == cudaSuccess) e = build_rvs_table(h);
  if (e == cudaSuccess) e = cudaMemset(h->exr, 0, nlev * sizeof(double));
  if (e == cudaSuccess) e = cudaMemset(h->mlp_dev, 0, sizeof(MlpPacked));
  if (e == cudaSuccess && h->dQ) e = cudaMemset(h->dQ, 0, n6 * sizeof(double));
  if (e == cudaSuccess && h->dQ32) e = cudaMemset(h->dQ32, 0, (size_t)Es * np32(mesh->N) * 6 * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(h->Q[0], 0, n6 * sizeof(double));
  if (e != cudaSuccess) {
    cmles_destroy(h);
    return CMLES_ERR_CUDA;
  }
  if (!lateral) h->K.tau_col = nullptr;
  if (h->curved) {
    h->K.curved = 1;
    h->K.geo32 = h->geo32;
    h->K.node32 = h->node32;
    if (build_curved(h) != CMLES_OK) {
      cmles_destroy(h);
      return CMLES_ERR_CUDA;
    }
  }
  *out = h;
  return CMLES_OK;
}

int cmles_host::lsrk_tables(cmles_handle h, const double **A, const double **B) {
  const bool l14 = h->prm.integrator == CMLES_LSRK144;
  *A = l14 ? kLsrk14A : kLsrkA;
  *B = l14 ? kLsrk14B : kLsrkB;
  return l14 ? 14 : 5;
}

extern "C" {

cmles_status cmles_create(const cmles_mesh *mesh, const cmles_params *params, cmles_handle *out) {
  return create_handle(mesh, params, nullptr, out);
}

cmles_status cmles_destroy(cmles_handle h) {
  if (!h) return CMLES_ERR_ARG;
  if (h->d2h_stream) cudaStreamSynchronize(h->d2h_stream);  // a download still writing host memory
  for (auto &t : h->timed) {
    cudaEventDestroy(t.a);
    cudaEventDestroy(t.b);
  }
  void *bufs[] = {h->Q[0],   h->Q[1],    h->dQ,      h->F2,      h->TH64[0], h->TH64[1],  h->rho_r,    h->p_r,
                  h->qt_r,   h->tau_lev, h->tau_col, h->wq,      h->flags,   h->partials, h->budget_out,
                  h->prof,   h->S32[0],  h->S32[1],  h->dQ32,    h->D32,     h->F2_32,    h->lev32,
                  h->TH32[0], h->TH32[1], h->dH32,   h->qref64,  h->mlp_dev, h->geo32,    h->node32,
                  h->wJn,    h->rvs_tab, h->exr};
  for (void *b : bufs)
    if (b) cudaFree(b);
  for (double *b : h->hv_buf)
    if (b) cudaFree(b);
  if (h->hv_tab) cudaFree(h->hv_tab);
  if (h->Qstage) cudaFree(h->Qstage);
  if (h->d2h_stream) {
    for (cudaEvent_t ev : h->fetch_ev)
      if (ev) cudaEventDestroy(ev);
    if (h->fetch_start_ev) cudaEventDestroy(h->fetch_start_ev);
    if (h->fetch_done_ev) cudaEventDestroy(h->fetch_done_ev);
    cudaStreamDestroy(h->d2h_stream);
  }
  if (h->staged_ev) cudaEventDestroy(h->staged_ev);
  if (h->compute_ev) cudaEventDestroy(h->compute_ev);
  if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
  delete h;
  return CMLES_OK;
}

const char *cmles_last_error_message(cmles_handle h) { return h ? h->err.c_str() : "null handle"; }

cmles_status cmles_set_stream(cmles_handle h, void *stream) {
  if (!h) return CMLES_ERR_ARG;
  h->stream = (cudaStream_t)stream;
  return CMLES_OK;
}

cmles_status cmles_set_reference(cmles_handle h, const double *rho_r, const double *p_r, const double *qt_r,
                                 size_t n) {
  if (!h || !rho_r || !p_r) return fail(h, CMLES_ERR_ARG, "cmles_set_reference: null array");
  if (h->curved) {
    if (n != (size_t)h->nodes) return fail(h, CMLES_ERR_ARG, "cmles_set_reference: expected one value per node");
    return curved_reference(h, rho_r, p_r, qt_r);
  }
  const size_t nlev = (size_t)h->mesh.nez * h->Nq;
  if (n != nlev) return fail(h, CMLES_ERR_ARG, "cmles_set_reference: expected one value per node level");
  // levels (ez, N) and (ez+1, 0) are the same height: the physical profile
  // must agree there; the total-water offset is taken from the lower element
  const int Nq0 = h->Nq;
  for (int ez = 0; ez + 1 < h->mesh.nez; ++ez) {
    const size_t a = (size_t)ez * Nq0 + Nq0 - 1, b = (size_t)(ez + 1) * Nq0;
    if (fabs(rho_r[a] - rho_r[b]) > 1e-12 * fabs(rho_r[a]) || fabs(p_r[a] - p_r[b]) > 1e-12 * fabs(p_r[a]))
      return fail(h, CMLES_ERR_ARG, "cmles_set_reference: levels of equal height differ");
  }
  std::vector<double> qcanon(nlev, 0.0);
  if (qt_r) {
    for (size_t l = 0; l < nlev; ++l) qcanon[l] = qt_r[l];
    for (int ez = 0; ez + 1 < h->mesh.nez; ++ez) qcanon[(size_t)(ez + 1) * Nq0] = qcanon[(size_t)ez * Nq0 + Nq0 - 1];
    qt_r = qcanon.data();
  }
  CK(cudaMemcpyAsync(h->rho_r, rho_r, nlev * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(h->p_r, p_r, nlev * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  h->ref_rho_h.assign(rho_r, rho_r + nlev);
  h->ref_p_h.assign(p_r, p_r + nlev);
  if (qt_r)
    h->ref_qt_h.assign(qt_r, qt_r + nlev);
  else
    h->ref_qt_h.assign(nlev, 0.0);
  h->hv_dt = -1.0;  // the HEVI tables depend on the reference
  {
    std::vector<double> ex(nlev);
    for (size_t l = 0; l < nlev; ++l) ex[l] = exp(-h->K.kappa * log(p_r[l] / h->prm.p0));
    CK(cudaMemcpy(h->exr, ex.data(), nlev * sizeof(double), cudaMemcpyHostToDevice));
  }
  if (qt_r)
    CK(cudaMemcpyAsync(h->qt_r, qt_r, nlev * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  else
    CK(cudaMemsetAsync(h->qt_r, 0, nlev * sizeof(double), h->stream));
  // FP32-path tables from the reference profile, built in FP64:
  // Q_ref = (rho_r, 0, 0, 0, rho e_r, rho q_r) with T_r = p_r / (rho_r R_m,r),
  // rho e_r = rho_r (I(T_r, q_r, 0) + g z), H_r = rho e_r + p_r, h_r = H_r/rho_r,
  // theta_v,r = T_r (p0/p_r)^kappa R_m,r / R_d, and the derivatives of h_r and
  // theta_v,r along z within each element (D applied to the level values).
  const cmles_params &p = h->prm;
  const KParams &K = h->K;
  std::vector<float> lev(nlev * L_NF, 0.0f), dH((size_t)h->mesh.nez * h->Nq * h->Nq);
  std::vector<double> qref(nlev * 4, 0.0), hr(nlev), thvr(nlev), tau(nlev);
  CK(cudaMemcpy(tau.data(), h->tau_lev, nlev * sizeof(double), cudaMemcpyDeviceToHost));
  for (size_t l = 0; l < nlev; ++l) {
    const double q = qt_r ? qt_r[l] : 0.0;
    const double z = level_z(h, (int)l);
    const double Rm = p.Rd * (1.0 - q) + p.Rv * q;
    const double Tr = p_r[l] / (rho_r[l] * Rm);
    const double I = (1.0 - q) * p.cvd * (Tr - p.T0) + q * (p.cvv * (Tr - p.T0) + K.Iv0);
    const double rhoe = rho_r[l] * (I + p.g * z);
    qref[l * 4 + 0] = rho_r[l];
    qref[l * 4 + 1] = rhoe;
    qref[l * 4 + 2] = rho_r[l] * q;
    hr[l] = (rhoe + p_r[l]) / rho_r[l];
    thvr[l] = Tr * pow(p.p0 / p_r[l], K.kappa) * Rm / p.Rd;
    float *L = &lev[l * L_NF];
    L[L_RHO] = (float)rho_r[l];
    L[L_RHOQ] = (float)(rho_r[l] * q);
    L[L_T] = (float)Tr;
    L[L_T_T0] = (float)(Tr - p.T0);
    L[L_GZ] = (float)(p.g * z);
    L[L_P] = (float)p_r[l];
    L[L_H] = (float)(rhoe + p_r[l]);
    L[L_HM] = (float)hr[l];
    L[L_THV] = (float)thvr[l];
    L[L_RHORM] = (float)(rho_r[l] * Rm);
    L[L_TAU] = (float)tau[l];
    L[L_QM] = (float)q;
    L[L_RVS] = (float)rhovsat64(h, Tr);
  }
  const int Nq = h->Nq;
  // The FP32 shadow holds deviations from the reference of its node's level,
  // and a face task takes the reference values of its own face node for the
  // neighbour's node, which across an element face sits at the same height.
  // Across a periodic wrap in z the two nodes are the bottom and the top
  // level, so their reference states (including rho e_r with its g z) must
  // be equal: a profile that repeats, as with g = 0.
  if (h->fp32 && h->mesh.periodic[2]) {
    const size_t top = nlev - 1;
    auto differ = [](double a, double b) { return fabs(a - b) > 1e-12 * fmax(fabs(a), fabs(b)) + 1e-300; };
    if (differ(rho_r[0], rho_r[top]) || differ(p_r[0], p_r[top]) || differ(qref[1], qref[top * 4 + 1]) ||
        differ(qref[2], qref[top * 4 + 2]))
      return fail(h, CMLES_ERR_ARG,
                  "cmles_set_reference: periodic z on the FP32 path needs a reference state that repeats across "
                  "the wrap (with g = 0)");
  }
  for (int ez = 0; ez < h->mesh.nez; ++ez)
    for (int k = 0; k < Nq; ++k) {
      double dh = 0.0, dth = 0.0, dq = 0.0;
      for (int m = 0; m < Nq; ++m) {
        dq += h->D[k * Nq + m] * (qt_r ? qt_r[ez * Nq + m] : 0.0);
        dh += h->D[k * Nq + m] * hr[ez * Nq + m];
        dth += h->D[k * Nq + m] * thvr[ez * Nq + m];
        dH[(size_t)ez * Nq * Nq + k * Nq + m] =
            (float)((qref[(ez * Nq + m) * 4 + 1] + p_r[ez * Nq + m]) - (qref[(ez * Nq + k) * 4 + 1] + p_r[ez * Nq + k]));
      }
      lev[(ez * Nq + k) * L_NF + L_DZ_HM] = (float)(K.jac[2] * dh);
      lev[(ez * Nq + k) * L_NF + L_DZ_THV] = (float)(K.jac[2] * dth);
      lev[(ez * Nq + k) * L_NF + L_DZ_Q] = (float)(K.jac[2] * dq);
    }
  CK(cudaMemcpy(h->lev32, lev.data(), lev.size() * sizeof(float), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(h->dH32, dH.data(), dH.size() * sizeof(float), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(h->qref64, qref.data(), qref.size() * sizeof(double), cudaMemcpyHostToDevice));
  CK(cudaStreamSynchronize(h->stream));
  h->have_ref = true;
  h->shadow_valid = false;
  return CMLES_OK;
}

cmles_status cmles_init_case(cmles_handle h, const cmles_case *c) {
  if (!h || !c) return fail(h, CMLES_ERR_ARG, "cmles_init_case: null argument");
  {
    cmles_status st = order_after_fetch(h);
    if (st != CMLES_OK) return st;
  }
  if (h->curved) {
    // flow over the terrain (case 3): dry, constant Brunt-Vaisala frequency
    // (Eqs. pressure_hs_brunt and the ideal gas law), uniform velocity u0
    if (c->id != 3) return fail(h, CMLES_ERR_ARG, "cmles_init_case: warped meshes support case 3 only");
    const cmles_params &p = h->prm;
    const double cpd = p.cvd + p.Rd, kappa = p.Rd / cpd, N2 = c->NBV * c->NBV;
    const size_t nn = (size_t)h->nodes;
    std::vector<double> Q(nn * 6), rr(nn), pr(nn);
    for (long long e = 0; e < h->E; ++e)
      for (int n = 0; n < h->Np; ++n) {
        const size_t g = (size_t)e * h->Np + n;
        const double z = h->hz_[g];
        const double th = c->theta0 * exp(N2 * z / p.g);
        const double pi = 1.0 + p.g * p.g / (cpd * c->theta0 * N2) * (exp(-z * N2 / p.g) - 1.0);
        const double pp = p.p0 * pow(pi, cpd / p.Rd);
        const double T = th * pow(pp / p.p0, kappa);
        const double rho = pp / (p.Rd * T);
        const double ke = 0.5 * (c->u0[0] * c->u0[0] + c->u0[1] * c->u0[1] + c->u0[2] * c->u0[2]);
        double *q = &Q[(size_t)e * 6 * h->Np + n];
        q[0] = rho;
        q[h->Np] = rho * c->u0[0];
        q[2 * h->Np] = rho * c->u0[1];
        q[3 * h->Np] = rho * c->u0[2];
        q[4 * h->Np] = rho * (p.cvd * (T - p.T0) + ke + p.g * z);
        q[5 * h->Np] = 0.0;
        rr[g] = rho;
        pr[g] = pp;
      }
    cmles_status st = curved_reference(h, rr.data(), pr.data(), nullptr);
    if (st != CMLES_OK) return st;
    CK(cudaMemcpy(h->Q[0], Q.data(), Q.size() * sizeof(double), cudaMemcpyHostToDevice));
    h->cur = 0;
    h->shadow_valid = false;
    h->time = 0.0;
    h->steps = 0;
    return CMLES_OK;
  }
  if (c->id != 1 && c->id != 2 && c->id != 5 && c->id != 11)
    return fail(h, CMLES_ERR_ARG, "cmles_init_case: case id not available on flat meshes");
  const cmles_params &p = h->prm;
  const int nlev = h->mesh.nez * h->Nq;
  const double cpd = p.cvd + p.Rd, kappa = p.Rd / cpd;
  const double Lz = h->mesh.Lz;
  // background theta and q_t profiles
  auto theta_of = [&](double z) {
    if (c->id == 2) return z <= c->z_ml ? c->theta0 : c->theta0 + c->dthdz_above * (z - c->z_ml);
    if (c->id == 5) return c->theta0 * exp(c->NBV * c->NBV * z / p.g);
    return c->theta0;
  };
  auto qt_of = [&](double z) {
    if (!c->moist) return 0.0;
    if (c->id == 2)
      return z <= c->z_ml ? c->qt_sfc + (c->qt_ml - c->qt_sfc) * z / c->z_ml
                          : c->qt_ml + (c->qt_top - c->qt_ml) * (z - c->z_ml) / (Lz - c->z_ml);
    if (c->id == 5) return c->qt_sfc * exp(-z / c->qt_H);
    return 0.0;
  };
  // hydrostatic balance dp/dz = -g p / (R_m T), T = theta (p/p0)^kappa, q_l = 0
  auto rhs = [&](double z, double pp) {
    const double T = theta_of(z) * pow(pp / p.p0, kappa);
    const double q = qt_of(z);
    return -p.g * pp / ((p.Rd * (1.0 - q) + p.Rv * q) * T);
  };
  auto rk4 = [&](double z, double pp, double hh) {
    const double k1 = rhs(z, pp), k2 = rhs(z + 0.5 * hh, pp + 0.5 * hh * k1);
    const double k3 = rhs(z + 0.5 * hh, pp + 0.5 * hh * k2), k4 = rhs(z + hh, pp + hh * k3);
    return pp + hh / 6.0 * (k1 + 2.0 * k2 + 2.0 * k3 + k4);
  };
  const bool integrate = c->id == 2 || (c->id == 5 && c->moist);
  std::vector<double> grid;
  const double h0 = 0.5;
  if (integrate) {
    double zmax = 0.0;
    for (int l = 0; l < nlev; ++l) zmax = fmax(zmax, level_z(h, l));
    const int M = (int)ceil(zmax / h0) + 2;
    grid.resize(M + 1);
    grid[0] = p.p0;
    for (int m = 0; m < M; ++m) grid[m + 1] = rk4(m * h0, grid[m], h0);
  }
  std::vector<double> th(nlev), qt(nlev), pr(nlev), rr(nlev);
  for (int l = 0; l < nlev; ++l) {
    const double z = level_z(h, l);
    double pp;
    if (c->id == 1 || c->id == 11) {
      pp = p.p0 * pow(1.0 - p.g / (cpd * c->theta0) * z, cpd / p.Rd);  // Eq. pressureDistrib
    } else if (!integrate) {                                            // Eq. pressure_hs_brunt
      const double N2 = c->NBV * c->NBV;
      const double pi = 1.0 + p.g * p.g / (cpd * c->theta0 * N2) * (exp(-z * N2 / p.g) - 1.0);
      pp = p.p0 * pow(pi, cpd / p.Rd);
    } else {
      int m = (int)floor(z / h0);
      if (m < 0) m = 0;
      if (m > (int)grid.size() - 1) m = (int)grid.size() - 1;
      const double zm = m * h0;
      pp = z == zm ? grid[m] : rk4(zm, grid[m], z - zm);
    }
    th[l] = theta_of(z);
    qt[l] = qt_of(z);
    pr[l] = pp;
    const double T = th[l] * pow(pp / p.p0, kappa);
    rr[l] = pp / ((p.Rd * (1.0 - qt[l]) + p.Rv * qt[l]) * T);
  }
  cmles_status st = cmles_set_reference(h, rr.data(), pr.data(), qt.data(), nlev);
  if (st != CMLES_OK) return st;
  double *dth = nullptr, *dqt = nullptr, *dpr = nullptr, *dmodes = nullptr;
  CK(cudaMalloc(&dth, nlev * sizeof(double)));
  CK(cudaMalloc(&dqt, nlev * sizeof(double)));
  CK(cudaMalloc(&dpr, nlev * sizeof(double)));
  CK(cudaMemcpy(dth, th.data(), nlev * sizeof(double), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(dqt, qt.data(), nlev * sizeof(double), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(dpr, pr.data(), nlev * sizeof(double), cudaMemcpyHostToDevice));
  if (c->nmodes > 0 && c->modes) {
    CK(cudaMalloc(&dmodes, (size_t)c->nmodes * 7 * sizeof(double)));
    CK(cudaMemcpy(dmodes, c->modes, (size_t)c->nmodes * 7 * sizeof(double), cudaMemcpyHostToDevice));
  }
  CaseDev cd;
  memset(&cd, 0, sizeof(cd));
  cd.id = c->id;
  cd.seed = c->seed;
  cd.dtheta = c->dtheta;
  cd.r0 = c->r0;
  cd.xc = c->xc;
  cd.yc = c->yc;
  cd.zc = c->zc;
  cd.noise_theta = c->noise_theta;
  cd.noise_qt = c->noise_qt;
  cd.noise_zmax = c->noise_zmax;
  for (int k = 0; k < 3; ++k) cd.u0[k] = c->u0[k];
  cd.moist = c->moist;
  cd.nmodes = dmodes ? c->nmodes : 0;
  cd.modes = dmodes;
  cd.theta_lev = dth;
  cd.qt_lev = dqt;
  cd.pref_lev = dpr;
  {
    LaunchScope ls(h, 2, 1);
    CK(launch_init_state(h->Q[0], cd, h->K, h->N, h->stream));
  }
  h->cur = 0;
  h->shadow_valid = false;
  CK(cudaStreamSynchronize(h->stream));
  cudaFree(dth);
  cudaFree(dqt);
  cudaFree(dpr);
  if (dmodes) cudaFree(dmodes);
  h->time = 0.0;
  h->steps = 0;
  return CMLES_OK;
}

cmles_status cmles_fetch_state_host(cmles_handle h, double *Q_host) {
  if (!h || !Q_host) return fail(h, CMLES_ERR_ARG, "cmles_fetch_state_host: null argument");
  if (!h->d2h_stream) {
    CK(cudaStreamCreateWithFlags(&h->d2h_stream, cudaStreamNonBlocking));
    for (cudaEvent_t &ev : h->fetch_ev) CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&h->fetch_start_ev, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&h->fetch_done_ev, cudaEventDisableTiming));
  }
  // after the work queued on the handle's stream, and after an uncommitted
  // staged upload, which may still be reading this host buffer
  CK(cudaEventRecord(h->fetch_start_ev, h->stream));
  CK(cudaStreamWaitEvent(h->d2h_stream, h->fetch_start_ev, 0));
  if (h->staged) CK(cudaStreamWaitEvent(h->d2h_stream, h->staged_ev, 0));
  const double *src = h->Q[h->cur];
  const size_t n = (size_t)h->nodes * 6;
  for (int i = 0; i < kFetchChunks; ++i) {
    size_t lo, hi;
    fetch_chunk(n, i, lo, hi);
    if (hi > lo)
      CK(cudaMemcpyAsync(Q_host + lo, src + lo, (hi - lo) * sizeof(double), cudaMemcpyDeviceToHost, h->d2h_stream));
    CK(cudaEventRecord(h->fetch_ev[i], h->d2h_stream));
  }
  CK(cudaEventRecord(h->fetch_done_ev, h->d2h_stream));
  h->fetch_src = src;
  h->fetch_host = Q_host;
  h->fetch_pending = true;
  h->fetch_unordered = true;
  return CMLES_OK;
}

cmles_status cmles_wait_fetch(cmles_handle h) {
  if (!h) return CMLES_ERR_ARG;
  if (!h->fetch_pending) return CMLES_OK;
  CK(cudaEventSynchronize(h->fetch_done_ev));
  h->fetch_pending = false;
  return CMLES_OK;
}

cmles_status cmles_set_state(cmles_handle h, const double *Q_dev) {
  if (!h || !Q_dev) return fail(h, CMLES_ERR_ARG, "cmles_set_state: null argument");
  {
    cmles_status st = order_after_fetch(h);
    if (st != CMLES_OK) return st;
  }
  CK(cudaMemcpyAsync(h->Q[h->cur], Q_dev, (size_t)h->nodes * 6 * sizeof(double), cudaMemcpyDeviceToDevice,
                     h->stream));
  h->shadow_valid = false;
  return CMLES_OK;
}

cmles_status cmles_get_state(cmles_handle h, double *Q_dev) {
  if (!h || !Q_dev) return fail(h, CMLES_ERR_ARG, "cmles_get_state: null argument");
  CK(cudaMemcpyAsync(Q_dev, h->Q[h->cur], (size_t)h->nodes * 6 * sizeof(double), cudaMemcpyDeviceToDevice,
                     h->stream));
  return CMLES_OK;
}

cmles_status cmles_set_state_host(cmles_handle h, const double *Q_host) {
  if (!h || !Q_host) return fail(h, CMLES_ERR_ARG, "cmles_set_state_host: null argument");
  {
    cmles_status st = order_after_fetch(h);
    if (st != CMLES_OK) return st;
  }
  // a download into this host buffer completes before it is read
  if (h->fetch_pending && h->fetch_host == Q_host) CK(cudaStreamWaitEvent(h->stream, h->fetch_done_ev, 0));
  CK(cudaMemcpyAsync(h->Q[h->cur], Q_host, (size_t)h->nodes * 6 * sizeof(double), cudaMemcpyHostToDevice,
                     h->stream));
  CK(cudaStreamSynchronize(h->stream));
  h->shadow_valid = false;
  return CMLES_OK;
}

cmles_status cmles_stage_state_host(cmles_handle h, const double *Q_host) {
  if (!h || !Q_host) return fail(h, CMLES_ERR_ARG, "cmles_stage_state_host: null argument");
  if (!h->Qstage) {
    cmles_status st = dalloc(h, (void **)&h->Qstage, (size_t)h->nodes * 6 * sizeof(double));
    if (st != CMLES_OK) return st;
    CK(cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&h->staged_ev, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&h->compute_ev, cudaEventDisableTiming));
  }
  // the staging buffer may have held the state of work still queued on the
  // handle's stream: the copy waits for that work, not for later launches
  CK(cudaEventRecord(h->compute_ev, h->stream));
  CK(cudaStreamWaitEvent(h->copy_stream, h->compute_ev, 0));
  // ... and for a host download still reading the staging buffer (the state
  // before a commit)
  if (h->fetch_unordered && h->fetch_src == h->Qstage) CK(cudaStreamWaitEvent(h->copy_stream, h->fetch_done_ev, 0));
  const size_t n = (size_t)h->nodes * 6;
  if (h->fetch_pending && h->fetch_host == Q_host) {
    // the host buffer is being written by the latest download: upload each
    // chunk as soon as it has arrived, so that the two directions overlap
    for (int i = 0; i < kFetchChunks; ++i) {
      size_t lo, hi;
      fetch_chunk(n, i, lo, hi);
      CK(cudaStreamWaitEvent(h->copy_stream, h->fetch_ev[i], 0));
      if (hi > lo)
        CK(cudaMemcpyAsync(h->Qstage + lo, Q_host + lo, (hi - lo) * sizeof(double), cudaMemcpyHostToDevice,
                           h->copy_stream));
    }
  } else {
    // an earlier download into this buffer has completed before the latest one
    if (h->fetch_pending) CK(cudaStreamWaitEvent(h->copy_stream, h->fetch_done_ev, 0));
    CK(cudaMemcpyAsync(h->Qstage, Q_host, n * sizeof(double), cudaMemcpyHostToDevice, h->copy_stream));
  }
  CK(cudaEventRecord(h->staged_ev, h->copy_stream));
  h->staged = true;
  return CMLES_OK;
}

cmles_status cmles_commit_staged_state(cmles_handle h) {
  if (!h) return CMLES_ERR_ARG;
  if (!h->staged) return fail(h, CMLES_ERR_STATE, "cmles_commit_staged_state: nothing staged");
  {
    cmles_status st = order_after_fetch(h);
    if (st != CMLES_OK) return st;
  }
  CK(cudaStreamWaitEvent(h->stream, h->staged_ev, 0));
  std::swap(h->Q[h->cur], h->Qstage);
  h->staged = false;
  h->shadow_valid = false;
  return CMLES_OK;
}

cmles_status cmles_get_state_host(cmles_handle h, double *Q_host) {
  if (!h || !Q_host) return fail(h, CMLES_ERR_ARG, "cmles_get_state_host: null argument");
  // a download into this host buffer lands first
  if (h->fetch_pending && h->fetch_host == Q_host) CK(cudaStreamWaitEvent(h->stream, h->fetch_done_ev, 0));
  CK(cudaMemcpyAsync(Q_host, h->Q[h->cur], (size_t)h->nodes * 6 * sizeof(double), cudaMemcpyDeviceToHost,
                     h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return CMLES_OK;
}

cmles_status cmles_tendency(cmles_handle h, const double *Q_dev, double *RHS_dev) {
  if (!h || !Q_dev || !RHS_dev) return fail(h, CMLES_ERR_ARG, "cmles_tendency: null argument");
  if (!h->have_ref) return fail(h, CMLES_ERR_STATE, "cmles_tendency: reference state not set");
  if (h->prm.closure == CMLES_CLOSURE_MLP && !h->have_mlp)
    return fail(h, CMLES_ERR_STATE, "cmles_tendency: closure weights not set");
  StageCoef sc = {0.0, 0.0, 0.0, 0, 0.f, 0.f, 0.f, 1};
  if (h->fp32) {
    // shadow of Q_dev into the idle shadow buffer; the handle's state is untouched
    cmles_status st = write_shadow(h, Q_dev, 1 - h->scur);
    if (st != CMLES_OK) return st;
    return run_stage_pair32(h, 1 - h->scur, RHS_dev, sc, false);
  }
  // the thermodynamic fields of Q_dev into the idle buffer
  cmles_status st = write_thermo64(h, Q_dev, h->TH64[1 - h->cur]);
  if (st != CMLES_OK) return st;
  return run_stage_pair(h, Q_dev, h->TH64[1 - h->cur], nullptr, nullptr, RHS_dev, sc, false);
}

// HEVI stage buffers and, for the current step, the vertical operator's
// tables (rebuilt when dt or the reference changes).
cmles_status ensure_hevi(cmles_handle h) {
  const size_t n6 = (size_t)h->nodes * 6;
  for (double *&b : h->hv_buf)
    if (!b) {
      cmles_status st = dalloc(h, (void **)&b, n6 * sizeof(double));
      if (st != CMLES_OK) return st;
    }
  if (h->hv_dt == h->prm.dt) return CMLES_OK;
  const int nez = h->mesh.nez, Nq = h->Nq, nlev = nez * Nq;
  HeviSetup S{};
  S.N = h->N;
  S.nez = nez;
  S.hz = h->K.hz;
  for (int a = 0; a < Nq; ++a) S.w[a] = h->w[a];
  for (int a = 0; a < Nq * Nq; ++a) S.D[a] = h->D[a];
  std::vector<double> z(nlev);
  for (int l = 0; l < nlev; ++l) z[l] = level_z(h, l);
  S.rho_r = h->ref_rho_h.data();
  S.p_r = h->ref_p_h.data();
  S.qt_r = h->ref_qt_h.data();
  S.z = z.data();
  S.g = h->prm.g;
  S.Rd = h->prm.Rd;
  S.Rv = h->prm.Rv;
  S.cvd = h->prm.cvd;
  S.cvv = h->prm.cvv;
  S.T0 = h->prm.T0;
  S.Iv0 = h->prm.Lv0 - h->prm.Rv * h->prm.T0;
  S.dtg = h->prm.dt * (1.0 - 1.0 / sqrt(2.0));
  HeviHost H;
  if (!hevi_build(S, H)) return fail(h, CMLES_ERR_ARG, "HEVI: I - dt gamma L could not be factored");
  const size_t nt = H.tab.size();
  if (!h->hv_tab) {
    cmles_status st = dalloc(h, (void **)&h->hv_tab, (nt + (size_t)nlev * 4) * sizeof(double));
    if (st != CMLES_OK) return st;
  }
  CK(cudaMemcpy(h->hv_tab, H.tab.data(), nt * sizeof(double), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(h->hv_tab + nt, H.lev.data(), (size_t)nlev * 4 * sizeof(double), cudaMemcpyHostToDevice));
  h->hv_T = HeviTables{h->hv_tab, h->hv_tab + nt, H.lift, S.dtg};
  h->hv_dt = h->prm.dt;
  return CMLES_OK;
}

// f(Y) for the HEVI stages, Y an FP64 state: the FP64 kernels, or on the
// FP32 path the FP32 kernels on Y's shadow (built in the idle shadow buffer).
cmles_status hevi_tendency(cmles_handle h, const double *Y, double *R) {
  const StageCoef sc = {0.0, 0.0, 0.0, 0, 0.f, 0.f, 0.f, 1};
  if (!h->fp32) {
    cmles_status st = write_thermo64(h, Y, h->TH64[1 - h->cur]);
    if (st != CMLES_OK) return st;
    return run_stage_pair(h, Y, h->TH64[1 - h->cur], nullptr, nullptr, R, sc, false);
  }
  cmles_status st = write_shadow(h, Y, 1 - h->scur);
  if (st != CMLES_OK) return st;
  return run_stage_pair32(h, 1 - h->scur, R, sc, false);
}

// One ARK2 step (Giraldo, Kelly & Constantinescu 2013) with the vertical
// linear operator L implicit: stage s solves
//   Y_s - dt gamma L(Y_s) = Q + dt sum_{j<s} (Ae_sj f_j + (Ai_sj - Ae_sj) L_j),
// f_j = f(Y_j), L_j = L(Y_j); then Q <- Q + dt sum_j b_j f_j.
cmles_status run_ark2_hevi(cmles_handle h) {
  const double g = 1.0 - 1.0 / sqrt(2.0), d = 1.0 / (2.0 * sqrt(2.0)), al = (3.0 + 2.0 * sqrt(2.0)) / 6.0;
  double *R0 = h->hv_buf[0], *R1 = h->hv_buf[1], *R2 = h->hv_buf[2], *L0 = h->hv_buf[3], *L1 = h->hv_buf[4];
  double *B = h->hv_buf[5], *Y = h->hv_buf[6];
  // the FP32 path keeps one FP64 state: its update is made in place
  double *Qn = h->Q[h->cur];
  double *Qo = h->fp32 ? Qn : h->Q[1 - h->cur];
  const double dt = h->prm.dt;
  const long long count = (long long)h->nodes * 6;
  cmles_status st;
  // stage 1: Y_1 = Q
  if ((st = hevi_tendency(h, Qn, R0)) != CMLES_OK) return st;
  {
    LaunchScope ls(h, 2, 3);
    CK(launch_hevi_apply(Qn, L0, h->hv_T, h->K, h->stream));
    // stage 2: Ae_21 = 2 gamma, Ai_21 = gamma
    CK(launch_lincomb(B, Qn, LinComb{2, dt, {2.0 * g, g - 2.0 * g, 0.0, 0.0}, {R0, L0, nullptr, nullptr}}, count,
                      h->stream));
    CK(launch_hevi_solve(B, Y, h->hv_T, h->K, h->stream));
  }
  if ((st = hevi_tendency(h, Y, R1)) != CMLES_OK) return st;
  {
    LaunchScope ls(h, 2, 3);
    CK(launch_hevi_apply(Y, L1, h->hv_T, h->K, h->stream));
    // stage 3: Ae_3 = (1 - alpha, alpha), Ai_3 = (delta, delta)
    CK(launch_lincomb(B, Qn, LinComb{4, dt, {1.0 - al, al, d - (1.0 - al), d - al}, {R0, R1, L0, L1}}, count,
                      h->stream));
    CK(launch_hevi_solve(B, Y, h->hv_T, h->K, h->stream));
  }
  if ((st = hevi_tendency(h, Y, R2)) != CMLES_OK) return st;
  {
    LaunchScope ls(h, 2, 1);
    CK(launch_lincomb(Qo, Qn, LinComb{3, dt, {d, d, g, 0.0}, {R0, R1, R2, nullptr}}, count, h->stream));
  }
  // the shadow (FP32) or the thermodynamic fields (FP64) of the new state are
  // built when next needed
  h->shadow_valid = false;
  if (!h->fp32) h->cur = 1 - h->cur;
  return CMLES_OK;
}

cmles_status cmles_step(cmles_handle h, int nsteps) {
  if (!h || nsteps < 0) return fail(h, CMLES_ERR_ARG, "cmles_step: bad argument");
  if (!h->have_ref) return fail(h, CMLES_ERR_STATE, "cmles_step: reference state not set");
  if (h->prm.closure == CMLES_CLOSURE_MLP && !h->have_mlp)
    return fail(h, CMLES_ERR_STATE, "cmles_step: closure weights not set");
  {
    cmles_status st = order_after_fetch(h);
    if (st != CMLES_OK) return st;
  }
  {
    cmles_status st = ensure_shadow(h);
    if (st != CMLES_OK) return st;
  }
  if (h->prm.integrator == CMLES_ARK2_HEVI) {
    cmles_status st = ensure_hevi(h);
    if (st != CMLES_OK) return st;
    for (int s = 0; s < nsteps; ++s) {
      if ((st = run_ark2_hevi(h)) != CMLES_OK) return st;
      if (h->prm.filter_order > 0 && (st = apply_expfilter(h)) != CMLES_OK) return st;
      h->steps += 1;
      h->time += h->prm.dt;
    }
    return CMLES_OK;
  }
  const bool l14 = h->prm.integrator == CMLES_LSRK144;
  const int nst = l14 ? 14 : 5;
  const double *TA = l14 ? kLsrk14A : kLsrkA, *TB = l14 ? kLsrk14B : kLsrkB;
  for (int s = 0; s < nsteps; ++s) {
    for (int k = 0; k < nst; ++k) {
      StageCoef sc = {TA[k], TB[k], h->prm.dt, k == nst - 1, (float)TA[k], (float)TB[k], (float)h->prm.dt,
                      TA[k] == 0.0};
      cmles_status st;
      if (h->fp32) {
        st = run_stage_pair32(h, h->scur, nullptr, sc, true);
        h->scur = 1 - h->scur;
      } else {
        st = run_stage_pair(h, h->Q[h->cur], h->TH64[h->cur], h->Q[1 - h->cur], h->TH64[1 - h->cur], h->dQ, sc,
                            true);
        h->cur = 1 - h->cur;
      }
      if (st != CMLES_OK) return st;
    }
    if (h->prm.filter_order > 0) {
      cmles_status st = apply_expfilter(h);
      if (st != CMLES_OK) return st;
    }
    h->steps += 1;
    h->time += h->prm.dt;
  }
  return CMLES_OK;
}

cmles_status cmles_filter(cmles_handle h) {
  if (!h) return CMLES_ERR_ARG;
  if (h->prm.filter_order <= 0) return fail(h, CMLES_ERR_ARG, "cmles_filter: filter_order is 0");
  {
    cmles_status st = order_after_fetch(h);
    if (st != CMLES_OK) return st;
  }
  return apply_expfilter(h);
}

cmles_status cmles_diagnostics(cmles_handle h, cmles_diag *out) {
  if (!h || !out) return fail(h, CMLES_ERR_ARG, "cmles_diagnostics: null argument");
  const double J = h->K.hx * h->K.hy * h->K.hz / 8.0;
  {
    LaunchScope ls(h, 2, 2);
    CK(launch_budgets(h->Q[h->cur], h->E, h->Np, h->wq, J, h->partials, h->budget_nblocks, h->budget_out,
                      h->stream, h->curved ? h->wJn : nullptr));
  }
  double res[7];
  int flags[16];
  CK(cudaMemcpyAsync(res, h->budget_out, 7 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemcpyAsync(flags, h->flags, 16 * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemsetAsync(h->flags, 0, 16 * sizeof(int), h->stream));
  CK(cudaStreamSynchronize(h->stream));
  for (int v = 0; v < 6; ++v) out->budget[v] = res[v];
  out->nonfinite = res[6] > 0.0 ? 1 : 0;
  out->satadj_failures = flags[0];
  out->tc_timeouts = flags[1];
  out->cold_saturated = flags[2];
  out->time = h->time;
  out->steps = h->steps;
  if (out->nonfinite) return fail(h, CMLES_ERR_NONFINITE, "state holds non-finite values");
  if (out->satadj_failures) return fail(h, CMLES_ERR_SATADJ, "saturation adjustment did not converge");
  if (out->tc_timeouts)
    return fail(h, CMLES_ERR_TIMEOUT, "a tensor-core completion wait gave up; the results since the previous "
                                      "report are invalid");
  return CMLES_OK;
}

cmles_status cmles_profiles(cmles_handle h, double *out_host) {
  if (!h || !out_host) return fail(h, CMLES_ERR_ARG, "cmles_profiles: null argument");
  if (h->curved) return fail(h, CMLES_ERR_ARG, "cmles_profiles: flat meshes only");
  const int nlev = h->mesh.nez * h->Nq;
  CK(cudaMemsetAsync(h->prof, 0, (size_t)nlev * 12 * sizeof(double), h->stream));
  {
    LaunchScope ls(h, 2, 2);
    CK(launch_profiles(h->Q[h->cur], h->K, h->N, h->prof, 0, h->stream));
    CK(launch_profiles(h->Q[h->cur], h->K, h->N, h->prof, 1, h->stream));
  }
  std::vector<double> a((size_t)nlev * 12);
  CK(cudaMemcpyAsync(a.data(), h->prof, a.size() * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  for (int l = 0; l < nlev; ++l) {
    const double *s = &a[(size_t)l * 12];
    double *o = out_host + (size_t)l * 11;
    o[0] = s[1] / s[0];
    o[1] = s[2] / s[1];
    o[2] = s[3] / s[1];
    o[3] = s[4] / s[1];
    o[4] = s[5] / s[1];
    o[5] = s[6] / s[1];
    o[6] = s[7] / s[1];
    o[7] = s[9] / s[1];
    o[8] = s[10] / s[1];
    o[9] = s[11] / s[1];
    o[10] = s[8] / s[1];
  }
  return CMLES_OK;
}

cmles_status cmles_set_closure_weights(cmles_handle h, const float *params_host, size_t n) {
  if (!h || !params_host) return fail(h, CMLES_ERR_ARG, "cmles_set_closure_weights: null argument");
  if (n != (size_t)kMlpParams)
    return fail(h, CMLES_ERR_ARG, "cmles_set_closure_weights: expected " + std::to_string(kMlpParams) + " values");
  h->mlp.assign(params_host, params_host + n);
  MlpPacked pk;
  pack_mlp_host(params_host, &pk);
  CK(cudaMemcpyAsync(h->mlp_dev, &pk, sizeof(pk), cudaMemcpyHostToDevice, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  h->have_mlp = true;
  return CMLES_OK;
}

cmles_status cmles_set_closure_weights_device(cmles_handle h, const float *params_dev) {
  if (!h || !params_dev) return fail(h, CMLES_ERR_ARG, "cmles_set_closure_weights_device: null argument");
  {
    LaunchScope ls(h, 2, 1);
    CK(launch_pack_mlp(params_dev, h->mlp_dev, h->stream));
  }
  h->have_mlp = true;
  return CMLES_OK;
}

cmles_status cmles_closure_samples(cmles_handle h, int factor, float *X_dev, float *T_dev, float *thv_dev,
                                   long long capacity, long long *n_out) {
  if (!h || !X_dev || !T_dev || factor < 1) return fail(h, CMLES_ERR_ARG, "cmles_closure_samples: bad argument");
  if (h->curved) return fail(h, CMLES_ERR_ARG, "cmles_closure_samples: flat meshes only");
  const cmles_mesh &m = h->mesh;
  if (m.nex % factor || m.ney % factor || m.nez % factor)
    return fail(h, CMLES_ERR_ARG, "cmles_closure_samples: element counts must be multiples of factor");
  const long long nc = (long long)(m.nex / factor) * (m.ney / factor) * (m.nez / factor) * h->Np;
  if (n_out) *n_out = nc;
  if (capacity < nc) return fail(h, CMLES_ERR_ARG, "cmles_closure_samples: output capacity too small");
  {
    LaunchScope ls(h, 2, 3);
    CK(launch_closure_samples(h->Q[h->cur], h->K, h->N, h->xi.data(), h->w.data(), h->D.data(), factor,
                              m.periodic, X_dev, T_dev, thv_dev, nc, h->stream));
  }
  return CMLES_OK;
}

cmles_status cmles_enable_timing(cmles_handle h, int enable) {
  if (!h) return CMLES_ERR_ARG;
  h->timing = enable != 0;
  return CMLES_OK;
}

cmles_status cmles_kernel_times(cmles_handle h, long long count[3], double ms[3], long long *launches) {
  if (!h) return CMLES_ERR_ARG;
  CK(cudaStreamSynchronize(h->stream));
  for (auto &t : h->timed) {
    float m = 0.f;
    cudaEventElapsedTime(&m, t.a, t.b);
    h->tcount[t.kind] += 1;
    h->tms[t.kind] += m;
    cudaEventDestroy(t.a);
    cudaEventDestroy(t.b);
  }
  h->timed.clear();
  for (int k = 0; k < 3; ++k) {
    if (count) count[k] = h->tcount[k];
    if (ms) ms[k] = h->tms[k];
    h->tcount[k] = 0;
    h->tms[k] = 0.0;
  }
  if (launches) *launches = h->launches;
  return CMLES_OK;
}

long long cmles_launch_count(cmles_handle h) { return h ? h->launches : -1; }

cmles_status cmles_hevi_operator(cmles_handle h, const double *Q_dev, double *out_dev) {
  if (!h || !Q_dev || !out_dev) return fail(h, CMLES_ERR_ARG, "cmles_hevi_operator: null argument");
  if (h->prm.integrator != CMLES_ARK2_HEVI) return fail(h, CMLES_ERR_STATE, "cmles_hevi_operator: not a HEVI handle");
  if (!h->have_ref) return fail(h, CMLES_ERR_STATE, "cmles_hevi_operator: reference state not set");
  cmles_status st = ensure_hevi(h);
  if (st != CMLES_OK) return st;
  LaunchScope ls(h, 2, 1);
  CK(launch_hevi_apply(Q_dev, out_dev, h->hv_T, h->K, h->stream));
  return CMLES_OK;
}

cmles_status cmles_hevi_solve(cmles_handle h, const double *B_dev, double *Y_dev) {
  if (!h || !B_dev || !Y_dev || B_dev == Y_dev) return fail(h, CMLES_ERR_ARG, "cmles_hevi_solve: bad argument");
  if (h->prm.integrator != CMLES_ARK2_HEVI) return fail(h, CMLES_ERR_STATE, "cmles_hevi_solve: not a HEVI handle");
  if (!h->have_ref) return fail(h, CMLES_ERR_STATE, "cmles_hevi_solve: reference state not set");
  cmles_status st = ensure_hevi(h);
  if (st != CMLES_OK) return st;
  LaunchScope ls(h, 2, 1);
  CK(launch_hevi_solve(B_dev, Y_dev, h->hv_T, h->K, h->stream));
  return CMLES_OK;
}

cmles_status cmles_test_stall_tc(cmles_handle h, int enable) {
  if (!h) return CMLES_ERR_ARG;
  if (enable < 0 || enable > 2) return fail(h, CMLES_ERR_ARG, "cmles_test_stall_tc: mode must be 0, 1 or 2");
  if (enable == 2 && h->N > 4)
    return fail(h, CMLES_ERR_ARG, "cmles_test_stall_tc: mode 2 has its test instance for N <= 4 only");
  h->tc_stall = enable;
  h->K.tc_stall = h->tc_stall;
  return CMLES_OK;
}
long long cmles_num_elements(cmles_handle h) { return h ? h->E : -1; }
long long cmles_num_nodes(cmles_handle h) { return h ? h->nodes : -1; }
long long cmles_device_bytes(cmles_handle h) { return h ? h->bytes : -1; }

}  // extern "C"
