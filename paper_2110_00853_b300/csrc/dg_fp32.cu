// FP32 DG right-hand side kernels with FP64 accumulation (CMLES_FP32_ACC64).
//
// Same two passes as the FP64 path (Sec. 3.1, Eq. matrixProblem), evaluated
// in FP32 on a shadow state stored as the deviation from the hydrostatic
// reference of its node level, s = Q - Q_ref(z) with
// Q_ref = (rho_r, 0, 0, 0, rho e_r, rho q_r); the subtraction is done in FP64
// when the shadow is written.  Every quantity whose full value is large next
// to its variation is evaluated in deviation form, which is exact algebra:
//   * temperature: rho c_vm (T - T_r) from the deviations of rho I, rho and
//     rho q_t (internal-energy balance of Eq. internal_energies);
//     saturation adjustment (Eq. sat_adjustment) as Newton on T - T_r with the
//     residual written relative to the reference identity;
//   * pressure: p - p_r = [rho R_m] (T - T_r) + ([rho R_m] - [rho R_m]_r) T_r
//     (Eq. eos), so the reference subtraction never cancels in FP32;
//   * h_tot, q_t and theta_v as deviations, with the reference parts' derivatives
//     (D applied to the level values in FP64) added to the gradient;
//   * the energy flux (rho e + p) u = H_r u + H' u: along x and y H_r is
//     constant on the derivative line and factors out; along z the line
//     differences H_r(m) - H_r(k) come from an FP64-built table.
// The LSRK register dQ is FP32.  Within a step the stage increments B_s dQ_s
// are summed in FP32 into D (relative to the increments, not to the state)
// and the shadow is advanced by them; the last stage adds D to the FP64 state
// Q once per step and rewrites the shadow from it.  On B300, where FP64 runs
// at 1/64 of the FP32 rate, four FP64 operations per variable and stage took
// a fifth of the flux pass.  Element traversal: 4 x 4 column tiles.
// The thermodynamics (temperature, saturation adjustment, pressure) runs once
// per node and state, in the kernel that writes the state: the flux pass for
// the state it advances to, the shadow kernel otherwise.  It stores p', the
// sound speed, h' and theta_v' (TH, four planes per element) for the flux
// pass and the gradient pass of the next stage, so that neither evaluates it
// again for its own nodes or its neighbours' face nodes.
#include "common.cuh"
#include "dg32_parts.cuh"
#include "launch.h"
#include "mlp.cuh"
#include "thermo32.cuh"

namespace cmles {

// CL: 1 Smagorinsky-Lilly, 3 Vreman (both with the Richardson correction),
// 2 learned closure
// (tensor-core MLP on the velocity and theta_v gradients and Delta).
// HOOK: the instance launched only under test hook 2 (cmles_test_stall_tc),
// whose first MMA completion wait gives up at once.
// One thread per node: NP = np32(N) threads per CTA (128 up to N = 4, then
// (N+1)^3 rounded up to a warp), the FP32 arrays padded to NP nodes per
// element.  The learned closure evaluates the CTA's rows in TT tiles of 128.
template <int N, int CL, bool HOOK = false>
__global__ void __launch_bounds__(np32(N), N > 4 ? 1 : (CL == 2 ? 6 : 8))
    k_grad32(const float *__restrict__ S, const float *__restrict__ TH, float *__restrict__ F2, const KParams P) {
  constexpr int Nq = N + 1, Np = Nq * Nq * Nq, Nf = Nq * Nq, NP = np32(N), TT = (NP + 127) / 128;
  // the gradient fields (own and neighbour face nodes) share their storage
  // with the closure network's A operand, which is written only after every
  // thread has finished its gradient
  constexpr bool DYN = grad32_dyn_bytes(N, CL) > 0;
  __shared__ float sD[Nq * Nq];
  __shared__ __align__(128) uint8_t sUst[DYN ? 16 : grad32_ubytes(N, CL)];
  extern __shared__ __align__(16) uint8_t sDynG32[];
  uint8_t *sU = DYN ? align128(sDynG32) : sUst;
  __shared__ int sNb[6];
  __shared__ __align__(16) uint8_t sMlpRaw[CL == 2 ? sizeof(MlpTc) : 16];
  __shared__ __align__(8) uint64_t sBar[2];
  __shared__ uint32_t sSlot;
  float(*sG)[NP] = reinterpret_cast<float(*)[NP]>(sU);
  float(*sGf)[6][Nf] = reinterpret_cast<float(*)[6][Nf]>(sU + 6 * NP * 4);
  __nv_bfloat16 *sA = reinterpret_cast<__nv_bfloat16 *>(sU);
  const KF &F = P.f;
  const int t = threadIdx.x;
  if (t < Nq * Nq) sD[t] = (float)P.D[t];
  const MlpTc &W = *reinterpret_cast<const MlpTc *>(sMlpRaw);
  TcState tcs;
  int stalled = 0;
  if (CL == 2) stalled = learned_setup<HOOK>(P, sMlpRaw, sBar, &sSlot, tcs, tc_cols_for(TT));
  const int i = t % Nq, j = (t / Nq) % Nq, k = t / Nf;
  // the element a CTA visits and its face neighbours, found by six lanes of
  // warp 0 one element ahead (during the previous element's last phase) and
  // shared, rather than by every thread
  __shared__ int sEl[3];
  if (t < 6 && blockIdx.x < P.E) next_element(P, blockIdx.x, sEl, sNb);
  __syncthreads();
  for (int g = blockIdx.x; g < P.E; g += gridDim.x) {
    const int e = sEl[0], ez = sEl[1];
    float sv[6], G[6];
    const float *L = P.lev32 + (size_t)(ez * Nq + (k < Nq ? k : 0)) * L_NF;
    if (t < Np) {
#pragma unroll
      for (int v = 0; v < 6; ++v) sv[v] = S[((size_t)e * 6 + v) * NP + t];
      // h' and theta_v' come with the state (its producer ran the
      // thermodynamics); u and q' are formed here exactly as there
      const float rinv = fdiv(1.0f, L[L_RHO] + sv[0]);
      G[0] = sv[1] * rinv;
      G[1] = sv[2] * rinv;
      G[2] = sv[3] * rinv;
      G[3] = TH[((size_t)e * 4 + 2) * NP + t];
      G[4] = (sv[5] - L[L_QM] * sv[0]) * rinv;
      G[5] = TH[((size_t)e * 4 + 3) * NP + t];
#pragma unroll
      for (int v = 0; v < 6; ++v) sG[v][t] = G[v];
    }
    __syncthreads();
    {
      // the 6 Nf face nodes, at most two per thread (task t and t + NP),
      // with the loads of both in flight before either is finished
      static_assert(6 * Nf <= 2 * NP, "two face nodes per thread at most");
      float ra[7], rb[7];
      const int tb = t + NP;
      auto load = [&](int task, float (&raw)[7]) {
        const int f = task / Nf, fn = task - f * Nf;
        const int nb = sNb[f];
        if (nb >= 0) face_load(S, TH, nb, face_node<Nq>(f >> 1, (f & 1) ? 0 : N, fn % Nq, fn / Nq), raw, NP);
      };
      auto finish = [&](int task, const float (&raw)[7]) {
        const int f = task / Nf, fn = task - f * Nf;
        const int d = f >> 1, t1 = fn % Nq, t2 = fn / Nq;
        if (sNb[f] < 0) {
          // a wall: the mirror state (normal velocity reversed), so that the
          // lift below is the same formula on every face
          const int n = face_node<Nq>(d, (f & 1) ? N : 0, t1, t2);
#pragma unroll
          for (int v = 0; v < 6; ++v)
            sGf[f][v][fn] = (v == d || (v < 3 && ((P.noslip >> f) & 1))) ? -sG[v][n] : sG[v][n];
          return;
        }
        // the shared face node has the same height, hence the same level values
        const float *Lf = P.lev32 + (size_t)(ez * Nq + (d == 2 ? (f & 1 ? N : 0) : t2)) * L_NF;
        float gf[6];
        face_finish(raw, Lf[L_RHO], Lf[L_QM], gf);
#pragma unroll
        for (int v = 0; v < 6; ++v) sGf[f][v][fn] = gf[v];
      };
      if (t < 6 * Nf) load(t, ra);
      if (tb < 6 * Nf) load(tb, rb);
      if (t < 6 * Nf) finish(t, ra);
      if (tb < 6 * Nf) finish(tb, rb);
    }
    __syncthreads();
    float gr[6][3];
    float nut = 0.f, Dt = 0.f;
    if (t < Np) {
#pragma unroll
      for (int v = 0; v < 6; ++v) {
        float a0 = 0.f, a1 = 0.f, a2 = 0.f;
#pragma unroll
        for (int m = 0; m < Nq; ++m) {
          a0 += sD[i * Nq + m] * sG[v][m + Nq * (j + Nq * k)];
          a1 += sD[j * Nq + m] * sG[v][i + Nq * (m + Nq * k)];
          a2 += sD[k * Nq + m] * sG[v][i + Nq * (j + Nq * m)];
        }
        gr[v][0] = F.jac[0] * a0;
        gr[v][1] = F.jac[1] * a1;
        gr[v][2] = F.jac[2] * a2;
      }
      // reference parts of h_tot, q_t and theta_v: derivative along z only
      gr[3][2] += L[L_DZ_HM];
      gr[4][2] += L[L_DZ_Q];
      gr[5][2] += L[L_DZ_THV];
      // the lift of the face averages on the node's x, y and z faces (the
      // mirror state on walls), without branches: factor 0 inside
      {
        const float Lx = i == 0 ? -F.lift[0] : (i == N ? F.lift[0] : 0.f);
        const float Ly = j == 0 ? -F.lift[1] : (j == N ? F.lift[1] : 0.f);
        const float Lz = k == 0 ? -F.lift[2] : (k == N ? F.lift[2] : 0.f);
        const float *gx = &sGf[i == N ? 1 : 0][0][j + Nq * k];
        const float *gy = &sGf[j == N ? 3 : 2][0][i + Nq * k];
        const float *gz = &sGf[k == N ? 5 : 4][0][i + Nq * j];
#pragma unroll
        for (int v = 0; v < 6; ++v) {
          gr[v][0] += Lx * (0.5f * (G[v] + gx[v * Nf]) - G[v]);
          gr[v][1] += Ly * (0.5f * (G[v] + gy[v * Nf]) - G[v]);
          gr[v][2] += Lz * (0.5f * (G[v] + gz[v * Nf]) - G[v]);
        }
      }

      if ((CL == 1 && P.closure == 1) || CL == 3)
        eddy_nu<CL == 3 ? 3 : 1>(gr, F.CsDelta2, L[L_THV] + G[5], F, P.richardson, nut, Dt);
    }
    // the learned closure on the tensor cores, row t = node t
    if (CL == 2) learned_nu<HOOK, TT>(W, sA, tcs, gr, F.Delta, t < Np, nut, Dt);
    if (t < Np) write_f2(F2, e, t, L[L_RHO] + sv[0], nut, Dt, gr, sv, G, NP);
    if (t < 6 && g + (int)gridDim.x < P.E) next_element(P, g + gridDim.x, sEl, sNb);
    __syncthreads();
  }
  if (CL == 2) {
    if (stalled) tcs.err = 1;
    tc_teardown(tcs, P.flags + 1, tc_cols_for(TT));
  }
}

// UPD: 0 right-hand side only; 1 LSRK stage, the step's increment
// D = sum_s B_s dQ_s carried in FP32 and the shadow advanced by B_s dQ_s;
// 2 last stage of the step, Q = Q_step_start + D added in FP64 and the shadow
// rewritten from it.  With UPD 1 and 2 the new shadow's thermodynamic fields
// go to THout.  p' and c of the input state come from TH.  FL: numerical
// flux of F1, 0 Rusanov, 1 HLLC, 2 Roe.  One thread per node, NP = np32(N)
// threads per CTA.
// The flux pass's 27 node planes (total fluxes, state, velocity) take
// 27 * 4 * np32(N) bytes of shared memory: static up to N = 6, dynamic at
// N = 7 (55 KB, beyond the 48 KB of static shared memory).
__host__ __device__ constexpr int rhs32_dyn_bytes(int N) { return 27 * 4 * np32(N) > 40 * 1024 ? 27 * 4 * np32(N) : 0; }

template <int N, int UPD, int FL>
__global__ void __launch_bounds__(np32(N), N > 4 ? 1 : (FL == 0 ? 7 : 6))
    k_rhs32(const float *__restrict__ S, const float *__restrict__ F2, const float *__restrict__ TH,
            float *__restrict__ dQ, double *__restrict__ Q64, float *__restrict__ Sout, float *__restrict__ THout,
            double *__restrict__ Rout, const StageCoef sc, const KParams P) {
  constexpr int Nq = N + 1, Np = Nq * Nq * Nq, Nf = Nq * Nq, NP = np32(N);
  constexpr bool DYN = rhs32_dyn_bytes(N) > 0;
  __shared__ float sD[Nq * Nq];
  __shared__ float sFst[DYN ? 1 : 18 * NP];
  __shared__ float sSst[DYN ? 1 : 6 * NP];
  __shared__ float sUst[DYN ? 1 : 3 * NP];
  extern __shared__ __align__(16) float sDyn32[];
  float(*sF)[3][NP] = reinterpret_cast<float(*)[3][NP]>(DYN ? sDyn32 : sFst);
  float(*sS)[NP] = reinterpret_cast<float(*)[NP]>(DYN ? sDyn32 + 18 * NP : sSst);
  float(*sU)[NP] = reinterpret_cast<float(*)[NP]>(DYN ? sDyn32 + 24 * NP : sUst);
  __shared__ float sLf[6][6][Nf];
  __shared__ int sNb[6];
  // the drag law's C_d |u_p| u_p of the bottom face nodes, from the nodes of
  // the first interior layer above them
  __shared__ float sDrag[2][Nf];
  const KF &F = P.f;
  const int t = threadIdx.x;
  if (t < Nq * Nq) sD[t] = (float)P.D[t];
  const int i = t % Nq, j = (t / Nq) % Nq, k = t / Nf;
  int fail = 0;
  // the element and its neighbours, found one element ahead by six lanes
  __shared__ int sEl[3];
  if (t < 6 && blockIdx.x < P.E) next_element(P, blockIdx.x, sEl, sNb);
  __syncthreads();
  for (int g = blockIdx.x; g < P.E; g += gridDim.x) {
    const int e = sEl[0], ez = sEl[1], ex = sEl[2];
    const float *L = P.lev32 + (size_t)(ez * Nq + (k < Nq ? k : 0)) * L_NF;
    float sv[6];
    // the update's inputs, loaded with the element's first loads so that
    // their latency overlaps the flux computation (the first stage has A = 0
    // and starts the step: no register or increment to read)
    float dq0[6], D0[6];
    double q0[6];
    if (UPD && t < Np) stage_inputs<UPD>(P, sc, dQ, Q64, e, t, Np, dq0, D0, q0, NP);
    if (t < Np) {
#pragma unroll
      for (int v = 0; v < 6; ++v) {
        sv[v] = S[((size_t)e * 6 + v) * NP + t];
        sS[v][t] = sv[v];
      }
      const float pp = TH[((size_t)e * 4) * NP + t];
      const float rho = L[L_RHO] + sv[0];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        float f[6];
        flux1_dev32(sv, L[L_RHO], L[L_RHOQ], pp, d, f);
        const float *g2 = F2 + ((size_t)e * 15 + d * 5) * NP + t;
        const float c0 = g2[0];
        sF[0][d][t] = f[0] + c0;
        sF[1][d][t] = f[1] + g2[1 * NP];
        sF[2][d][t] = f[2] + g2[2 * NP];
        sF[3][d][t] = f[3] + g2[3 * NP];
        sF[4][d][t] = f[4] + g2[4 * NP];
        sF[5][d][t] = f[5] + c0;
        sU[d][t] = fdiv(sv[1 + d], rho);
      }
      if (k == 1 && F.drag_cd > 0.f && sNb[4] < 0) {
        const float ux = sU[0][t], uy = sU[1][t];
        const float c = F.drag_cd * sqrtf(ux * ux + uy * uy);
        sDrag[0][i + Nq * j] = c * ux;
        sDrag[1][i + Nq * j] = c * uy;
      }
    }
    __syncthreads();
    for (int task = t; task < 6 * Nf; task += blockDim.x) {
      const int f = task / Nf, fn = task - f * Nf;
      const int d = f >> 1, t1 = fn % Nq, t2 = fn / Nq;
      const int a = (f & 1) ? N : 0;
      const float sg = (f & 1) ? 1.f : -1.f;
      const int n = face_node<Nq>(d, a, t1, t2);
      const float *Lf = P.lev32 + (size_t)(ez * Nq + (d == 2 ? a : t2)) * L_NF;
      const float rho_r = Lf[L_RHO], rhoq_r = Lf[L_RHOQ];
      float sm[6], sp[6];
#pragma unroll
      for (int v = 0; v < 6; ++v) sm[v] = sS[v][n];
      const float cm = TH[((size_t)e * 4 + 1) * NP + n];
      const int nb = sNb[f];
      if (FL == 0 && nb >= 0) {
        // Rusanov across an interior face.  The own node's total normal flux
        // n.(F1 + F2) is sF from the first phase, so the lifted jump
        // n.F_- - F* is 1/2 n.(F_- - F_+) - 1/2 lambda (s_- - s_+) and only
        // the neighbour's F1 is evaluated here (1 % of the pass).
        const int nn = face_node<Nq>(d, N - a, t1, t2);
#pragma unroll
        for (int v = 0; v < 6; ++v) sp[v] = S[((size_t)nb * 6 + v) * NP + nn];
        const float pp = TH[((size_t)nb * 4) * NP + nn];
        const float cp = TH[((size_t)nb * 4 + 1) * NP + nn];
        const float *g2p = F2 + ((size_t)nb * 15 + d * 5) * NP + nn;
        float fp[6];
        flux1_dev32(sp, rho_r, rhoq_r, pp, d, fp);
        fp[0] += g2p[0];
        fp[1] += g2p[1 * NP];
        fp[2] += g2p[2 * NP];
        fp[3] += g2p[3 * NP];
        fp[4] += g2p[4 * NP];
        fp[5] += g2p[0];
        const float smd = d == 0 ? sm[1] : (d == 1 ? sm[2] : sm[3]);
        const float spd = d == 0 ? sp[1] : (d == 1 ? sp[2] : sp[3]);
        const float um = fdiv(smd, rho_r + sm[0]), up = fdiv(spd, rho_r + sp[0]);
        const float lam = fmaxf(fabsf(um) + cm, fabsf(up) + cp);
        const float hs = 0.5f * sg;
#pragma unroll
        for (int v = 0; v < 6; ++v) {
          float r = hs * (sF[v][d][n] - fp[v]) - 0.5f * lam * (sm[v] - sp[v]);
          if (v == 4) r += hs * Lf[L_H] * (um - up);  // reference part of the energy flux
          sLf[f][v][fn] = F.lift[d] * r;
        }
        continue;
      }
      const float pm = TH[((size_t)e * 4) * NP + n];
      float pp, cp, f2s[5];
      if (nb >= 0) {
        const int nn = face_node<Nq>(d, N - a, t1, t2);
#pragma unroll
        for (int v = 0; v < 6; ++v) sp[v] = S[((size_t)nb * 6 + v) * NP + nn];
        pp = TH[((size_t)nb * 4) * NP + nn];
        cp = TH[((size_t)nb * 4 + 1) * NP + nn];
        const float *g2m = F2 + ((size_t)e * 15 + d * 5) * NP + n;
        const float *g2p = F2 + ((size_t)nb * 15 + d * 5) * NP + nn;
#pragma unroll
        for (int c = 0; c < 5; ++c) f2s[c] = 0.5f * (sg * g2m[c * NP] + sg * g2p[c * NP]);
      } else {
#pragma unroll
        for (int v = 0; v < 6; ++v) sp[v] = sm[v];
        // (no-slip: u_bc = 0, every velocity component reversed)
        const bool ns = (P.noslip >> f) & 1;
        sp[1] = (ns || d == 0) ? -sm[1] : sm[1];
        sp[2] = (ns || d == 1) ? -sm[2] : sm[2];
        sp[3] = (ns || d == 2) ? -sm[3] : sm[3];
        pp = pm;
        cp = cm;
#pragma unroll
        for (int c = 0; c < 5; ++c) f2s[c] = 0.f;
        if (f == 4 && P.surface_flux) {
          f2s[0] = -F.E_water;
          f2s[4] = -F.E_energy;
        }
        if (f == 4 && F.drag_cd > 0.f) {
          // drag law (Eq. drag_law) on the flat bottom: outward flux
          // rho C_d |u_p| u_p of the horizontal momentum, C_d |u_p| u_p from
          // the first phase
          const float rw = rho_r + sm[0];
          f2s[1] = rw * sDrag[0][fn];
          f2s[2] = rw * sDrag[1][fn];
        }
      }
      float fm[6], fp[6], f1s[6];
      flux1_dev32(sm, rho_r, rhoq_r, pm, d, fm);
      flux1_dev32(sp, rho_r, rhoq_r, pp, d, fp);
      const float smd = d == 0 ? sm[1] : (d == 1 ? sm[2] : sm[3]);
      const float spd = d == 0 ? sp[1] : (d == 1 ? sp[2] : sp[3]);
      const float um = fdiv(smd, rho_r + sm[0]), up = fdiv(spd, rho_r + sp[0]);
      // reference part of the energy flux (H_r u.n is not in fm, fp): the
      // own node's H_r (u-.n) minus that of the numerical flux
      float ref4;
      if (FL == 1) {
        // HLLC: n.F1(Y_K) + S_K (U*_K - U_K), full states from the deviations
        const float rM = rho_r + sm[0], rP = rho_r + sp[0];
        const float iM = fdiv(1.0f, rM), iP = fdiv(1.0f, rP);
        const float uM[3] = {sm[1] * iM, sm[2] * iM, sm[3] * iM}, uP[3] = {sp[1] * iP, sp[2] * iP, sp[3] * iP};
        const float Er = Lf[L_H] - Lf[L_P];  // rho e_r
        const float nrm[3] = {d == 0 ? sg : 0.f, d == 1 ? sg : 0.f, d == 2 ? sg : 0.f};
        float J[6];
        const int K = hllc_jump<float>(rM, uM, (rhoq_r + sm[5]) * iM, (Er + sm[4]) * iM, Lf[L_P] + pm, cm, rP, uP,
                                       (rhoq_r + sp[5]) * iP, (Er + sp[4]) * iP, Lf[L_P] + pp, cp, pp - pm, nrm, J);
#pragma unroll
        for (int v = 0; v < 6; ++v) f1s[v] = sg * (K ? fp[v] : fm[v]) + J[v];
        ref4 = K ? sg * Lf[L_H] * (um - up) : 0.f;
      } else if (FL == 2) {
        // Roe: 1/2 n.(F1- + F1+) - 1/2 |A| (Y+ - Y-), full states from the deviations
        const float rM = rho_r + sm[0], rP = rho_r + sp[0];
        const float iM = fdiv(1.0f, rM), iP = fdiv(1.0f, rP);
        const float uM[3] = {sm[1] * iM, sm[2] * iM, sm[3] * iM}, uP[3] = {sp[1] * iP, sp[2] * iP, sp[3] * iP};
        const float nrm[3] = {d == 0 ? sg : 0.f, d == 1 ? sg : 0.f, d == 2 ? sg : 0.f};
        float dY[6], D[6];
#pragma unroll
        for (int v = 0; v < 6; ++v) dY[v] = sp[v] - sm[v];
        const RoeConst<float> rk = {F.Rd, F.Rv - F.Rd, F.cvd, F.cvv - F.cvd, F.T0, F.Iv0};
        roe_dissipation<float>(rM, uM, (rhoq_r + sm[5]) * iM, (Lf[L_H] + sm[4] + pm) * iM, rP, uP,
                               (rhoq_r + sp[5]) * iP, (Lf[L_H] + sp[4] + pp) * iP, dY, Lf[L_GZ], nrm, rk, D);
#pragma unroll
        for (int v = 0; v < 6; ++v) f1s[v] = 0.5f * (sg * fm[v] + sg * fp[v]) - 0.5f * D[v];
        ref4 = 0.5f * sg * Lf[L_H] * (um - up);
      } else {
        const float lam = fmaxf(fabsf(um) + cm, fabsf(up) + cp);
#pragma unroll
        for (int v = 0; v < 6; ++v) f1s[v] = 0.5f * (sg * fm[v] + sg * fp[v]) + 0.5f * lam * (sm[v] - sp[v]);
        ref4 = 0.5f * sg * Lf[L_H] * (um - up);
      }
      const int c_of_v[6] = {0, 1, 2, 3, 4, 0};
#pragma unroll
      for (int v = 0; v < 6; ++v) {
        float r = sg * sF[v][d][n] - (f1s[v] + f2s[c_of_v[v]]);
        if (v == 4) r += ref4;
        sLf[f][v][fn] = F.lift[d] * r;
      }
    }
    __syncthreads();
    if (t < Np) {
      // the lifted face terms of the node's x, y and z faces, without
      // branches: weight 1 on a face, 0 (on any valid entry) inside
      const float wx = (i == 0 || i == N) ? 1.f : 0.f, wy = (j == 0 || j == N) ? 1.f : 0.f,
                  wz = (k == 0 || k == N) ? 1.f : 0.f;
      const float *lx = &sLf[i == N ? 1 : 0][0][j + Nq * k];
      const float *ly = &sLf[j == N ? 3 : 2][0][i + Nq * k];
      const float *lz = &sLf[k == N ? 5 : 4][0][i + Nq * j];
      float R[6];
#pragma unroll
      for (int v = 0; v < 6; ++v) {
        float a0 = 0.f, a1 = 0.f, a2 = 0.f;
#pragma unroll
        for (int m = 0; m < Nq; ++m) {
          a0 += sD[i * Nq + m] * sF[v][0][m + Nq * (j + Nq * k)];
          a1 += sD[j * Nq + m] * sF[v][1][i + Nq * (m + Nq * k)];
          a2 += sD[k * Nq + m] * sF[v][2][i + Nq * (j + Nq * m)];
        }
        float r = -(F.jac[0] * a0 + F.jac[1] * a1 + F.jac[2] * a2);
        r = fmaf(wx, lx[v * Nf], r);
        r = fmaf(wy, ly[v * Nf], r);
        r = fmaf(wz, lz[v * Nf], r);
        R[v] = r;
      }
      {
        // divergence of H_r u: H_r(k) D u along x and y, and along z
        // H_r(k) D w + sum_m D_km (H_r(m) - H_r(k)) w_m
        float ux = 0.f, vy = 0.f, wz = 0.f, wdh = 0.f;
        const float *dH = P.dH32 + (size_t)ez * Nq * Nq + k * Nq;
#pragma unroll
        for (int m = 0; m < Nq; ++m) {
          ux += sD[i * Nq + m] * sU[0][m + Nq * (j + Nq * k)];
          vy += sD[j * Nq + m] * sU[1][i + Nq * (m + Nq * k)];
          const float wm = sU[2][i + Nq * (j + Nq * m)];
          wz += sD[k * Nq + m] * wm;
          wdh += sD[k * Nq + m] * dH[m] * wm;
        }
        R[4] -= L[L_H] * (F.jac[0] * ux + F.jac[1] * vy + F.jac[2] * wz) + F.jac[2] * wdh;
      }
      float tau = L[L_TAU];
      if (P.tau_col) tau = fmaxf(tau, (float)P.tau_col[(ex + P.gx0) * Nq + i]);
      momentum_sources(sv, L[L_RHO] + sv[0], tau, F, R);
      float sn[6];
      stage_update<UPD>(P, sc, R, dq0, D0, q0, sv, P.qref64 + (size_t)(ez * Nq + k) * 4, 1, dQ, Q64, Sout, Rout, e,
                        t, Np, sn, NP);
      // the thermodynamics of the new state, for the next stage's two passes
      if (UPD) thermo_store32(P, L, sn, THout, e, t, fail, NP);
    }
    if (t < 6 && g + (int)gridDim.x < P.E) next_element(P, g + gridDim.x, sEl, sNb);
    __syncthreads();
  }
  report_thermo_flags(P, fail);
}

// Shadow of an FP64 state: s = (float)(Q - Q_ref(level)), subtraction in
// FP64, with its thermodynamic fields.  Q64 null: the shadow S is given and
// only its thermodynamic fields are written.  np: padded nodes per element
// of the FP32 arrays.
__global__ void k_shadow32(const double *__restrict__ Q64, float *__restrict__ S, float *__restrict__ TH,
                           const KParams P, int Np, int Nq, int np) {
  const long long n = (long long)P.E * Np;
  int fail = 0;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
    const long long g = q / Np;
    const int node = (int)(q - g * Np);
    int ex, ey, ez;
    const long long e = element_lin(P, g, ex, ey, ez);
    const int k = node / (Nq * Nq);
    const double *qr = P.qref64 + (size_t)(ez * Nq + k) * 4;
    float s[6];
#pragma unroll
    for (int v = 0; v < 6; ++v) {
      if (Q64) {
        const double ref = v == 0 ? qr[0] : (v == 4 ? qr[1] : (v == 5 ? qr[2] : 0.0));
        s[v] = (float)(Q64[(e * 6 + v) * Np + node] - ref);
        S[(e * 6 + v) * np + node] = s[v];
      } else {
        s[v] = S[(e * 6 + v) * np + node];
      }
    }
    thermo_store32(P, P.lev32 + (size_t)(ez * Nq + k) * L_NF, s, TH, (size_t)e, node, fail, np);
  }
  report_thermo_flags(P, fail);
}

cudaError_t launch_shadow32(const double *Q64, float *S, float *TH, const KParams &P, int N, cudaStream_t s) {
  const int Nq = N + 1, Np = Nq * Nq * Nq;
  long long nodes = (long long)P.E * Np;
  int blocks = (int)((nodes + 255) / 256);
  if (blocks > 148 * 32) blocks = 148 * 32;
  k_shadow32<<<blocks, 256, 0, s>>>(Q64, S, TH, P, Np, Nq, np32(N));
  return cudaGetLastError();
}

template <int N, int CL>
static void grad32_instance(const float *S, const float *TH, float *F2, const KParams &P, cudaStream_t s) {
  static int grid = 0;
  constexpr int dyn = grad32_dyn_bytes(N, CL);
  if (!grid) {
    if (dyn > 0)
      cudaFuncSetAttribute((const void *)k_grad32<N, CL>, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
    grid = CL == 2 ? grid_for_tc((const void *)k_grad32<N, CL>, 1 << 30, tc_cols_for((np32(N) + 127) / 128),
                                 np32(N), dyn)
                   : grid_for((const void *)k_grad32<N, CL>, 1 << 30, 0, np32(N));
  }
  // the test instance of hook 2 is built for the 128-thread CTAs
  if constexpr (CL == 2 && N <= 4) {
    if (P.tc_stall == 2) {
      static int hgrid = 0;
      if (!hgrid) hgrid = grid_for_tc((const void *)k_grad32<N, 2, true>, 1 << 30, kTcCols);
      k_grad32<N, 2, true><<<hgrid < P.E ? hgrid : P.E, 128, 0, s>>>(S, TH, F2, P);
      return;
    }
  }
  k_grad32<N, CL><<<grid < P.E ? grid : P.E, np32(N), dyn, s>>>(S, TH, F2, P);
}

template <int N>
static void grad32_order(const float *S, const float *TH, float *F2, const KParams &P, cudaStream_t s) {
  if (P.closure == 2)
    grad32_instance<N, 2>(S, TH, F2, P, s);
  else if (P.closure == 3)
    grad32_instance<N, 3>(S, TH, F2, P, s);
  else
    grad32_instance<N, 1>(S, TH, F2, P, s);
}

// the flat-mesh kernels are instantiated for the orders 1 .. 7 (one thread
// per node, np32(N) threads per CTA and padded nodes per element)
cudaError_t launch_grad32(const float *S, const float *TH, float *F2, const KParams &P, cudaStream_t s) {
  switch (P.N) {
    case 1: grad32_order<1>(S, TH, F2, P, s); break;
    case 2: grad32_order<2>(S, TH, F2, P, s); break;
    case 3: grad32_order<3>(S, TH, F2, P, s); break;
    case 4: grad32_order<4>(S, TH, F2, P, s); break;
    case 5: grad32_order<5>(S, TH, F2, P, s); break;
    case 6: grad32_order<6>(S, TH, F2, P, s); break;
    case 7: grad32_order<7>(S, TH, F2, P, s); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <int N, int UPD, int FL>
static void k_rhs32_instance(const float *S, const float *F2, const float *TH, float *dQ, double *Q64, float *Sout,
                             float *THout, double *Rout, const StageCoef &sc, const KParams &P, cudaStream_t s) {
  static int grid = 0;
  constexpr int smem = rhs32_dyn_bytes(N);
  if (!grid) {
    if (smem > 0)
      cudaFuncSetAttribute((const void *)k_rhs32<N, UPD, FL>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    grid = grid_for((const void *)k_rhs32<N, UPD, FL>, 1 << 30, smem, np32(N));
  }
  k_rhs32<N, UPD, FL><<<grid < P.E ? grid : P.E, np32(N), smem, s>>>(S, F2, TH, dQ, Q64, Sout, THout, Rout, sc, P);
}

template <int N, int FL>
static void k_rhs32_dispatch(const float *S, const float *F2, const float *TH, float *dQ, double *Q64, float *Sout,
                             float *THout, double *Rout, const StageCoef &sc, bool update, const KParams &P,
                             cudaStream_t s) {
  if (!update)
    k_rhs32_instance<N, 0, FL>(S, F2, TH, dQ, Q64, Sout, THout, Rout, sc, P, s);
  else if (sc.last)
    k_rhs32_instance<N, 2, FL>(S, F2, TH, dQ, Q64, Sout, THout, Rout, sc, P, s);
  else
    k_rhs32_instance<N, 1, FL>(S, F2, TH, dQ, Q64, Sout, THout, Rout, sc, P, s);
}

template <int N>
static void rhs32_order(const float *S, const float *F2, const float *TH, float *dQ, double *Q64, float *Sout,
                        float *THout, double *Rout, const StageCoef &sc, bool update, const KParams &P,
                        cudaStream_t s) {
  if (P.flux == 2)
    k_rhs32_dispatch<N, 2>(S, F2, TH, dQ, Q64, Sout, THout, Rout, sc, update, P, s);
  else if (P.flux == 1)
    k_rhs32_dispatch<N, 1>(S, F2, TH, dQ, Q64, Sout, THout, Rout, sc, update, P, s);
  else
    k_rhs32_dispatch<N, 0>(S, F2, TH, dQ, Q64, Sout, THout, Rout, sc, update, P, s);
}

cudaError_t launch_rhs32(const float *S, const float *F2, const float *TH, float *dQ, double *Q64, float *Sout,
                         float *THout, double *Rout, const StageCoef &sc, bool update, const KParams &P,
                         cudaStream_t s) {
  switch (P.N) {
    case 1: rhs32_order<1>(S, F2, TH, dQ, Q64, Sout, THout, Rout, sc, update, P, s); break;
    case 2: rhs32_order<2>(S, F2, TH, dQ, Q64, Sout, THout, Rout, sc, update, P, s); break;
    case 3: rhs32_order<3>(S, F2, TH, dQ, Q64, Sout, THout, Rout, sc, update, P, s); break;
    case 4: rhs32_order<4>(S, F2, TH, dQ, Q64, Sout, THout, Rout, sc, update, P, s); break;
    case 5: rhs32_order<5>(S, F2, TH, dQ, Q64, Sout, THout, Rout, sc, update, P, s); break;
    case 6: rhs32_order<6>(S, F2, TH, dQ, Q64, Sout, THout, Rout, sc, update, P, s); break;
    case 7: rhs32_order<7>(S, F2, TH, dQ, Q64, Sout, THout, Rout, sc, update, P, s); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace cmles
