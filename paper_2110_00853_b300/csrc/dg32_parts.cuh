// Device functions shared by the FP32 passes on flat meshes (dg_fp32.cu) and
// on curvilinear meshes (dg_curved32.cu): the closures of the gradient pass
// (Sec. 4: Smagorinsky-Lilly with the Richardson correction and Vreman; the
// learned closure on the tensor cores, which extends Sec. 4), the diffusive
// flux F2 they feed, the primitives of a neighbour's face node, and the
// sources and LSRK stage update that end the flux pass.  The two files differ only in geometry:
// constant axis-aligned metric terms and level tables on flat meshes,
// per-node metric terms and tables on curvilinear ones.
#pragma once

#include "common.cuh"
#include "mlp.cuh"
#include "thermo32.cuh"

namespace cmles {

// Set-up of the learned closure in a CTA: the network's weights to shared
// memory, the TMEM columns and the MMA completion barrier (sBar[0]); sBar[1]
// serves test hook 1, a bounded wait that nothing arrives on.  Returns 1 when
// that wait ran out (reported like a failed MMA wait; the work stays intact).
// HOOK instances (test hook 2) give up their first MMA completion wait at
// once, while the MMA is in flight.  All threads must call it.
// ncols: TMEM columns of the CTA (tc_cols_for its row tiles).
template <bool HOOK>
__device__ __forceinline__ int learned_setup(const KParams &P, uint8_t *sMlpRaw, uint64_t *sBar, uint32_t *sSlot,
                                             TcState &tcs, uint32_t ncols = kTcCols) {
  const int t = threadIdx.x;
  const uint4 *src = reinterpret_cast<const uint4 *>(&P.mlp->tc);
  uint4 *dst = reinterpret_cast<uint4 *>(sMlpRaw);
  for (int q = t; q < (int)(sizeof(MlpTc) / 16); q += blockDim.x) dst[q] = src[q];
  fence_proxy_async_smem();
  if (t == 0) mbar_init(&sBar[1], 1);
  tc_setup(tcs, sSlot, &sBar[0], ncols);
  int stalled = 0;
  if (P.tc_stall == 1 && !mbar_wait_bounded(&sBar[1], 0, 1 << 14)) stalled = 1;
  if (HOOK) tcs.hook = 1;
  __syncwarp();
  return stalled;
}

// The learned closure (an extension of Sec. 4): the network's inputs are
// the nine velocity gradients, the three theta_v gradients and Delta, scaled;
// its two outputs, rectified and scaled, are nu_t and the eddy diffusivity D_t.  Row
// t of the tensor-core evaluation is node t; rows without a node (valid
// false) carry zeros.  The A operand overwrites shared storage that the
// gradient fields occupied, hence the block barrier before it is written.
// All threads must call it.  T: row tiles of 128 rows (CTAs of more than 128
// threads, N > 4).
template <bool HOOK, int T = 1>
__device__ __forceinline__ void learned_nu(const MlpTc &W, __nv_bfloat16 *sA, TcState &tcs, const float (&gr)[6][3],
                                           float Delta, bool valid, float &nut, float &Dt) {
  float x[kMlpIn];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) x[3 * a + b] = valid ? gr[a][b] * W.in_scale[3 * a + b] : 0.f;
#pragma unroll
  for (int b = 0; b < 3; ++b) x[9 + b] = valid ? gr[5][b] * W.in_scale[9 + b] : 0.f;
  x[12] = valid ? Delta * W.in_scale[12] : 0.f;
  __syncthreads();
  mlp_tc_put_input<T>(sA, x);
  float y0, y1;
  mlp_tc_forward<HOOK, T>(W, sA, tcs, y0, y1);
  if (valid) {
    nut = W.out_scale[0] * fmaxf(y0, 0.f);
    Dt = W.out_scale[1] * fmaxf(y1, 0.f);
  }
}

// Shared memory of a gradient pass: the gradient fields of the element and
// its face neighbours (6 np32(N) + 36 (N+1)^2 floats), which the learned
// closure's A operand overwrites (T = np32(N) / 128 row tiles of kTcAElems
// BF16 elements).  Static up to N = 4; with the learned closure above it
// (40 to 80 KB) dynamic, 128 bytes more for the alignment of the operand.
__host__ __device__ constexpr int grad32_ubytes(int N, int CL) {
  return (CL == 2 && (np32(N) + 127) / 128 * kTcAElems * 2 > (6 * np32(N) + 36 * (N + 1) * (N + 1)) * 4)
             ? (np32(N) + 127) / 128 * kTcAElems * 2
             : (6 * np32(N) + 36 * (N + 1) * (N + 1)) * 4;
}
__host__ __device__ constexpr int grad32_dyn_bytes(int N, int CL) {
  return CL == 2 && N > 4 ? grad32_ubytes(N, CL) + 128 : 0;
}
__device__ __forceinline__ uint8_t *align128(uint8_t *p) {
  return reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(p) + 127) & ~(uintptr_t)127);
}

// Eddy viscosity and diffusivity of the algebraic closures from the
// gradients gr[v][m] (v: u, v, w, h', q', theta_v; m: x, y, z).  CL 1:
// Smagorinsky-Lilly, nu_t = (C_s Delta)^2 |S| with |S| = sqrt(2 S_ij S_ij)
// (Eq. smago); CL 3: Vreman (Eq. vreman-sgs).  With the Richardson
// correction (Eq. richardson) nu_t is scaled by (1 - Ri/Pr_t)^(1/4) for
// Ri = g (d theta_v/dz) / (theta_v |S|^2) > 0, and 0 beyond Ri = Pr_t.
// D_t = nu_t / Pr_t.
template <int CL>
__device__ __forceinline__ void eddy_nu(const float (&gr)[6][3], float CsDelta2, float thv, const KF &F,
                                        int richardson, float &nut, float &Dt) {
  float S2 = 0.f;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const float Sab = 0.5f * (gr[a][b] + gr[b][a]);
      S2 += Sab * Sab;
    }
  const float Smag2 = 2.0f * S2;
  if (CL == 1)
    nut = Smag2 > 0.0f ? CsDelta2 * sqrtf(Smag2) : 0.0f;
  else
    nut = vreman_nu<float>(gr, F.vr_c, F.vr_d2);
  if (richardson && Smag2 > 0.0f) {
    const float Ri = fdiv(F.g * gr[5][2], thv * Smag2);
    if (Ri > 0.0f) {
      const float a = 1.0f - Ri * F.inv_Prt;
      nut *= a > 0.0f ? sqrtf(sqrtf(a)) : 0.0f;
    }
  }
  Dt = nut * F.inv_Prt;
}

// The diffusive flux F2 of node t (Eqs. stress_tensor, diff_moisture_flux,
// diff_energy_flux; in deviation form) along x, y and z: -rho D_t dq/dx_d for the water, the subgrid stress
// tau_dj = -2 rho nu_t S_dj plus the water's momentum, and the energy's
// -rho D_t dh/dx_d + tau_dj u_j.  Planes d * 5 + c of the element's 15, np
// padded nodes each.
__device__ __forceinline__ void write_f2(float *__restrict__ F2, size_t e, int t, float rho, float nut, float Dt,
                                         const float (&gr)[6][3], const float (&sv)[6], const float (&G)[6],
                                         int np = kNP) {
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const float di = -Dt * gr[4][d];
    float rt[3];
#pragma unroll
    for (int b = 0; b < 3; ++b) rt[b] = -2.0f * rho * nut * (0.5f * (gr[d][b] + gr[b][d]));
    float *o = F2 + (e * 15 + d * 5) * np + t;
    o[0] = rho * di;
    o[1 * np] = rt[0] + di * sv[1];
    o[2 * np] = rt[1] + di * sv[2];
    o[3 * np] = rt[2] + di * sv[3];
    o[4 * np] = -rho * Dt * gr[3][d] + (rt[0] * G[0] + rt[1] * G[1] + rt[2] * G[2]);
  }
}

// The gradient pass's fields (u, v, w, h', q', theta_v') at node nn of
// element nb, formed from its state and thermodynamic planes exactly as for
// an own node; rho_r and q_r are the reference values at that node's height.
// In two steps, so that a thread can have the loads of two face nodes in
// flight: face_load gathers the seven values (rho', rho u, rho v, rho w,
// rho q_t', h', theta_v'), face_finish forms the fields.
__device__ __forceinline__ void face_load(const float *__restrict__ S, const float *__restrict__ TH, size_t nb, int nn,
                                          float (&raw)[7], int np = kNP) {
#pragma unroll
  for (int v = 0; v < 4; ++v) raw[v] = S[(nb * 6 + v) * np + nn];
  raw[4] = S[(nb * 6 + 5) * np + nn];
  raw[5] = TH[(nb * 4 + 2) * np + nn];
  raw[6] = TH[(nb * 4 + 3) * np + nn];
}
__device__ __forceinline__ void face_finish(const float (&raw)[7], float rho_r, float q_r, float (&gf)[6]) {
  const float rinv = fdiv(1.0f, rho_r + raw[0]);
  gf[0] = raw[1] * rinv;
  gf[1] = raw[2] * rinv;
  gf[2] = raw[3] * rinv;
  gf[3] = raw[5];
  gf[4] = (raw[4] - q_r * raw[0]) * rinv;
  gf[5] = raw[6];
}
__device__ __forceinline__ void face_primitives(const float *__restrict__ S, const float *__restrict__ TH, size_t nb,
                                                int nn, float rho_r, float q_r, float (&gf)[6], int np = kNP) {
  float raw[7];
  face_load(S, TH, nb, nn, raw, np);
  face_finish(raw, rho_r, q_r, gf);
}

// Sources of the momentum equations (Sec. 2, momentum balance): buoyancy of
// the density deviation, the sponge's relaxation toward u_relax at rate tau
// (Eq. sponge), and the Coriolis force -2 Omega x (rho u).
__device__ __forceinline__ void momentum_sources(const float (&sv)[6], float rho, float tau, const KF &F,
                                                 float (&R)[6]) {
  float Sr[3];
  Sr[0] = -tau * (sv[1] - rho * F.u_relax[0]);
  Sr[1] = -tau * (sv[2] - rho * F.u_relax[1]);
  Sr[2] = -sv[0] * F.g - tau * (sv[3] - rho * F.u_relax[2]);
  Sr[0] -= 2.0f * (F.Omega[1] * sv[3] - F.Omega[2] * sv[2]);
  Sr[1] -= 2.0f * (F.Omega[2] * sv[1] - F.Omega[0] * sv[3]);
  Sr[2] -= 2.0f * (F.Omega[0] * sv[2] - F.Omega[1] * sv[1]);
  R[1] += Sr[0];
  R[2] += Sr[1];
  R[3] += Sr[2];
}

// The update inputs of node t, loaded early so that their latency overlaps
// the flux computation: the register dQ and the step's increment D (none in
// the first stage, A = 0), and in the last stage the FP64 state.  Np: nodes
// per element of the FP64 state, np: padded nodes per element of the FP32
// arrays.
template <int UPD>
__device__ __forceinline__ void stage_inputs(const KParams &P, const StageCoef &sc, const float *__restrict__ dQ,
                                             const double *__restrict__ Q64, size_t e, int t, int Np, float (&dq0)[6],
                                             float (&D0)[6], double (&q0)[6], int np = kNP) {
#pragma unroll
  for (int v = 0; v < 6; ++v) {
    const size_t i32 = (e * 6 + v) * np + t;
    dq0[v] = sc.first ? 0.f : dQ[i32];
    D0[v] = sc.first ? 0.f : P.D32[i32];
    if (UPD == 2) q0[v] = Q64[(e * 6 + v) * Np + t];
  }
}

// The end of the flux pass at node t (Sec. 3.2, low-storage Runge-Kutta):
// UPD 0 writes the tendency R in FP64; UPD 1 forms dQ = A dQ + dt R, adds
// B dQ to the step's FP32 increment D and to the shadow; UPD 2 (last stage)
// adds D + B dQ to the FP64 state and writes the shadow anew from it, relative
// to the reference values qr[0], qr[qs], qr[2 qs] (rho, rho e, rho q_t).  sn:
// the new shadow node, whose thermodynamics the caller stores.
template <int UPD>
__device__ __forceinline__ void stage_update(const KParams &P, const StageCoef &sc, const float (&R)[6],
                                             const float (&dq0)[6], const float (&D0)[6], const double (&q0)[6],
                                             const float (&s_old)[6], const double *qr, int qs, float *__restrict__ dQ,
                                             double *__restrict__ Q64, float *__restrict__ Sout,
                                             double *__restrict__ Rout, size_t e, int t, int Np, float (&sn)[6],
                                             int np = kNP) {
#pragma unroll
  for (int v = 0; v < 6; ++v) {
    const size_t i64 = (e * 6 + v) * Np + t;
    if (UPD) {
      const size_t i32 = (e * 6 + v) * np + t;
      const float dq = sc.Af * dq0[v] + sc.dtf * R[v];
      const float Bdq = sc.Bf * dq;
      if (UPD == 1) {
        dQ[i32] = dq;
        P.D32[i32] = D0[v] + Bdq;
        sn[v] = s_old[v] + Bdq;
      } else {
        // the register is not read again before the next step's first stage
        const double qn = q0[v] + (double)(D0[v] + Bdq);
        Q64[i64] = qn;
        const double ref = v == 0 ? qr[0] : (v == 4 ? qr[qs] : (v == 5 ? qr[2 * qs] : 0.0));
        sn[v] = (float)(qn - ref);
      }
      Sout[i32] = sn[v];
    } else {
      Rout[i64] = (double)R[v];
    }
  }
}

}  // namespace cmles
