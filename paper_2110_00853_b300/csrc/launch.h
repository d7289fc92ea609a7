// Host-side launchers of the cmles kernels (internal to the library).
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "common.cuh"

namespace cmles {

// persistent grid: the resident CTAs per SM of fn (threads per CTA, dynamic
// shared memory smem) times the SMs, at most E
int grid_for(const void *fn, int E, size_t smem, int threads = 128);
int grid_for_tc(const void *fn, int E, int tmem_cols, int threads = 128, size_t dyn_smem = 0);

// FP64 path (dg_fp64.cu).  TH: the state's thermodynamic fields (p - p_r, c,
// h_tot, theta_v; four planes per element), written with the state (the flux
// pass with update for Qout, launch_thermo64 otherwise) and read by the next
// two passes.
cudaError_t launch_thermo64(const double *Q, double *TH, const KParams &P, int N, cudaStream_t s);
cudaError_t launch_grad64(const double *Q, const double *TH, double *F2, const KParams &P, cudaStream_t s);
cudaError_t launch_rhs64(const double *Q, const double *F2, const double *TH, double *dQ, double *Qout,
                         double *THout, const StageCoef &sc, bool update, const KParams &P, cudaStream_t s);

// FP32 path with FP64 accumulation (dg_fp32.cu); FP32 arrays padded to 128
// nodes.  TH: the state's thermodynamic fields (p', c, h', theta_v'; four
// planes per element), written with the state (shadow kernel, or the flux
// pass for the state it advances to) and read by the next two passes.
// launch_shadow32[c] with Q64 null writes only TH for the given shadow S.
cudaError_t launch_shadow32(const double *Q64, float *S, float *TH, const KParams &P, int N, cudaStream_t s);
cudaError_t launch_grad32(const float *S, const float *TH, float *F2, const KParams &P, cudaStream_t s);
cudaError_t launch_rhs32(const float *S, const float *F2, const float *TH, float *dQ, double *Q64, float *Sout,
                         float *THout, double *Rout, const StageCoef &sc, bool update, const KParams &P,
                         cudaStream_t s);

// FP32 path on curvilinear (warped) meshes (dg_curved32.cu)
// per-node table of a warped mesh: fields per node (kCurvedNF), and the slots
// of the per-element filter width Delta, (C_s Delta)^2 and Vreman's squared
// directional lengths (three slots)
enum { kCurvedNF = 27, kCurvedDelta = 22, kCurvedCsd2 = 23, kCurvedVr = 24 };
cudaError_t launch_shadow32c(const double *Q64, float *S, float *TH, const KParams &P, int N, cudaStream_t s);
cudaError_t launch_grad32c(const float *S, const float *TH, float *F2, const KParams &P, cudaStream_t s);
cudaError_t launch_rhs32c(const float *S, const float *F2, const float *TH, float *dQ, double *Q64, float *Sout,
                          float *THout, double *Rout, const StageCoef &sc, bool update, const KParams &P,
                          cudaStream_t s);

// Exponential modal filter (expfilter.cu): F is the 1D filter matrix
// (row-major (N+1)^2), mask selects momentum components (bits 1..3); S32,
// when not null, is the FP32 shadow to rewrite for the filtered variables.
struct ExpFilter {
  double F[kMaxQ * kMaxQ];
  int mask;
};
cudaError_t launch_expfilter(double *Q, float *S32, const ExpFilter &F, int N, int E, cudaStream_t s);

// HEVI (hevi.cu): the vertical linear operator's element blocks and the
// factors of I - dt gamma L, built on the host, used by the line kernels.
struct HeviTables {
  const double *tab;  // [nez][513]: L's diagonal and face blocks, G and E's columns (hevi.cu)
  const double *lev;  // [nez (N+1)][4]: rho_r, rho e_r, c_r, unused
  double lift, dtg;   // 2 / (h_z w_0), dt gamma
};
struct HeviSetup {
  int N, nez;
  double hz, w[kMaxQ], D[kMaxQ * kMaxQ];
  const double *rho_r, *p_r, *qt_r, *z;  // per level node (nez (N+1)); qt_r may be null (0)
  double g, Rd, Rv, cvd, cvv, T0, Iv0, dtg;
};
struct HeviHost {
  std::vector<double> Lb, Gf, Ef, lev;  // full blocks of L, G and E; level values
  std::vector<double> tab;              // the kernels' packed per-level table
  double lift = 0.0;
};
bool hevi_build(const HeviSetup &S, HeviHost &H);
cudaError_t launch_hevi_apply(const double *Q, double *out, const HeviTables &T, const KParams &P, cudaStream_t s);
cudaError_t launch_hevi_solve(const double *B, double *Y, const HeviTables &T, const KParams &P, cudaStream_t s);
// out = Q + dt sum_k c[k] X[k], k < n <= 4, over count doubles
struct LinComb {
  int n;
  double dt, c[4];
  const double *X[4];
};
cudaError_t launch_lincomb(double *out, const double *Q, const LinComb &lc, long long count, cudaStream_t s);

// Learned closure network (mlp.cu)
struct MlpPacked;
void pack_mlp_host(const float *params, MlpPacked *out);
cudaError_t launch_pack_mlp(const float *params_dev, MlpPacked *out, cudaStream_t s);

// Closure training samples from a fine run (filter.cu)
cudaError_t launch_closure_samples(const double *Q, const KParams &P, int N, const double *xi, const double *w,
                                   const double *D, int factor, const int periodic[3], float *X, float *T,
                                   float *thv, long long ncoarse, cudaStream_t s);

// Diagnostics and set-up (aux_kernels.cu)
// Budgets: partial sums per block into partials[nblocks][7] (6 integrals and a
// non-finite count), then a single-block pass in fixed order into out[7].
int budget_blocks(long long nodes);
// wJn: optional per-node w_n J_n (curvilinear meshes); otherwise wq[n] * J.
// pnex > 0: Q is a partition's storage (pnex x pney interior columns with a
// ghost element on each side in x and y), summed over the interior.
cudaError_t launch_budgets(const double *Q, long long E, int Np, const double *wq, double J, double *partials,
                           int nblocks, double *out, cudaStream_t s, const double *wJn = nullptr, int pnex = 0,
                           int pney = 0);

struct CaseDev {
  int id;
  unsigned long long seed;
  double dtheta, r0, xc, yc, zc, noise_theta, noise_qt, noise_zmax;
  double u0[3];
  int moist;
  int nmodes;
  const double *modes;  // device
  const double *theta_lev, *qt_lev, *pref_lev;  // per level background theta, q_t and pressure
};
cudaError_t launch_init_state(double *Q, const CaseDev &c, const KParams &P, int N, cudaStream_t s);

// Favre profiles: accum[level][12] of quadrature-weighted horizontal sums.
cudaError_t launch_profiles(const double *Q, const KParams &P, int N, double *accum, int pass, cudaStream_t s);

}  // namespace cmles
