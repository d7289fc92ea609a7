// Set-up and diagnostic kernels of the cmles CUDA path: FP64 domain budgets
// (the integrals of Sec. 6), Favre horizontal means (App. C) and the
// synthetic initial states.
#include <math.h>

#include "common.cuh"
#include "launch.h"
#include "thermo.cuh"

namespace cmles {

// ------------------------------------------------------------------ budgets

constexpr int kBudgetThreads = 256;

int budget_blocks(long long nodes) {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  long long want = (nodes + kBudgetThreads - 1) / kBudgetThreads;
  long long cap = (long long)nsm * 8;
  return (int)(want < cap ? (want < 1 ? 1 : want) : cap);
}

// Quadrature sums sum_e sum_n w_n J Q_v with LGL weights w_n = w_i w_j w_k
// and the constant element Jacobian J of a flat mesh, plus a count of
// non-finite entries.  Fixed grid and fixed reduction order: deterministic.
// On a partition (pnex > 0) the E = pnex x pney x nez elements are the
// interior of a storage block with one ghost element on each side in x and y.
__global__ void __launch_bounds__(kBudgetThreads) k_budget_partial(const double *__restrict__ Q, long long E,
                                                                   int Np, const double *__restrict__ wq,
                                                                   double J, double *__restrict__ partials,
                                                                   const double *__restrict__ wJn, int pnex,
                                                                   int pney) {
  double acc[7] = {0, 0, 0, 0, 0, 0, 0};
  const long long nodes = E * Np;
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < nodes;
       g += (long long)gridDim.x * blockDim.x) {
    const long long ei = g / Np;
    const int n = (int)(g - ei * Np);
    long long e = ei;
    if (pnex > 0) {
      const long long ex = ei % pnex, ey = (ei / pnex) % pney, ez = ei / ((long long)pnex * pney);
      e = (ex + 1) + (pnex + 2) * ((ey + 1) + (long long)(pney + 2) * ez);
    }
    const double w = wJn ? wJn[g] : wq[n] * J;
#pragma unroll
    for (int v = 0; v < 6; ++v) {
      const double q = Q[(e * 6 + v) * Np + n];
      acc[v] += w * q;
      if (!isfinite(q)) acc[6] += 1.0;
    }
  }
  __shared__ double red[7][kBudgetThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int v = 0; v < 7; ++v) {
    double x = acc[v];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) red[v][warp] = x;
  }
  __syncthreads();
  if (threadIdx.x < 7) {
    double x = 0.0;
    for (int w = 0; w < kBudgetThreads / 32; ++w) x += red[threadIdx.x][w];
    partials[(size_t)blockIdx.x * 7 + threadIdx.x] = x;
  }
}

__global__ void k_budget_final(const double *__restrict__ partials, int nblocks, double *__restrict__ out) {
  if (threadIdx.x < 7) {
    double x = 0.0;
    for (int b = 0; b < nblocks; ++b) x += partials[(size_t)b * 7 + threadIdx.x];
    out[threadIdx.x] = x;
  }
}

cudaError_t launch_budgets(const double *Q, long long E, int Np, const double *wq, double J, double *partials,
                           int nblocks, double *out, cudaStream_t s, const double *wJn, int pnex, int pney) {
  k_budget_partial<<<nblocks, kBudgetThreads, 0, s>>>(Q, E, Np, wq, J, partials, wJn, pnex, pney);
  k_budget_final<<<1, 32, 0, s>>>(partials, nblocks, out);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ profiles

// pass 0: per level sums of w, w rho, w rho theta, w rho q_t, w rho q_l,
//         w rho u, w rho v, w rho w, w rho theta_l;
// pass 1: w rho w'^2, w rho w' theta', w rho w' q_t' with the pass-0 means
//         (accum[level][9..11] read back from the finished pass 0).
template <bool MOIST>
__global__ void k_profiles(const double *__restrict__ Q, const KParams P, int N, double *__restrict__ accum,
                           int pass) {
  const int Nq = N + 1, Np = Nq * Nq * Nq;
  const long long nodes = (long long)P.E * Np;
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < nodes;
       g += (long long)gridDim.x * blockDim.x) {
    const long long e = g / Np;
    const int n = (int)(g - e * Np);
    const int i = n % Nq, j = (n / Nq) % Nq, k = n / (Nq * Nq);
    const int ez = (int)(e / ((long long)P.nex * P.ney));
    const int lev = ez * Nq + k;
    double Y[6];
    for (int v = 0; v < 6; ++v) Y[v] = Q[(e * 6 + v) * Np + n];
    Th64 s;
    int fail = 0;
    thermo64<MOIST>(P, Y, node_z(P, ez, k), ez * Nq + k, s, fail);
    const double th = s.thv * P.Rd / (P.Rd * (1.0 - s.q) + P.Rv * (s.q - s.ql));
    const double w = P.w[i] * P.w[j];
    double *a = accum + (size_t)lev * 12;
    if (pass == 0) {
      const double thl = th * (1.0 - P.Lv0 * s.ql / (P.cpd * s.T));
      atomicAdd(a + 0, w);
      atomicAdd(a + 1, w * Y[0]);
      atomicAdd(a + 2, w * Y[0] * th);
      atomicAdd(a + 3, w * Y[5]);
      atomicAdd(a + 4, w * Y[0] * s.ql);
      atomicAdd(a + 5, w * Y[1]);
      atomicAdd(a + 6, w * Y[2]);
      atomicAdd(a + 7, w * Y[3]);
      atomicAdd(a + 8, w * Y[0] * thl);
    } else {
      const double wbar = a[7] / a[1], thbar = a[2] / a[1], qbar = a[3] / a[1];
      const double wp = s.u[2] - wbar;
      atomicAdd(a + 9, w * Y[0] * wp * wp);
      atomicAdd(a + 10, w * Y[0] * wp * (th - thbar));
      atomicAdd(a + 11, w * Y[0] * wp * (s.q - qbar));
    }
  }
}

cudaError_t launch_profiles(const double *Q, const KParams &P, int N, double *accum, int pass, cudaStream_t s) {
  long long nodes = (long long)P.E * (N + 1) * (N + 1) * (N + 1);
  int blocks = (int)((nodes + 255) / 256);
  if (blocks > 148 * 16) blocks = 148 * 16;
  if (P.moist)
    k_profiles<true><<<blocks, 256, 0, s>>>(Q, P, N, accum, pass);
  else
    k_profiles<false><<<blocks, 256, 0, s>>>(Q, P, N, accum, pass);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ initial states

// SplitMix64 (Steele, Lea & Flood 2014), output number `counter` of the
// stream seeded with `seed`, mapped to a double in [0, 1) from its top 53 bits.
__device__ __forceinline__ double splitmix_uniform(unsigned long long seed, unsigned long long counter) {
  unsigned long long z = seed + (counter + 1ULL) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  z ^= z >> 31;
  return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

// One thread per node: background theta, q_t and hydrostatic pressure of the
// node level, perturbations of the case (bubble, random-phase velocity sum with FP32
// cosines and FP64 accumulation, seeded noise), then T = theta (p/p0)^kappa, rho = p/(R_m T) with
// q_l = 0, rho e = rho (I + |u|^2/2 + g z).
__global__ void k_init_state(double *__restrict__ Q, const CaseDev c, const KParams P, int N) {
  const int Nq = N + 1, Np = Nq * Nq * Nq;
  const long long nodes = (long long)P.E * Np;
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < nodes;
       g += (long long)gridDim.x * blockDim.x) {
    const long long e = g / Np;
    const int n = (int)(g - e * Np);
    const int i = n % Nq, j = (n / Nq) % Nq, k = n / (Nq * Nq);
    const int ex = (int)(e % P.nex), ey = (int)((e / P.nex) % P.ney), ez = (int)(e / ((long long)P.nex * P.ney));
    const double x = P.x0 + (ex + 0.5 * (P.xi[i] + 1.0)) * P.hx;
    const double y = P.y0 + (ey + 0.5 * (P.xi[j] + 1.0)) * P.hy;
    const double z = node_z(P, ez, k);
    const int lev = ez * Nq + k;
    double th = c.theta_lev[lev], qt = c.qt_lev[lev];
    const double p = c.pref_lev[lev];
    double u[3] = {c.u0[0], c.u0[1], c.u0[2]};
    if (c.id == 1) {
      const double dx = x - c.xc, dy = y - c.yc, dz = z - c.zc;
      const double r = sqrt(dx * dx + dy * dy + dz * dz);
      if (r <= c.r0) {
        const double cs = cos(M_PI * r / (2.0 * c.r0));
        th += c.dtheta * cs * cs;
      }
    }
    if (c.id == 11) {  // density current: theta_c/2 (1 + cos(pi r)), r <= 1
      const double ax = (x - c.xc) / c.r0, az = (z - c.zc) / (0.5 * c.r0);
      const double r = sqrt(ax * ax + az * az);
      if (r <= 1.0) th += 0.5 * c.dtheta * (1.0 + cos(M_PI * r));
    }
    if (c.nmodes > 0) {
      double su = 0.0, sv = 0.0, sw = 0.0;
      for (int m = 0; m < c.nmodes; ++m) {
        const double *md = c.modes + (size_t)m * 7;
        // phase reduced to [-pi, pi] in FP64 before the FP32 cosine
        const double ph64 = md[0] * x + md[1] * y + md[2] * z + md[6];
        const float ph = (float)(ph64 - 6.283185307179586 * rint(ph64 * 0.15915494309189535));
        const float cs = cosf(ph);
        su += md[3] * cs;
        sv += md[4] * cs;
        sw += md[5] * cs;
      }
      u[0] += su;
      u[1] += sv;
      u[2] += sw;
    }
    if (z <= c.noise_zmax) {
      th += c.noise_theta * (2.0 * splitmix_uniform(c.seed, 4ULL * g + 0) - 1.0);
      if (c.moist) qt += c.noise_qt * (2.0 * splitmix_uniform(c.seed, 4ULL * g + 1) - 1.0);
    }
    const double T = th * exp(P.kappa * log(p / P.p0));
    const double Rm = P.Rd * (1.0 - qt) + P.Rv * qt;
    const double rho = p / (Rm * T);
    const double I = (1.0 - qt) * P.cvd * (T - P.T0) + qt * (P.cvv * (T - P.T0) + P.Iv0);
    const double ke = 0.5 * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    double *q = Q + (size_t)e * 6 * Np + n;
    q[0] = rho;
    q[1 * Np] = rho * u[0];
    q[2 * Np] = rho * u[1];
    q[3 * Np] = rho * u[2];
    q[4 * Np] = rho * (I + ke + P.g * z);
    q[5 * Np] = rho * qt;
  }
}

cudaError_t launch_init_state(double *Q, const CaseDev &c, const KParams &P, int N, cudaStream_t s) {
  long long nodes = (long long)P.E * (N + 1) * (N + 1) * (N + 1);
  int blocks = (int)((nodes + 255) / 256);
  if (blocks > 148 * 32) blocks = 148 * 32;
  k_init_state<<<blocks, 256, 0, s>>>(Q, c, P, N);
  return cudaGetLastError();
}

}  // namespace cmles
