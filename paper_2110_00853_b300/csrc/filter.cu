// Training samples for the learned SGS closure from a fine-resolution run.
//
// The paper has no learned closure; these are the targets of its extension,
// a 4x box filter: the fine field is averaged with a top-hat of width
// Delta_c = H_c / N (the coarse node spacing, 4 fine node spacings for a
// factor-4 coarsening) centred on every node of the coarse mesh, using the
// fine LGL quadrature weights.  From the filtered moments
//   tau_ij  = <u_i u_j> - <u_i><u_j>,   tau_thj = <u_j th> - <u_j><th>,
//   S_ij    = (<d_j u_i> + <d_i u_j>)/2,   g_j = <d_j th>   (th = theta_v),
// the least-squares eddy viscosity and diffusivity are
//   nu* = max(0, -tau:S / (2 S:S)),   kappa* = max(0, -tau_th.g / |g|^2),
// and the network inputs are the filtered velocity gradients (9), the
// filtered theta_v gradient (3) and Delta_c.  Fine-node derivatives are the
// element-local LGL derivatives (the BR1 face term is left out here).  Fine
// nodes on a shared face count once per element; a node within 1e-9
// (relative) of the box edge counts as inside.  The primitive fields are kept
// in FP64 (scratch memory of the call): the subgrid moments are small
// differences of large ones (<u u> - <u><u>), which FP32 inputs would leave
// with only a few correct digits.
#include <math.h>
#include <string.h>

#include "cmles.h"
#include "common.cuh"
#include "launch.h"
#include "thermo.cuh"

namespace cmles {

// u, v, w, theta_v at every fine node (FP64 thermodynamics), [E][4][Np].
template <bool MOIST>
__global__ void k_primitives(const double *__restrict__ Q, double *__restrict__ prim, const KParams P, int N) {
  const int Nq = N + 1, Np = Nq * Nq * Nq;
  const long long nodes = (long long)P.E * Np;
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < nodes;
       g += (long long)gridDim.x * blockDim.x) {
    const long long e = g / Np;
    const int n = (int)(g - e * Np);
    const int k = n / (Nq * Nq);
    const int ez = (int)(e / ((long long)P.nex * P.ney));
    double Y[6];
    for (int v = 0; v < 6; ++v) Y[v] = Q[(e * 6 + v) * Np + n];
    Th64 s;
    int fail = 0;
    thermo64<MOIST>(P, Y, node_z(P, ez, k), ez * Nq + k, s, fail);
    double *o = prim + e * 4 * Np + n;
    o[0] = s.u[0];
    o[Np] = s.u[1];
    o[2 * Np] = s.u[2];
    o[3 * Np] = s.thv;
  }
}

struct FilterGeom {
  int nex, ney, nez, factor, N, periodic[3];
  double x0, y0, z0, h[3];
  double xi[kMaxQ], w[kMaxQ], D[kMaxQ * kMaxQ];
  double Delta_c;
};

__global__ void k_filter_samples(const double *__restrict__ prim, const FilterGeom G, float *__restrict__ X,
                                 float *__restrict__ T, float *__restrict__ thv, long long ncoarse) {
  const int N = G.N, Nq = N + 1, Np = Nq * Nq * Nq;
  const int cnx = G.nex / G.factor, cny = G.ney / G.factor;
  const int nel[3] = {G.nex, G.ney, G.nez};
  const double org[3] = {G.x0, G.y0, G.z0};
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < ncoarse;
       q += (long long)gridDim.x * blockDim.x) {
    const long long ce = q / Np;
    const int n = (int)(q - ce * Np);
    const int cidx[3] = {(int)(ce % cnx), (int)((ce / cnx) % cny), (int)(ce / ((long long)cnx * cny))};
    const int nidx[3] = {n % Nq, (n / Nq) % Nq, n / (Nq * Nq)};
    double xc[3], b[3];
    int lo[3], hi[3];
    for (int d = 0; d < 3; ++d) {
      const double H = G.factor * G.h[d];
      xc[d] = org[d] + (cidx[d] + 0.5 * (G.xi[nidx[d]] + 1.0)) * H;
      b[d] = 0.5 * H / N * (1.0 + 1e-9);
      lo[d] = (int)floor((xc[d] - b[d] - org[d]) / G.h[d]);
      hi[d] = (int)floor((xc[d] + b[d] - org[d]) / G.h[d]);
      if (!G.periodic[d]) {
        lo[d] = max(lo[d], 0);
        hi[d] = min(hi[d], nel[d] - 1);
      }
    }
    double W = 0, su[3] = {0, 0, 0}, suu[6] = {0, 0, 0, 0, 0, 0}, sth = 0, suth[3] = {0, 0, 0};
    double sdu[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, sdth[3] = {0, 0, 0};
    for (int fz = lo[2]; fz <= hi[2]; ++fz)
      for (int fy = lo[1]; fy <= hi[1]; ++fy)
        for (int fx = lo[0]; fx <= hi[0]; ++fx) {
          const int f[3] = {fx, fy, fz};
          int fw[3];
          for (int d = 0; d < 3; ++d) fw[d] = ((f[d] % nel[d]) + nel[d]) % nel[d];
          const long long fe = fw[0] + (long long)G.nex * (fw[1] + (long long)G.ney * fw[2]);
          const double *pe = prim + fe * 4 * Np;
          for (int c = 0; c < Nq; ++c)
            for (int bb = 0; bb < Nq; ++bb)
              for (int a = 0; a < Nq; ++a) {
                const int ab[3] = {a, bb, c};
                bool in = true;
                for (int d = 0; d < 3; ++d) {
                  const double xf = org[d] + (f[d] + 0.5 * (G.xi[ab[d]] + 1.0)) * G.h[d];
                  if (fabs(xf - xc[d]) > b[d]) in = false;
                }
                if (!in) continue;
                const int node = a + Nq * (bb + Nq * c);
                const double w = G.w[a] * G.w[bb] * G.w[c];
                double val[4];
                for (int v = 0; v < 4; ++v) val[v] = pe[v * Np + node];
                // element-local derivatives of u, v, w, theta_v
                double dv[4][3];
                for (int v = 0; v < 4; ++v)
                  for (int d = 0; d < 3; ++d) {
                    double acc = 0.0;
                    for (int m = 0; m < Nq; ++m) {
                      int t3[3] = {a, bb, c};
                      t3[d] = m;
                      acc += G.D[ab[d] * Nq + m] * pe[v * Np + t3[0] + Nq * (t3[1] + Nq * t3[2])];
                    }
                    dv[v][d] = 2.0 / G.h[d] * acc;
                  }
                W += w;
                for (int i = 0; i < 3; ++i) {
                  su[i] += w * val[i];
                  suth[i] += w * val[i] * val[3];
                  sdth[i] += w * dv[3][i];
                  for (int j = 0; j < 3; ++j) sdu[3 * i + j] += w * dv[i][j];
                }
                suu[0] += w * val[0] * val[0];
                suu[1] += w * val[1] * val[1];
                suu[2] += w * val[2] * val[2];
                suu[3] += w * val[0] * val[1];
                suu[4] += w * val[0] * val[2];
                suu[5] += w * val[1] * val[2];
                sth += w * val[3];
              }
        }
    const double iW = 1.0 / W;
    double ub[3], tau[3][3], S[3][3], gth[3], gu[9];
    for (int i = 0; i < 3; ++i) ub[i] = su[i] * iW;
    const int pi[6] = {0, 1, 2, 0, 0, 1}, pj[6] = {0, 1, 2, 1, 2, 2};
    for (int p = 0; p < 6; ++p) {
      const double t = suu[p] * iW - ub[pi[p]] * ub[pj[p]];
      tau[pi[p]][pj[p]] = tau[pj[p]][pi[p]] = t;
    }
    for (int k = 0; k < 9; ++k) gu[k] = sdu[k] * iW;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) S[i][j] = 0.5 * (gu[3 * i + j] + gu[3 * j + i]);
    double tS = 0, SS = 0, tg = 0, gg = 0;
    const double thb = sth * iW;
    for (int i = 0; i < 3; ++i) {
      gth[i] = sdth[i] * iW;
      const double tth = suth[i] * iW - ub[i] * thb;
      tg += tth * gth[i];
      gg += gth[i] * gth[i];
      for (int j = 0; j < 3; ++j) {
        tS += tau[i][j] * S[i][j];
        SS += S[i][j] * S[i][j];
      }
    }
    const double nu = SS > 0.0 ? fmax(0.0, -tS / (2.0 * SS)) : 0.0;
    const double ka = gg > 0.0 ? fmax(0.0, -tg / gg) : 0.0;
    float *x = X + q * 13;
    for (int k = 0; k < 9; ++k) x[k] = (float)gu[k];
    for (int k = 0; k < 3; ++k) x[9 + k] = (float)gth[k];
    x[12] = (float)G.Delta_c;
    T[q * 2] = (float)nu;
    T[q * 2 + 1] = (float)ka;
    if (thv) thv[q] = (float)thb;
  }
}

cudaError_t launch_closure_samples(const double *Q, const KParams &P, int N, const double *xi, const double *w,
                                   const double *D, int factor, const int periodic[3], float *X, float *T,
                                   float *thv, long long ncoarse, cudaStream_t s) {
  const int Nq = N + 1, Np = Nq * Nq * Nq;
  double *prim = nullptr;
  cudaError_t e = cudaMallocAsync((void **)&prim, (size_t)P.E * 4 * Np * sizeof(double), s);
  if (e != cudaSuccess) return e;
  const long long nodes = (long long)P.E * Np;
  int blocks = (int)((nodes + 255) / 256);
  if (blocks > 148 * 32) blocks = 148 * 32;
  if (P.moist)
    k_primitives<true><<<blocks, 256, 0, s>>>(Q, prim, P, N);
  else
    k_primitives<false><<<blocks, 256, 0, s>>>(Q, prim, P, N);
  FilterGeom G;
  memset(&G, 0, sizeof(G));
  G.nex = P.nex;
  G.ney = P.ney;
  G.nez = P.nez;
  G.factor = factor;
  G.N = N;
  for (int d = 0; d < 3; ++d) G.periodic[d] = periodic[d];
  G.x0 = P.x0;
  G.y0 = P.y0;
  G.z0 = P.z0;
  G.h[0] = P.hx;
  G.h[1] = P.hy;
  G.h[2] = P.hz;
  for (int a = 0; a < Nq; ++a) {
    G.xi[a] = xi[a];
    G.w[a] = w[a];
    for (int b = 0; b < Nq; ++b) G.D[a * Nq + b] = D[a * Nq + b];
  }
  G.Delta_c = cbrt(factor * P.hx * factor * P.hy * factor * P.hz) / N;
  int cb = (int)((ncoarse + 127) / 128);
  if (cb > 148 * 16) cb = 148 * 16;
  k_filter_samples<<<cb, 128, 0, s>>>(prim, G, X, T, thv, ncoarse);
  e = cudaGetLastError();
  cudaFreeAsync(prim, s);
  return e;
}

}  // namespace cmles
