// HEVI time stepping (Sec. 3.2: horizontally explicit, vertically implicit;
// flat meshes, walls at the bottom and top).  The stages' tendencies come
// from the DG kernels of the handle's precision; the operator, the line
// solves and the stage combinations are FP64.
//
// The implicit part L is the vertical acoustic-gravity operator linearised
// about the hydrostatic reference (rho_r, p_r, total water q_r) and the rest
// state, with the equation of state of unsaturated air at rest and fixed
// q_r, linear in (rho, rho e): p = R_m T_0 rho + kappa_m (rho e - rho Phi - rho q_r I_v0),
// kappa_m = R_m / c_vm.  On the deviations y = (rho - rho_r, rho w, rho e - rho e_r),
//   L y = -d F(y)/dz + (0, -g rho', 0),  F = (rho w, a rho' + kappa_m (rho e)', h_r rho w),
//   a = R_m T_0 - kappa_m (Phi + q_r I_v0),  h_r = (rho e_r + p_r)/rho_r,
//   rho e_r = rho_r (c_vm (T_r - T_0) + q_r I_v0 + Phi),  T_r = p_r / (rho_r R_m),
// in strong-form nodal DG along z with a Rusanov flux at the reference sound
// speed c_r (walls mirror rho w); the horizontal momentum and rho q_t keep
// only that flux's dissipation on the z-faces.  The same operator holds on
// every vertical line, so its element blocks (3 (N+1) x 3 (N+1) for the three
// coupled unknowns at the N + 1 LGL levels of an element, 15 x 15 at N = 4)
// are assembled once on the host, and I - dt gamma L is factored there by block Gaussian elimination
// of the block-tridiagonal line matrix.  The kernels below apply L and solve
// with the factors, one thread per vertical line of nodes.
#include <math.h>

#include <utility>
#include <vector>

#include "common.cuh"
#include "launch.h"

namespace cmles {

// coupled unknowns per element on a line: N + 1 levels x (rho', rho w, rho e')
__host__ __device__ constexpr int hevi_hb(int N) { return 3 * (N + 1); }

template <int Nq>
__device__ __forceinline__ void hevi_line(const KParams &P, long long line, int &ex, int &ey, int &n0) {
  const int ij = (int)(line % (Nq * Nq));
  const long long col = line / (Nq * Nq);
  ex = (int)(col % P.nex);
  ey = (int)(col / P.nex);
  n0 = ij;  // i + Nq j: the line's node index at level k is n0 + Nq^2 k
}

// Per-level table layout (doubles), HB = hevi_hb(N): the diagonal block of L
// (HB x HB), the two face-coupling blocks of L (3 x 3: rows of the element's
// bottom level against the lower element's top level, rows of the top level
// against the upper element's bottom level; every other entry of L's
// off-diagonal blocks is zero), the inverse G of the elimination's diagonal
// block (HB x HB) and the three nonzero columns of the back-substitution
// block E = G C^M (HB x 3).  At N = 4: offsets 0, 225, 234, 243, 468, stride 513.
__host__ __device__ constexpr int hevi_tB(int) { return 0; }
__host__ __device__ constexpr int hevi_tA(int N) { return hevi_hb(N) * hevi_hb(N); }
__host__ __device__ constexpr int hevi_tC(int N) { return hevi_tA(N) + 9; }
__host__ __device__ constexpr int hevi_tG(int N) { return hevi_tC(N) + 9; }
__host__ __device__ constexpr int hevi_tE(int N) { return hevi_tG(N) + hevi_hb(N) * hevi_hb(N); }
__host__ __device__ constexpr int hevi_stride(int N) { return hevi_tE(N) + 3 * hevi_hb(N); }

// out = L (Q - Q_ref) on every vertical line (all six components).
template <int N>
__global__ void k_hevi_apply(const double *__restrict__ Q, double *__restrict__ out, const HeviTables T,
                             const KParams P) {
  constexpr int Nq = N + 1, Np = Nq * Nq * Nq, Nf = Nq * Nq, kHB = hevi_hb(N), kTB = hevi_tB(N),
                kTA = hevi_tA(N), kTC = hevi_tC(N), kTStride = hevi_stride(N), kTop = 3 * N;
  const long long nlines = (long long)P.nex * P.ney * Nf;
  const size_t slab = (size_t)P.nex * P.ney;
  for (long long line = blockIdx.x * (long long)blockDim.x + threadIdx.x; line < nlines;
       line += (long long)gridDim.x * blockDim.x) {
    int ex, ey, n0;
    hevi_line<Nq>(P, line, ex, ey, n0);
    const size_t e0 = (size_t)ex + (size_t)P.nex * ey;
    auto load = [&](int ez, double *y) {
      const size_t e = e0 + slab * ez;
#pragma unroll
      for (int k = 0; k < Nq; ++k) {
        const int n = n0 + Nf * k, lev = ez * Nq + k;
        y[3 * k + 0] = Q[(e * 6 + 0) * Np + n] - T.lev[4 * lev + 0];
        y[3 * k + 1] = Q[(e * 6 + 3) * Np + n];
        y[3 * k + 2] = Q[(e * 6 + 4) * Np + n] - T.lev[4 * lev + 1];
      }
    };
    double yc[kHB], yn[kHB], ytop_prev[3] = {0.0, 0.0, 0.0};
    load(0, yc);
    for (int ez = 0; ez < P.nez; ++ez) {
      if (ez + 1 < P.nez) load(ez + 1, yn);
      const double *Tz = T.tab + (size_t)ez * kTStride;
      double r[kHB];
#pragma unroll
      for (int a = 0; a < kHB; ++a) {
        double s = 0.0;
#pragma unroll
        for (int b = 0; b < kHB; ++b) s += Tz[kTB + a * kHB + b] * yc[b];
        r[a] = s;
      }
      if (ez > 0)
#pragma unroll
        for (int a = 0; a < 3; ++a)
          r[a] += Tz[kTA + 3 * a] * ytop_prev[0] + Tz[kTA + 3 * a + 1] * ytop_prev[1] + Tz[kTA + 3 * a + 2] * ytop_prev[2];
      if (ez + 1 < P.nez)
#pragma unroll
        for (int a = 0; a < 3; ++a)
          r[kTop + a] += Tz[kTC + 3 * a] * yn[0] + Tz[kTC + 3 * a + 1] * yn[1] + Tz[kTC + 3 * a + 2] * yn[2];
      const size_t e = e0 + slab * ez;
#pragma unroll
      for (int k = 0; k < Nq; ++k) {
        const int n = n0 + Nf * k;
        out[(e * 6 + 0) * Np + n] = r[3 * k + 0];
        out[(e * 6 + 3) * Np + n] = r[3 * k + 1];
        out[(e * 6 + 4) * Np + n] = r[3 * k + 2];
        // horizontal momentum and rho q_t: dissipation on the element's z-faces
        const int vs[3] = {1, 2, 5};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          double o = 0.0;
          const double q = Q[(e * 6 + vs[c]) * Np + n];
          if (k == Nq - 1 && ez + 1 < P.nez) {
            const size_t eu = e + slab;
            o = -T.lift * 0.5 * T.lev[4 * (ez * Nq + k) + 2] * (q - Q[(eu * 6 + vs[c]) * Np + n0]);
          } else if (k == 0 && ez > 0) {
            const size_t ed = e - slab;
            o = -T.lift * 0.5 * T.lev[4 * (ez * Nq + k) + 2] * (q - Q[(ed * 6 + vs[c]) * Np + n0 + Nf * (Nq - 1)]);
          }
          out[(e * 6 + vs[c]) * Np + n] = o;
        }
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) ytop_prev[c] = yc[kTop + c];
#pragma unroll
      for (int a = 0; a < kHB; ++a) yc[a] = yn[a];
    }
  }
}

// Y = Q_ref + (I - dt gamma L)^-1 (B - Q_ref) on every vertical line.
template <int N>
__global__ void k_hevi_solve(const double *__restrict__ Bv, double *__restrict__ Y, const HeviTables T,
                             const KParams P) {
  constexpr int Nq = N + 1, Np = Nq * Nq * Nq, Nf = Nq * Nq, kHB = hevi_hb(N), kTA = hevi_tA(N),
                kTG = hevi_tG(N), kTE = hevi_tE(N), kTStride = hevi_stride(N), kTop = 3 * N;
  const long long nlines = (long long)P.nex * P.ney * Nf;
  const size_t slab = (size_t)P.nex * P.ney;
  for (long long line = blockIdx.x * (long long)blockDim.x + threadIdx.x; line < nlines;
       line += (long long)gridDim.x * blockDim.x) {
    int ex, ey, n0;
    hevi_line<Nq>(P, line, ex, ey, n0);
    const size_t e0 = (size_t)ex + (size_t)P.nex * ey;
    // forward sweep of the block elimination: y_ez = G_ez (b_ez - A^M_ez y_ez-1)
    // with A^M = -dt gamma A^L (nonzero on the face levels only); y kept in Y
    // (as deviations) until the back sweep
    double ytop[3] = {0.0, 0.0, 0.0};
    for (int ez = 0; ez < P.nez; ++ez) {
      const size_t e = e0 + slab * ez;
      const double *Tz = T.tab + (size_t)ez * kTStride;
      double r[kHB];
#pragma unroll
      for (int k = 0; k < Nq; ++k) {
        const int n = n0 + Nf * k, lev = ez * Nq + k;
        r[3 * k + 0] = Bv[(e * 6 + 0) * Np + n] - T.lev[4 * lev + 0];
        r[3 * k + 1] = Bv[(e * 6 + 3) * Np + n];
        r[3 * k + 2] = Bv[(e * 6 + 4) * Np + n] - T.lev[4 * lev + 1];
      }
      if (ez > 0)
#pragma unroll
        for (int a = 0; a < 3; ++a)
          r[a] += T.dtg * (Tz[kTA + 3 * a] * ytop[0] + Tz[kTA + 3 * a + 1] * ytop[1] + Tz[kTA + 3 * a + 2] * ytop[2]);
      double y[kHB];
#pragma unroll
      for (int a = 0; a < kHB; ++a) {
        double s = 0.0;
#pragma unroll
        for (int b = 0; b < kHB; ++b) s += Tz[kTG + a * kHB + b] * r[b];
        y[a] = s;
      }
#pragma unroll
      for (int k = 0; k < Nq; ++k) {
        const int n = n0 + Nf * k;
        Y[(e * 6 + 0) * Np + n] = y[3 * k + 0];
        Y[(e * 6 + 3) * Np + n] = y[3 * k + 1];
        Y[(e * 6 + 4) * Np + n] = y[3 * k + 2];
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) ytop[c] = y[kTop + c];
    }
    // back sweep: x_ez = y_ez - E_ez x_ez+1 (E nonzero in the columns of the
    // upper element's bottom level), then Y = Q_ref + x
    double xbot[3] = {0.0, 0.0, 0.0};
    for (int ez = P.nez - 1; ez >= 0; --ez) {
      const size_t e = e0 + slab * ez;
      const double *Tz = T.tab + (size_t)ez * kTStride;
      double x[kHB];
#pragma unroll
      for (int k = 0; k < Nq; ++k) {
        const int n = n0 + Nf * k;
        x[3 * k + 0] = Y[(e * 6 + 0) * Np + n];
        x[3 * k + 1] = Y[(e * 6 + 3) * Np + n];
        x[3 * k + 2] = Y[(e * 6 + 4) * Np + n];
      }
      if (ez + 1 < P.nez)
#pragma unroll
        for (int a = 0; a < kHB; ++a)
          x[a] -= Tz[kTE + 3 * a] * xbot[0] + Tz[kTE + 3 * a + 1] * xbot[1] + Tz[kTE + 3 * a + 2] * xbot[2];
#pragma unroll
      for (int k = 0; k < Nq; ++k) {
        const int n = n0 + Nf * k, lev = ez * Nq + k;
        Y[(e * 6 + 0) * Np + n] = T.lev[4 * lev + 0] + x[3 * k + 0];
        Y[(e * 6 + 3) * Np + n] = x[3 * k + 1];
        Y[(e * 6 + 4) * Np + n] = T.lev[4 * lev + 1] + x[3 * k + 2];
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) xbot[c] = x[c];
    }
    // horizontal momentum and rho q_t: each z-face couples only its two face
    // nodes, (1 + a) q_t - a q_b = b_t and -a q_t + (1 + a) q_b = b_b with
    // a = dt gamma lift c_r / 2; every other node keeps B
    const int vs[3] = {1, 2, 5};
    for (int ez = 0; ez < P.nez; ++ez) {
      const size_t e = e0 + slab * ez;
#pragma unroll
      for (int c = 0; c < 3; ++c)
        for (int k = 1; k < Nq - 1; ++k) {
          const int n = n0 + Nf * k;
          Y[(e * 6 + vs[c]) * Np + n] = Bv[(e * 6 + vs[c]) * Np + n];
        }
      if (ez == 0)
        for (int c = 0; c < 3; ++c) Y[(e * 6 + vs[c]) * Np + n0] = Bv[(e * 6 + vs[c]) * Np + n0];
      if (ez + 1 == P.nez) {
        const int n = n0 + Nf * (Nq - 1);
        for (int c = 0; c < 3; ++c) Y[(e * 6 + vs[c]) * Np + n] = Bv[(e * 6 + vs[c]) * Np + n];
      } else {
        const size_t eu = e + slab;
        const int nt = n0 + Nf * (Nq - 1), nb = n0;
        const double a = T.dtg * T.lift * 0.5 * T.lev[4 * (ez * Nq + Nq - 1) + 2];
        const double inv = 1.0 / (1.0 + 2.0 * a);
        for (int c = 0; c < 3; ++c) {
          const double bt = Bv[(e * 6 + vs[c]) * Np + nt], bb = Bv[(eu * 6 + vs[c]) * Np + nb];
          Y[(e * 6 + vs[c]) * Np + nt] = ((1.0 + a) * bt + a * bb) * inv;
          Y[(eu * 6 + vs[c]) * Np + nb] = (a * bt + (1.0 + a) * bb) * inv;
        }
      }
    }
  }
}

// out = Q + dt sum_k c_k X_k (elementwise, up to four terms); out may be Q.
__global__ void k_lincomb(double *out, const double *Q, LinComb lc, long long count) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < count;
       q += (long long)gridDim.x * blockDim.x) {
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (k < lc.n) s += lc.c[k] * lc.X[k][q];
    out[q] = Q[q] + lc.dt * s;
  }
}

static int line_grid(long long nlines) {
  long long b = (nlines + 127) / 128;
  return (int)(b < 148 * 16 ? b : 148 * 16);
}

// one thread per vertical line of nodes, (N+1)^2 lines per element column;
// the line kernels are instantiated for the orders 1 .. 7
template <int N>
static void hevi_apply_order(const double *Q, double *out, const HeviTables &T, const KParams &P, cudaStream_t s) {
  const long long nlines = (long long)P.nex * P.ney * (N + 1) * (N + 1);
  k_hevi_apply<N><<<line_grid(nlines), 128, 0, s>>>(Q, out, T, P);
}
template <int N>
static void hevi_solve_order(const double *B, double *Y, const HeviTables &T, const KParams &P, cudaStream_t s) {
  const long long nlines = (long long)P.nex * P.ney * (N + 1) * (N + 1);
  k_hevi_solve<N><<<line_grid(nlines), 128, 0, s>>>(B, Y, T, P);
}

cudaError_t launch_hevi_apply(const double *Q, double *out, const HeviTables &T, const KParams &P, cudaStream_t s) {
  switch (P.N) {
    case 1: hevi_apply_order<1>(Q, out, T, P, s); break;
    case 2: hevi_apply_order<2>(Q, out, T, P, s); break;
    case 3: hevi_apply_order<3>(Q, out, T, P, s); break;
    case 4: hevi_apply_order<4>(Q, out, T, P, s); break;
    case 5: hevi_apply_order<5>(Q, out, T, P, s); break;
    case 6: hevi_apply_order<6>(Q, out, T, P, s); break;
    case 7: hevi_apply_order<7>(Q, out, T, P, s); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_hevi_solve(const double *B, double *Y, const HeviTables &T, const KParams &P, cudaStream_t s) {
  switch (P.N) {
    case 1: hevi_solve_order<1>(B, Y, T, P, s); break;
    case 2: hevi_solve_order<2>(B, Y, T, P, s); break;
    case 3: hevi_solve_order<3>(B, Y, T, P, s); break;
    case 4: hevi_solve_order<4>(B, Y, T, P, s); break;
    case 5: hevi_solve_order<5>(B, Y, T, P, s); break;
    case 6: hevi_solve_order<6>(B, Y, T, P, s); break;
    case 7: hevi_solve_order<7>(B, Y, T, P, s); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_lincomb(double *out, const double *Q, const LinComb &lc, long long count, cudaStream_t s) {
  long long b = (count + 255) / 256;
  k_lincomb<<<(int)(b < 148 * 32 ? b : 148 * 32), 256, 0, s>>>(out, Q, lc, count);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- host side

namespace {

// inverse of an n x n matrix (row-major) by Gauss-Jordan elimination with
// partial pivoting; false if a pivot vanishes
bool invert(int n, const double *M, double *inv) {
  std::vector<double> a(M, M + n * n);
  for (int i = 0; i < n * n; ++i) inv[i] = 0.0;
  for (int i = 0; i < n; ++i) inv[i * n + i] = 1.0;
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (fabs(a[r * n + c]) > fabs(a[piv * n + c])) piv = r;
    if (a[piv * n + c] == 0.0) return false;
    if (piv != c)
      for (int k = 0; k < n; ++k) {
        std::swap(a[c * n + k], a[piv * n + k]);
        std::swap(inv[c * n + k], inv[piv * n + k]);
      }
    const double d = 1.0 / a[c * n + c];
    for (int k = 0; k < n; ++k) {
      a[c * n + k] *= d;
      inv[c * n + k] *= d;
    }
    for (int r = 0; r < n; ++r)
      if (r != c && a[r * n + c] != 0.0) {
        const double f = a[r * n + c];
        for (int k = 0; k < n; ++k) {
          a[r * n + k] -= f * a[c * n + k];
          inv[r * n + k] -= f * inv[c * n + k];
        }
      }
  }
  return true;
}

}  // namespace

bool hevi_build(const HeviSetup &S, HeviHost &H) {
  const int N = S.N, Nq = N + 1, kHB = hevi_hb(N), kTB = hevi_tB(N), kTA = hevi_tA(N), kTC = hevi_tC(N),
            kTG = hevi_tG(N), kTE = hevi_tE(N), kTStride = hevi_stride(N), kTop = 3 * N;
  const int nez = S.nez, nlev = nez * Nq;
  const double jz = 2.0 / S.hz;
  H.lift = 2.0 / (S.hz * S.w[0]);
  H.lev.assign((size_t)nlev * 4, 0.0);
  std::vector<double> a(nlev), hr(nlev), cr(nlev), kap(nlev);
  for (int l = 0; l < nlev; ++l) {
    const double rr = S.rho_r[l], pr = S.p_r[l], phi = S.g * S.z[l], q = S.qt_r ? S.qt_r[l] : 0.0;
    const double Rm = (1.0 - q) * S.Rd + q * S.Rv, cvm = (1.0 - q) * S.cvd + q * S.cvv;
    kap[l] = Rm / cvm;
    const double rer = rr * (cvm * (pr / (rr * Rm) - S.T0) + q * S.Iv0 + phi);
    a[l] = Rm * S.T0 - kap[l] * (phi + q * S.Iv0);
    hr[l] = (rer + pr) / rr;
    cr[l] = sqrt((1.0 + kap[l]) * pr / rr);
    H.lev[4 * l + 0] = rr;
    H.lev[4 * l + 1] = rer;
    H.lev[4 * l + 2] = cr[l];
  }
  // blocks of L: [ez][sub, diag, super][kHB x kHB], row/col index 3 k + c
  H.Lb.assign((size_t)nez * 3 * kHB * kHB, 0.0);
  auto dF = [&](int l, int c, int cc) {  // d F_c / d y_cc at level node l
    if (c == 0) return cc == 1 ? 1.0 : 0.0;
    if (c == 1) return cc == 0 ? a[l] : (cc == 2 ? kap[l] : 0.0);
    return cc == 1 ? hr[l] : 0.0;
  };
  for (int ez = 0; ez < nez; ++ez) {
    double *A = H.Lb.data() + (size_t)ez * 3 * kHB * kHB, *B = A + kHB * kHB, *C = B + kHB * kHB;
    for (int k = 0; k < Nq; ++k) {
      for (int m = 0; m < Nq; ++m) {
        const int lm = ez * Nq + m;
        for (int c = 0; c < 3; ++c)
          for (int cc = 0; cc < 3; ++cc) B[(3 * k + c) * kHB + 3 * m + cc] += -jz * S.D[k * Nq + m] * dF(lm, c, cc);
      }
      B[(3 * k + 1) * kHB + 3 * k + 0] += -S.g;
      for (int side = 0; side < 2; ++side) {
        if ((side == 0 && k != 0) || (side == 1 && k != N)) continue;
        const double nz = side == 0 ? -1.0 : 1.0;
        const int l = ez * Nq + k;
        const bool wall = side == 0 ? ez == 0 : ez == nez - 1;
        for (int c = 0; c < 3; ++c)
          for (int cc = 0; cc < 3; ++cc) {
            const double d = c == cc ? 1.0 : 0.0;
            // lift (nz F(y-)/2 - nz F(y+)/2 - c_r (y- - y+)/2)
            B[(3 * k + c) * kHB + 3 * k + cc] += H.lift * (0.5 * nz * dF(l, c, cc) - 0.5 * cr[l] * d);
            if (wall) {
              const double R = cc == 1 ? -1.0 : 1.0;  // y+ = R y-
              B[(3 * k + c) * kHB + 3 * k + cc] += H.lift * (-0.5 * nz * dF(l, c, cc) * R + 0.5 * cr[l] * d * R);
            } else {
              double *X = side == 0 ? A : C;
              const int kp = side == 0 ? N : 0;
              X[(3 * k + c) * kHB + 3 * kp + cc] += H.lift * (-0.5 * nz * dF(l, c, cc) + 0.5 * cr[l] * d);
            }
          }
      }
    }
  }
  // block elimination of M = I - dtg L: S_0 = B^M_0, S_ez = B^M_ez - A^M_ez E_ez-1,
  // G_ez = S_ez^-1, E_ez = G_ez C^M_ez
  H.Gf.assign((size_t)nez * kHB * kHB, 0.0);
  H.Ef.assign((size_t)nez * kHB * kHB, 0.0);
  std::vector<double> Sm(kHB * kHB);
  for (int ez = 0; ez < nez; ++ez) {
    const double *A = H.Lb.data() + (size_t)ez * 3 * kHB * kHB, *B = A + kHB * kHB, *C = B + kHB * kHB;
    for (int i = 0; i < kHB; ++i)
      for (int j = 0; j < kHB; ++j) Sm[i * kHB + j] = (i == j ? 1.0 : 0.0) - S.dtg * B[i * kHB + j];
    if (ez > 0) {
      const double *Ep = H.Ef.data() + (size_t)(ez - 1) * kHB * kHB;
      for (int i = 0; i < kHB; ++i)
        for (int j = 0; j < kHB; ++j) {
          double s = 0.0;
          for (int k = 0; k < kHB; ++k) s += (-S.dtg * A[i * kHB + k]) * Ep[k * kHB + j];
          Sm[i * kHB + j] -= s;
        }
    }
    double *G = H.Gf.data() + (size_t)ez * kHB * kHB;
    if (!invert(kHB, Sm.data(), G)) return false;
    double *E = H.Ef.data() + (size_t)ez * kHB * kHB;
    for (int i = 0; i < kHB; ++i)
      for (int j = 0; j < kHB; ++j) {
        double s = 0.0;
        for (int k = 0; k < kHB; ++k) s += G[i * kHB + k] * (-S.dtg * C[k * kHB + j]);
        E[i * kHB + j] = s;
      }
  }
  // the kernels' per-level table; the face-coupling blocks must be the only
  // nonzeros of L's off-diagonal blocks and of E
  H.tab.assign((size_t)nez * kTStride, 0.0);
  for (int ez = 0; ez < nez; ++ez) {
    const double *A = H.Lb.data() + (size_t)ez * 3 * kHB * kHB, *B = A + kHB * kHB, *C = B + kHB * kHB;
    const double *G = H.Gf.data() + (size_t)ez * kHB * kHB, *E = H.Ef.data() + (size_t)ez * kHB * kHB;
    double *Tz = H.tab.data() + (size_t)ez * kTStride;
    for (int i = 0; i < kHB * kHB; ++i) {
      Tz[kTB + i] = B[i];
      Tz[kTG + i] = G[i];
    }
    for (int i = 0; i < kHB; ++i)
      for (int j = 0; j < kHB; ++j) {
        const bool a_face = i < 3 && j >= kTop, c_face = i >= kTop && j < 3, e_col = j < 3;
        if ((A[i * kHB + j] != 0.0 && !a_face) || (C[i * kHB + j] != 0.0 && !c_face) ||
            (E[i * kHB + j] != 0.0 && !e_col))
          return false;
        if (a_face) Tz[kTA + 3 * i + (j - kTop)] = A[i * kHB + j];
        if (c_face) Tz[kTC + 3 * (i - kTop) + j] = C[i * kHB + j];
        if (e_col) Tz[kTE + 3 * i + j] = E[i * kHB + j];
      }
  }
  return true;
}

}  // namespace cmles
