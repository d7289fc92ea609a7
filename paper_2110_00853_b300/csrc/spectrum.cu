// Kinetic-energy spectrum of the handle's state (cmles_spectrum): the
// turbulence diagnostic of Sec. 5.5 (a Fourier transform of the velocity
// field), on the nodal DG field of a mesh periodic in x and y.
//
//   1. velocity u_i = (rho u_i) / rho at the nodes;
//   2. uniform resampling: N points per element and direction at the cell
//      centres xi_s = -1 + (2 s + 1) / N of the reference interval (never on
//      an element face), M_x = nex N, M_y = ney N points per level and
//      M_z = nez N levels; the value at a point is the element's Lagrange
//      polynomial of degree N in each direction;
//   3. per level, the discrete Fourier coefficients
//      u^(p, q) = 1/(M_x M_y) sum_ij u_ij exp(-2 pi i (p i / M_x + q j / M_y)),
//      as two passes of direct sums with a table of cos and sin (FP64): along
//      x for p = 0 .. M_x/2 (the field is real: negative p mirror positive
//      ones), then along y;
//   4. shell s = round(L sqrt((p / L_x)^2 + (q / L_y)^2)), L = max(L_x, L_y);
//   5. E(s) = level average of the shell sums of (|u^|^2 + |v^|^2 + |w^|^2)/2,
//      each p in (0, M_x/2) counted twice for its mirror -p.
// The grid, the two transforms and the shell sums use scratch device memory
// allocated on the handle's stream for the call.
#include <math.h>

#include <vector>

#include "handle.h"

using namespace cmles_host;

namespace {

struct SpecGeom {
  int nex, ney, nez, N, Mx, My, Mz, nshell;
  double Lx, Ly;
  double xi[kMaxQ];     // LGL nodes
  double lag[kMaxQ * kMaxQ];  // lag[s][a] = l_a(xi_s), the N sample points of an element
};

// Steps 1-2: thread per grid point (c = all three components at once).
__global__ void k_spec_resample(const double *__restrict__ Q, const SpecGeom G, double *__restrict__ U) {
  const int N = G.N, Nq = N + 1, Np = Nq * Nq * Nq;
  const long long total = (long long)G.Mx * G.My * G.Mz;
  const long long plane = (long long)G.Mx * G.My;
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += (long long)gridDim.x * blockDim.x) {
    const int ix = (int)(g % G.Mx), iy = (int)((g / G.Mx) % G.My), iz = (int)(g / plane);
    const int ex = ix / N, sx = ix - ex * N, ey = iy / N, sy = iy - ey * N, ez = iz / N, sz = iz - ez * N;
    const long long e = ex + (long long)G.nex * (ey + (long long)G.ney * ez);
    const double *q = Q + e * 6 * Np;
    double acc[3] = {0.0, 0.0, 0.0};
    for (int c = 0; c < Nq; ++c) {
      const double lz = G.lag[sz * Nq + c];
      for (int b = 0; b < Nq; ++b) {
        const double lyz = G.lag[sy * Nq + b] * lz;
        for (int a = 0; a < Nq; ++a) {
          const double w = G.lag[sx * Nq + a] * lyz;
          const int n = a + Nq * (b + Nq * c);
          const double ir = 1.0 / q[n];
          acc[0] += w * q[Np + n] * ir;
          acc[1] += w * q[2 * Np + n] * ir;
          acc[2] += w * q[3 * Np + n] * ir;
        }
      }
    }
    for (int k = 0; k < 3; ++k) U[k * total + g] = acc[k];
  }
}

// Step 3a: X[c][l][j][p] = sum_i U[c][l][j][i] e^{-2 pi i p i / M_x}, p <= M_x/2.
__global__ void k_spec_dft_x(const double *__restrict__ U, const double2 *__restrict__ twx, const SpecGeom G,
                             double2 *__restrict__ X) {
  const int P = G.Mx / 2 + 1;
  const long long rows = 3LL * G.Mz * G.My;
  const long long total = rows * P;
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += (long long)gridDim.x * blockDim.x) {
    const int p = (int)(g % P);
    const long long r = g / P;
    const double *u = U + r * G.Mx;
    double re = 0.0, im = 0.0;
    int idx = 0;  // p i mod M_x
    for (int i = 0; i < G.Mx; ++i) {
      const double2 t = twx[idx];  // (cos, -sin) of 2 pi idx / M_x
      re += u[i] * t.x;
      im += u[i] * t.y;
      idx += p;
      if (idx >= G.Mx) idx -= G.Mx;
    }
    X[g] = make_double2(re, im);
  }
}

// Step 3b: Y[c][l][q][p] = sum_j X[c][l][j][p] e^{-2 pi i q j / M_y}.
__global__ void k_spec_dft_y(const double2 *__restrict__ X, const double2 *__restrict__ twy, const SpecGeom G,
                             double2 *__restrict__ Y) {
  const int P = G.Mx / 2 + 1;
  const long long total = 3LL * G.Mz * G.My * P;
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += (long long)gridDim.x * blockDim.x) {
    const int p = (int)(g % P);
    const int q = (int)((g / P) % G.My);
    const long long cl = g / ((long long)P * G.My);
    const double2 *x = X + cl * G.My * P + p;
    double re = 0.0, im = 0.0;
    int idx = 0;  // q j mod M_y
    for (int j = 0; j < G.My; ++j) {
      const double2 a = x[(long long)j * P], t = twy[idx];
      re += a.x * t.x - a.y * t.y;
      im += a.x * t.y + a.y * t.x;
      idx += q;
      if (idx >= G.My) idx -= G.My;
    }
    Y[g] = make_double2(re, im);
  }
}

// Steps 4-5: thread per (level, q, p) of the half spectrum, its energy added
// to its level's shell sum El[l][s] (FP64 atomics: the order of the additions
// varies, their rounding is below the diagnostic's use).
__global__ void k_spec_shells(const double2 *__restrict__ Y, const SpecGeom G, double *__restrict__ El) {
  const int P = G.Mx / 2 + 1;
  const long long total = (long long)G.Mz * G.My * P;
  const double L = G.Lx > G.Ly ? G.Lx : G.Ly;
  const double norm = 1.0 / ((double)G.Mx * G.My);
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += (long long)gridDim.x * blockDim.x) {
    const int p = (int)(g % P);
    const int q = (int)((g / P) % G.My);
    const int l = (int)(g / ((long long)P * G.My));
    const int qs = q < (G.My + 1) / 2 ? q : q - G.My;  // the signed index (numpy's ordering)
    const double kx = p / G.Lx, ky = qs / G.Ly;
    const int s = (int)rint(L * sqrt(kx * kx + ky * ky));
    if (s >= G.nshell) continue;
    // p in (0, M_x/2) stands for itself and the mirror (-p, -q); for even M_x
    // the Nyquist column p = M_x/2 is counted once
    const double mult = (p == 0 || 2 * p == G.Mx) ? 1.0 : 2.0;
    double e = 0.0;
    for (int c = 0; c < 3; ++c) {
      const double2 y = Y[(((long long)c * G.Mz + l) * G.My + q) * P + p];
      e += y.x * y.x + y.y * y.y;
    }
    atomicAdd(&El[(long long)l * G.nshell + s], 0.5 * mult * e * norm * norm);
  }
}

int blocks_of(long long n) {
  long long b = (n + 255) / 256;
  if (b > 148 * 16) b = 148 * 16;
  return (int)(b < 1 ? 1 : b);
}

}  // namespace

extern "C" cmles_status cmles_spectrum(cmles_handle h, int nshell, double *E_host) {
  if (!h || !E_host || nshell < 1) return fail(h, CMLES_ERR_ARG, "cmles_spectrum: bad argument");
  if (h->curved || h->part) return fail(h, CMLES_ERR_ARG, "cmles_spectrum: flat whole meshes only");
  const cmles_mesh &m = h->mesh;
  if (!m.periodic[0] || !m.periodic[1])
    return fail(h, CMLES_ERR_ARG, "cmles_spectrum: the mesh must be periodic in x and y");
  SpecGeom G;
  memset(&G, 0, sizeof(G));
  G.nex = m.nex;
  G.ney = m.ney;
  G.nez = m.nez;
  G.N = h->N;
  G.Mx = m.nex * h->N;
  G.My = m.ney * h->N;
  G.Mz = m.nez * h->N;
  G.nshell = nshell;
  G.Lx = m.Lx;
  G.Ly = m.Ly;
  const int Nq = h->Nq;
  for (int a = 0; a < Nq; ++a) G.xi[a] = h->xi[a];
  for (int s = 0; s < h->N; ++s) {
    const double x = -1.0 + (2.0 * s + 1.0) / h->N;
    for (int a = 0; a < Nq; ++a) {
      double l = 1.0;
      for (int b = 0; b < Nq; ++b)
        if (b != a) l *= (x - h->xi[b]) / (h->xi[a] - h->xi[b]);
      G.lag[s * Nq + a] = l;
    }
  }
  const long long pts = (long long)G.Mx * G.My * G.Mz, P = G.Mx / 2 + 1;
  double *U = nullptr, *El = nullptr;
  double2 *X = nullptr, *Y = nullptr, *twx = nullptr, *twy = nullptr;
  cudaStream_t s = h->stream;
  cudaError_t e = cudaSuccess;
  auto alloc = [&](void **p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMallocAsync(p, bytes, s);
  };
  alloc((void **)&U, (size_t)pts * 3 * sizeof(double));
  alloc((void **)&X, (size_t)3 * G.Mz * G.My * P * sizeof(double2));
  alloc((void **)&Y, (size_t)3 * G.Mz * G.My * P * sizeof(double2));
  alloc((void **)&twx, (size_t)G.Mx * sizeof(double2));
  alloc((void **)&twy, (size_t)G.My * sizeof(double2));
  alloc((void **)&El, (size_t)G.Mz * nshell * sizeof(double));
  std::vector<double2> hx(G.Mx), hy(G.My);
  for (int i = 0; i < G.Mx; ++i) hx[i] = make_double2(cos(2.0 * M_PI * i / G.Mx), -sin(2.0 * M_PI * i / G.Mx));
  for (int j = 0; j < G.My; ++j) hy[j] = make_double2(cos(2.0 * M_PI * j / G.My), -sin(2.0 * M_PI * j / G.My));
  std::vector<double> el((size_t)G.Mz * nshell);
  if (e == cudaSuccess) e = cudaMemcpyAsync(twx, hx.data(), hx.size() * sizeof(double2), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(twy, hy.data(), hy.size() * sizeof(double2), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(El, 0, (size_t)G.Mz * nshell * sizeof(double), s);
  if (e == cudaSuccess) {
    LaunchScope ls(h, 2, 4);
    k_spec_resample<<<blocks_of(pts), 256, 0, s>>>(h->Q[h->cur], G, U);
    k_spec_dft_x<<<blocks_of(3 * G.Mz * G.My * P), 256, 0, s>>>(U, twx, G, X);
    k_spec_dft_y<<<blocks_of(3 * G.Mz * G.My * P), 256, 0, s>>>(X, twy, G, Y);
    k_spec_shells<<<blocks_of((long long)G.Mz * G.My * P), 256, 0, s>>>(Y, G, El);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(el.data(), El, el.size() * sizeof(double), cudaMemcpyDeviceToHost, s);
  void *bufs[] = {U, X, Y, twx, twy, El};
  for (void *b : bufs)
    if (b) cudaFreeAsync(b, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(h, CMLES_ERR_CUDA, std::string("cmles_spectrum: ") + cudaGetErrorString(e));
  for (int k = 0; k < nshell; ++k) {
    double acc = 0.0;
    for (int l = 0; l < G.Mz; ++l) acc += el[(size_t)l * nshell + k];
    E_host[k] = acc / G.Mz;
  }
  return CMLES_OK;
}
