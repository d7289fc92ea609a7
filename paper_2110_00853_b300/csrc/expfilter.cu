// Exponential modal filter (Eq. exponential_filter) on the momentum.
//
// In each element and along each direction the nodal values are mapped to
// Legendre modes, mode k is scaled by sigma(k/N) = exp(-alpha (k/N)^s) and
// mapped back: one (N+1) x (N+1) matrix F = V diag(sigma) V^-1 applied along
// x, then y, then z.  The momentum has a zero balanced background, so the
// filter acts on the prognostic values themselves.  One CTA per element (grid
// stride), the element's variable staged in shared memory between the three
// passes; the FP32 shadow of a filtered variable is rewritten alongside.
#include "launch.h"

namespace cmles {

// threads per CTA: one per node (128 up to N = 4), as many as the FP32
// arrays' padded nodes per element
__host__ __device__ constexpr int filter_block(int N) { return np32(N); }

template <int N>
__global__ void __launch_bounds__(filter_block(N)) k_expfilter(double *__restrict__ Q, float *__restrict__ S32,
                                                               const ExpFilter Fm, int E) {
  constexpr int Nq = N + 1, Np = Nq * Nq * Nq;
  __shared__ double sF[Nq * Nq];
  __shared__ double a[Np], b[Np];
  const int t = threadIdx.x;
  if (t < Nq * Nq) sF[t] = Fm.F[t];
  const int i = t % Nq, j = (t / Nq) % Nq, k = t / (Nq * Nq);
  __syncthreads();
  for (int e = blockIdx.x; e < E; e += gridDim.x) {
    for (int v = 1; v <= 3; ++v) {
      if (!(Fm.mask & (1 << v))) continue;
      double *q = Q + ((size_t)e * 6 + v) * Np;
      if (t < Np) a[t] = q[t];
      __syncthreads();
      if (t < Np) {
        double r = 0.0;
#pragma unroll
        for (int m = 0; m < Nq; ++m) r += sF[i * Nq + m] * a[m + Nq * (j + Nq * k)];
        b[t] = r;
      }
      __syncthreads();
      if (t < Np) {
        double r = 0.0;
#pragma unroll
        for (int m = 0; m < Nq; ++m) r += sF[j * Nq + m] * b[i + Nq * (m + Nq * k)];
        a[t] = r;
      }
      __syncthreads();
      if (t < Np) {
        double r = 0.0;
#pragma unroll
        for (int m = 0; m < Nq; ++m) r += sF[k * Nq + m] * a[i + Nq * (j + Nq * m)];
        q[t] = r;
        if (S32) S32[((size_t)e * 6 + v) * np32(N) + t] = (float)r;
      }
      __syncthreads();
    }
  }
}

template <int N>
static void expfilter_order(double *Q, float *S32, const ExpFilter &F, int E, cudaStream_t s) {
  static int grid = 0;
  if (!grid) grid = grid_for((const void *)k_expfilter<N>, 1 << 30, 0, filter_block(N));
  k_expfilter<N><<<grid < E ? grid : E, filter_block(N), 0, s>>>(Q, S32, F, E);
}

cudaError_t launch_expfilter(double *Q, float *S32, const ExpFilter &F, int N, int E, cudaStream_t s) {
  switch (N) {
    case 1: expfilter_order<1>(Q, S32, F, E, s); break;
    case 2: expfilter_order<2>(Q, S32, F, E, s); break;
    case 3: expfilter_order<3>(Q, S32, F, E, s); break;
    case 4: expfilter_order<4>(Q, S32, F, E, s); break;
    case 5: expfilter_order<5>(Q, S32, F, E, s); break;
    case 6: expfilter_order<6>(Q, S32, F, E, s); break;
    case 7: expfilter_order<7>(Q, S32, F, E, s); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace cmles
