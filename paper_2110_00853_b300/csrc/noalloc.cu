// Allocation-free variant of the budget reduction (cmles_budgets_noalloc).
//
// Some callers cannot call cudaMalloc: applications that hand all device
// memory to their own pool allocator and forbid allocations outside it, and
// time-stepping loops that cannot afford the implicit device-wide
// synchronisation of cudaMalloc/cudaFree.  For them this entry point computes
// the same FP64 quadrature budgets as cmles_diagnostics from a caller-owned
// state, writing into a caller-owned output, with its block partial sums kept
// in the file-scope device array below instead of a handle's buffer.
//
// The array is shared by every call in the process (and every GPU that loads
// the library holds one copy until exit).  Its device address is looked up
// once per device and cached; it belongs to that device's primary context,
// so after cudaDeviceReset the library must be unloaded and loaded again (a
// new process) before this entry point is used on that device.  Each block
// overwrites its own slots before they are read, so nothing needs clearing
// between calls, but calls that overlap on the GPU race on the array and
// must be serialised by the caller (same stream, or ordered by events).
#include <math.h>

#include <mutex>

#include "cmles.h"

namespace {

constexpr int kElemsPerBlock = 64;
constexpr int kMaxBlocks = 32768;  // at most kMaxBlocks * kElemsPerBlock = 2,097,152 elements
constexpr int kThreads = 256;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_budget_partials[kMaxBlocks * 8];

struct QuadWeights {
  double w[512];  // w_i w_j w_k, (N+1)^3 <= 512
};

// Block b sums w_n J Q_v over the nodes of elements [64 b, 64 b + 64) and
// counts non-finite entries; one slot of 8 doubles per block.
__global__ void __launch_bounds__(kThreads) k_budget_noalloc_partial(const double *__restrict__ Q, long long E,
                                                                     int Np, const QuadWeights W, double J,
                                                                     double *__restrict__ partials) {
  const long long e0 = (long long)blockIdx.x * kElemsPerBlock;
  long long e1 = e0 + kElemsPerBlock;
  if (e1 > E) e1 = E;
  const long long n0 = e0 * Np, n1 = e1 * Np;
  double acc[7] = {0, 0, 0, 0, 0, 0, 0};
  for (long long g = n0 + threadIdx.x; g < n1; g += kThreads) {
    const long long e = g / Np;
    const int n = (int)(g - e * Np);
    const double w = W.w[n] * J;
#pragma unroll
    for (int v = 0; v < 6; ++v) {
      const double q = Q[(e * 6 + v) * Np + n];
      acc[v] += w * q;
      if (!isfinite(q)) acc[6] += 1.0;
    }
  }
  __shared__ double red[7][kThreads / 32];
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
    for (int w = 0; w < kThreads / 32; ++w) x += red[threadIdx.x][w];
    partials[(size_t)blockIdx.x * 8 + threadIdx.x] = x;
  }
}

__global__ void k_budget_noalloc_final(const double *__restrict__ partials, int nblocks, double *__restrict__ out) {
  if (threadIdx.x < 7) {
    double x = 0.0;
    for (int b = 0; b < nblocks; ++b) x += partials[(size_t)b * 8 + threadIdx.x];
    out[threadIdx.x] = x;
  }
}

// LGL quadrature weights without heap use: nodes by Newton on
// (1 - x^2) P_N'(x) = N (P_{N-1} - x P_N), weights 2 / (N (N+1) P_N^2).
void lgl_weights_fixed(int N, double *w) {
  for (int i = 0; i <= N; ++i) {
    double x = -cos(M_PI * i / N);
    double PN = 1.0, PNm1 = 0.0;
    for (int it = 0; it < 200; ++it) {
      double pm = 1.0, p = x;
      for (int k = 1; k < N; ++k) {
        const double pn = ((2.0 * k + 1.0) * x * p - k * pm) / (k + 1.0);
        pm = p;
        p = pn;
      }
      PN = p;
      PNm1 = pm;
      if (i == 0 || i == N) break;
      const double step = (PNm1 - x * PN) / ((N + 1.0) * PN);
      x += step;
      if (fabs(step) < 1e-17) break;
    }
    w[i] = 2.0 / (N * (N + 1.0) * PN * PN);
  }
}

std::mutex g_mutex;
double *g_scratch[kMaxDevices] = {nullptr};

}  // namespace

extern "C" cmles_status cmles_budgets_noalloc(const double *Q_dev, long long num_elements, int N, double jacobian,
                                              double *out_dev, void *stream) {
  if (!Q_dev || !out_dev) return CMLES_ERR_ARG;
  if (N < 1 || N > 7) return CMLES_ERR_ARG;
  if (num_elements < 1 || num_elements > (long long)kMaxBlocks * kElemsPerBlock) return CMLES_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return CMLES_ERR_CUDA;
  double *scratch = nullptr;
  {
    // once per device, with that device current: the device address of the
    // file-scope array (its host-side name is only a stand-in)
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch[dev]) {
      void *ptr = nullptr;
      if (cudaGetSymbolAddress(&ptr, g_budget_partials) != cudaSuccess || !ptr) return CMLES_ERR_CUDA;
      g_scratch[dev] = (double *)ptr;
    }
    scratch = g_scratch[dev];
  }
  const int Nq = N + 1;
  int Np = Nq * Nq * Nq;
  double w1[8];
  lgl_weights_fixed(N, w1);
  QuadWeights W;
  for (int k = 0; k < Nq; ++k)
    for (int j = 0; j < Nq; ++j)
      for (int i = 0; i < Nq; ++i) W.w[i + Nq * (j + Nq * k)] = w1[i] * w1[j] * w1[k];
  int nblocks = (int)((num_elements + kElemsPerBlock - 1) / kElemsPerBlock);
  cudaStream_t s = (cudaStream_t)stream;
  // the status of each launch is taken from cudaLaunchKernel itself, not
  // from cudaGetLastError, so an earlier non-sticky error of other code on
  // this thread is neither reported here nor cleared (a sticky fault of the
  // context is reported by every call)
  long long E = num_elements;
  void *args1[] = {(void *)&Q_dev, (void *)&E, (void *)&Np, (void *)&W, (void *)&jacobian, (void *)&scratch};
  if (cudaLaunchKernel((const void *)k_budget_noalloc_partial, dim3(nblocks), dim3(kThreads), args1, 0, s) !=
      cudaSuccess)
    return CMLES_ERR_CUDA;
  void *args2[] = {(void *)&scratch, (void *)&nblocks, (void *)&out_dev};
  if (cudaLaunchKernel((const void *)k_budget_noalloc_final, dim3(1), dim3(32), args2, 0, s) != cudaSuccess)
    return CMLES_ERR_CUDA;
  return CMLES_OK;
}
