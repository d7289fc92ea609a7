// Learned-closure network: weight packing, batched inference, BF16
// tensor-core training step (forward, backward, weight gradients) and Adam.
//
// Loss: L = 1/(2n) sum_s |y_s - t_s|^2 over the n samples of a call.
// Backward (per sample, FP32 with BF16 tensor-core products):
//   dy = (y - t)/n,  dh2 = W3^T dy,  da2 = dh2 * silu'(a2),
//   dh1 = W2^T da2,  da1 = dh1 * silu'(a1),  silu'(a) = s (1 + a (1 - s)),
//   gW3 += dy h2^T, gW2 += da2 h1^T, gW1 += da1 x^T, gb_l += da_l.
// One CTA of 128 threads handles 128 samples per iteration (one row per
// thread for pointwise work, 4 warps x 32 rows for the mma.sync products) and
// keeps its gradient partial sums in shared memory until the end.
#include <string.h>

#include "cmles.h"
#include "common.cuh"
#include "launch.h"
#include "mlp.cuh"

namespace cmles {

// ------------------------------------------------------------------ packing

// Entry (row, k) of the tensor-core operand of layer l (0, 1, 2) from the
// FP32 parameter vector: the weight for k < K_in, then the bias split as
// hi + mid + lo on k = K_in .. K_in + 2, zero elsewhere.
__host__ __device__ inline __nv_bfloat16 tc_weight(const float *p, int l, int row, int k) {
  const int kin = l == 0 ? kMlpIn : kMlpH, nout = l == 2 ? kMlpOut : kMlpH;
  if (row >= nout) return __float2bfloat16_rn(0.f);
  if (k < kin) {
    const int off = l == 0 ? kMlpOffW1 : (l == 1 ? kMlpOffW2 : kMlpOffW3);
    return __float2bfloat16_rn(p[off + row * kin + k]);
  }
  if (k >= kin + 3) return __float2bfloat16_rn(0.f);
  const float b = p[(l == 0 ? kMlpOffB1 : (l == 1 ? kMlpOffB2 : kMlpOffB3)) + row];
  const __nv_bfloat16 hi = __float2bfloat16_rn(b);
  const float r1 = b - __bfloat162float(hi);
  const __nv_bfloat16 mid = __float2bfloat16_rn(r1);
  if (k == kin) return hi;
  if (k == kin + 1) return mid;
  return __float2bfloat16_rn(r1 - __bfloat162float(mid));
}

// Fill entry q of the three tensor-core operand arrays (q < the largest).
__host__ __device__ inline void tc_fill(const float *p, MlpTc *o, int q) {
  const int c = q & 7, r = (q >> 3) & 7;
  if (q < kMlpH * 8 * kTcKG1) {
    const int kg = (q >> 6) % kTcKG1, rg = (q >> 6) / kTcKG1;
    o->W1[q] = tc_weight(p, 0, rg * 8 + r, kg * 8 + c);
  }
  if (q < kMlpH * 8 * kTcKG) {
    const int kg = (q >> 6) % kTcKG, rg = (q >> 6) / kTcKG;
    o->W2[q] = tc_weight(p, 1, rg * 8 + r, kg * 8 + c);
  }
  if (q < kTcN3 * 8 * kTcKG) {
    const int kg = (q >> 6) % kTcKG, rg = (q >> 6) / kTcKG;
    o->W3[q] = tc_weight(p, 2, rg * 8 + r, kg * 8 + c);
  }
  if (q < kMlpInPad) o->in_scale[q] = q < kMlpIn ? p[kMlpOffIn + q] : 0.f;
  if (q < 4) o->out_scale[q] = q < 2 ? p[kMlpOffOut + q] : 0.f;
}

void pack_mlp_host(const float *p, MlpPacked *o) {
  memset(o, 0, sizeof(*o));
  for (int n = 0; n < kMlpH; ++n)
    for (int k = 0; k < kMlpIn; ++k) o->W1[n * kLdW1 + k] = __float2bfloat16_rn(p[kMlpOffW1 + n * kMlpIn + k]);
  for (int n = 0; n < kMlpH; ++n)
    for (int k = 0; k < kMlpH; ++k) o->W2[n * kLdW + k] = __float2bfloat16_rn(p[kMlpOffW2 + n * kMlpH + k]);
  for (int n = 0; n < kMlpOut; ++n)
    for (int k = 0; k < kMlpH; ++k) o->W3[n * kLdW + k] = __float2bfloat16_rn(p[kMlpOffW3 + n * kMlpH + k]);
  for (int n = 0; n < kMlpH; ++n) {
    o->b1[n] = p[kMlpOffB1 + n];
    o->b2[n] = p[kMlpOffB2 + n];
  }
  o->b3[0] = p[kMlpOffB3];
  o->b3[1] = p[kMlpOffB3 + 1];
  for (int k = 0; k < kMlpIn; ++k) o->in_scale[k] = p[kMlpOffIn + k];
  o->out_scale[0] = p[kMlpOffOut];
  o->out_scale[1] = p[kMlpOffOut + 1];
  for (int q = 0; q < kMlpH * 8 * kTcKG; ++q) tc_fill(p, &o->tc, q);
}

__global__ void k_pack_mlp(const float *__restrict__ p, MlpPacked *__restrict__ o) {
  const int t = threadIdx.x + blockIdx.x * blockDim.x, nt = blockDim.x * gridDim.x;
  for (int q = t; q < kMlpH * kLdW1; q += nt) {
    const int n = q / kLdW1, k = q % kLdW1;
    o->W1[q] = __float2bfloat16_rn(k < kMlpIn ? p[kMlpOffW1 + n * kMlpIn + k] : 0.f);
  }
  for (int q = t; q < kMlpH * kLdW; q += nt) {
    const int n = q / kLdW, k = q % kLdW;
    o->W2[q] = __float2bfloat16_rn(k < kMlpH ? p[kMlpOffW2 + n * kMlpH + k] : 0.f);
  }
  for (int q = t; q < kMlpOutPad * kLdW; q += nt) {
    const int n = q / kLdW, k = q % kLdW;
    o->W3[q] = __float2bfloat16_rn(n < kMlpOut && k < kMlpH ? p[kMlpOffW3 + n * kMlpH + k] : 0.f);
  }
  for (int q = t; q < kMlpH; q += nt) {
    o->b1[q] = p[kMlpOffB1 + q];
    o->b2[q] = p[kMlpOffB2 + q];
  }
  for (int q = t; q < kMlpOutPad; q += nt) o->b3[q] = q < kMlpOut ? p[kMlpOffB3 + q] : 0.f;
  for (int q = t; q < kMlpInPad; q += nt) o->in_scale[q] = q < kMlpIn ? p[kMlpOffIn + q] : 0.f;
  if (t < 2) o->out_scale[t] = p[kMlpOffOut + t];
  for (int q = t; q < kMlpH * 8 * kTcKG; q += nt) tc_fill(p, &o->tc, q);
}

cudaError_t launch_pack_mlp(const float *params_dev, MlpPacked *out, cudaStream_t s) {
  k_pack_mlp<<<8, 256, 0, s>>>(params_dev, out);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ inference

// One CTA of 128 threads per 128 rows, on the tensor cores (tcgen05); a CTA
// loops over row blocks.  err_count: CTAs whose tensor-core wait gave up.
__global__ void __launch_bounds__(128) k_mlp_forward(const MlpPacked *__restrict__ Wg, const float *__restrict__ X,
                                                     float *__restrict__ Y, long long n, int *err_count) {
  __shared__ __align__(16) uint8_t sWraw[sizeof(MlpTc)];
  __shared__ __align__(128) __nv_bfloat16 sA[kTcAElems];
  __shared__ __align__(8) uint64_t sBar;
  __shared__ uint32_t sSlot;
  const int t = threadIdx.x;
  for (int q = t; q < (int)(sizeof(MlpTc) / 16); q += 128)
    reinterpret_cast<uint4 *>(sWraw)[q] = reinterpret_cast<const uint4 *>(&Wg->tc)[q];
  fence_proxy_async_smem();
  TcState st;
  tc_setup(st, &sSlot, &sBar);
  const MlpTc &W = *reinterpret_cast<const MlpTc *>(sWraw);
  for (long long b = (long long)blockIdx.x * 128; b < n; b += (long long)gridDim.x * 128) {
    const long long s = b + t;
    float x[kMlpIn];
#pragma unroll
    for (int k = 0; k < kMlpIn; ++k) x[k] = s < n ? X[s * kMlpIn + k] : 0.f;
    mlp_tc_put_input(sA, x);
    float y0, y1;
    mlp_tc_forward(W, sA, st, y0, y1);
    if (s < n) {
      Y[s * 2 + 0] = y0;
      Y[s * 2 + 1] = y1;
    }
  }
  tc_teardown(st, err_count);
}

// ------------------------------------------------------------------ training

struct TrainSmem {
  MlpPacked W;
  __nv_bfloat16 W2T[kMlpH * kLdW];      // W2^T: [in][out], row stride kLdW
  __nv_bfloat16 X[128 * kMlpInPad];     // inputs, row-major
  __nv_bfloat16 XT[kMlpInPad * 128];    // inputs, [feature][sample]
  float A1[128 * kMlpH], A2[128 * kMlpH];  // pre-activations
  float Y[128 * 2], DY[128 * 2];
  __nv_bfloat16 DA2[128 * kMlpH];       // da2, row-major
  __nv_bfloat16 DA2T[kMlpH * 128];      // da2, [unit][sample]
  __nv_bfloat16 DA1T[kMlpH * 128];      // da1, [unit][sample]
  __nv_bfloat16 H1T[kMlpH * 128];       // h1 = silu(a1), [unit][sample]
  float g[kMlpNet];                     // gradient partial sums (parameter-vector layout)
  float loss;
};

__device__ __forceinline__ float dsilu(float a) {
  const float sg = __fdividef(1.0f, 1.0f + __expf(-a));
  return sg * (1.0f + a * (1.0f - sg));
}

__global__ void __launch_bounds__(128) k_mlp_train(const MlpPacked *__restrict__ Wg, const float *__restrict__ X,
                                                   const float *__restrict__ T, long long n,
                                                   float *__restrict__ grad, float *__restrict__ loss) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  TrainSmem &S = *reinterpret_cast<TrainSmem *>(smem_raw);
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5, g = lane >> 2, c = lane & 3;
  for (int q = t; q < (int)(sizeof(MlpPacked) / 16); q += 128)
    reinterpret_cast<uint4 *>(&S.W)[q] = reinterpret_cast<const uint4 *>(Wg)[q];
  for (int q = t; q < kMlpNet; q += 128) S.g[q] = 0.f;
  if (t == 0) S.loss = 0.f;
  __syncthreads();
  for (int q = t; q < kMlpH * kMlpH; q += 128) {
    const int o = q / kMlpH, i = q % kMlpH;
    S.W2T[i * kLdW + o] = S.W.W2[o * kLdW + i];
  }
  __syncthreads();
  const float inv_n = 1.0f / (float)n;
  for (long long b = (long long)blockIdx.x * 128; b < n; b += (long long)gridDim.x * 128) {
    const long long s = b + t;
    const bool valid = s < n;
    // inputs (bf16), row-major and transposed
    {
      uint32_t *xr = reinterpret_cast<uint32_t *>(S.X + t * kMlpInPad);
      float x[kMlpInPad];
#pragma unroll
      for (int k = 0; k < kMlpInPad; ++k) x[k] = (valid && k < kMlpIn) ? X[s * kMlpIn + k] : 0.f;
#pragma unroll
      for (int q = 0; q < kMlpInPad / 2; ++q) xr[q] = pack_bf16(x[2 * q], x[2 * q + 1]);
#pragma unroll
      for (int k = 0; k < kMlpInPad; ++k) S.XT[k * 128 + t] = __float2bfloat16_rn(x[k]);
    }
    __syncwarp();
    mlp_warp_forward(S.W, S.X, S.Y, 32 * warp, S.A1, S.A2, kMlpH);
    __syncthreads();
    // output error, loss, gW3 and gb3 pieces
    float dy0 = 0.f, dy1 = 0.f;
    if (valid) {
      const float r0 = S.Y[2 * t] - T[s * 2], r1 = S.Y[2 * t + 1] - T[s * 2 + 1];
      atomicAdd(&S.loss, 0.5f * (r0 * r0 + r1 * r1) * inv_n);
      dy0 = r0 * inv_n;
      dy1 = r1 * inv_n;
    }
    S.DY[2 * t] = dy0;
    S.DY[2 * t + 1] = dy1;
    __syncthreads();
    {
      // thread t: output unit o = t / 64, hidden unit i = t % 64
      const int o = t >> 6, i = t & 63;
      float acc = 0.f, accb = 0.f;
      for (int r = 0; r < 128; ++r) {
        const float d = S.DY[2 * r + o];
        acc += d * silu(S.A2[r * kMlpH + i]);
        accb += d;
      }
      S.g[kMlpOffW3 + o * kMlpH + i] += acc;
      if (i == 0) S.g[kMlpOffB3 + o] += accb;
    }
    // da2 = (W3^T dy) * silu'(a2): thread per sample
    for (int i = 0; i < kMlpH; ++i) {
      const float w0 = __bfloat162float(S.W.W3[0 * kLdW + i]), w1 = __bfloat162float(S.W.W3[1 * kLdW + i]);
      const float da = (w0 * dy0 + w1 * dy1) * dsilu(S.A2[t * kMlpH + i]);
      const __nv_bfloat16 db = __float2bfloat16_rn(da);
      S.DA2[t * kMlpH + i] = db;
      S.DA2T[i * 128 + t] = db;
      atomicAdd(&S.g[kMlpOffB2 + i], da);
    }
    // h1^T (bf16)
    for (int i = 0; i < kMlpH; ++i) S.H1T[i * 128 + t] = __float2bfloat16_rn(silu(S.A1[t * kMlpH + i]));
    __syncthreads();
    // dh1 = da2 W2 (per warp: its 32 rows), then da1 = dh1 * silu'(a1)
#pragma unroll 1
    for (int mt = 0; mt < 2; ++mt) {
      const int rb = 32 * warp + 16 * mt;
      uint32_t a[4][4];
#pragma unroll
      for (int kt = 0; kt < 4; ++kt) {
        a[kt][0] = ld_u32(S.DA2 + (rb + g) * kMlpH + 16 * kt + 2 * c);
        a[kt][1] = ld_u32(S.DA2 + (rb + g + 8) * kMlpH + 16 * kt + 2 * c);
        a[kt][2] = ld_u32(S.DA2 + (rb + g) * kMlpH + 16 * kt + 2 * c + 8);
        a[kt][3] = ld_u32(S.DA2 + (rb + g + 8) * kMlpH + 16 * kt + 2 * c + 8);
      }
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) {
        float d[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int kt = 0; kt < 4; ++kt)
          mma_bf16_16816(d, a[kt], ld_u32(S.W2T + (8 * nt + g) * kLdW + 16 * kt + 2 * c),
                         ld_u32(S.W2T + (8 * nt + g) * kLdW + 16 * kt + 2 * c + 8));
        const int col = 8 * nt + 2 * c;
        const int rows[2] = {rb + g, rb + g + 8};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            const int r = rows[h], cc = col + e;
            const float da = d[2 * h + e] * dsilu(S.A1[r * kMlpH + cc]);
            S.DA1T[cc * 128 + r] = __float2bfloat16_rn(b + r < n ? da : 0.f);
            if (b + r < n) atomicAdd(&S.g[kMlpOffB1 + cc], da);
          }
        }
      }
    }
    __syncthreads();
    // gW2 = da2^T h1 (warp w: output rows 16w..16w+15), K = 128 samples
    {
      const int ob = 16 * warp;
      float acc[8][4];
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
#pragma unroll 2
      for (int kt = 0; kt < 8; ++kt) {
        uint32_t a[4];
        a[0] = ld_u32(S.DA2T + (ob + g) * 128 + 16 * kt + 2 * c);
        a[1] = ld_u32(S.DA2T + (ob + g + 8) * 128 + 16 * kt + 2 * c);
        a[2] = ld_u32(S.DA2T + (ob + g) * 128 + 16 * kt + 2 * c + 8);
        a[3] = ld_u32(S.DA2T + (ob + g + 8) * 128 + 16 * kt + 2 * c + 8);
#pragma unroll
        for (int nt = 0; nt < 8; ++nt)
          mma_bf16_16816(acc[nt], a, ld_u32(S.H1T + (8 * nt + g) * 128 + 16 * kt + 2 * c),
                         ld_u32(S.H1T + (8 * nt + g) * 128 + 16 * kt + 2 * c + 8));
      }
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) {
        const int col = 8 * nt + 2 * c;
        S.g[kMlpOffW2 + (ob + g) * kMlpH + col] += acc[nt][0];
        S.g[kMlpOffW2 + (ob + g) * kMlpH + col + 1] += acc[nt][1];
        S.g[kMlpOffW2 + (ob + g + 8) * kMlpH + col] += acc[nt][2];
        S.g[kMlpOffW2 + (ob + g + 8) * kMlpH + col + 1] += acc[nt][3];
      }
      // gW1 = da1^T x, 2 n-tiles of 8 inputs (13 used)
      float acc1[2][4];
#pragma unroll
      for (int nt = 0; nt < 2; ++nt) acc1[nt][0] = acc1[nt][1] = acc1[nt][2] = acc1[nt][3] = 0.f;
#pragma unroll 2
      for (int kt = 0; kt < 8; ++kt) {
        uint32_t a[4];
        a[0] = ld_u32(S.DA1T + (ob + g) * 128 + 16 * kt + 2 * c);
        a[1] = ld_u32(S.DA1T + (ob + g + 8) * 128 + 16 * kt + 2 * c);
        a[2] = ld_u32(S.DA1T + (ob + g) * 128 + 16 * kt + 2 * c + 8);
        a[3] = ld_u32(S.DA1T + (ob + g + 8) * 128 + 16 * kt + 2 * c + 8);
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
          mma_bf16_16816(acc1[nt], a, ld_u32(S.XT + (8 * nt + g) * 128 + 16 * kt + 2 * c),
                         ld_u32(S.XT + (8 * nt + g) * 128 + 16 * kt + 2 * c + 8));
      }
#pragma unroll
      for (int nt = 0; nt < 2; ++nt) {
        const int col = 8 * nt + 2 * c;
        if (col < kMlpIn) {
          S.g[kMlpOffW1 + (ob + g) * kMlpIn + col] += acc1[nt][0];
          S.g[kMlpOffW1 + (ob + g + 8) * kMlpIn + col] += acc1[nt][2];
        }
        if (col + 1 < kMlpIn) {
          S.g[kMlpOffW1 + (ob + g) * kMlpIn + col + 1] += acc1[nt][1];
          S.g[kMlpOffW1 + (ob + g + 8) * kMlpIn + col + 1] += acc1[nt][3];
        }
      }
    }
    __syncthreads();
  }
  for (int q = t; q < kMlpNet; q += 128) atomicAdd(&grad[q], S.g[q]);
  if (t == 0) atomicAdd(loss, S.loss);
}

// Adam (Kingma & Ba 2015) on the network parameters of the FP32 vector.
__global__ void k_mlp_adam(float *__restrict__ p, const float *__restrict__ gr, float *__restrict__ m,
                           float *__restrict__ v, int count, float lr, float b1, float b2, float eps, float c1,
                           float c2) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= count) return;
  const float gq = gr[q];
  const float mq = b1 * m[q] + (1.0f - b1) * gq;
  const float vq = b2 * v[q] + (1.0f - b2) * gq * gq;
  m[q] = mq;
  v[q] = vq;
  p[q] -= lr * (mq / c1) / (sqrtf(vq / c2) + eps);
}

static int train_grid() {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  return nsm;
}

}  // namespace cmles

using namespace cmles;

extern "C" {

cmles_status cmles_mlp_forward(const float *params_dev, const float *X_dev, float *Y_dev, long long n, void *stream) {
  if (n == 0) return CMLES_OK;  // an empty batch: nothing to read or write
  if (!params_dev || !X_dev || !Y_dev || n < 0) return CMLES_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  MlpPacked *pk = nullptr;
  const size_t bytes = sizeof(MlpPacked) + 16;
  if (cudaMallocAsync((void **)&pk, bytes, s) != cudaSuccess) return CMLES_ERR_OOM;
  int *err = reinterpret_cast<int *>(reinterpret_cast<char *>(pk) + sizeof(MlpPacked));
  cudaMemsetAsync(err, 0, sizeof(int), s);
  k_pack_mlp<<<8, 256, 0, s>>>(params_dev, pk);
  static int grid = 0;
  if (!grid) grid = grid_for_tc((const void *)k_mlp_forward, 1 << 30, kTcCols);
  long long blocks = (n + 127) / 128;
  if (blocks > grid) blocks = grid;
  k_mlp_forward<<<(int)blocks, 128, 0, s>>>(pk, X_dev, Y_dev, n, err);
  int err_h = 0;
  const cudaError_t e1 = cudaGetLastError();
  const cudaError_t e2 = cudaMemcpyAsync(&err_h, err, sizeof(int), cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(pk, s);
  const cudaError_t e3 = cudaStreamSynchronize(s);
  if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) return CMLES_ERR_CUDA;
  return err_h ? CMLES_ERR_TIMEOUT : CMLES_OK;
}

cmles_status cmles_mlp_loss_grad(const float *params_dev, const float *X_dev, const float *T_dev, long long n,
                                 float *grad_dev, float *loss_dev, void *stream) {
  if (!params_dev || !X_dev || !T_dev || !grad_dev || !loss_dev || n <= 0) return CMLES_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  static bool attr = false;
  const int smem = (int)sizeof(TrainSmem);
  if (!attr) {
    if (cudaFuncSetAttribute(k_mlp_train, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
      return CMLES_ERR_CUDA;
    attr = true;
  }
  MlpPacked *pk = nullptr;
  if (cudaMallocAsync((void **)&pk, sizeof(MlpPacked), s) != cudaSuccess) return CMLES_ERR_OOM;
  k_pack_mlp<<<8, 256, 0, s>>>(params_dev, pk);
  cudaMemsetAsync(grad_dev, 0, kMlpNet * sizeof(float), s);
  cudaMemsetAsync(loss_dev, 0, sizeof(float), s);
  long long blocks = (n + 127) / 128;
  const int cap = train_grid();
  if (blocks > cap) blocks = cap;
  k_mlp_train<<<(int)blocks, 128, smem, s>>>(pk, X_dev, T_dev, n, grad_dev, loss_dev);
  cudaFreeAsync(pk, s);
  return cudaGetLastError() == cudaSuccess ? CMLES_OK : CMLES_ERR_CUDA;
}

cmles_status cmles_mlp_adam(float *params_dev, const float *grad_dev, float *m_dev, float *v_dev, int t, float lr,
                            float beta1, float beta2, float eps, void *stream) {
  if (!params_dev || !grad_dev || !m_dev || !v_dev || t < 1) return CMLES_ERR_ARG;
  const float c1 = 1.0f - powf(beta1, (float)t), c2 = 1.0f - powf(beta2, (float)t);
  k_mlp_adam<<<(kMlpNet + 255) / 256, 256, 0, (cudaStream_t)stream>>>(params_dev, grad_dev, m_dev, v_dev, kMlpNet,
                                                                      lr, beta1, beta2, eps, c1, c2);
  return cudaGetLastError() == cudaSuccess ? CMLES_OK : CMLES_ERR_CUDA;
}

}  // extern "C"
