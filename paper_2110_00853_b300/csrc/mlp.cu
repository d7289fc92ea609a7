// Learned-closure network: weight packing, batched inference, BF16
// tensor-core training step (forward, backward, weight gradients) and Adam.
//
// Loss: L = 1/(2n) sum_s |y_s - t_s|^2 over the n samples of a call.
// Backward (per sample, FP32 with BF16 tensor-core products):
//   dy = (y - t)/n,  dh2 = W3^T dy,  da2 = dh2 * silu'(a2),
//   dh1 = W2^T da2,  da1 = dh1 * silu'(a1),  silu'(a) = s (1 + a (1 - s)),
//   gW3 += dy h2^T, gW2 += da2 h1^T, gW1 += da1 x^T, gb_l += da_l.
// One CTA of 128 threads handles 128 samples per iteration (one sample per
// thread for pointwise work; the products on the tcgen05 tensor cores) and
// keeps its gradient partial sums in shared memory and Tensor Memory until
// the end.
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

// Row-major BF16 copies of W2 and W3, entry q of [out][in].
__host__ __device__ inline void rowmajor_fill(const float *p, MlpPacked *o, int q) {
  if (q < kMlpH * kMlpH) o->W2[q] = __float2bfloat16_rn(p[kMlpOffW2 + q]);
  if (q < kMlpOut * kMlpH) o->W3[q] = __float2bfloat16_rn(p[kMlpOffW3 + q]);
}

void pack_mlp_host(const float *p, MlpPacked *o) {
  memset(o, 0, sizeof(*o));
  for (int q = 0; q < kMlpH * kMlpH; ++q) rowmajor_fill(p, o, q);
  for (int q = 0; q < kMlpH * 8 * kTcKG; ++q) tc_fill(p, &o->tc, q);
}

__global__ void k_pack_mlp(const float *__restrict__ p, MlpPacked *__restrict__ o) {
  const int t = threadIdx.x + blockIdx.x * blockDim.x, nt = blockDim.x * gridDim.x;
  for (int q = t; q < kMlpH * kMlpH; q += nt) rowmajor_fill(p, o, q);
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

// One CTA of 128 threads per SM; each iteration takes 128 samples (thread t
// owns sample t) through the forward pass and the backward products on the
// tcgen05 tensor cores, with every accumulator in Tensor Memory:
//   forward  a1 = W1 x + b1, a2 = W2 h1 + b2, y = W3 h2 + b3 (biases folded
//            as in inference); a1 stays in TMEM for the backward pass;
//   dh1      = da2 W2 (M = 128 samples, N = 64, K = 64);
//   gW2     += da2^T h1 and gW1 += da1^T x (K = 128 samples), accumulated in
//            TMEM over all the CTA's iterations: one A operand holds da2^T
//            (rows 0..63) and da1^T (rows 64..127), so each product is one
//            M = 128 chain whose other half is discarded.
// gW3, the bias gradients and the loss are FP32 sums in shared memory.
constexpr uint32_t kTrCols = 512;  // TMEM columns (one CTA per SM)
constexpr int kTrA1 = 0, kTrA2 = 64, kTrY = 128, kTrDH1 = 192, kTrGW2 = 256, kTrGW1 = 320;

struct TrainSmem {
  MlpTc W;                           // forward B operands
  __nv_bfloat16 Aop[kTcAElems];      // forward A operand, 128 x 80
  __nv_bfloat16 W2T[kMlpH * kMlpH];  // B of dh1: [in][out], 8 groups
  __nv_bfloat16 DA2[128 * kMlpH];    // A of dh1: [sample][out], 8 groups
  __nv_bfloat16 AC[128 * 128];       // A of gW2 / gW1: [da2^T; da1^T], [unit][sample], 16 groups
  __nv_bfloat16 H1T[kMlpH * 128];    // B of gW2: [in unit][sample], 16 groups
  __nv_bfloat16 XT[16 * 128];        // B of gW1: [input][sample], 16 groups
  float A2[128 * kMlpH];             // layer-2 pre-activations
  float DY[128 * 2];
  float W3f[kMlpOut * kMlpH];        // W3 (its BF16 values)
  float g[kMlpNet];                  // gradient partial sums (parameter-vector layout)
  float loss;
  uint64_t bar;
  uint32_t slot;
};

__device__ __forceinline__ float dsilu(float a) {
  const float sg = __fdividef(1.0f, 1.0f + __expf(-a));
  return sg * (1.0f + a * (1.0f - sg));
}

__global__ void __launch_bounds__(128) k_mlp_train(const MlpPacked *__restrict__ Wg, const float *__restrict__ X,
                                                   const float *__restrict__ T, long long n,
                                                   float *__restrict__ grad, float *__restrict__ loss,
                                                   int *err_count) {
  extern __shared__ __align__(128) uint8_t smem_raw[];
  TrainSmem &S = *reinterpret_cast<TrainSmem *>(smem_raw);
  const int t = threadIdx.x, warp = t >> 5;
  for (int q = t; q < (int)(sizeof(MlpTc) / 16); q += 128)
    reinterpret_cast<uint4 *>(&S.W)[q] = reinterpret_cast<const uint4 *>(&Wg->tc)[q];
  for (int q = t; q < kMlpH * kMlpH; q += 128) {
    const int in = q / kMlpH, out = q % kMlpH;
    S.W2T[tc_off(in, out, 8)] = Wg->W2[out * kMlpH + in];
  }
  for (int q = t; q < kMlpOut * kMlpH; q += 128)
    S.W3f[q] = __bfloat162float(Wg->W3[q]);
  for (int q = t; q < kMlpNet; q += 128) S.g[q] = 0.f;
  if (t == 0) S.loss = 0.f;
  fence_proxy_async_smem();
  TcState st;
  tc_setup(st, &S.slot, &S.bar, kTrCols);
  const uint32_t lane_base = st.tmem + ((uint32_t)(t & ~31) << 16);
  constexpr uint32_t kSboA = 8 * 16 * kTcKG, kSbo1 = 8 * 16 * kTcKG1, kSbo8 = 8 * 16 * 8, kSbo16 = 8 * 16 * 16;
  const float inv_n = 1.0f / (float)n;
  bool first = true;
  for (long long b = (long long)blockIdx.x * 128; b < n; b += (long long)gridDim.x * 128) {
    const long long s = b + t;
    const bool valid = s < n;
    float x[kMlpIn];
#pragma unroll
    for (int k = 0; k < kMlpIn; ++k) x[k] = valid ? X[s * kMlpIn + k] : 0.f;
    mlp_tc_put_input(S.Aop, x);
#pragma unroll
    for (int k = 0; k < 16; ++k) S.XT[tc_off(k, t, 16)] = __float2bfloat16_rn(k < kMlpIn ? x[k] : 0.f);
    // ---- forward, layer 1 (a1 kept in TMEM)
    tc_group_open();
    if (t == 0 && !st.err) {
      tc_fence_after_sync();
      tc_mma(st.tmem + kTrA1, tc_sdesc(S.Aop, 128, kSboA), tc_sdesc(S.W.W1, 128, kSbo1), tc_idesc_bf16(128, kMlpH),
             0u);
    }
    tc_group_close(st);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      float v[32];
      tc_ld32(lane_base + kTrA1 + 32 * h, v);
      uint32_t w[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        w[q] = silu2_bf16(v[2 * q], v[2 * q + 1]);
        S.H1T[tc_off(32 * h + 2 * q, t, 16)] = __ushort_as_bfloat16((unsigned short)(w[q] & 0xFFFFu));
        S.H1T[tc_off(32 * h + 2 * q + 1, t, 16)] = __ushort_as_bfloat16((unsigned short)(w[q] >> 16));
      }
#pragma unroll
      for (int kk = 0; kk < 4; ++kk)
        *reinterpret_cast<uint4 *>(S.Aop + tc_off(t, 32 * h + 8 * kk, kTcKG)) =
            make_uint4(w[4 * kk], w[4 * kk + 1], w[4 * kk + 2], w[4 * kk + 3]);
    }
    // ---- layer 2 (a2 to shared memory)
    tc_group_open();
    if (t == 0 && !st.err) {
      tc_fence_after_sync();
#pragma unroll
      for (int ks = 0; ks < kTcKG / 2; ++ks)
        tc_mma(st.tmem + kTrA2, tc_sdesc(S.Aop + ks * 128, 128, kSboA), tc_sdesc(S.W.W2 + ks * 128, 128, kSboA),
               tc_idesc_bf16(128, kMlpH), ks > 0 ? 1u : 0u);
    }
    tc_group_close(st);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      float v[32];
      tc_ld32(lane_base + kTrA2 + 32 * h, v);
      uint32_t w[16];
#pragma unroll
      for (int q = 0; q < 32; ++q) S.A2[t * kMlpH + 32 * h + q] = v[q];
#pragma unroll
      for (int q = 0; q < 16; ++q) w[q] = silu2_bf16(v[2 * q], v[2 * q + 1]);
#pragma unroll
      for (int kk = 0; kk < 4; ++kk)
        *reinterpret_cast<uint4 *>(S.Aop + tc_off(t, 32 * h + 8 * kk, kTcKG)) =
            make_uint4(w[4 * kk], w[4 * kk + 1], w[4 * kk + 2], w[4 * kk + 3]);
    }
    // ---- layer 3
    tc_group_open();
    if (t == 0 && !st.err) {
      tc_fence_after_sync();
#pragma unroll
      for (int ks = 0; ks < kTcKG / 2; ++ks)
        tc_mma(st.tmem + kTrY, tc_sdesc(S.Aop + ks * 128, 128, kSboA), tc_sdesc(S.W.W3 + ks * 128, 128, kSboA),
               tc_idesc_bf16(128, kTcN3), ks > 0 ? 1u : 0u);
    }
    tc_group_close(st);
    float y0, y1;
    tc_ld2(lane_base + kTrY, y0, y1);
    // output error and loss
    float dy0 = 0.f, dy1 = 0.f;
    if (valid) {
      const float r0 = y0 - T[s * 2], r1 = y1 - T[s * 2 + 1];
      atomicAdd(&S.loss, 0.5f * (r0 * r0 + r1 * r1) * inv_n);
      dy0 = r0 * inv_n;
      dy1 = r1 * inv_n;
    }
    S.DY[2 * t] = dy0;
    S.DY[2 * t + 1] = dy1;
    __syncthreads();
    {
      // gW3 and gb3: thread t takes output unit o = t / 64, hidden unit i = t % 64
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
    // da2 = (W3^T dy) * silu'(a2) for sample t
    for (int i = 0; i < kMlpH; ++i) {
      const float da = (S.W3f[i] * dy0 + S.W3f[kMlpH + i] * dy1) * dsilu(S.A2[t * kMlpH + i]);
      const __nv_bfloat16 db = __float2bfloat16_rn(da);
      S.DA2[tc_off(t, i, 8)] = db;
      S.AC[tc_off(i, t, 16)] = db;
      atomicAdd(&S.g[kMlpOffB2 + i], da);
    }
    // ---- dh1 = da2 W2
    tc_group_open();
    if (t == 0 && !st.err) {
      tc_fence_after_sync();
#pragma unroll
      for (int ks = 0; ks < 4; ++ks)
        tc_mma(st.tmem + kTrDH1, tc_sdesc(S.DA2 + ks * 128, 128, kSbo8), tc_sdesc(S.W2T + ks * 128, 128, kSbo8),
               tc_idesc_bf16(128, kMlpH), ks > 0 ? 1u : 0u);
    }
    tc_group_close(st);
    // da1 = dh1 * silu'(a1) for sample t (zero for the padding samples)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      float dh[32], a1[32];
      tc_ld32(lane_base + kTrDH1 + 32 * h, dh);
      tc_ld32(lane_base + kTrA1 + 32 * h, a1);
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        const float da = valid ? dh[q] * dsilu(a1[q]) : 0.f;
        S.AC[tc_off(kMlpH + 32 * h + q, t, 16)] = __float2bfloat16_rn(da);
        if (valid) atomicAdd(&S.g[kMlpOffB1 + 32 * h + q], da);
      }
    }
    // ---- gW2 += da2^T h1 and gW1 += da1^T x over the 128 samples
    tc_group_open();
    if (t == 0 && !st.err) {
      tc_fence_after_sync();
#pragma unroll
      for (int ks = 0; ks < 8; ++ks)
        tc_mma(st.tmem + kTrGW2, tc_sdesc(S.AC + ks * 128, 128, kSbo16), tc_sdesc(S.H1T + ks * 128, 128, kSbo16),
               tc_idesc_bf16(128, kMlpH), (!first || ks > 0) ? 1u : 0u);
#pragma unroll
      for (int ks = 0; ks < 8; ++ks)
        tc_mma(st.tmem + kTrGW1, tc_sdesc(S.AC + ks * 128, 128, kSbo16), tc_sdesc(S.XT + ks * 128, 128, kSbo16),
               tc_idesc_bf16(128, 16), (!first || ks > 0) ? 1u : 0u);
    }
    tc_group_close(st);
    first = false;
  }
  // weight gradients out of TMEM: gW2 in rows 0..63 (warps 0, 1), gW1 in rows
  // 64..127 (warps 2, 3)
  if (!first) {
    if (warp < 2) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        float v[32];
        tc_ld32(lane_base + kTrGW2 + 32 * h, v);
#pragma unroll
        for (int q = 0; q < 32; ++q) S.g[kMlpOffW2 + t * kMlpH + 32 * h + q] += v[q];
      }
    } else {
      float v[32];
      tc_ld32(lane_base + kTrGW1, v);
#pragma unroll
      for (int k = 0; k < kMlpIn; ++k) S.g[kMlpOffW1 + (t - kMlpH) * kMlpIn + k] += v[k];
    }
  }
  __syncthreads();
  for (int q = t; q < kMlpNet; q += 128) atomicAdd(&grad[q], S.g[q]);
  if (t == 0) atomicAdd(loss, S.loss);
  tc_teardown(st, err_count, kTrCols);
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
  if (cudaMallocAsync((void **)&pk, sizeof(MlpPacked) + 16, s) != cudaSuccess) return CMLES_ERR_OOM;
  int *err = reinterpret_cast<int *>(reinterpret_cast<char *>(pk) + sizeof(MlpPacked));
  cudaMemsetAsync(err, 0, sizeof(int), s);
  k_pack_mlp<<<8, 256, 0, s>>>(params_dev, pk);
  cudaMemsetAsync(grad_dev, 0, kMlpNet * sizeof(float), s);
  cudaMemsetAsync(loss_dev, 0, sizeof(float), s);
  long long blocks = (n + 127) / 128;
  const int cap = train_grid();
  if (blocks > cap) blocks = cap;
  // one CTA per SM (its shared memory exceeds half the SM's), so its 512
  // Tensor Memory columns are always free
  k_mlp_train<<<(int)blocks, 128, smem, s>>>(pk, X_dev, T_dev, n, grad_dev, loss_dev, err);
  int err_h = 0;
  const cudaError_t e1 = cudaGetLastError();
  const cudaError_t e2 = cudaMemcpyAsync(&err_h, err, sizeof(int), cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(pk, s);
  const cudaError_t e3 = cudaStreamSynchronize(s);
  if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) return CMLES_ERR_CUDA;
  return err_h ? CMLES_ERR_TIMEOUT : CMLES_OK;
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
