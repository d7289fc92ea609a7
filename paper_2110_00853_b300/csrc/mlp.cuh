// Learned SGS closure network on tensor cores: 13 -> 64 -> 64 -> 2, SiLU
// hidden activations, BF16 weights and activations, FP32 accumulation.
// (The paper has no learned closure; this network extends its Sec. 4, with
// Smagorinsky-Lilly kept as fallback.)
//
// Inference (inside the gradient passes, and cmles_mlp_forward) and training
// (cmles_mlp_loss_grad) run on the tcgen05 tensor cores: one CTA per 128
// rows, thread t owning row t, operands in shared memory and accumulators in
// Tensor Memory (primitives in tc.cuh).
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

#include "tc.cuh"

namespace cmles {

constexpr int kMlpIn = 13, kMlpH = 64, kMlpOut = 2;
constexpr int kMlpInPad = 16;
// FP32 parameter vector: W1[64][13], b1[64], W2[64][64], b2[64], W3[2][64],
// b3[2], in_scale[13], out_scale[2]
constexpr int kMlpOffW1 = 0, kMlpOffB1 = 832, kMlpOffW2 = 896, kMlpOffB2 = 4992, kMlpOffW3 = 5056,
              kMlpOffB3 = 5184, kMlpOffIn = 5186, kMlpOffOut = 5199, kMlpParams = 5201, kMlpNet = 5186;

// Tensor-core (tcgen05) copy of the network used by the forward passes:
// the weights as K-major B operands in the core-matrix layout of tc.cuh,
// with the biases folded into the contraction.  Layer 1 has K = 16: the 13
// inputs and three columns on which the A operand holds 1 and W1 holds the
// bias b1 split as hi + mid + lo, three BF16 numbers whose sum is the FP32
// bias to 2^-27 relative.  Layers 2 and 3 have K = 80: the 64 hidden units,
// one group of 8 columns that holds (1, 1, 1, 0, ...) in A and the split
// bias in W, and one zero group (K steps of 16).  Layer 3 has N = 16 with
// output rows 2..15 zero.
constexpr int kTcKG1 = 2, kTcKG = 10, kTcN3 = 16;
struct __align__(16) MlpTc {
  __nv_bfloat16 W1[kMlpH * 8 * kTcKG1];   // [n/8][k/8][n%8][k%8]
  __nv_bfloat16 W2[kMlpH * 8 * kTcKG];
  __nv_bfloat16 W3[kTcN3 * 8 * kTcKG];
  float in_scale[kMlpInPad], out_scale[4];
};

// Packed device copy used by the kernels (16-byte aligned, size a multiple of
// 16 so that it can be staged into shared memory with 16-byte copies): the
// tensor-core forward operands, and W2, W3 row-major ([out][in], BF16) from
// which the training kernel builds its backward operands.
struct __align__(16) MlpPacked {
  __nv_bfloat16 W2[kMlpH * kMlpH];
  __nv_bfloat16 W3[kMlpOut * kMlpH];
  MlpTc tc;
};

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t *>(&v);
}

// SiLU with the fast exponential and division (relative error ~1e-6, far
// below the BF16 rounding of the activation that follows); for x -> -inf the
// fast division by +inf returns 0, the limit of x sigma(x).
__device__ __forceinline__ float silu(float x) { return __fdividef(x, 1.0f + __expf(-x)); }

// SiLU of the pair (x0, x1) packed as BF16x2, for the hidden activations of
// the forward pass: x sigma(x) = x / (1 + 2^(-x log2 e)), with the multiplies
// and the add done two at a time by the packed FP32 instructions (f32x2, one
// instruction for both values, each rounded as the scalar operation) and the
// exponential and reciprocal on the MUFU unit (flush-to-zero; relative error
// a few 1e-7, far below the BF16 rounding that follows).  For x -> -inf the
// reciprocal of +inf is 0, the limit of x sigma(x); for x -> +inf it is x.
__device__ __forceinline__ uint32_t silu2_bf16(float x0, float x1) {
  uint64_t xv, t, dv, rv, hv;
  asm("mov.b64 %0, {%1, %2};" : "=l"(xv) : "f"(x0), "f"(x1));
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(t) : "l"(xv), "l"(0xBFB8AA3BBFB8AA3Bull));  // -log2(e) twice
  float t0, t1, e0, e1, r0, r1, h0, h1;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(t0), "=f"(t1) : "l"(t));
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e0) : "f"(t0));
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e1) : "f"(t1));
  asm("mov.b64 %0, {%1, %2};" : "=l"(dv) : "f"(e0), "f"(e1));
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(dv) : "l"(dv), "l"(0x3F8000003F800000ull));  // + (1, 1)
  float d0, d1;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(d0), "=f"(d1) : "l"(dv));
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r0) : "f"(d0));
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r1) : "f"(d1));
  asm("mov.b64 %0, {%1, %2};" : "=l"(rv) : "f"(r0), "f"(r1));
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(hv) : "l"(xv), "l"(rv));
  asm("mov.b64 {%0, %1}, %2;" : "=f"(h0), "=f"(h1) : "l"(hv));
  return pack_bf16(h0, h1);
}

// ---------------------------------------------------------------------------
// Inference on the fifth-generation tensor cores (tcgen05): one CTA of 128
// threads evaluates 128 rows, thread t owning row t.  Each layer is one MMA
// chain of M = 128 rows issued by thread 0 (A: the rows' inputs or hidden
// activations in shared memory; B: the layer's weights in shared memory;
// D: 64 FP32 columns of Tensor Memory), whose completion arrives on an
// mbarrier; every thread then reads its row of D from TMEM (lane t), applies
// SiLU and writes the BF16 activations back as the next layer's A operand.
//
// The A buffer holds 128 rows x 80 columns (kTcKG groups): columns 64..66 are
// the bias columns (1.0) of layers 2 and 3 and 67..79 are zero; the layer-1
// inputs occupy columns 0..15 (13 inputs, then three 1.0 bias columns).

constexpr int kTcAElems = 128 * 8 * kTcKG;  // A buffer, BF16 elements (20 KB)
constexpr int kTcCols = 64;                 // TMEM columns per CTA (per row tile)
// TMEM columns of a CTA with T row tiles of 128 rows: 64 per tile, the
// allocation rounded up to a power of two
__host__ __device__ constexpr int tc_cols_for(int T) { return T <= 1 ? 64 : (T == 2 ? 128 : 256); }
constexpr int kTcWaitLimit = 1 << 20;       // mbarrier tries before giving up

struct TcState {
  uint32_t tmem;    // TMEM base address of this CTA's columns
  uint64_t *mbar;   // MMA completion barrier (shared memory)
  uint32_t parity;  // parity of the next phase to complete
  int err;          // sticky: a wait gave up (results of this CTA invalid)
  int hook;         // test hook (instances built for it only): the next wait gives up at once
};

// The committed phase that thread 0 has not seen complete, as 1 + its
// parity (0: none), kept in shared memory rather than in registers: it is
// written only when a wait gives up and read only by the tear-down.
__device__ __forceinline__ uint32_t &tc_pending() {
  __shared__ uint32_t pending;
  return pending;
}

// Write this thread's row of the A buffer for layer 1: the 13 inputs (BF16),
// the three bias columns, and the bias and zero groups of layers 2 and 3
// (columns 64..79; rewritten every time, so the buffer may share storage
// with other data between calls).  With T row tiles (CTAs of more than 128
// threads) thread t writes row t % 128 of tile t / 128, the tiles kTcAElems
// apart.
template <int T = 1>
__device__ __forceinline__ void mlp_tc_put_input(__nv_bfloat16 *A, const float x[kMlpIn]) {
  const int t = T > 1 ? (int)(threadIdx.x & 127) : (int)threadIdx.x;
  if (T > 1) A += (threadIdx.x >> 7) * kTcAElems;
  const uint32_t one2 = pack_bf16(1.0f, 1.0f);
  *reinterpret_cast<uint4 *>(A + tc_off(t, 0, kTcKG)) =
      make_uint4(pack_bf16(x[0], x[1]), pack_bf16(x[2], x[3]), pack_bf16(x[4], x[5]), pack_bf16(x[6], x[7]));
  *reinterpret_cast<uint4 *>(A + tc_off(t, 8, kTcKG)) =
      make_uint4(pack_bf16(x[8], x[9]), pack_bf16(x[10], x[11]), pack_bf16(x[12], 1.0f), one2);
  *reinterpret_cast<uint4 *>(A + tc_off(t, 64, kTcKG)) = make_uint4(one2, pack_bf16(1.0f, 0.0f), 0u, 0u);
  *reinterpret_cast<uint4 *>(A + tc_off(t, 72, kTcKG)) = make_uint4(0u, 0u, 0u, 0u);
}

// Set-up of a CTA's tensor-core state: TMEM columns (allocated by warp 0)
// and the MMA completion barrier (initialised by thread 0).  All threads must
// call it; it ends with a block barrier.
__device__ __forceinline__ void tc_setup(TcState &s, uint32_t *slot, uint64_t *mbar, uint32_t ncols = kTcCols) {
  if (threadIdx.x < 32) tc_alloc(slot, ncols);
  if (threadIdx.x == 0) {
    mbar_init(mbar, 1);
    tc_pending() = 0u;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  tc_fence_before_sync();
  __syncthreads();
  tc_fence_after_sync();
  s.tmem = *slot;
  s.mbar = mbar;
  s.parity = 0;
  s.err = 0;
  s.hook = 0;
}

// Wait (bounded) for the MMAs thread 0 has committed.  A wait that gives up
// sets the sticky error flag; thread 0 records the phase it has not seen
// complete, which the tear-down waits for before freeing the columns.  Once
// the flag is set thread 0 issues and commits nothing more and later waits
// make one try, so a failing CTA runs through its remaining work quickly (its
// results are reported invalid).  HOOK instances (test hook 2) give up on
// their first wait at once (s.hook).
template <bool HOOK = false>
__device__ __forceinline__ void tc_wait_group(TcState &s) {
  bool ok;
  if (HOOK && s.hook) {
    s.hook = 0;
    ok = false;
  } else {
    ok = mbar_wait_bounded(s.mbar, s.parity, s.err ? 1 : kTcWaitLimit);
  }
  if (!ok) {
    if (!s.err && threadIdx.x == 0) tc_pending() = 1u + s.parity;
    s.err = 1;
  }
  s.parity ^= 1u;
  __syncwarp();  // the TMEM loads that follow are warp-collective
  tc_fence_after_sync();
}

// Tear-down: thread 0 waits (bounded) for a committed phase it has not seen
// complete (commits complete in order and thread 0 commits nothing after a
// wait gave up, so that phase is the last one), so that no MMA of the CTA
// still runs when the TMEM columns are freed; the CTA is counted once in
// *err_count if any of its waits gave up.  All threads must call it.
__device__ __forceinline__ void tc_teardown(TcState &s, int *err_count, uint32_t ncols = kTcCols) {
  tc_fence_before_sync();
  const int any_err = __syncthreads_or(s.err);
  if (threadIdx.x == 0) {
    const uint32_t pend = tc_pending();
    if (pend) mbar_wait_bounded(s.mbar, pend - 1u, kTcWaitLimit);
  }
  tc_fence_before_sync();
  __syncthreads();
  if (threadIdx.x < 32) {
    tc_fence_after_sync();
    tc_dealloc(s.tmem, ncols);
  }
  if (threadIdx.x == 0 && any_err) atomicAdd(err_count, 1);
}

// One MMA group of the CTA: every thread makes its shared-memory operand
// writes visible to the tensor core and meets the others (tc_group_open);
// thread 0 then issues the group's MMAs unless one of its waits has given up;
// tc_group_close commits them to the barrier and waits for their completion
// in every thread (tc_wait_group).
__device__ __forceinline__ void tc_group_open() {
  fence_proxy_async_smem();
  tc_fence_before_sync();
  __syncthreads();
}
__device__ __forceinline__ void tc_group_close(TcState &s) {
  if (threadIdx.x == 0 && !s.err) tc_commit(s.mbar);
  tc_wait_group(s);
}

// Forward pass of the CTA's 128 T rows; (y0, y1) of this thread's row.  All
// threads must call it (it contains block barriers).  The A buffer's
// layer-1 columns must have been written by every thread and the bias and
// zero groups (columns 64..79) set.  T row tiles (CTAs of more than 128
// threads): thread 0 issues one chain per tile, tile q's A operand kTcAElems
// elements after tile 0's and its accumulator in TMEM columns 64 q ..
// 64 q + 63; thread t owns row t % 128 of tile t / 128, which its warp reads
// in TMEM lane t % 128 (warp w reads lanes 32 (w % 4) .. 32 (w % 4) + 31).
// Rows of the last tile beyond the CTA's threads are never written or read;
// an MMA row depends on its own A row only.
template <bool HOOK = false, int T = 1>
__device__ __forceinline__ void mlp_tc_forward(const MlpTc &W, __nv_bfloat16 *A, TcState &s, float &y0,
                                               float &y1) {
  const int t = threadIdx.x;
  const int row = T > 1 ? (t & 127) : t;
  const uint32_t lane_base = s.tmem + ((uint32_t)(row & ~31) << 16) + (T > 1 ? (uint32_t)(t >> 7) * kTcCols : 0u);
  __nv_bfloat16 *Arow = T > 1 ? A + (t >> 7) * kTcAElems : A;
  constexpr uint32_t kSboA = 8 * 16 * kTcKG, kSbo1 = 8 * 16 * kTcKG1;
#pragma unroll 1
  for (int layer = 0; layer < 3; ++layer) {
    fence_proxy_async_smem();
    tc_fence_before_sync();
    __syncthreads();
    if (t == 0 && !s.err) {
      tc_fence_after_sync();
#pragma unroll
      for (int q = 0; q < T; ++q) {
        const __nv_bfloat16 *Aq = A + q * kTcAElems;
        const uint32_t dq = s.tmem + (uint32_t)q * kTcCols;
        if (layer == 0) {
          tc_mma(dq, tc_sdesc(Aq, 128, kSboA), tc_sdesc(W.W1, 128, kSbo1), tc_idesc_bf16(128, kMlpH), 0u);
        } else {
          const __nv_bfloat16 *B = layer == 1 ? W.W2 : W.W3;
          const uint32_t idesc = tc_idesc_bf16(128, layer == 1 ? kMlpH : kTcN3);
#pragma unroll
          for (int ks = 0; ks < kTcKG / 2; ++ks)
            tc_mma(dq, tc_sdesc(Aq + ks * 128, 128, kSboA), tc_sdesc(B + ks * 128, 128, kSboA), idesc,
                   ks > 0 ? 1u : 0u);
        }
      }
      tc_commit(s.mbar);
    }
    tc_wait_group<HOOK>(s);
    // the test instance reads no TMEM once its wait gave up (its MMA may
    // still be writing it) and leaves the drain to the tear-down
    const bool skip = HOOK && s.err;
    if (layer < 2) {
      // eight columns per TMEM load: the gradient pass that calls this holds
      // its gradients across the network at its 80-register limit, and
      // smaller batches leave the SiLU more registers (32 columns per load:
      // 21.1 ms per pass on the 256M-node box, 16: 20.9, 8: 20.7, 4: 20.7)
#pragma unroll
      for (int h = 0; h < 8; ++h) {
        float v[8];
        if (skip) {
#pragma unroll
          for (int q = 0; q < 8; ++q) v[q] = 0.f;
        } else {
          tc_ld8(lane_base + 8 * h, v);
        }
        uint32_t w[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) w[q] = silu2_bf16(v[2 * q], v[2 * q + 1]);
        *reinterpret_cast<uint4 *>(Arow + tc_off(row, 8 * h, kTcKG)) = make_uint4(w[0], w[1], w[2], w[3]);
      }
    } else if (skip) {
      y0 = y1 = 0.f;
    } else {
      tc_ld2(lane_base, y0, y1);
    }
  }
}

}  // namespace cmles
