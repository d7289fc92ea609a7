// Learned SGS closure network on tensor cores: 13 -> 64 -> 64 -> 2, SiLU
// hidden activations, BF16 weights and activations, FP32 accumulation.
// (The paper has no learned closure; this network extends its Sec. 4, with
// Smagorinsky-Lilly kept as fallback.)
//
// One warp evaluates 32 rows (two m16 tiles) with mma.sync m16n8k16 BF16.
// The accumulator fragment of two neighbouring n8 tiles is exactly the A
// fragment of the next layer's k16 tile, so hidden activations never leave
// registers.  Weights are stored out-major with the input index contiguous
// (W[n][k]), which is the k-contiguous B layout the instruction wants.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace cmles {

constexpr int kMlpIn = 13, kMlpH = 64, kMlpOut = 2;
constexpr int kMlpInPad = 16, kMlpOutPad = 8;
// FP32 parameter vector: W1[64][13], b1[64], W2[64][64], b2[64], W3[2][64],
// b3[2], in_scale[13], out_scale[2]
constexpr int kMlpOffW1 = 0, kMlpOffB1 = 832, kMlpOffW2 = 896, kMlpOffB2 = 4992, kMlpOffW3 = 5056,
              kMlpOffB3 = 5184, kMlpOffIn = 5186, kMlpOffOut = 5199, kMlpParams = 5201, kMlpNet = 5186;

// Row stride of W2 and W3 in the packed copy: 72 BF16 = 144 B, so the eight
// rows g = 0..7 that one B-fragment load touches start in eight different
// 4-bank groups (a 128 B stride would put all eight on the same banks).
constexpr int kLdW = 72;
// Row stride of W1: 24 BF16 = 48 B, so that eight consecutive rows fall in
// eight different 16-byte bank groups for ldmatrix (32 B would pair them).
constexpr int kLdW1 = 24;

// Packed device copy used by the kernels (16-byte aligned, size a multiple of
// 16 so that it can be staged into shared memory with 16-byte copies).
struct __align__(16) MlpPacked {
  __nv_bfloat16 W1[kMlpH * kLdW1];       // [64][24], k >= 13 zero
  __nv_bfloat16 W2[kMlpH * kLdW];        // [64][72], k >= 64 zero
  __nv_bfloat16 W3[kMlpOutPad * kLdW];   // [8][72], n >= 2 or k >= 64 zero
  float b1[kMlpH], b2[kMlpH], b3[kMlpOutPad];
  float in_scale[kMlpInPad], out_scale[2];
};

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t *>(&v);
}

__device__ __forceinline__ void mma_bf16_16816(float d[4], const uint32_t a[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
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

__device__ __forceinline__ uint32_t ld_u32(const __nv_bfloat16 *p) { return *reinterpret_cast<const uint32_t *>(p); }

// ldmatrix: four (x4) or two (x2) 8x8 BF16 tiles from shared memory; lane l
// gives the address of row l % 8 of tile l / 8 (16-byte aligned), and
// register m of lane (g, c) receives elements 2c, 2c + 1 of row g of tile m,
// which for a weight tile stored [n][k] is the B fragment of mma m16n8k16.
__device__ __forceinline__ void ldsm_x4(uint32_t r[4], const __nv_bfloat16 *p) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}
__device__ __forceinline__ void ldsm_x2(uint32_t r[2], const __nv_bfloat16 *p) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];\n" : "=r"(r[0]), "=r"(r[1]) : "r"(a));
}

// Forward pass of the 32 rows [r0, r0 + 32) of X (bf16 [rows][16], shared
// memory) by one warp; writes Y[row][0..1] (FP32, shared memory).
// Optionally stores the pre-activations of both hidden layers (FP32,
// [rows][64] each) for the backward pass.
__device__ __forceinline__ void mlp_warp_forward(const MlpPacked &W, const __nv_bfloat16 *X, float *Y, int r0,
                                                 float *A1 = nullptr, float *A2 = nullptr, int lda = 0) {
  const int lane = threadIdx.x & 31, g = lane >> 2, c = lane & 3;
#pragma unroll 1
  for (int mt = 0; mt < 2; ++mt) {
    const int rb = r0 + 16 * mt;
    uint32_t a[4];
    a[0] = ld_u32(X + (rb + g) * kMlpInPad + 2 * c);
    a[1] = ld_u32(X + (rb + g + 8) * kMlpInPad + 2 * c);
    a[2] = ld_u32(X + (rb + g) * kMlpInPad + 2 * c + 8);
    a[3] = ld_u32(X + (rb + g + 8) * kMlpInPad + 2 * c + 8);
    // layer 1: 8 n-tiles, one k-tile; outputs repacked as 4 k-tiles of layer 2
    uint32_t h1[4][4];
    // ldmatrix row address of this lane: tile lane / 8, row lane % 8
    const int lr = lane & 7, lt = lane >> 3;
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      float d[4];
      d[0] = d[2] = W.b1[8 * nt + 2 * c];
      d[1] = d[3] = W.b1[8 * nt + 2 * c + 1];
      uint32_t b[2];
      ldsm_x2(b, W.W1 + (8 * nt + lr) * kLdW1 + 8 * (lt & 1));
      mma_bf16_16816(d, a, b[0], b[1]);
      if (A1) {
        A1[(rb + g) * lda + 8 * nt + 2 * c] = d[0];
        A1[(rb + g) * lda + 8 * nt + 2 * c + 1] = d[1];
        A1[(rb + g + 8) * lda + 8 * nt + 2 * c] = d[2];
        A1[(rb + g + 8) * lda + 8 * nt + 2 * c + 1] = d[3];
      }
      const int kt = nt >> 1, hi = nt & 1;
      h1[kt][0 + 2 * hi] = silu2_bf16(d[0], d[1]);
      h1[kt][1 + 2 * hi] = silu2_bf16(d[2], d[3]);
    }
    // layer 2 and 3
    float y[4] = {0.f, 0.f, 0.f, 0.f};
    y[0] = y[2] = W.b3[2 * c];
    y[1] = y[3] = W.b3[2 * c + 1];
    uint32_t h2[4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      float d[4];
      d[0] = d[2] = W.b2[8 * nt + 2 * c];
      d[1] = d[3] = W.b2[8 * nt + 2 * c + 1];
#pragma unroll
      for (int kp = 0; kp < 2; ++kp) {
        // tiles: (k-tile 2kp, low 8), (2kp, high 8), (2kp+1, low), (2kp+1, high)
        uint32_t b[4];
        ldsm_x4(b, W.W2 + (8 * nt + lr) * kLdW + 32 * kp + 8 * lt);
        mma_bf16_16816(d, h1[2 * kp], b[0], b[1]);
        mma_bf16_16816(d, h1[2 * kp + 1], b[2], b[3]);
      }
      if (A2) {
        A2[(rb + g) * lda + 8 * nt + 2 * c] = d[0];
        A2[(rb + g) * lda + 8 * nt + 2 * c + 1] = d[1];
        A2[(rb + g + 8) * lda + 8 * nt + 2 * c] = d[2];
        A2[(rb + g + 8) * lda + 8 * nt + 2 * c + 1] = d[3];
      }
      const int hi = nt & 1;
      h2[0 + 2 * hi] = silu2_bf16(d[0], d[1]);
      h2[1 + 2 * hi] = silu2_bf16(d[2], d[3]);
      if (hi) {  // a full k-tile of layer 3 is ready
        const int kt = nt >> 1;
        uint32_t b[2];
        ldsm_x2(b, W.W3 + lr * kLdW + 16 * kt + 8 * (lt & 1));
        mma_bf16_16816(y, h2, b[0], b[1]);
      }
    }
    if (c == 0) {
      Y[(rb + g) * 2 + 0] = y[0];
      Y[(rb + g) * 2 + 1] = y[1];
      Y[(rb + g + 8) * 2 + 0] = y[2];
      Y[(rb + g + 8) * 2 + 1] = y[3];
    }
  }
}

}  // namespace cmles
