// Learned reconstruction selector: a 15 -> 32 -> 32 -> 1 perceptron with GELU
// (tanh form) that reads the compressed consecutive variations of three
// characteristic fields over a face's six-cell stencil and predicts whether
// WENO5-JS is needed or the linear 5th-order reconstruction suffices for the
// acoustic and entropy fields (the shear fields keep WENO5).  The paper has no
// selector; it is the learned component of this GPU design, with WENO5-JS as
// its fallback and as the reference its labels and error are measured against.
//
// Inference runs on the tensor cores: a warp evaluates 32 faces at once as a
// 32 x 16 @ 16 x 32 -> 32 x 32 @ 32 x 32 -> 32 x 32 @ 32 x 8 chain of
// mma.sync.m16n8k16 (BF16 operands, FP32 accumulation).  Biases enter as the
// accumulator's initial value; the FP32 result fragments of one layer are
// packed to BF16, passed through the GELU in packed BF16 arithmetic
// (tanh.approx.bf16x2), and reused directly as the A fragments of the next
// layer.
//
// Parameters (FP32 master copy, MRB_MLP_NPARAM = 1601 floats): W1[32][15],
// b1[32], W2[32][32], b2[32], w3[32], b3.  The kernels round the weights to
// BF16 when they stage them.
#pragma once

#include <cuda_bf16.h>

#include "kernels.cuh"

namespace mrb {

constexpr int MLP_IN = 15, MLP_H = 32;
constexpr int MLP_NPARAM = MLP_H * MLP_IN + MLP_H + MLP_H * MLP_H + MLP_H + MLP_H + 1;   // 1601
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + MLP_H * MLP_IN, OFF_W2 = OFF_B1 + MLP_H, OFF_B2 = OFF_W2 + MLP_H * MLP_H,
              OFF_W3 = OFF_B2 + MLP_H, OFF_B3 = OFF_W3 + MLP_H;
// B-fragment table in shared memory: layer 1 (4 n-tiles x 1 k-step), layer 2
// (4 x 2), layer 3 (1 x 2); 32 lanes x 2 registers each
constexpr int FRAG_L1 = 0, FRAG_L2 = FRAG_L1 + 4 * 1 * 64, FRAG_L3 = FRAG_L2 + 4 * 2 * 64, FRAG_N = FRAG_L3 + 1 * 2 * 64;
constexpr float GELU_K0 = 0.7978845608028654f, GELU_K1 = 0.044715f;

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ float bf16_round(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

__device__ __forceinline__ void mma_bf16_16816(float c[4], const uint32_t a[4], const uint32_t b[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Twice the GELU (tanh form) of two pre-activations, z (1 + tanh(k0 (z +
// k1 z^3))), in packed BF16 arithmetic; the result is the packed BF16 A
// operand of the next layer, whose weights carry the GELU's factor 1/2
// (mlp_bval).  Scaling by a power of two is exact in BF16, so the layer's
// products and sums are bitwise those of 1/2 z (1 + tanh(...)) with the
// unscaled weights, one multiplication fewer per pair.
__device__ __forceinline__ uint32_t gelu2_bf16(float z0, float z1) {
  const __nv_bfloat162 z = __floats2bfloat162_rn(z0, z1);
  const __nv_bfloat162 k0 = __float2bfloat162_rn(GELU_K0), k01 = __float2bfloat162_rn(GELU_K0 * GELU_K1);
  const __nv_bfloat162 z2 = __hmul2(z, z);
  const __nv_bfloat162 arg = __hmul2(__hfma2(z2, k01, k0), z);   // k0 (z + k1 z^3)
  uint32_t th;
  asm("tanh.approx.bf16x2 %0, %1;" : "=r"(th) : "r"(*reinterpret_cast<const uint32_t*>(&arg)));
  const __nv_bfloat162 out = __hfma2(*reinterpret_cast<const __nv_bfloat162*>(&th), z, z);
  return *reinterpret_cast<const uint32_t*>(&out);
}

// Weight element B(k, n) of layer L as the B operand (k = input, n = output);
// layers 2 and 3 read doubled activations (gelu2_bf16) and take half weights.
__device__ __forceinline__ float mlp_bval(const float* __restrict__ P, int L, int k, int n) {
  if (L == 1) return (k < MLP_IN) ? P[OFF_W1 + n * MLP_IN + k] : 0.f;
  if (L == 2) return 0.5f * P[OFF_W2 + n * MLP_H + k];
  return (n == 0) ? 0.5f * P[OFF_W3 + k] : 0.f;
}

// Build the per-lane B fragments of all three layers (BF16) into `frag`
// (FRAG_N uint32 in shared memory); called by all threads of the CTA.
__device__ __forceinline__ void mlp_stage_fragments(const float* __restrict__ P, uint32_t* frag) {
  for (int e = threadIdx.x; e < FRAG_N / 2; e += blockDim.x) {
    int L, base, rem;
    if (e < FRAG_L2 / 2) { L = 1; base = FRAG_L1; rem = e; }
    else if (e < FRAG_L3 / 2) { L = 2; base = FRAG_L2; rem = e - FRAG_L2 / 2; }
    else { L = 3; base = FRAG_L3; rem = e - FRAG_L3 / 2; }
    const int nk = (L == 1) ? 1 : 2;
    const int lane = rem % 32, tk = rem / 32;           // tk = ntile * nk + kstep
    const int nt = tk / nk, ks = tk % nk;
    const int g = lane >> 2, t = lane & 3;
    const int n = nt * 8 + g, k0 = ks * 16 + 2 * t;
    frag[base + 2 * rem] = pack_bf16(mlp_bval(P, L, k0, n), mlp_bval(P, L, k0 + 1, n));
    frag[base + 2 * rem + 1] = pack_bf16(mlp_bval(P, L, k0 + 8, n), mlp_bval(P, L, k0 + 9, n));
  }
}

// Logits of 32 samples held by one warp.  rows: per-warp shared scratch of
// 32 x 9 uint32 (row r = the 16 BF16 features of sample r in 8 words + pad);
// each lane has written its own row before the call.  Returns lane's logit.
__device__ __forceinline__ float mlp_warp_logit(const float* __restrict__ P, const uint32_t* __restrict__ frag,
                                                uint32_t* rows, float* logit_sh) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  __syncwarp();
#pragma unroll 1
  for (int mt = 0; mt < 2; ++mt) {
    uint32_t a[4];
    a[0] = rows[(16 * mt + g) * 9 + t];
    a[1] = rows[(16 * mt + g + 8) * 9 + t];
    a[2] = rows[(16 * mt + g) * 9 + 4 + t];
    a[3] = rows[(16 * mt + g + 8) * 9 + 4 + t];
    // layer 1
    float c1[4][4];
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      const float b0 = P[OFF_B1 + nt * 8 + 2 * t], b1 = P[OFF_B1 + nt * 8 + 2 * t + 1];
      c1[nt][0] = b0; c1[nt][1] = b1; c1[nt][2] = b0; c1[nt][3] = b1;
      const uint32_t bf[2] = {frag[FRAG_L1 + 2 * (nt * 32 + lane)], frag[FRAG_L1 + 2 * (nt * 32 + lane) + 1]};
      mma_bf16_16816(c1[nt], a, bf);
    }
    uint32_t a2[2][4];
#pragma unroll
    for (int ks = 0; ks < 2; ++ks) {
      a2[ks][0] = gelu2_bf16(c1[2 * ks][0], c1[2 * ks][1]);
      a2[ks][1] = gelu2_bf16(c1[2 * ks][2], c1[2 * ks][3]);
      a2[ks][2] = gelu2_bf16(c1[2 * ks + 1][0], c1[2 * ks + 1][1]);
      a2[ks][3] = gelu2_bf16(c1[2 * ks + 1][2], c1[2 * ks + 1][3]);
    }
    // layer 2
    float c2[4][4];
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      const float b0 = P[OFF_B2 + nt * 8 + 2 * t], b1 = P[OFF_B2 + nt * 8 + 2 * t + 1];
      c2[nt][0] = b0; c2[nt][1] = b1; c2[nt][2] = b0; c2[nt][3] = b1;
#pragma unroll
      for (int ks = 0; ks < 2; ++ks) {
        const int fi = FRAG_L2 + 2 * ((nt * 2 + ks) * 32 + lane);
        const uint32_t bf[2] = {frag[fi], frag[fi + 1]};
        mma_bf16_16816(c2[nt], a2[ks], bf);
      }
    }
    uint32_t a3[2][4];
#pragma unroll
    for (int ks = 0; ks < 2; ++ks) {
      a3[ks][0] = gelu2_bf16(c2[2 * ks][0], c2[2 * ks][1]);
      a3[ks][1] = gelu2_bf16(c2[2 * ks][2], c2[2 * ks][3]);
      a3[ks][2] = gelu2_bf16(c2[2 * ks + 1][0], c2[2 * ks + 1][1]);
      a3[ks][3] = gelu2_bf16(c2[2 * ks + 1][2], c2[2 * ks + 1][3]);
    }
    // layer 3 (output column 0)
    const float b3 = P[OFF_B3];
    float c3[4] = {b3, b3, b3, b3};
#pragma unroll
    for (int ks = 0; ks < 2; ++ks) {
      const int fi = FRAG_L3 + 2 * (ks * 32 + lane);
      const uint32_t bf[2] = {frag[fi], frag[fi + 1]};
      mma_bf16_16816(c3, a3[ks], bf);
    }
    if (t == 0) {
      logit_sh[16 * mt + g] = c3[0];
      logit_sh[16 * mt + g + 8] = c3[2];
    }
  }
  __syncwarp();
  const float z = logit_sh[lane];
  __syncwarp();
  return z;
}

// Write 15 features (+ zero pad) of this lane's face as BF16 into its row.
__device__ __forceinline__ void mlp_put_row(uint32_t* rows, const float f[15]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int w = 0; w < 7; ++w) rows[lane * 9 + w] = pack_bf16(f[2 * w], f[2 * w + 1]);
  rows[lane * 9 + 7] = pack_bf16(f[14], 0.f);
}

// One feature per consecutive variation d of a characteristic field over the
// six-cell stencil (cells i-2 .. i+3), compressed as
// sign(d) log10(1 + 1e6 |d|) / 8.
__device__ __forceinline__ float compress_diff(float d) {
  const float a = 0.125f * __log10f(fmaf(1e6f, fabsf(d), 1.f));
  return copysignf(a, d);
}

}  // namespace mrb
