// Learned reconstruction selector: training-data generation from the solver's
// own faces, training (forward and backward of the BF16-operand perceptron
// with FP32 accumulation, Adam), and tensor-core inference.  See learned.cuh.
#include <cstring>
#include <algorithm>

#include "learned.cuh"
#include "mrb.h"
#include "stage_f32.cuh"

namespace mrb {

// ---------------------------------------------------------------- labels
// Label: 1 when any reconstruction of fields 0, 1, 4 the face performs
// differs between WENO5 and the linear scheme by more than both tau_lab times
// its largest |input| and the absolute floor 1e-6.
__device__ __forceinline__ int face_label_f32(const float* __restrict__ S, int c0, int st, Rot R, const RoeF& e,
                                              float tau_lab) {
  float Ur[6][5], Fr[6][5];
#pragma unroll
  for (int m = 0; m < 6; ++m) cell_uf(S, c0 + m * st, R, Ur[m], Fr[m]);
  int lab = 0;
  auto check = [&](float a, float b, float c, float d, float ee) {
    const float sc = fmaxf(fmaxf(fabsf(a), fabsf(b)), fmaxf(fmaxf(fabsf(c), fabsf(d)), fabsf(ee)));
    if (fabsf(weno5f(a, b, c, d, ee) - linear5f(a, b, c, d, ee)) > fmaxf(tau_lab * sc, 1e-6f)) lab = 1;
  };
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    if (k == 2 || k == 3) continue;   // shear fields are not selected
    float l[5], G[6], V[6];
    lrow_f32(e, k, l);
#pragma unroll
    for (int m = 0; m < 6; ++m) {
      V[m] = fmaf(l[0], Ur[m][0], fmaf(l[1], Ur[m][1], fmaf(l[2], Ur[m][2], fmaf(l[3], Ur[m][3], l[4] * Ur[m][4]))));
      G[m] = fmaf(l[0], Fr[m][0], fmaf(l[1], Fr[m][1], fmaf(l[2], Fr[m][2], fmaf(l[3], Fr[m][3], l[4] * Fr[m][4]))));
    }
    float lL, lR, lt;
    if (k == 0 || k == 4) {
      const float sg = (k == 0) ? 1.f : -1.f;
      lL = fmaf(-sg, e.cL, e.unL);
      lR = fmaf(-sg, e.cR, e.unR);
      lt = fmaf(-sg, e.c, e.un);
    } else {
      lL = e.unL;
      lR = e.unR;
      lt = e.un;
    }
    if (lL > 0.f && lR > 0.f && lt > 0.f) {
      check(G[0], G[1], G[2], G[3], G[4]);
    } else if (lL < 0.f && lR < 0.f && lt < 0.f) {
      check(G[5], G[4], G[3], G[2], G[1]);
    } else {
      const float ha = 0.5f * fmaxf(fabsf(lL), fabsf(lR));
      float fp[6], fm[6];
#pragma unroll
      for (int m = 0; m < 6; ++m) {
        fp[m] = fmaf(0.5f, G[m], ha * V[m]);
        fm[m] = fmaf(0.5f, G[m], -ha * V[m]);
      }
      check(fp[0], fp[1], fp[2], fp[3], fp[4]);
      check(fm[5], fm[4], fm[3], fm[2], fm[1]);
    }
  }
  return lab;
}

constexpr int FACES_PER_LEAF = 3 * 17 * 256;   // 13056

// Every stride-th face (global id = leaf * 13056 + direction * 4352 + index in
// the block's canonical face order) -> features [n][16], labels [n] and the
// face id.  Work items are (leaf, z-slab) as in the stage kernel.
__device__ __forceinline__ void sample_dir(int D, const RegionSrc& RS, float* __restrict__ S, int li, int z0,
                                           float g, float B, float gm1, float tau_lab, int64_t stride,
                                           float* __restrict__ feats, uint8_t* __restrict__ labels,
                                           int64_t* __restrict__ where, int64_t cap) {
  load_region_f32(D, RS, S, z0, g, B, gm1);
  __syncthreads();
  const int nf = region_faces(D);
  const int st = region_stride(D);
  for (int f = threadIdx.x; f < nf; f += blockDim.x) {
    int fa, c0, ta, tb;
    face_of(D, f, z0, fa, c0, ta, tb);
    if (D == 2 && fa == SF_TZ && z0 + SF_TZ != NB) continue;   // the next slab owns this face plane
    const int canon = (D == 0) ? z0 * 16 * 17 + f : (D == 1 ? z0 * 17 * 16 + f : z0 * 256 + f);
    const int64_t id = (int64_t)li * FACES_PER_LEAF + D * 4352 + canon;
    if (id % stride) continue;
    const int64_t o = id / stride;
    if (o >= cap) continue;
    const Rot R = rot_of(D);
    const RoeF e = roe_f32(S, c0 + 2 * st, c0 + 3 * st, gm1, g, B, R);
    float fe[15];
    face_features_f32(S, c0, st, R, e, fe);
#pragma unroll
    for (int q = 0; q < 15; ++q) feats[o * 16 + q] = fe[q];
    feats[o * 16 + 15] = 0.f;
    labels[o] = (uint8_t)face_label_f32(S, c0, st, R, e, tau_lab);
    if (where) where[o] = id;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(SF_THREADS) k_face_samples(Topo t, Phys p, Pool pool, int cur, float tau_lab,
                                                             int64_t stride, float* __restrict__ feats,
                                                             uint8_t* __restrict__ labels, int64_t* __restrict__ where,
                                                             int64_t cap) {
  extern __shared__ __align__(16) float smp_smem[];
  const int nitems = t.cnt[CNT_NLEAVES] * SF_NSLAB;
  const float g = (float)p.gamma, B = (float)p.B, gm1 = (float)(p.gamma - 1.0);
  for (int w = blockIdx.x; w < nitems; w += gridDim.x) {
    const int li = w / SF_NSLAB, z0 = (w % SF_NSLAB) * SF_TZ;
    // the block's own records and stored halo (filled by the caller), no
    // neighbour reads
    const int slot = t.slot[t.leaves[li]];
    RegionSrc RS;
    RS.u = pool.bufp(cur) + (size_t)slot * SLOT_U;
    RS.sh = pool.shp(cur) ? pool.shp(cur) + (size_t)slot * SLOT_SH : nullptr;
#pragma unroll
    for (int q = 0; q < 6; ++q) RS.nsh[q] = nullptr;
#pragma unroll 1
    for (int D = 0; D < 3; ++D)
      sample_dir(D, RS, smp_smem, li, z0, g, B, gm1, tau_lab, stride, feats, labels, where, cap);
  }
}

void launch_face_samples(const Topo& t, const Phys& p, const Pool& pool, int cur, float tau_lab, int64_t stride,
                         float* feats, uint8_t* labels, int64_t* where, int64_t cap, cudaStream_t st) {
  const size_t smem = sizeof(float) * SF_NREC * SF_REG;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_face_samples, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = true;
  }
  k_face_samples<<<sm_count() * 2, SF_THREADS, smem, st>>>(t, p, pool, cur, tau_lab, stride, feats, labels, where,
                                                            cap);
  ++g_kernel_launches;
}

// ---------------------------------------------------------------- training
constexpr int TR_T = 128;                 // samples per tile = threads per CTA
constexpr int TR_GRID_MAX = 512;
constexpr int TR_LD = 33;                  // padded row length of the activation tiles
constexpr size_t TR_SMEM = sizeof(float) * (MLP_NPARAM + (MLP_NPARAM + 1) + TR_T * 16 + 6 * TR_T * TR_LD + TR_T);

__device__ __forceinline__ float gelu_acc(float z) {
  const float t = tanhf(GELU_K0 * (z + GELU_K1 * z * z * z));
  return 0.5f * z * (1.f + t);
}

__device__ __forceinline__ float gelu_grad_acc(float z) {
  const float t = tanhf(GELU_K0 * (z + GELU_K1 * z * z * z));
  return 0.5f * (1.f + t) + 0.5f * z * (1.f - t * t) * GELU_K0 * (1.f + 3.f * GELU_K1 * z * z);
}

// Per CTA: forward and backward of its sample tiles (one thread per sample),
// then each thread sums its gradient entries over the tile's samples in a
// fixed order.  Writes the CTA's gradient and loss sums to work[cta].
__global__ void __launch_bounds__(TR_T) k_mlp_grad(const float* __restrict__ P, const float* __restrict__ X,
                                                   const uint8_t* __restrict__ Y, int64_t n, float posw,
                                                   float* __restrict__ work) {
  extern __shared__ __align__(16) float tr[];
  float* Wr = tr;                               // weights rounded to BF16, biases FP32
  float* gacc = Wr + MLP_NPARAM;                // gradient + loss accumulator
  float* xs = gacc + MLP_NPARAM + 1;            // [T][16]
  float* h1 = xs + TR_T * 16;                   // [T][33]
  float* h2 = h1 + TR_T * TR_LD;
  float* d1 = h2 + TR_T * TR_LD;
  float* d2 = d1 + TR_T * TR_LD;
  float* z1 = d2 + TR_T * TR_LD;                // pre-activations [T][33]
  float* z2 = z1 + TR_T * TR_LD;
  float* d3 = z2 + TR_T * TR_LD;                // [T]
  for (int e = threadIdx.x; e < MLP_NPARAM; e += blockDim.x) {
    const bool is_bias = (e >= OFF_B1 && e < OFF_W2) || (e >= OFF_B2 && e < OFF_W3) || e == OFF_B3;
    Wr[e] = is_bias ? P[e] : bf16_round(P[e]);
  }
  for (int e = threadIdx.x; e <= MLP_NPARAM; e += blockDim.x) gacc[e] = 0.f;
  __syncthreads();
  const float inv_n = 1.0f / (float)n;
  const int64_t ntiles = (n + TR_T - 1) / TR_T;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int s = threadIdx.x;
    const int64_t gi = tile * TR_T + s;
    const bool act = gi < n;
    float x[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) x[k] = (act && k < MLP_IN) ? bf16_round(X[gi * 16 + k]) : 0.f;
#pragma unroll
    for (int k = 0; k < 16; ++k) xs[s * 16 + k] = x[k];
#pragma unroll 1
    for (int o = 0; o < MLP_H; ++o) {
      float a = Wr[OFF_B1 + o];
#pragma unroll
      for (int k = 0; k < MLP_IN; ++k) a = fmaf(Wr[OFF_W1 + o * MLP_IN + k], x[k], a);
      z1[s * TR_LD + o] = a;
      h1[s * TR_LD + o] = bf16_round(gelu_acc(a));
    }
#pragma unroll 1
    for (int o = 0; o < MLP_H; ++o) {
      float a = Wr[OFF_B2 + o];
#pragma unroll 8
      for (int k = 0; k < MLP_H; ++k) a = fmaf(Wr[OFF_W2 + o * MLP_H + k], h1[s * TR_LD + k], a);
      z2[s * TR_LD + o] = a;
      h2[s * TR_LD + o] = bf16_round(gelu_acc(a));
    }
    float z3 = Wr[OFF_B3];
#pragma unroll 8
    for (int k = 0; k < MLP_H; ++k) z3 = fmaf(Wr[OFF_W3 + k], h2[s * TR_LD + k], z3);
    float dz3 = 0.f, loss = 0.f;
    if (act) {
      const float y = (float)Y[gi];
      const float w = (y > 0.5f) ? posw : 1.f;
      loss = w * (fmaxf(z3, 0.f) - z3 * y + log1pf(expf(-fabsf(z3))));
      const float sig = 1.f / (1.f + expf(-z3));
      dz3 = w * (sig - y) * inv_n;
    }
    d3[s] = dz3;
#pragma unroll 1
    for (int o = 0; o < MLP_H; ++o) d2[s * TR_LD + o] = dz3 * Wr[OFF_W3 + o] * gelu_grad_acc(z2[s * TR_LD + o]);
#pragma unroll 1
    for (int k = 0; k < MLP_H; ++k) {
      float a = 0.f;
#pragma unroll 8
      for (int o = 0; o < MLP_H; ++o) a = fmaf(Wr[OFF_W2 + o * MLP_H + k], d2[s * TR_LD + o], a);
      d1[s * TR_LD + k] = a * gelu_grad_acc(z1[s * TR_LD + k]);
    }
    // loss of the tile in a fixed order (thread 0)
    xs[s * 16 + 15] = loss;
    __syncthreads();
    if (threadIdx.x == 0) {
      float ls = 0.f;
      for (int q = 0; q < TR_T; ++q) ls += xs[q * 16 + 15];
      gacc[MLP_NPARAM] += ls;
    }
    // gradient entries, each summed over the tile's samples by one thread
    for (int e = threadIdx.x; e < MLP_NPARAM; e += blockDim.x) {
      float a = 0.f;
      if (e < OFF_B1) {
        const int o = e / MLP_IN, k = e % MLP_IN;
        for (int q = 0; q < TR_T; ++q) a = fmaf(d1[q * TR_LD + o], (k == 15) ? 0.f : xs[q * 16 + k], a);
      } else if (e < OFF_W2) {
        const int o = e - OFF_B1;
        for (int q = 0; q < TR_T; ++q) a += d1[q * TR_LD + o];
      } else if (e < OFF_B2) {
        const int o = (e - OFF_W2) / MLP_H, k = (e - OFF_W2) % MLP_H;
        for (int q = 0; q < TR_T; ++q) a = fmaf(d2[q * TR_LD + o], h1[q * TR_LD + k], a);
      } else if (e < OFF_W3) {
        const int o = e - OFF_B2;
        for (int q = 0; q < TR_T; ++q) a += d2[q * TR_LD + o];
      } else if (e < OFF_B3) {
        const int k = e - OFF_W3;
        for (int q = 0; q < TR_T; ++q) a = fmaf(d3[q], h2[q * TR_LD + k], a);
      } else {
        for (int q = 0; q < TR_T; ++q) a += d3[q];
      }
      gacc[e] += a;
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e <= MLP_NPARAM; e += blockDim.x) work[(size_t)blockIdx.x * (MLP_NPARAM + 1) + e] = gacc[e];
}

// Sum the CTA partials in order; optional gradient/loss outputs; Adam step.
__global__ void k_mlp_adam(float* __restrict__ P, float* __restrict__ m, float* __restrict__ v, int t_step,
                           const float* __restrict__ work, int nblk, float lr, float* __restrict__ loss_out,
                           float* __restrict__ grad_out, int64_t n) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e > MLP_NPARAM) return;
  float gsum = 0.f;
  for (int b = 0; b < nblk; ++b) gsum += work[(size_t)b * (MLP_NPARAM + 1) + e];
  if (e == MLP_NPARAM) {
    if (loss_out) *loss_out = gsum / (float)n;
    return;
  }
  if (grad_out) grad_out[e] = gsum;
  if (lr <= 0.f) return;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float mm = b1 * m[e] + (1.f - b1) * gsum;
  const float vv = b2 * v[e] + (1.f - b2) * gsum * gsum;
  m[e] = mm;
  v[e] = vv;
  const float mh = mm / (1.f - powf(b1, (float)t_step));
  const float vh = vv / (1.f - powf(b2, (float)t_step));
  P[e] -= lr * mh / (sqrtf(vh) + eps);
}

// ---------------------------------------------------------------- inference
// One warp per 32 samples, tensor-core layers (learned.cuh).
__global__ void __launch_bounds__(256) k_mlp_logits(const float* __restrict__ P, const float* __restrict__ X,
                                                    int64_t n, float* __restrict__ out) {
  __shared__ uint32_t frag[FRAG_N];
  __shared__ uint32_t rows[8][32 * 9];
  __shared__ float lsh[8][32];
  mlp_stage_fragments(P, frag);
  __syncthreads();
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t nw = (n + 31) / 32;
  for (int64_t wb = (int64_t)blockIdx.x * 8 + wid; wb < nw; wb += (int64_t)gridDim.x * 8) {
    const int64_t i = wb * 32 + lane;
    float f[15];
#pragma unroll
    for (int q = 0; q < 15; ++q) f[q] = (i < n) ? X[i * 16 + q] : 0.f;
    mlp_put_row(rows[wid], f);
    const float z = mlp_warp_logit(P, frag, rows[wid], lsh[wid]);
    if (i < n) out[i] = z;
  }
}

}  // namespace mrb

// ------------------------------------------------------------------ C ABI
using namespace mrb;

extern "C" int mrb_mlp_logits(const float* params_dev, const float* feats_dev, int64_t n, float* logits_dev,
                              void* stream) {
  if (!params_dev || n < 0 || (n > 0 && (!feats_dev || !logits_dev))) return MRB_EINVAL;
  if (n == 0) return MRB_OK;
  const int64_t nw = (n + 31) / 32;
  const int grid = (int)std::min<int64_t>((nw + 7) / 8, (int64_t)sm_count() * 8);
  k_mlp_logits<<<grid, 256, 0, (cudaStream_t)stream>>>(params_dev, feats_dev, n, logits_dev);
  ++g_kernel_launches;
  return cudaGetLastError() == cudaSuccess ? MRB_OK : MRB_ECUDA;
}

// ---------------------------------------------------------------- threshold
// Order statistics of the logits of label-1 samples by radix selection on
// the float's order-preserving 32-bit key, eight bits per pass (most
// significant first): each pass histograms the next digit of the keys that
// share the digits chosen so far.
__device__ __forceinline__ uint32_t order_key(float x) {
  const uint32_t b = __float_as_uint(x);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
static float key_value(uint32_t k) {
  const uint32_t b = (k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k;
  float x;
  std::memcpy(&x, &b, sizeof x);
  return x;
}

__global__ void __launch_bounds__(256) k_key_hist(const float* __restrict__ z, const uint8_t* __restrict__ y,
                                                  int64_t n, uint32_t prefix, int shift,
                                                  unsigned long long* __restrict__ hist) {
  __shared__ unsigned int h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (!y[i]) continue;
    const uint32_t k = order_key(z[i]);
    if (shift < 24 && (k >> (shift + 8)) != (prefix >> (shift + 8))) continue;
    atomicAdd(&h[(k >> shift) & 255u], 1u);
  }
  __syncthreads();
  if (h[threadIdx.x]) atomicAdd(&hist[threadIdx.x], (unsigned long long)h[threadIdx.x]);
}

// The kth smallest (from 0) label-1 logit; *m receives the number of label-1
// samples (from the first pass).
static int select_kth(const float* z, const uint8_t* y, int64_t n, int64_t kth, unsigned long long* hist,
                      cudaStream_t st, float* out, int64_t* m) {
  const int grid = (int)std::min<int64_t>((n + 255) / 256, (int64_t)sm_count() * 4);
  uint32_t prefix = 0;
  unsigned long long h[256];
  for (int shift = 24; shift >= 0; shift -= 8) {
    if (cudaMemsetAsync(hist, 0, 256 * sizeof(unsigned long long), st) != cudaSuccess) return MRB_ECUDA;
    k_key_hist<<<grid, 256, 0, st>>>(z, y, n, prefix, shift, hist);
    ++g_kernel_launches;
    if (cudaMemcpyAsync(h, hist, sizeof h, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return MRB_ECUDA;
    if (shift == 24) {
      int64_t total = 0;
      for (int d = 0; d < 256; ++d) total += (int64_t)h[d];
      *m = total;
      if (kth >= total) return MRB_EINVAL;
    }
    int d = 0;
    for (; d < 256; ++d) {
      if (kth < (int64_t)h[d]) break;
      kth -= (int64_t)h[d];
    }
    prefix |= (uint32_t)d << shift;
  }
  *out = key_value(prefix);
  return MRB_OK;
}

extern "C" int mrb_mlp_threshold(const float* logits_dev, const uint8_t* labels_dev, int64_t n, double q,
                                 uint64_t* work_dev, float* tau_out, void* stream) {
  if (!tau_out || n < 0 || !(q >= 0.0 && q <= 1.0) || (n > 0 && (!logits_dev || !labels_dev || !work_dev)))
    return MRB_EINVAL;
  *tau_out = 0.f;
  if (n == 0) return MRB_OK;
  cudaStream_t st = (cudaStream_t)stream;
  unsigned long long* hist = reinterpret_cast<unsigned long long*>(work_dev);
  // count the label-1 samples with a first selection of the smallest one
  float lo = 0.f;
  int64_t m = 0;
  int rc = select_kth(logits_dev, labels_dev, n, 0, hist, st, &lo, &m);
  if (rc == MRB_EINVAL && m == 0) return MRB_OK;     // no label-1 sample: threshold 0
  if (rc != MRB_OK) return rc;
  // linear interpolation between the order statistics around (m - 1) q
  const double pos = (double)(m - 1) * q;
  const int64_t k = (int64_t)pos;
  const float frac = (float)(pos - (double)k);
  float a = lo, b = lo;
  if (k > 0 && (rc = select_kth(logits_dev, labels_dev, n, k, hist, st, &a, &m)) != MRB_OK) return rc;
  b = a;
  if (k + 1 < m && (rc = select_kth(logits_dev, labels_dev, n, k + 1, hist, st, &b, &m)) != MRB_OK) return rc;
  *tau_out = a + frac * (b - a);
  return MRB_OK;
}

extern "C" int mrb_mlp_train_step(float* params_dev, float* adam_m_dev, float* adam_v_dev, int32_t t_step,
                                  const float* feats_dev, const uint8_t* labels_dev, int64_t n, float pos_weight,
                                  float lr, float* work_dev, float* loss_dev, float* grad_dev, void* stream) {
  if (!params_dev || !work_dev || n <= 0 || !feats_dev || !labels_dev) return MRB_EINVAL;
  if (lr > 0.f && (!adam_m_dev || !adam_v_dev || t_step < 1)) return MRB_EINVAL;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TR_SMEM);
    attr = true;
  }
  const int64_t ntiles = (n + TR_T - 1) / TR_T;
  const int grid = (int)std::min<int64_t>(ntiles, (int64_t)std::min(TR_GRID_MAX, sm_count() * 3));
  cudaStream_t st = (cudaStream_t)stream;
  k_mlp_grad<<<grid, TR_T, TR_SMEM, st>>>(params_dev, feats_dev, labels_dev, n, pos_weight, work_dev);
  k_mlp_adam<<<(MLP_NPARAM + 1 + 255) / 256, 256, 0, st>>>(params_dev, adam_m_dev, adam_v_dev, t_step, work_dev, grid,
                                                           lr, loss_dev, grad_dev, n);
  g_kernel_launches += 2;
  return cudaGetLastError() == cudaSuccess ? MRB_OK : MRB_ECUDA;
}
