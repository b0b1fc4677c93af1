// Mixed-precision fused stage kernel (MRB_FP32_ACC64): characteristic WENO5-JS
// with the Roe / local Lax-Friedrichs switch (Sec. 2.2 of arXiv:2012.04385) in
// FP32, flux differences accumulated per cell in FP32, and the Runge-Kutta
// stage update of the FP64 state with one FP64 addition per value.  The same
// kernel template covers the other reconstructions (TENO5, WENO-AO(5,3),
// linear, the learned selector), the LLF and HLLC flux schemes and the
// viscous terms (see rec5 and MODE).
//
// Work item = (leaf, z-slab of 16 x 16 x 4 cells); a CTA of 256 threads loops
// over items.  Every node keeps FP32 primitive records (rho, vx, vy, vz, p, E)
// of its internal cells beside its FP64 state, written by the previous
// stage's update; the kernel copies the records of a region into shared
// memory with 16-byte asynchronous copies (the block's own stored halo,
// converted from FP64, where a face has no same-level neighbour): for the x
// and y directions one region holds the slab with 3 cells on each side in x
// and in y, for z the slab with 3 planes below and above.  One thread per
// face then computes the face flux from six records (velocity read in the
// direction's frame: normal, tangential 1, tangential 2), writes it to shared
// memory (and, on the block boundary, to the block's face buffers), and each
// thread adds the flux differences of the four cells of its (i, j) column.
// The x and y faces form one loop of 2 x 1088 faces (34 warps each, so every
// warp has one direction).  Reciprocals and square roots use the fast
// hardware approximations; WENO5 works on the consecutive differences of its
// five values and needs one reciprocal: omega_k = d_k P_k / sum_j d_j P_j with
// P_k the product of the other two (eps + beta)^2.
//
// The update keeps the stage's increment u^(s) - u^n of every cell in FP32
// (pool.dl).  With a_s + b_s = 1 the Shu-Osher stage u^(s+1) = a_s u^n + b_s
// (u^(s) + dt L) is u^n + b_s (increment + dt L): the new increment is formed
// in FP32 and added to u^n in FP64, one FP64 operation per value, where the
// FP64 pipe (1/64 of the FP32 rate on GB300) is the update's bottleneck.
#pragma once

#include "convert.cuh"
#include "kernels.cuh"
#include "learned.cuh"

namespace mrb {

constexpr int SF_TZ = 4;
constexpr int SF_NSLAB = NB / SF_TZ;
constexpr int SF_THREADS = 256;
constexpr int SF_REG = NB * NB * (SF_TZ + 6);            // record slots: the z region, 2560 cells
constexpr int SF_XY = 24 * 22 * SF_TZ;                   // x-y region (corners unused): 2112 slots
constexpr int SF_NFX = 17 * 16 * SF_TZ;                  // x (and y) faces of a slab: 1088
constexpr int SF_NFZ = NB * NB * (SF_TZ + 1);            // z faces of a slab: 1280
constexpr int SF_FMAX = 2 * SF_NFX;                      // face-flux slots: the x-y loop, 2176
constexpr int SF_NREC = 6;                                // rho, vx, vy, vz, p, E
constexpr size_t SF_SMEM = sizeof(float) * (SF_NREC * SF_REG + NV * SF_FMAX);
// learned selector at stage 0 (one direction at a time, face-flux rows of
// SF_NFZ): records, face fluxes, B fragments, per-warp feature rows and logits
constexpr size_t SF_SMEM_LEARNED = sizeof(float) * (SF_NREC * SF_REG + NV * SF_NFZ) +
                                   sizeof(uint32_t) * (FRAG_N + (SF_THREADS / 32) * 32 * 9) +
                                   sizeof(float) * SF_THREADS;


__device__ __forceinline__ float frcp(float x) { return __fdividef(1.0f, x); }

// Three-way select by direction (D = 0, 1, 2).
__device__ __forceinline__ float sel3(int D, float a, float b, float c) { return D == 0 ? a : (D == 1 ? b : c); }
__device__ __forceinline__ int sel3i(int D, int a, int b, int c) { return D == 0 ? a : (D == 1 ? b : c); }

// WENO5-JS on the differences da = a-b, db = b-c, dc = c-d, dd = d-e; the
// smoothness indicators are scaled by 12 (beta' = 13 t1^2 + 3 t2^2) together
// with eps' = 12 eps, which leaves the weights unchanged, and the candidate
// stencils are written as c + (linear combination of differences) / 6.
__device__ __forceinline__ float weno5f(float a, float b, float c, float d, float e) {
  const float da = a - b, db = b - c, dc = c - d, dd = d - e;
  const float eps12 = 12e-6f;
  float t1 = da - db, t2 = fmaf(-3.f, db, da);
  float s0 = fmaf(13.f * t1, t1, fmaf(3.f * t2, t2, eps12));
  t1 = db - dc;
  t2 = db + dc;
  float s1 = fmaf(13.f * t1, t1, fmaf(3.f * t2, t2, eps12));
  t1 = dc - dd;
  t2 = fmaf(3.f, dc, -dd);
  float s2 = fmaf(13.f * t1, t1, fmaf(3.f * t2, t2, eps12));
  s0 *= s0;
  s1 *= s1;
  s2 *= s2;
  const float w0 = 0.1f * (s1 * s2), w1 = 0.6f * (s0 * s2), w2 = 0.3f * (s0 * s1);
  const float e0 = fmaf(2.f, da, -5.f * db), e1 = fmaf(-2.f, dc, -db), e2 = fmaf(-4.f, dc, dd);
  return fmaf(fmaf(w0, e0, fmaf(w1, e1, w2 * e2)), frcp(6.f * (w0 + w1 + w2)), c);
}

// Packed FP32 pairs (fma / add / sub / mul .rn.ftz.f32x2: two lanes' IEEE
// operations in one instruction, flushing subnormals like the scalar FP32
// code built with -ftz).
__device__ __forceinline__ float2 f2s(float x) { return make_float2(x, x); }
__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c) {
  float2 r;
  asm("{.reg .b64 ra, rb, rc, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n mov.b64 rc, {%6, %7};\n"
      " fma.rn.ftz.f32x2 rd, ra, rb, rc;\n mov.b64 {%0, %1}, rd;}"
      : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return r;
}
__device__ __forceinline__ float2 f2add(float2 a, float2 b) {
  float2 r;
  asm("{.reg .b64 ra, rb, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n add.rn.ftz.f32x2 rd, ra, rb;\n"
      " mov.b64 {%0, %1}, rd;}" : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) {
  float2 r;
  asm("{.reg .b64 ra, rb, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n sub.rn.ftz.f32x2 rd, ra, rb;\n"
      " mov.b64 {%0, %1}, rd;}" : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}
__device__ __forceinline__ float2 f2mul(float2 a, float2 b) {
  float2 r;
  asm("{.reg .b64 ra, rb, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n mul.rn.ftz.f32x2 rd, ra, rb;\n"
      " mov.b64 {%0, %1}, rd;}" : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}

// Two WENO5 reconstructions in packed pairs, lane by lane the operations of
// weno5f: where weno5f negates an operand (3 dc - dd, -2 dc - db) the pair
// forms the exact negation instead (dd - 3 dc only enters squared; -e1 meets
// -w1 in the product and w0 - (-w1) = w0 + w1), so every lane's result is
// weno5f's bit for bit.
__device__ __forceinline__ float2 weno5f2(float2 a, float2 b, float2 c, float2 d, float2 e) {
  const float2 da = f2sub(a, b), db = f2sub(b, c), dc = f2sub(c, d), dd = f2sub(d, e);
  const float2 eps12 = f2s(12e-6f);
  float2 t1 = f2sub(da, db), t2 = f2fma(f2s(-3.f), db, da);
  float2 s0 = f2fma(f2mul(f2s(13.f), t1), t1, f2fma(f2mul(f2s(3.f), t2), t2, eps12));
  t1 = f2sub(db, dc);
  t2 = f2add(db, dc);
  float2 s1 = f2fma(f2mul(f2s(13.f), t1), t1, f2fma(f2mul(f2s(3.f), t2), t2, eps12));
  t1 = f2sub(dc, dd);
  t2 = f2fma(f2s(-3.f), dc, dd);
  float2 s2 = f2fma(f2mul(f2s(13.f), t1), t1, f2fma(f2mul(f2s(3.f), t2), t2, eps12));
  s0 = f2mul(s0, s0);
  s1 = f2mul(s1, s1);
  s2 = f2mul(s2, s2);
  const float2 w0 = f2mul(f2s(0.1f), f2mul(s1, s2)), nw1 = f2mul(f2s(-0.6f), f2mul(s0, s2));
  const float2 w2 = f2mul(f2s(0.3f), f2mul(s0, s1));
  const float2 e0 = f2fma(f2s(2.f), da, f2mul(f2s(-5.f), db)), ne1 = f2fma(f2s(2.f), dc, db);
  const float2 e2 = f2fma(f2s(-4.f), dc, dd);
  const float2 num = f2fma(w0, e0, f2fma(nw1, ne1, f2mul(w2, e2)));
  const float2 den = f2mul(f2s(6.f), f2add(f2sub(w0, nw1), w2));
  return f2fma(num, make_float2(frcp(den.x), frcp(den.y)), c);
}

// TENO5 (Fu, Hu & Adams 2016) on the differences, with the smoothness
// indicators scaled by 12 as in weno5f: stencil k is kept when gamma_k >=
// C_T sum gamma, gamma_k = (1 + tau5 / (beta_k + eps))^6, tau5 = |beta0 -
// beta2|, C_T = 1e-5; the comparison uses gamma_k / max gamma (no overflow)
// and eps = 1e-30 (a normal FP32 number).  Kept stencils take the linear
// weights, renormalised.
__device__ __forceinline__ float teno5f(float a, float b, float c, float d, float e) {
  const float da = a - b, db = b - c, dc = c - d, dd = d - e;
  const float eps = 1e-30f;
  float t1 = da - db, t2 = fmaf(-3.f, db, da);
  const float s0 = fmaf(13.f * t1, t1, 3.f * t2 * t2);
  t1 = db - dc;
  t2 = db + dc;
  const float s1 = fmaf(13.f * t1, t1, 3.f * t2 * t2);
  t1 = dc - dd;
  t2 = fmaf(3.f, dc, -dd);
  const float s2 = fmaf(13.f * t1, t1, 3.f * t2 * t2);
  const float tau = fabsf(s0 - s2);
  const float r0 = fmaf(tau, frcp(s0 + eps), 1.f), r1 = fmaf(tau, frcp(s1 + eps), 1.f), r2 = fmaf(tau, frcp(s2 + eps), 1.f);
  const float inv = frcp(fmaxf(r0, fmaxf(r1, r2)));
  float g0 = r0 * inv, g1 = r1 * inv, g2 = r2 * inv;
  g0 = g0 * g0 * g0;
  g1 = g1 * g1 * g1;
  g2 = g2 * g2 * g2;
  g0 *= g0;
  g1 *= g1;
  g2 *= g2;
  const float lim = 1e-5f * (g0 + g1 + g2);
  const float w0 = (g0 < lim) ? 0.f : 0.1f, w1 = (g1 < lim) ? 0.f : 0.6f, w2 = (g2 < lim) ? 0.f : 0.3f;
  const float e0 = fmaf(2.f, da, -5.f * db), e1 = fmaf(-2.f, dc, -db), e2 = fmaf(-4.f, dc, dd);
  return fmaf(fmaf(w0, e0, fmaf(w1, e1, w2 * e2)), frcp(6.f * (w0 + w1 + w2)), c);
}

// WENO-AO(5,3) (Balsara, Garain & Shu 2016) on the differences, smoothness
// indicators (the parabolas' and the quartic's) scaled by 12 with eps' = 12
// eps, eps = 1e-12; linear weights from gamma_hi = gamma_lo = 0.85; weights
// gamma_k (1 + r_k^2), r_k = tau / (beta_k + eps), evaluated as gamma_k (1/M^2
// + (r_k/M)^2) with M = max(1, max r_k) (no overflow; same normalised weights).
// The value is c + [(w5/g5)(e5/60 - sum g_k e_k/6) + sum w_k e_k/6] / sum w,
// e_k the parabolas' and e5 the quartic's offsets from c times 6 and 60.
__device__ __forceinline__ float wenoao5f(float a, float b, float c, float d, float e) {
  const float da = a - b, db = b - c, dc = c - d, dd = d - e;
  const float eps12 = 12e-12f;
  float t1 = da - db, t2 = fmaf(-3.f, db, da);
  const float s0 = fmaf(13.f * t1, t1, 3.f * t2 * t2);
  t1 = db - dc;
  t2 = db + dc;
  const float s1 = fmaf(13.f * t1, t1, 3.f * t2 * t2);
  t1 = dc - dd;
  t2 = fmaf(3.f, dc, -dd);
  const float s2 = fmaf(13.f * t1, t1, 3.f * t2 * t2);
  // Legendre coefficients of the quartic on the middle cell
  const float ae = da + db + dc + dd, bd = db + dc;   // a - e, b - d
  const float u1 = fmaf(11.f / 120.f, ae, (-82.f / 120.f) * bd);
  const float u2 = (fmaf(-3.f, da, 3.f * dd) + 37.f * (db - dc)) * (1.f / 56.f);
  const float u3 = fmaf(-1.f / 12.f, ae, (2.f / 12.f) * bd);
  const float u4 = (fmaf(-3.f, db - dc, da) - dd) * (1.f / 24.f);
  const float x1 = fmaf(0.1f, u3, u1), x2 = fmaf(123.f / 455.f, u4, u2);
  const float s5 = 12.f * fmaf(x1, x1, fmaf(13.f / 3.f * x2, x2, fmaf(781.f / 20.f * u3, u3, (1421461.f / 2275.f) * u4 * u4)));
  const float tau = (fabsf(s5 - s0) + fabsf(s5 - s1) + fabsf(s5 - s2)) * (1.f / 3.f);
  const float r0 = tau * frcp(s0 + eps12), r1 = tau * frcp(s1 + eps12), r2 = tau * frcp(s2 + eps12);
  const float r5 = tau * frcp(s5 + eps12);
  const float M = fmaxf(1.f, fmaxf(fmaxf(r0, r1), fmaxf(r2, r5))), iM = frcp(M);
  const float iM2 = iM * iM;
  const float y0 = r0 * iM, y1 = r1 * iM, y2 = r2 * iM, y5 = r5 * iM;
  constexpr float g5 = 0.85f, g1 = 0.15f * 0.85f, g0 = 0.5f * 0.15f * 0.15f;
  const float w0 = g0 * fmaf(y0, y0, iM2), w1 = g1 * fmaf(y1, y1, iM2), w2 = g0 * fmaf(y2, y2, iM2);
  const float w5 = g5 * fmaf(y5, y5, iM2);
  const float e0 = fmaf(2.f, da, -5.f * db), e1 = fmaf(-2.f, dc, -db), e2 = fmaf(-4.f, dc, dd);
  const float e5 = fmaf(2.f, da, fmaf(-11.f, db, fmaf(-24.f, dc, 3.f * dd)));
  const float hi = fmaf(e5, 1.f / 60.f, -(1.f / 6.f) * fmaf(g0, e0 + e2, g1 * e1));
  const float num = fmaf(w5 * (1.f / g5), hi, (1.f / 6.f) * fmaf(w0, e0, fmaf(w1, e1, w2 * e2)));
  return fmaf(num, frcp(w0 + w1 + w2 + w5), c);
}

__device__ __forceinline__ float linear5f(float a, float b, float c, float d, float e) {
  // (2a - 13b + 47c + 27d - 3e) / 60
  return fmaf(2.f / 60.f, a, fmaf(-13.f / 60.f, b, fmaf(47.f / 60.f, c, fmaf(27.f / 60.f, d, (-3.f / 60.f) * e))));
}

// Record offsets of the velocity components in the direction frame of D:
// normal, tangential 1, tangential 2 (x: vx, vy, vz; y: vy, vz, vx; z: vz, vx, vy).
struct Rot {
  int n, t1, t2;
};
__device__ __forceinline__ Rot rot_of(int D) {
  return Rot{(1 + D) * SF_REG, (1 + (D + 1) % 3) * SF_REG, (1 + (D + 2) % 3) * SF_REG};
}

// Roe average of the face between the records at cl and cr (direction frame)
// and the cell eigenvalue ingredients of the two face cells.
struct RoeF {
  float un, ut1, ut2, H, q2, c, ic, b1, b2, hb1, unL, unR, cL, cR;
};

__device__ __forceinline__ RoeF roe_f32(const float* __restrict__ S, int cl, int cr, float gm1, float g, float B,
                                        Rot R) {
  RoeF e;
  const float rL = S[cl], rR = S[cr];
  const float pL = S[4 * SF_REG + cl], pR = S[4 * SF_REG + cr];
  e.unL = S[R.n + cl];
  e.unR = S[R.n + cr];
  // sqrt(rho) weights, H = (E + p) / rho, c = sqrt(gamma (p + B) / rho)
  const float rsL = rsqrtf(rL), rsR = rsqrtf(rR);
  e.cL = sqrtf(g * (pL + B)) * rsL;
  e.cR = sqrtf(g * (pR + B)) * rsR;
  const float sL = rL * rsL, sR = rR * rsR;
  const float iden = frcp(sL + sR);
  e.un = fmaf(sL, e.unL, sR * e.unR) * iden;
  e.ut1 = fmaf(sL, S[R.t1 + cl], sR * S[R.t1 + cr]) * iden;
  e.ut2 = fmaf(sL, S[R.t2 + cl], sR * S[R.t2 + cr]) * iden;
  e.H = fmaf(S[5 * SF_REG + cl] + pL, rsL, (S[5 * SF_REG + cr] + pR) * rsR) * iden;
  e.q2 = fmaf(e.un, e.un, fmaf(e.ut1, e.ut1, e.ut2 * e.ut2));
  const float c2 = gm1 * fmaf(-0.5f, e.q2, e.H);
  e.ic = rsqrtf(c2);
  e.c = c2 * e.ic;
  e.b1 = gm1 * e.ic * e.ic;
  e.b2 = 0.5f * e.b1 * e.q2;
  e.hb1 = 0.5f * e.b1;
  return e;
}

// Left eigenvector k (rotated frame): rows 0 and 4 the acoustic fields, 1 the
// entropy field, 2 and 3 the shear fields.
__device__ __forceinline__ void lrow_f32(const RoeF& e, int k, float l[5]) {
  if (k == 0 || k == 4) {
    const float sg = (k == 0) ? 1.f : -1.f;
    l[0] = fmaf(0.5f * sg * e.un, e.ic, 0.5f * e.b2);
    l[1] = fmaf(-e.hb1, e.un, -0.5f * sg * e.ic);
    l[2] = -e.hb1 * e.ut1;
    l[3] = -e.hb1 * e.ut2;
    l[4] = e.hb1;
  } else if (k == 1) {
    l[0] = 1.f - e.b2;
    l[1] = e.b1 * e.un;
    l[2] = e.b1 * e.ut1;
    l[3] = e.b1 * e.ut2;
    l[4] = -e.b1;
  } else {
    l[0] = -((k == 2) ? e.ut1 : e.ut2);
    l[1] = 0.f;
    l[2] = (k == 2) ? 1.f : 0.f;
    l[3] = (k == 3) ? 1.f : 0.f;
    l[4] = 0.f;
  }
}

// Conserved state and physical flux of the record at c in the direction frame
// (index 1 normal, 2 and 3 tangential).
__device__ __forceinline__ void cell_uf(const float* __restrict__ S, int c, Rot R, float U[5], float F[5]) {
  const float r = S[c], un = S[R.n + c], u1 = S[R.t1 + c], u2 = S[R.t2 + c];
  const float p = S[4 * SF_REG + c], E = S[5 * SF_REG + c];
  const float mn = r * un;
  U[0] = r;
  U[1] = mn;
  U[2] = r * u1;
  U[3] = r * u2;
  U[4] = E;
  F[0] = mn;
  F[1] = fmaf(mn, un, p);
  F[2] = mn * u1;
  F[3] = mn * u2;
  F[4] = un * (E + p);
}

// Conserved states and physical fluxes of two records (ca, cb) in packed
// pairs, lane by lane cell_uf's operations.
__device__ __forceinline__ void cell_uf2(const float* __restrict__ S, int ca, int cb, Rot R, float Ua[5], float Ub[5],
                                         float Fa[5], float Fb[5]) {
  const float2 r = make_float2(S[ca], S[cb]), un = make_float2(S[R.n + ca], S[R.n + cb]);
  const float2 u1 = make_float2(S[R.t1 + ca], S[R.t1 + cb]), u2 = make_float2(S[R.t2 + ca], S[R.t2 + cb]);
  const float2 p = make_float2(S[4 * SF_REG + ca], S[4 * SF_REG + cb]);
  const float2 E = make_float2(S[5 * SF_REG + ca], S[5 * SF_REG + cb]);
  const float2 mn = f2mul(r, un), U2 = f2mul(r, u1), U3 = f2mul(r, u2);
  const float2 F1 = f2fma(mn, un, p), F2 = f2mul(mn, u1), F3 = f2mul(mn, u2), F4 = f2mul(un, f2add(E, p));
  Ua[0] = r.x; Ub[0] = r.y;
  Ua[1] = mn.x; Ub[1] = mn.y;
  Ua[2] = U2.x; Ub[2] = U2.y;
  Ua[3] = U3.x; Ub[3] = U3.y;
  Ua[4] = E.x; Ub[4] = E.y;
  Fa[0] = mn.x; Fb[0] = mn.y;
  Fa[1] = F1.x; Fb[1] = F1.y;
  Fa[2] = F2.x; Fb[2] = F2.y;
  Fa[3] = F3.x; Fb[3] = F3.y;
  Fa[4] = F4.x; Fb[4] = F4.y;
}

// Kernel variants: MODE 0 WENO5, 2 linear, 4 TENO5, 1 learned selector at stage 0
// (WENO5 fluxes; the selector is evaluated on the same faces and its
// decisions stored), 3 learned selector at stages 1 and 2 (the stored
// decision of each face picks linear or WENO5 for fields 0, 1, 4).
// MODE 5 is WENO-AO(5,3).  Bits 3-4 of MODE select the flux scheme (0 Roe
// with the LLF fallback, 1 LLF on every field, 2 HLLC) for MODES 0, 2, 4, 5;
// bit 5 adds the viscous (Navier-Stokes) face fluxes.
template <int MODE>
__device__ __forceinline__ float rec5(bool lin, float a, float b, float c, float d, float e) {
  constexpr int REC = MODE & 7;
  if (REC == 2) return linear5f(a, b, c, d, e);
  if (REC == 4) return teno5f(a, b, c, d, e);
  if (REC == 5) return wenoao5f(a, b, c, d, e);
  if (REC != 3) return weno5f(a, b, c, d, e);
  return lin ? linear5f(a, b, c, d, e) : weno5f(a, b, c, d, e);
}

// Selector features from the characteristic fluxes g and variables v of
// fields 0, 1, 4 over the six stencil cells: the compressed consecutive
// variations s (|dg| + alpha_k |dv|) (alpha_k the field's LLF speed, s the
// sign of dg, of dv where dg is zero).
__device__ __forceinline__ void features_gv(const float (&g)[3][6], const float (&v)[3][6], const RoeF& e,
                                            float f[15]) {
  float alpha[3];
  alpha[0] = fmaxf(fabsf(e.unL - e.cL), fabsf(e.unR - e.cR));
  alpha[1] = fmaxf(fabsf(e.unL), fabsf(e.unR));
  alpha[2] = fmaxf(fabsf(e.unL + e.cL), fabsf(e.unR + e.cR));
#pragma unroll
  for (int q = 0; q < 3; ++q)
#pragma unroll
    for (int m = 1; m < 6; ++m) {
      const float dg = g[q][m] - g[q][m - 1], dv = v[q][m] - v[q][m - 1];
      const float mag = fmaf(alpha[q], fabsf(dv), fabsf(dg));
      f[5 * q + m - 1] = compress_diff((dg != 0.f) ? copysignf(mag, dg) : copysignf(mag, dv));
    }
}

// Characteristic values of fields 0, 1, 4 of a conserved (or flux) vector X,
// sharing the terms of the left eigenvector rows: l0 X = A + B, l4 X = A - B,
// l1 X = X0 - 2A with A = b2/2 X0 + b1/2 (X4 - un X1 - ut1 X2 - ut2 X3) and
// B = (un X0 - X1) / (2c).
__device__ __forceinline__ void char014(const float X[5], const RoeF& e, float& x0, float& x1, float& x4) {
  const float Sm = fmaf(e.un, X[1], fmaf(e.ut1, X[2], e.ut2 * X[3]));
  const float A = fmaf(0.5f * e.b2, X[0], e.hb1 * (X[4] - Sm));
  const float Bm = (0.5f * e.ic) * fmaf(e.un, X[0], -X[1]);
  x0 = A + Bm;
  x4 = A - Bm;
  x1 = fmaf(-2.f, A, X[0]);
}

// Characteristic fluxes of fields 0, 1, 4 of two cells in packed pairs,
// lane by lane the scalar evaluation: X4 = un (E + p) enters X4 - Sm as one
// fused multiply-add (-Sm formed exactly by negating its products), and
// x0, x4 = A -/+ B as fused multiply-adds.
__device__ __forceinline__ void char014f2(const float2 X[4], float2 un, float2 Ep, const RoeF& e, float2& x0,
                                          float2& x1, float2& x4) {
  const float2 nSm = f2fma(f2s(-e.un), X[1], f2fma(f2s(-e.ut1), X[2], f2mul(f2s(-e.ut2), X[3])));
  const float2 A = f2fma(f2s(0.5f * e.b2), X[0], f2mul(f2s(e.hb1), f2fma(un, Ep, nSm)));
  const float2 nt = f2fma(f2s(-e.un), X[0], X[1]);
  x0 = f2fma(f2s(-0.5f * e.ic), nt, A);
  x4 = f2fma(f2s(0.5f * e.ic), nt, A);
  x1 = f2fma(f2s(-2.f), A, X[0]);
}

// X += x times right eigenvector k of the face (columns r0 = (1, u-c, ut1,
// ut2, H-uc), r1 = (1, u, ut1, ut2, q2/2), r2 = (0, 0, 1, 0, ut1), r3 = (0, 0,
// 0, 1, ut2), r4 = (1, u+c, ut1, ut2, H+uc)).
__device__ __forceinline__ void add_rcol(const RoeF& e, int k, float x, float X[5]) {
  if (k == 0 || k == 4) {
    const float sg = (k == 0) ? -1.f : 1.f;
    X[0] += x;
    X[1] = fmaf(fmaf(sg, e.c, e.un), x, X[1]);
    X[2] = fmaf(e.ut1, x, X[2]);
    X[3] = fmaf(e.ut2, x, X[3]);
    X[4] = fmaf(fmaf(sg * e.un, e.c, e.H), x, X[4]);
  } else if (k == 1) {
    X[0] += x;
    X[1] = fmaf(e.un, x, X[1]);
    X[2] = fmaf(e.ut1, x, X[2]);
    X[3] = fmaf(e.ut2, x, X[3]);
    X[4] = fmaf(0.5f * e.q2, x, X[4]);
  } else if (k == 2) {
    X[2] += x;
    X[4] = fmaf(e.ut1, x, X[4]);
  } else {
    X[3] += x;
    X[4] = fmaf(e.ut2, x, X[4]);
  }
}

// Reconstructed face state usable by HLLC: rho > 0 and p + B > 0.
__device__ __forceinline__ bool admissible_f32(const float U[5], float gm1, float g, float B) {
  if (!(U[0] > 0.f)) return false;
  const float q2 = fmaf(U[1], U[1], fmaf(U[2], U[2], U[3] * U[3])) * frcp(U[0]);
  return fmaf(gm1, fmaf(-0.5f, q2, U[4]), -g * B) + B > 0.f;
}

// HLLC (Toro, Spruce & Speares 1994) between direction-frame states UL, UR:
// Einfeldt outer speeds from the Roe average of the two states, contact speed
// from the momentum balance, F_L / F*_L / F*_R / F_R by the sign pattern.
__device__ __forceinline__ void hllc_f32(const float UL[5], const float UR[5], float gm1, float g, float B,
                                         float F[5]) {
  const float rsL = rsqrtf(UL[0]), rsR = rsqrtf(UR[0]);
  const float irL = rsL * rsL, irR = rsR * rsR;
  const float uL = UL[1] * irL, vL = UL[2] * irL, wL = UL[3] * irL;
  const float uR = UR[1] * irR, vR = UR[2] * irR, wR = UR[3] * irR;
  const float pL = fmaf(gm1, fmaf(-0.5f * UL[0], fmaf(uL, uL, fmaf(vL, vL, wL * wL)), UL[4]), -g * B);
  const float pR = fmaf(gm1, fmaf(-0.5f * UR[0], fmaf(uR, uR, fmaf(vR, vR, wR * wR)), UR[4]), -g * B);
  const float cL = sqrtf(g * (pL + B) * irL), cR = sqrtf(g * (pR + B) * irR);
  const float sL = UL[0] * rsL, sR = UR[0] * rsR, iden = frcp(sL + sR);
  const float un = fmaf(sL, uL, sR * uR) * iden, ut1 = fmaf(sL, vL, sR * vR) * iden, ut2 = fmaf(sL, wL, sR * wR) * iden;
  const float H = fmaf(UL[4] + pL, rsL, (UR[4] + pR) * rsR) * iden;
  const float c = sqrtf(gm1 * fmaf(-0.5f, fmaf(un, un, fmaf(ut1, ut1, ut2 * ut2)), H));
  const float SL = fminf(uL - cL, un - c), SR = fmaxf(uR + cR, un + c);
  const float mL = UL[0] * (SL - uL), mR = UR[0] * (SR - uR);
  const float Ss = fmaf(uL, mL, fmaf(-uR, mR, pR - pL)) * frcp(mL - mR);
  const bool left = Ss >= 0.f;
  const float* U = left ? UL : UR;
  const float SK = (SL >= 0.f) ? 0.f : ((SR <= 0.f) ? 0.f : (left ? SL : SR));
  const float uK = left ? uL : uR, vK = left ? vL : vR, wK = left ? wL : wR, pK = left ? pL : pR;
  const float mK = left ? mL : mR, irK = left ? irL : irR;
  // upwind physical flux of the side the contact leaves behind x/t = 0
  const bool useL = (SL >= 0.f) || (SR > 0.f && left);
  const float* UK = useL ? UL : UR;
  const float uF = useL ? uL : uR, vF = useL ? vL : vR, wF = useL ? wL : wR, pF = useL ? pL : pR;
  F[0] = UK[1];
  F[1] = fmaf(UK[1], uF, pF);
  F[2] = UK[1] * vF;
  F[3] = UK[1] * wF;
  F[4] = uF * (UK[4] + pF);
  if (SK != 0.f) {
    const float fac = mK * frcp(SK - Ss);
    const float Es = fac * fmaf(Ss - uK, Ss + pK * frcp(mK), U[4] * irK);
    F[0] = fmaf(SK, fac - U[0], F[0]);
    F[1] = fmaf(SK, fmaf(fac, Ss, -U[1]), F[1]);
    F[2] = fmaf(SK, fmaf(fac, vK, -U[2]), F[2]);
    F[3] = fmaf(SK, fmaf(fac, wK, -U[3]), F[3]);
    F[4] = fmaf(SK, Es - U[4], F[4]);
  }
}

// True when the record at c equals the record at c0 in all six fields, read
// through cell_uf2's own expressions so that the loads are shared with it.
__device__ __forceinline__ bool same_record(const float* __restrict__ S, int c, int c0, Rot R) {
  return (S[c] == S[c0]) & (S[R.n + c] == S[R.n + c0]) & (S[R.t1 + c] == S[R.t1 + c0]) &
         (S[R.t2 + c] == S[R.t2 + c0]) & (S[4 * SF_REG + c] == S[4 * SF_REG + c0]) &
         (S[5 * SF_REG + c] == S[5 * SF_REG + c0]);
}

// Face flux between stencil cells 2 and 3 (cells at S index c0 + m*st, m = 0..5)
// from the FP32 records; result in the direction frame.  With FLAT, *flat
// tells whether the six records are identical, in which case every selector
// feature of the face is exactly zero (tested on the flux's own loads: a
// separate test that read the 36 values again cost the selector stage 12%).
template <int MODE, bool FLAT = false>
__device__ __forceinline__ void face_flux_f32(const float* __restrict__ S, int c0, int st, Rot R, float gm1, float g,
                                              float B, bool lin, float F[5], bool* flat = nullptr) {
  constexpr int FLUX = (MODE >> 3) & 3;
  float Ur[6][5], Fr[6][5];
#pragma unroll
  for (int m = 0; m < 6; m += 2) cell_uf2(S, c0 + m * st, c0 + (m + 1) * st, R, Ur[m], Ur[m + 1], Fr[m], Fr[m + 1]);
  if constexpr (FLAT) {
    bool fl = true;
#pragma unroll
    for (int m = 1; m < 6; ++m) fl = fl & same_record(S, c0 + m * st, c0, R);
    *flat = fl;
  }
  const RoeF e = roe_f32(S, c0 + 2 * st, c0 + 3 * st, gm1, g, B, R);
  if constexpr (FLUX == 2) {
    // HLLC: characteristic variables reconstructed from both sides, back to states
    float UL[5] = {0.f, 0.f, 0.f, 0.f, 0.f}, UR[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    float V[5][6];
#pragma unroll
    for (int m = 0; m < 6; ++m) {
      char014(Ur[m], e, V[0][m], V[1][m], V[4][m]);
      V[2][m] = fmaf(-e.ut1, Ur[m][0], Ur[m][2]);
      V[3][m] = fmaf(-e.ut2, Ur[m][0], Ur[m][3]);
    }
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      add_rcol(e, k, rec5<MODE>(false, V[k][0], V[k][1], V[k][2], V[k][3], V[k][4]), UL);
      add_rcol(e, k, rec5<MODE>(false, V[k][5], V[k][4], V[k][3], V[k][2], V[k][1]), UR);
    }
    if (!admissible_f32(UL, gm1, g, B) || !admissible_f32(UR, gm1, g, B)) {
#pragma unroll
      for (int j = 0; j < 5; ++j) {
        UL[j] = Ur[2][j];
        UR[j] = Ur[3][j];
      }
    }
    hllc_f32(UL, UR, gm1, g, B, F);
    return;
  }
  // characteristic fluxes of all fields (l2 F = F2 - ut1 F0, l3 F = F3 - ut2 F0)
  float Gall[5][6];
#pragma unroll
  for (int m = 0; m < 6; m += 2) {
    // two cells in packed pairs (flux components 0-3, and u_n, E + p for the
    // energy flux)
    float2 X[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) X[v] = make_float2(Fr[m][v], Fr[m + 1][v]);
    const int ca = c0 + m * st, cb = c0 + (m + 1) * st;
    const float2 un = make_float2(S[R.n + ca], S[R.n + cb]);
    const float2 Ep = make_float2(S[5 * SF_REG + ca] + S[4 * SF_REG + ca], S[5 * SF_REG + cb] + S[4 * SF_REG + cb]);
    float2 g0, g1, g4;
    char014f2(X, un, Ep, e, g0, g1, g4);
    const float2 g2 = f2fma(f2s(-e.ut1), X[0], X[2]), g3 = f2fma(f2s(-e.ut2), X[0], X[3]);
    Gall[0][m] = g0.x;
    Gall[0][m + 1] = g0.y;
    Gall[1][m] = g1.x;
    Gall[1][m + 1] = g1.y;
    Gall[2][m] = g2.x;
    Gall[2][m + 1] = g2.y;
    Gall[3][m] = g3.x;
    Gall[3][m + 1] = g3.y;
    Gall[4][m] = g4.x;
    Gall[4][m + 1] = g4.y;
  }
  float Fh0 = 0.f, Fh1 = 0.f, Fh2 = 0.f, Fh3 = 0.f, Fh4 = 0.f;
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    // the selector decides for the acoustic and entropy fields; shear fields keep WENO5
    const bool use_lin = (MODE == 3) && lin && (k == 0 || k == 1 || k == 4);
    float G[6];
#pragma unroll
    for (int m = 0; m < 6; ++m) G[m] = Gall[k][m];
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
    const bool pos = FLUX == 0 && lL > 0.f && lR > 0.f && lt > 0.f;
    const bool llf = FLUX == 1 || (!pos && !(lL < 0.f && lR < 0.f && lt < 0.f));
    // upwind: W+ of G (pos) or W- of G; LLF: W+ of (G + a V)/2 and W- of (G - a V)/2
    float gh;
    if (pos) {
      gh = rec5<MODE>(use_lin, G[0], G[1], G[2], G[3], G[4]);
    } else if (!llf) {
      gh = rec5<MODE>(use_lin, G[5], G[4], G[3], G[2], G[1]);
    } else {
      float l[5], V[6];
      lrow_f32(e, k, l);
      if (k == 2 || k == 3) {
        const int j = (k == 2) ? 2 : 3;
#pragma unroll
        for (int m = 0; m < 6; ++m) V[m] = fmaf(l[0], Ur[m][0], Ur[m][j]);
      } else {
#pragma unroll
        for (int m = 0; m < 6; ++m)
          V[m] = fmaf(l[0], Ur[m][0], fmaf(l[1], Ur[m][1], fmaf(l[2], Ur[m][2], fmaf(l[3], Ur[m][3], l[4] * Ur[m][4]))));
      }
      const float ha = 0.5f * fmaxf(fabsf(lL), fabsf(lR));
      float fp[6], fm[6];
#pragma unroll
      for (int m = 0; m < 6; ++m) {
        fp[m] = fmaf(0.5f, G[m], ha * V[m]);
        fm[m] = fmaf(0.5f, G[m], -ha * V[m]);
      }
      constexpr int REC = MODE & 7;
      if constexpr (REC == 0 || REC == 1 || REC == 3) {
        // the split's two WENO5 reconstructions as one packed evaluation
        if (REC == 3 && use_lin) {
          gh = linear5f(fp[0], fp[1], fp[2], fp[3], fp[4]) + linear5f(fm[5], fm[4], fm[3], fm[2], fm[1]);
        } else {
          const float2 r = weno5f2(make_float2(fp[0], fm[5]), make_float2(fp[1], fm[4]), make_float2(fp[2], fm[3]),
                                   make_float2(fp[3], fm[2]), make_float2(fp[4], fm[1]));
          gh = r.x + r.y;
        }
      } else {
        gh = rec5<MODE>(use_lin, fp[0], fp[1], fp[2], fp[3], fp[4]) + rec5<MODE>(use_lin, fm[5], fm[4], fm[3], fm[2], fm[1]);
      }
    }
    // F_hat = R g_hat, columns r0 = (1, u-c, ut1, ut2, H-uc), r1 = (1, u, ut1, ut2, q2/2),
    // r2 = (0, 0, 1, 0, ut1), r3 = (0, 0, 0, 1, ut2), r4 = (1, u+c, ut1, ut2, H+uc)
    if (k == 0 || k == 4) {
      const float sg = (k == 0) ? -1.f : 1.f;
      Fh0 += gh;
      Fh1 = fmaf(fmaf(sg, e.c, e.un), gh, Fh1);
      Fh2 = fmaf(e.ut1, gh, Fh2);
      Fh3 = fmaf(e.ut2, gh, Fh3);
      Fh4 = fmaf(fmaf(sg * e.un, e.c, e.H), gh, Fh4);
    } else if (k == 1) {
      Fh0 += gh;
      Fh1 = fmaf(e.un, gh, Fh1);
      Fh2 = fmaf(e.ut1, gh, Fh2);
      Fh3 = fmaf(e.ut2, gh, Fh3);
      Fh4 = fmaf(0.5f * e.q2, gh, Fh4);
    } else if (k == 2) {
      Fh2 += gh;
      Fh4 = fmaf(e.ut1, gh, Fh4);
    } else {
      Fh3 += gh;
      Fh4 = fmaf(e.ut2, gh, Fh4);
    }
  }
  F[0] = Fh0;
  F[1] = Fh1;
  F[2] = Fh2;
  F[3] = Fh3;
  F[4] = Fh4;
}

// Velocity of the stored cell s of a block's FP64 state, in FP32.
__device__ __forceinline__ void cell_vel_f32(const double* __restrict__ u, int s, float w[3]) {
  const float ir = frcp(d2f_fast(u[s]));
  w[0] = d2f_fast(u[NCELL + s]) * ir;
  w[1] = d2f_fast(u[2 * NCELL + s]) * ir;
  w[2] = d2f_fast(u[3 * NCELL + s]) * ir;
}

// F -= the viscous flux at the face between stored cells sL and sL + step_D
// of the block (FP64 state with halos, arithmetic in FP32), F in the
// direction frame of D: second-order compact gradients (normal derivative
// from the two face cells, tangential ones as the mean of their central
// differences), tau = mu (grad u + grad u^T) - 2/3 mu (div u) I, energy flux
// u_face . tau_D.
template <int D>
__device__ __forceinline__ void sub_viscous_f32(const double* __restrict__ u, int sL, float mu, float idx,
                                                float F[5]) {
  constexpr int step[3] = {1, NS, NS * NS};
  const int sR = sL + step[D];
  float uL[3], uR[3];
  cell_vel_f32(u, sL, uL);
  cell_vel_f32(u, sR, uR);
  float G[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i) G[i][D] = (uR[i] - uL[i]) * idx;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    if (j == D) continue;
    float a[3], b[3], c[3], e[3];
    cell_vel_f32(u, sL + step[j], a);
    cell_vel_f32(u, sL - step[j], b);
    cell_vel_f32(u, sR + step[j], c);
    cell_vel_f32(u, sR - step[j], e);
#pragma unroll
    for (int i = 0; i < 3; ++i) G[i][j] = ((a[i] - b[i]) + (c[i] - e[i])) * (0.25f * idx);
  }
  const float div = G[0][0] + G[1][1] + G[2][2];
  float tau[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) tau[i] = mu * (G[i][D] + G[D][i]);
  tau[D] = fmaf(-2.f / 3.f * mu, div, tau[D]);
  const float E = fmaf(0.5f * (uL[0] + uR[0]), tau[0],
                       fmaf(0.5f * (uL[1] + uR[1]), tau[1], 0.5f * (uL[2] + uR[2]) * tau[2]));
  F[1] -= tau[D];
  F[2] -= tau[(D + 1) % 3];
  F[3] -= tau[(D + 2) % 3];
  F[4] -= E;
}

// Selector features of the face between records c0+2st and c0+3st, for the
// stage-0 selector kernel and the training samples alike.  The characteristic
// fluxes of fields 0, 1, 4 are the face flux's own (two cells per packed
// instruction, bitwise the same values), so the features are those of the
// fluxes the kernel computes.
__device__ __forceinline__ void face_features_f32(const float* __restrict__ S, int c0, int st, Rot R, const RoeF& e,
                                                  float f[15]) {
  float g[3][6], v[3][6];
#pragma unroll
  for (int m = 0; m < 6; m += 2) {
    float Ua[5], Ub[5], Fa[5], Fb[5];
    cell_uf2(S, c0 + m * st, c0 + (m + 1) * st, R, Ua, Ub, Fa, Fb);
    float2 X[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) X[q] = make_float2(Fa[q], Fb[q]);
    const int ca = c0 + m * st, cb = c0 + (m + 1) * st;
    const float2 un = make_float2(S[R.n + ca], S[R.n + cb]);
    const float2 Ep = make_float2(S[5 * SF_REG + ca] + S[4 * SF_REG + ca], S[5 * SF_REG + cb] + S[4 * SF_REG + cb]);
    float2 g0, g1, g4;
    char014f2(X, un, Ep, e, g0, g1, g4);
    g[0][m] = g0.x;
    g[0][m + 1] = g0.y;
    g[1][m] = g1.x;
    g[1][m + 1] = g1.y;
    g[2][m] = g4.x;
    g[2][m + 1] = g4.y;
    char014(Ua, e, v[0][m], v[1][m], v[2][m]);
    char014(Ub, e, v[0][m + 1], v[1][m + 1], v[2][m + 1]);
  }
  features_gv(g, v, e, f);
}

// Region layouts of one slab (records in S, x fastest; rows of the x
// direction hold 24 slots, x = -4 .. 19, so that every run of four cells
// starting at a multiple of 4 is one 16-byte chunk in shared memory):
//   x region (MODE 1, D = 0): slot (kz * 16 + y) * 24 + x + 4, y in [0, 16);
//   y region (MODE 1, D = 1): slot (kz * 22 + y + 3) * 16 + x, y in [-3, 19);
//   z region (D = 2):         slot ((z - z0 + 3) * 16 + y) * 16 + x, z in [z0-3, z0+7);
//   x-y region (MODES 0, 2, 3): slot (kz * 22 + y + 3) * 24 + x + 4, x, y in
//   [-4, 20) x [-3, 19) except the corners (outside the block in both).
__device__ __forceinline__ int region_cells(int D) { return D == 2 ? SF_REG : (D == 0 ? 24 * 16 * SF_TZ : 22 * 16 * SF_TZ); }
__device__ __forceinline__ int region_faces(int D) { return D == 2 ? SF_NFZ : SF_NFX; }
__device__ __forceinline__ int region_stride(int D) { return sel3i(D, 1, 16, 256); }

// FP32 primitive record (rho, vx, vy, vz, p, E) of FP64 conserved values.
__device__ __forceinline__ void make_record(double r64, double mx64, double my64, double mz64, double E64, float g,
                                            float B, float gm1, float rec[6]) {
  const float r = d2f_fast(r64), mx = d2f_fast(mx64), my = d2f_fast(my64);
  const float mz = d2f_fast(mz64), E = d2f_fast(E64);
  const float ir = frcp(r);
  const float vx = mx * ir, vy = my * ir, vz = mz * ir;
  const float q2 = fmaf(vx, vx, fmaf(vy, vy, vz * vz));
  rec[0] = r;
  rec[1] = vx;
  rec[2] = vy;
  rec[3] = vz;
  rec[4] = fmaf(gm1, fmaf(-0.5f * r, q2, E), -g * B);
  rec[5] = E;
}

// One FP32 primitive record from the FP64 conserved state at s.
__device__ __forceinline__ void put_record(const double* __restrict__ src, int s, float* __restrict__ S, int idx,
                                           float g, float B, float gm1) {
  float rec[6];
  make_record(src[s], src[NCELL + s], src[2 * NCELL + s], src[3 * NCELL + s], src[4 * NCELL + s], g, B, gm1, rec);
#pragma unroll
  for (int f = 0; f < SF_NREC; ++f) S[f * SF_REG + idx] = rec[f];
}

// 16-byte asynchronous copy from global to shared memory (L2 only); both
// addresses 16-byte aligned.
__device__ __forceinline__ void cp_async16(float* smem, const float* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// Sources of a slab's region: the block's FP64 stage buffer (stored cells,
// for its predicted and boundary halo regions) and the FP32 records of the
// internal cells of the block and of its same-level face neighbours (x-, x+,
// y-, y+, z-, z+; null where there is none, and then the block's own halo
// is read).  sh is null when the context keeps no records: everything is
// then converted from the block's own stored cells.
struct RegionSrc {
  const double* u;
  const float* sh;
  const float* nsh[6];
};

// Source of the chunk of four cells along x from x0 at (y, z) in block
// coordinates (x0 a multiple of 4, at most one coordinate outside the block):
// the FP32 records of the block or of the same-level face neighbour on that
// side, or null (the block's own stored halo, converted from FP64).
__device__ __forceinline__ const float* chunk_src(const RegionSrc& R, int x0, int y, int z) {
  if (!R.sh) return nullptr;
  int side = -1;
  if (x0 < 0) side = 0;
  else if (x0 >= NB) side = 1;
  else if (y < 0) side = 2;
  else if (y >= NB) side = 3;
  else if (z < 0) side = 4;
  else if (z >= NB) side = 5;
  if (side < 0) return R.sh + (z * NB + y) * NB + x0;
  // (selects, not an indexed load: R stays in registers)
  const float* n = (side == 0) ? R.nsh[0]
                 : (side == 1) ? R.nsh[1]
                 : (side == 2) ? R.nsh[2]
                 : (side == 3) ? R.nsh[3]
                 : (side == 4) ? R.nsh[4] : R.nsh[5];
  if (!n) return nullptr;
  const int d = (side & 1) ? -NB : NB;
  if (side < 2) x0 += d;
  else if (side < 4) y += d;
  else z += d;
  return n + (z * NB + y) * NB + x0;
}

// The chunk at (x0, y, z) and the same chunk on the next nk - 1 planes (z + k,
// same source block) -> slots slot + k * slot_step of S: one 16-byte
// asynchronous copy per field and plane, or (own halo) four records
// converted from FP64.
__device__ __forceinline__ void chunk_planes(const RegionSrc& R, int x0, int y, int z, int nk, float* __restrict__ S,
                                             int slot, int slot_step, float g, float B, float gm1) {
  const float* src = chunk_src(R, x0, y, z);
  for (int k = 0; k < nk; ++k) {
    if (src) {
#pragma unroll
      for (int f = 0; f < SF_NREC; ++f)
        cp_async16(S + f * SF_REG + slot + k * slot_step, src + f * NINT + k * NB * NB);
    } else {
#pragma unroll
      for (int c = 0; c < 4; ++c) put_record(R.u, sidx(x0 + c, y, z + k), S, slot + k * slot_step + c, g, B, gm1);
    }
  }
}

// Stencil region of direction D for the slab at z0 -> records in S (layouts
// above).  Each thread owns one chunk position of a plane and copies it on
// a fixed set of planes; every copy has landed when the caller's next
// barrier is passed.
__device__ __forceinline__ void load_region_f32(int D, const RegionSrc& R, float* __restrict__ S, int z0, float g,
                                                float B, float gm1) {
  const int t = threadIdx.x;
  if (D == 0) {                 // 96 chunk positions per plane (16 rows of 6), two planes per thread
    if (t < 192) {
      const int c = t % 96, kz = t / 96, y = c / 6, q = c % 6;
      chunk_planes(R, 4 * q - 4, y, z0 + kz, 1, S, (kz * 16 + y) * 24 + 4 * q, 0, g, B, gm1);
      chunk_planes(R, 4 * q - 4, y, z0 + kz + 2, 1, S, ((kz + 2) * 16 + y) * 24 + 4 * q, 0, g, B, gm1);
    }
  } else if (D == 1) {          // 88 chunk positions per plane (22 rows of 4), two planes per thread
    if (t < 176) {
      const int c = t % 88, kz = t / 88, r = c / 4, q = c % 4;
      chunk_planes(R, 4 * q, r - 3, z0 + kz, 1, S, (kz * 22 + r) * 16 + 4 * q, 0, g, B, gm1);
      chunk_planes(R, 4 * q, r - 3, z0 + kz + 2, 1, S, ((kz + 2) * 22 + r) * 16 + 4 * q, 0, g, B, gm1);
    }
  } else {                      // 64 chunk positions per plane, planes t/64, +4, +8 (ten planes)
    const int c = t % 64, lane = t / 64, y = c / 4, q = c % 4;
    for (int zz = lane; zz < SF_TZ + 6; zz += 4)
      chunk_planes(R, 4 * q, y, z0 - 3 + zz, 1, S, (zz * 16 + y) * 16 + 4 * q, 0, g, B, gm1);
  }
  cp_async_wait_all();
}

// The x-y region of the slab at z0 (rows of 24 slots, the corners skipped).
__device__ __forceinline__ int xy_slot(int x, int y, int kz) { return (kz * 22 + y + 3) * 24 + x + 4; }

// 120 chunk positions per plane (16 rows of 6 chunks, 6 rows of 4); threads
// 0..239 own one position on two of the four planes.
__device__ __forceinline__ void load_xy_f32(const RegionSrc& R, float* __restrict__ S, int z0, float g, float B,
                                            float gm1) {
  const int t = threadIdx.x;
  if (t < 240) {
    const int c = t % 120, kz = 2 * (t / 120);
    int x0, y;
    if (c < 96) {               // rows y in [0, 16): x = -4 .. 19
      y = c / 6;
      x0 = 4 * (c % 6) - 4;
    } else {                    // rows y in [-3, 0) and [16, 19): x = 0 .. 15
      const int r = (c - 96) / 4;
      y = (r < 3) ? r - 3 : r + 13;
      x0 = 4 * ((c - 96) % 4);
    }
    chunk_planes(R, x0, y, z0 + kz, 2, S, xy_slot(x0, y, kz), xy_slot(0, 0, 1) - xy_slot(0, 0, 0), g, B, gm1);
  }
  cp_async_wait_all();
}

// Sources of the block at `slot` with its same-level face neighbours (stage
// buffer `cur`).
__device__ __forceinline__ RegionSrc region_src(const Topo& t, const Pool& pool, int cur, int node, int slot) {
  RegionSrc R;
  R.u = pool.bufp(cur) + (size_t)slot * SLOT_U;
  R.sh = pool.shp(cur) ? pool.shp(cur) + (size_t)slot * SLOT_SH : nullptr;
  const int rn[6] = {12, 14, 10, 16, 4, 22};
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    const int nb = R.sh ? t.nbr[(size_t)node * 27 + rn[q]] : -1;
    R.nsh[q] = (nb >= 0) ? pool.shp(cur) + (size_t)t.slot[nb] * SLOT_SH : nullptr;
  }
  return R;
}

// Face f of direction D in the slab (per-direction regions): first stencil
// record c0 and the face's position (fa along D; ta, tb the block-face
// coordinates of a boundary face).
__device__ __forceinline__ void face_of(int D, int f, int z0, int& fa, int& c0, int& ta, int& tb) {
  if (D == 0) {
    fa = f % 17;
    const int r = f / 17;                 // row = kz * 16 + j
    c0 = r * 24 + fa + 1;                 // cell x = fa - 3 at record index fa + 1
    ta = r % 16;
    tb = z0 + r / 16;
  } else if (D == 1) {
    const int i = f % 16, r = f / 16;     // r = kz * 17 + fa
    fa = r % 17;
    const int kz = r / 17;
    c0 = (kz * 22 + fa) * 16 + i;
    ta = i;
    tb = z0 + kz;
  } else {
    const int i = f % 16, j = (f / 16) % 16;
    fa = f / 256;
    c0 = (fa * 16 + j) * 16 + i;
    ta = i;
    tb = j;
  }
}

// Per-CTA state of the learned selector (MODES 1 and 3) and of the viscous
// variants (MODE bit 5).
struct LearnedCtx {
  const float* P;            // FP32 parameters (biases read from here)
  const uint32_t* frag;      // BF16 B fragments in shared memory
  uint32_t* rows;            // per-warp feature rows
  float* logit;              // per-warp logits
  float tau;                 // linear when logit < tau
  unsigned long long* count; // [0] faces sent to linear, [1] faces evaluated (nullable)
  uint32_t* bits;            // this block's decision words (SLOT_SEL)
  float z0;                  // the network's logit for all-zero features
  const uint32_t* selw;      // MODE 3: the slab's 108 decision words, staged in shared memory
  float mu, idx;             // viscous variants: dynamic viscosity and 1 / dx of the block
};

// Direction-frame flux components (normal, tangential 1, tangential 2) of
// direction D -> lab components x, y, z.
__device__ __forceinline__ void to_lab(int D, float n, float t1, float t2, float& x, float& y, float& z) {
  x = sel3(D, n, t2, t1);
  y = sel3(D, t1, n, t2);
  z = sel3(D, t2, t1, n);
}

// Store face f's flux (direction frame of D) into the flux slots (row length
// fstr per variable), and into
// the block's face buffer (lab frame, FP64) when the face is on the block
// boundary (gface 0 or 16 along D).
__device__ __forceinline__ void store_face(int D, const float F[5], float* __restrict__ Fs, int fstr, int f, int gface,
                                           int ta, int tb, double* __restrict__ fb) {
#pragma unroll
  for (int v = 0; v < 5; ++v) Fs[v * fstr + f] = F[v];
  if (gface == 0 || gface == NB) {
    const int side = 2 * D + (gface == NB ? 1 : 0);
    float Fl[5];
    Fl[0] = F[0];
    Fl[4] = F[4];
    to_lab(D, F[1], F[2], F[3], Fl[1], Fl[2], Fl[3]);
#pragma unroll
    for (int v = 0; v < 5; ++v) fb[((side * NV + v) * NB + tb) * NB + ta] = f2d_fast(Fl[v]);
  }
}

// acc[kz][.] += flux difference of direction D at column (ti, tj); lo, hi the
// slots of the cell's lower and upper faces.
__device__ __forceinline__ void add_diff(int D, const float* __restrict__ Fs, int fstr, int lo, int hi,
                                         float (&a)[NV]) {
  float d[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) d[v] = Fs[v * fstr + lo] - Fs[v * fstr + hi];
  float dx, dy, dz;
  to_lab(D, d[1], d[2], d[3], dx, dy, dz);
  a[0] += d[0];
  a[1] += dx;
  a[2] += dy;
  a[3] += dz;
  a[4] += d[4];
}

// Per-direction sweep (the stage-0 selector variant, MODE 1): region of D,
// faces with WENO5 fluxes and the selector's decisions, flux differences.
template <int MODE>
__device__ __forceinline__ void sweep_f32(int D, const Topo& t, const Pool& pool, int cur, int node, int slot,
                                          double* __restrict__ fb, float* __restrict__ S, float* __restrict__ Fs,
                                          int z0, float g, float B, float gm1, float (&acc)[SF_TZ][NV],
                                          const LearnedCtx& L, unsigned (&cnt)[2]) {   // cnt: the warp's census
  const int ti = threadIdx.x & 15, tj = threadIdx.x >> 4;
  // the x-y region serves the x and the y faces (loaded for D = 0 and kept
  // for D = 1), the z region the z faces
  if (D != 1) {
    if (D == 0) load_xy_f32(region_src(t, pool, cur, node, slot), S, z0, g, B, gm1);
    else load_region_f32(2, region_src(t, pool, cur, node, slot), S, z0, g, B, gm1);
    __syncthreads();
  }
  const int nf = region_faces(D);
  const int st = sel3i(D, 1, 24, 256);
  const Rot R = rot_of(D);
  const int nfr = ((nf + blockDim.x - 1) / blockDim.x) * blockDim.x;
  for (int f0 = threadIdx.x; f0 < nfr; f0 += blockDim.x) {
    const bool act = f0 < nf;
    const int f = act ? f0 : 0;
    int fa, c0, ta, tb;
    face_of(D, f, z0, fa, c0, ta, tb);
    if (D == 0) c0 = xy_slot(fa - 3, (f / 17) % 16, f / 17 / 16);
    else if (D == 1) c0 = xy_slot(f % 16, fa - 3, f / 16 / 17);
    // decision word of this warp's 32 consecutive faces
    uint32_t* word = L.bits + (z0 / SF_TZ) * 108 + D * 34 + (f0 >> 5);
    // WENO5 fluxes, then the selector's features of the same faces.  Flat
    // stencils have all-zero features, whose logit z0 is known: a warp
    // computes features and runs the tensor-core MLP only when one of its
    // faces is not flat (on the shock-bubble tree about 70% of the warps are
    // all flat), and its flat lanes skip the features
    float F[5], fe[15];
    bool flat = true;
    if (act) face_flux_f32<MODE, true>(S, c0, st, R, gm1, g, B, false, F, &flat);
    float z = L.z0;
    if (!__all_sync(0xffffffffu, flat)) {
      if (flat) {
#pragma unroll
        for (int q = 0; q < 15; ++q) fe[q] = 0.f;
      } else {
        const RoeF e = roe_f32(S, c0 + 2 * st, c0 + 3 * st, gm1, g, B, R);
        face_features_f32(S, c0, st, R, e, fe);
      }
      const int wid = threadIdx.x >> 5;
      mlp_put_row(L.rows + wid * 32 * 9, fe);
      z = mlp_warp_logit(L.P, L.frag, L.rows + wid * 32 * 9, L.logit + wid * 32);
    }
    const bool dl = act && (z < L.tau);
    const unsigned bl = __ballot_sync(0xffffffffu, dl), ba = __ballot_sync(0xffffffffu, act);
    // (a warp past the direction's last face writes nothing: its word index
    // would fall among the next direction's words)
    if ((threadIdx.x & 31) == 0 && ba) {
      *word = bl;
      cnt[0] += __popc(bl);
      cnt[1] += __popc(ba);
    }
    if (!act) continue;
    store_face(D, F, Fs, SF_NFZ, f, (D == 2) ? z0 + fa : fa, ta, tb, fb);
  }
  __syncthreads();
#pragma unroll
  for (int kz = 0; kz < SF_TZ; ++kz) {
    int lo, hi;
    if (D == 0) { lo = (kz * 16 + tj) * 17 + ti; hi = lo + 1; }
    else if (D == 1) { lo = (kz * 17 + tj) * 16 + ti; hi = lo + 16; }
    else { lo = (kz * 16 + tj) * 16 + ti; hi = lo + 256; }
    add_diff(D, Fs, SF_NFZ, lo, hi, acc[kz]);
  }
  __syncthreads();
}

// x and y directions of the slab together (MODES 0, 2, 3): one region, one
// loop over the 1088 x faces followed by the 1088 y faces, through a single
// call site of the face flux (the two directions differ only in the stencil
// stride and the rotation's offsets, so one inlined copy serves both; 1.5%
// faster than one copy per direction).
template <int MODE>
__device__ __forceinline__ void sweep_xy(const double* __restrict__ u, const Topo& t, const Pool& pool, int cur,
                                         int node, int slot, double* __restrict__ fb, float* __restrict__ S,
                                         float* __restrict__ Fs, int z0, float g, float B, float gm1,
                                         float (&acc)[SF_TZ][NV], const LearnedCtx& L) {
  const int ti = threadIdx.x & 15, tj = threadIdx.x >> 4;
  load_xy_f32(region_src(t, pool, cur, node, slot), S, z0, g, B, gm1);
  __syncthreads();
  for (int f = threadIdx.x; f < 2 * SF_NFX; f += blockDim.x) {
    float F[5];
    const bool isx = f < SF_NFX;          // warp-uniform (1088 = 34 warps)
    int fa, c0, ta, tb, st, wi;
    if (isx) {
      fa = f % 17;
      const int r = f / 17;               // r = kz * 16 + j
      c0 = xy_slot(fa - 3, r % 16, r / 16);
      ta = r % 16;
      tb = z0 + r / 16;
      st = 1;
      wi = f >> 5;
    } else {
      const int fy = f - SF_NFX;
      const int i = fy % 16, r = fy / 16; // r = kz * 17 + fa
      fa = r % 17;
      c0 = xy_slot(i, fa - 3, r / 17);
      ta = i;
      tb = z0 + r / 17;
      st = 24;
      wi = 34 + (fy >> 5);
    }
    const bool lin = (MODE == 3) && ((L.selw[wi] >> (threadIdx.x & 31)) & 1u);
    face_flux_f32<MODE>(S, c0, st, isx ? rot_of(0) : rot_of(1), gm1, g, B, lin, F);
    if (MODE & 32) {
      if (isx) sub_viscous_f32<0>(u, sidx(fa - 1, ta, tb), L.mu, L.idx, F);
      else sub_viscous_f32<1>(u, sidx(ta, fa - 1, tb), L.mu, L.idx, F);
    }
    store_face(isx ? 0 : 1, F, Fs, SF_FMAX, f, fa, ta, tb, fb);
  }
  __syncthreads();
#pragma unroll
  for (int kz = 0; kz < SF_TZ; ++kz) {
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[kz][v] = 0.f;
    const int lx = (kz * 16 + tj) * 17 + ti, ly = SF_NFX + (kz * 17 + tj) * 16 + ti;
    add_diff(0, Fs, SF_FMAX, lx, lx + 1, acc[kz]);
    add_diff(1, Fs, SF_FMAX, ly, ly + 16, acc[kz]);
  }
  __syncthreads();
}

// z direction of the slab (MODES 0, 2, 3).
template <int MODE>
__device__ __forceinline__ void sweep_z(const double* __restrict__ u, const Topo& t, const Pool& pool, int cur,
                                        int node, int slot, double* __restrict__ fb, float* __restrict__ S,
                                        float* __restrict__ Fs, int z0, float g, float B, float gm1,
                                        float (&acc)[SF_TZ][NV], const LearnedCtx& L) {
  const int ti = threadIdx.x & 15, tj = threadIdx.x >> 4;
  load_region_f32(2, region_src(t, pool, cur, node, slot), S, z0, g, B, gm1);
  __syncthreads();
  for (int f = threadIdx.x; f < SF_NFZ; f += blockDim.x) {
    const int i = f % 16, j = (f / 16) % 16, fa = f / 256;
    const int c0 = (fa * 16 + j) * 16 + i;
    const bool lin = (MODE == 3) && ((L.selw[68 + (f >> 5)] >> (threadIdx.x & 31)) & 1u);
    float F[5];
    face_flux_f32<MODE>(S, c0, 256, rot_of(2), gm1, g, B, lin, F);
    if (MODE & 32) sub_viscous_f32<2>(u, sidx(i, j, z0 + fa - 1), L.mu, L.idx, F);
    store_face(2, F, Fs, SF_FMAX, f, z0 + fa, i, j, fb);
  }
  __syncthreads();
#pragma unroll
  for (int kz = 0; kz < SF_TZ; ++kz) {
    const int lo = (kz * 16 + tj) * 16 + ti;
    add_diff(2, Fs, SF_FMAX, lo, lo + 256, acc[kz]);
  }
  __syncthreads();
}

template <int MODE>
__global__ void __launch_bounds__(SF_THREADS, 2)
    k_stage_f32(Topo t, Phys p, Pool pool, int cur, int stage, const double* __restrict__ dt,
                double* __restrict__ rhs_out, int level) {
  extern __shared__ __align__(16) float sf_smem[];
  float* S = sf_smem;
  float* Fs = sf_smem + SF_NREC * SF_REG;
  const int nitems = stage_nodes(t, level) * SF_NSLAB;
  const double* __restrict__ src = pool.bufp(cur);
  double* __restrict__ dst = pool.bufp(cur ^ 1);
  const float g = (float)p.gamma, B = (float)p.B, gm1 = (float)(p.gamma - 1.0);
  const int ti = threadIdx.x & 15, tj = threadIdx.x >> 4;
  __shared__ uint32_t sel_sh[108];
  LearnedCtx L{nullptr, nullptr, nullptr, nullptr, 0.f, nullptr, nullptr, 0.f, sel_sh, (float)p.mu, 0.f};
  if (MODE == 1) {
    uint32_t* frag = reinterpret_cast<uint32_t*>(Fs + NV * SF_NFZ);   // after one direction's face fluxes
    L.P = p.mlp;
    L.frag = frag;
    L.rows = frag + FRAG_N;
    L.logit = reinterpret_cast<float*>(L.rows + (SF_THREADS / 32) * 32 * 9);
    L.tau = p.mlp_tau;
    L.count = p.lin_count;
    mlp_stage_fragments(p.mlp, frag);
    __syncthreads();
    // logit of all-zero features (same value in every lane)
    if (threadIdx.x < 32) {
      const float zero[15] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      mlp_put_row(L.rows, zero);
      const float z = mlp_warp_logit(L.P, L.frag, L.rows, L.logit);
      if (threadIdx.x == 0) L.logit[SF_THREADS - 1] = z;
    }
    __syncthreads();
    L.z0 = L.logit[SF_THREADS - 1];
    __syncthreads();
  }
  const ItemRange IR = item_range(nitems, p.blocked);
  // selector census (faces sent to linear, faces evaluated), counted by each
  // warp's lane 0 and added to the two global counters once at the end: one
  // atomic pair per 32 faces, all on the same two addresses, serialised in L2
  // and held the kernel up once the all-flat warps had become cheap
  unsigned cnt[2] = {0u, 0u};
  for (int w = IR.first; w < IR.end; w += IR.step) {
    const int li = w / SF_NSLAB, z0 = (w % SF_NSLAB) * SF_TZ;
    const int node = stage_node(t, level, li);
    const int slot = t.slot[node];
    // the update's per-block scalars, loaded here so that their latency is
    // hidden behind the sweeps (after them in the register-bound selector
    // variant)
    int lvl = 0;
    double h = 0.0;
    if (MODE != 1) {
      lvl = t.level[node];
      h = dt ? node_dt(t, p, dt, node, level) : 0.0;
    }
    const double* __restrict__ u = src + (size_t)slot * SLOT_U;
    double* __restrict__ fb = pool.face + (size_t)slot * SLOT_F;
    if (MODE == 1 || MODE == 3) L.bits = pool.sel + (size_t)slot * SLOT_SEL;
    if (MODE & 32) L.idx = d2f_fast(ldexp(1.0 / p.dx0, t.level[node]));
    // the slab's decision words (read before the first barrier of the sweep)
    if (MODE == 3 && threadIdx.x < 108) sel_sh[threadIdx.x] = L.bits[(z0 / SF_TZ) * 108 + threadIdx.x];
    float acc[SF_TZ][NV];
    if (MODE == 1) {
      // with the selector inlined, one copy of the sweep (direction at run
      // time) keeps the kernel within the instruction cache
#pragma unroll
      for (int kz = 0; kz < SF_TZ; ++kz)
#pragma unroll
        for (int v = 0; v < NV; ++v) acc[kz][v] = 0.f;
#pragma unroll 1
      for (int D = 0; D < 3; ++D) sweep_f32<MODE>(D, t, pool, cur, node, slot, fb, S, Fs, z0, g, B, gm1, acc, L, cnt);
    } else {
      sweep_xy<MODE>(u, t, pool, cur, node, slot, fb, S, Fs, z0, g, B, gm1, acc, L);
      sweep_z<MODE>(u, t, pool, cur, node, slot, fb, S, Fs, z0, g, B, gm1, acc, L);
    }
    if (MODE == 1) {
      lvl = t.level[node];
      h = dt ? node_dt(t, p, dt, node, level) : 0.0;
    }
    // 1 / dx = 2^level / dx0 (exact power-of-two scaling, no division)
    const double idx_ = ldexp(p.inv_dx0, lvl);
    const double hdx = h * idx_;
    // the stage's increment is formed in FP32: b_s dt / dx (sum of flux
    // differences) at stage 0, b_s (previous increment + dt / dx sum) after it
    // (read in place of u^(s), in the low word of its operand's register);
    // with gravity the FP64 combination a_s u^n + b_s (u^(s) + dt L) is kept
    // and the increment taken from its result
    const double ka = kRkA[rk_row(p)][stage], kb = kRkB[rk_row(p)][stage];
    const float hf = d2f_fast(hdx), bhf = d2f_fast(kb * hdx), kbf = d2f_fast(kb);
    const bool incr = pool.dl && stage != 0 && !rhs_out && !p.has_grav;
    // the thread's four cells in groups of KC: every FP64 operand of a group is
    // loaded before its first store, so those loads are in flight together
    // (groups of one cell in the register-bound selector variant)
    constexpr int KC = (MODE == 1) ? 1 : SF_TZ;
#pragma unroll
    for (int k0 = 0; k0 < SF_TZ; k0 += KC) {
      double us[KC][NV], un[KC][NV];
#pragma unroll
      for (int c = 0; c < KC; ++c) {
        const int s = sidx(ti, tj, z0 + k0 + c), ii = iidx(ti, tj, z0 + k0 + c);
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          us[c][v] = incr ? __longlong_as_double((long long)(unsigned)__float_as_uint(
                                pool.dl[(size_t)slot * SLOT_N + v * NINT + ii]))
                           : u[v * NCELL + s];
          un[c][v] = (stage != 0 && !rhs_out) ? pool.un[(size_t)slot * SLOT_N + v * NINT + ii] : 0.0;
        }
      }
#pragma unroll
      for (int c = 0; c < KC; ++c) {
        const int kz = k0 + c, k = z0 + kz;
        const int s = sidx(ti, tj, k), ii = iidx(ti, tj, k);
        double S4[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
        if (p.has_grav) {
          const double rho = us[c][0], mx = us[c][1], my = us[c][2], mz = us[c][3];
          S4[1] = rho * p.grav[0];
          S4[2] = rho * p.grav[1];
          S4[3] = rho * p.grav[2];
          S4[4] = fma(mx, p.grav[0], fma(my, p.grav[1], mz * p.grav[2]));
        }
        if (rhs_out) {
#pragma unroll
          for (int v = 0; v < 5; ++v)
            rhs_out[((size_t)li * NV + v) * NINT + ii] = fma(f2d_fast(acc[kz][v]), idx_, S4[v]);
        } else {
          double* __restrict__ unb = pool.un + (size_t)slot * SLOT_N;
          float* __restrict__ dlw = pool.dl ? pool.dl + (size_t)slot * SLOT_N : nullptr;
          double* __restrict__ o = dst + (size_t)slot * SLOT_U;
          double o5[5];
#pragma unroll
          for (int v = 0; v < 5; ++v) {
            double out;
            if (stage == 0) {
              unb[v * NINT + ii] = us[c][v];
              const float d = acc[kz][v] * hf;
              out = us[c][v] + f2d_fast(d);
              if (p.has_grav) out = fma(h, S4[v], out);
              if (dlw) dlw[v * NINT + ii] = p.has_grav ? d2f_fast(out - us[c][v]) : d;
            } else if (incr) {
              const float dp = __uint_as_float((unsigned)__double_as_longlong(us[c][v]));
              const float d = fmaf(kbf, dp, acc[kz][v] * bhf);
              out = un[c][v] + f2d_fast(d);
              dlw[v * NINT + ii] = d;
            } else {
              double inc = f2d_fast(acc[kz][v] * bhf);
              if (p.has_grav) inc = fma(kb * h, S4[v], inc);
              out = fma(ka, un[c][v], fma(kb, us[c][v], inc));
              if (dlw) dlw[v * NINT + ii] = d2f_fast(out - un[c][v]);
            }
            o[v * NCELL + s] = out;
            o5[v] = out;
          }
          // the FP32 records of the new state, read by the next stage's regions
          if (pool.shp(cur ^ 1)) {
            float rec[6];
            make_record(o5[0], o5[1], o5[2], o5[3], o5[4], g, B, gm1, rec);
            float* __restrict__ shw = pool.shp(cur ^ 1) + (size_t)slot * SLOT_SH;
#pragma unroll
            for (int f = 0; f < SF_NREC; ++f) shw[f * NINT + ii] = rec[f];
          }
        }
      }
    }
  }
  if (MODE == 1 && L.count && (threadIdx.x & 31) == 0) {
    atomicAdd(&L.count[0], (unsigned long long)cnt[0]);
    atomicAdd(&L.count[1], (unsigned long long)cnt[1]);
  }
}

// Launch of one stage-kernel variant on a grid of (CTAs per SM) x SMs.
template <int MODE>
static void launch_stage_f32(const Topo& t, const Phys& p, const Pool& pool, int cur, int stage, const double* dt,
                             double* rhs_out, cudaStream_t st, int level) {
  const size_t smem = (MODE == 1) ? SF_SMEM_LEARNED : SF_SMEM;
  static int resident = 0;
  if (resident == 0) {
    cudaFuncSetAttribute(k_stage_f32<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_stage_f32<MODE>, SF_THREADS, smem);
    resident = sm_count() * (per_sm < 1 ? 1 : per_sm);
  }
  const int grid = resident * (g_tune.stage_waves < 1 ? 1 : g_tune.stage_waves);
  k_stage_f32<MODE><<<grid, SF_THREADS, smem, st>>>(t, p, pool, cur, stage, dt, rhs_out, level);
  ++g_kernel_launches;
}

}  // namespace mrb
