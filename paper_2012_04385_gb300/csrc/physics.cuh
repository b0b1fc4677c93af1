// Device physics of the block-based MR Euler method (arXiv:2012.04385):
// stiffened-gas EOS and Euler fluxes (Eq. Euler, Eq. StiffenedGas), the Roe
// eigensystem, WENO5-JS / TENO5 / WENO-AO(5,3) / linear 5th-order
// reconstruction in characteristic variables with the Roe / local
// Lax-Friedrichs switch per field, the standalone LLF and HLLC fluxes
// (Sec. 2.2), and the Navier-Stokes viscous flux.  The prediction of
// Eq. (Prediction) lives in mr.cuh.
//
// Every formula is written in one fixed evaluation order.  The FP64 kernels are
// compiled without FMA contraction (-fmad=false), so each double result is the
// correctly rounded value of that exact sequence of operations; the mixed
// kernels instantiate the same templates with R = float and may contract.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace mrb {

constexpr int NB = 16;                 // internal cells per block edge
constexpr int HW = 4;                  // halo width
constexpr int NS = NB + 2 * HW;        // 24 stored cells per edge
constexpr int NCELL = NS * NS * NS;    // 13824
constexpr int NINT = NB * NB * NB;     // 4096
constexpr int NV = 5;
constexpr int NFACE = NB * NB;         // 256
constexpr int SLOT_U = NV * NCELL;     // doubles per stage buffer
constexpr int SLOT_N = NV * NINT;      // doubles per u^n buffer
constexpr int SLOT_F = 6 * NV * NFACE; // doubles per face-flux set
constexpr int SLOT_SEL = 4 * (34 + 34 + 40);  // uint32 selector decision bits per block (4 z-slabs x 3 directions)
constexpr int SLOT_SH = 6 * NINT;      // floats per FP32 record set (mixed-precision path)

__host__ __device__ __forceinline__ int sidx(int i, int j, int k) { return ((k + HW) * NS + (j + HW)) * NS + (i + HW); }
__host__ __device__ __forceinline__ int iidx(int i, int j, int k) { return (k * NB + j) * NB + i; }

template <class R> __device__ __forceinline__ R rsqrt_(R x);
template <> __device__ __forceinline__ double rsqrt_<double>(double x) { return sqrt(x); }
template <> __device__ __forceinline__ float rsqrt_<float>(float x) { return sqrtf(x); }
template <class R> __device__ __forceinline__ R rabs(R x);
template <> __device__ __forceinline__ double rabs<double>(double x) { return fabs(x); }
template <> __device__ __forceinline__ float rabs<float>(float x) { return fabsf(x); }
template <class R> __device__ __forceinline__ R rmax(R a, R b);
template <> __device__ __forceinline__ double rmax<double>(double a, double b) { return fmax(a, b); }
template <> __device__ __forceinline__ float rmax<float>(float a, float b) { return fmaxf(a, b); }

// ---------------------------------------------------------------- EOS
template <class R> struct Prim {
  R rho, vel[3], p, c, E;
};

// p = (gamma - 1)(E - rho |v|^2 / 2) - gamma B,  c = sqrt(gamma (p + B) / rho)
template <class R> __device__ __forceinline__ Prim<R> prim_of(const R U[5], R g, R B) {
  Prim<R> q;
  q.rho = U[0];
  q.vel[0] = U[1] / q.rho;
  q.vel[1] = U[2] / q.rho;
  q.vel[2] = U[3] / q.rho;
  R q2 = (q.vel[0] * q.vel[0] + q.vel[1] * q.vel[1]) + q.vel[2] * q.vel[2];
  q.p = (g - R(1.0)) * (U[4] - R(0.5) * q.rho * q2) - g * B;
  q.c = rsqrt_<R>(g * (q.p + B) / q.rho);
  q.E = U[4];
  return q;
}

__host__ __device__ __forceinline__ int rot_axis(int d, int j) { return (d + j) % 3; }

// ---------------------------------------------------------------- WENO5-JS
// Jiang & Shu (1996): value at the right face of the middle cell of
// (a, b, c, d, e), epsilon = 1e-6, linear weights (0.1, 0.6, 0.3).
template <class R> __device__ __forceinline__ R weno5(R a, R b, R c, R d, R e) {
  const R eps = R(1e-6);
  R t1 = (a - R(2.0) * b) + c, t2 = (a - R(4.0) * b) + R(3.0) * c;
  R beta0 = R(13.0 / 12.0) * t1 * t1 + R(0.25) * t2 * t2;
  t1 = (b - R(2.0) * c) + d;
  t2 = b - d;
  R beta1 = R(13.0 / 12.0) * t1 * t1 + R(0.25) * t2 * t2;
  t1 = (c - R(2.0) * d) + e;
  t2 = (R(3.0) * c - R(4.0) * d) + e;
  R beta2 = R(13.0 / 12.0) * t1 * t1 + R(0.25) * t2 * t2;
  R a0 = R(0.1) / ((eps + beta0) * (eps + beta0));
  R a1 = R(0.6) / ((eps + beta1) * (eps + beta1));
  R a2 = R(0.3) / ((eps + beta2) * (eps + beta2));
  R sum = (a0 + a1) + a2;
  R q0 = ((R(2.0) * a - R(7.0) * b) + R(11.0) * c) / R(6.0);
  R q1 = ((-b + R(5.0) * c) + R(2.0) * d) / R(6.0);
  R q2 = ((R(2.0) * c + R(5.0) * d) - e) / R(6.0);
  return ((a0 * q0 + a1 * q1) + a2 * q2) / sum;
}

template <class R> __device__ __forceinline__ R linear5(R a, R b, R c, R d, R e) {
  R q0 = ((R(2.0) * a - R(7.0) * b) + R(11.0) * c) / R(6.0);
  R q1 = ((-b + R(5.0) * c) + R(2.0) * d) / R(6.0);
  R q2 = ((R(2.0) * c + R(5.0) * d) - e) / R(6.0);
  return (R(0.1) * q0 + R(0.6) * q1) + R(0.3) * q2;
}

// TENO5 (Fu, Hu & Adams 2016): the WENO5 stencils kept or dropped by a sharp
// cutoff C_T = 1e-5 on chi_k = gamma_k / sum gamma, gamma_k = (1 + tau5 /
// (beta_k + eps))^6, tau5 = |beta0 - beta2|, eps = 1e-40; the kept stencils
// combined with the linear weights, renormalised.
template <class R> __device__ __forceinline__ R teno5(R a, R b, R c, R d, R e) {
  const R eps = R(1e-40), CT = R(1e-5);
  R t1 = (a - R(2.0) * b) + c, t2 = (a - R(4.0) * b) + R(3.0) * c;
  R beta0 = R(13.0 / 12.0) * t1 * t1 + R(0.25) * t2 * t2;
  t1 = (b - R(2.0) * c) + d;
  t2 = b - d;
  R beta1 = R(13.0 / 12.0) * t1 * t1 + R(0.25) * t2 * t2;
  t1 = (c - R(2.0) * d) + e;
  t2 = (R(3.0) * c - R(4.0) * d) + e;
  R beta2 = R(13.0 / 12.0) * t1 * t1 + R(0.25) * t2 * t2;
  const R tau = fabs(beta0 - beta2);
  R r0 = R(1.0) + tau / (beta0 + eps), r1 = R(1.0) + tau / (beta1 + eps), r2 = R(1.0) + tau / (beta2 + eps);
  r0 = r0 * r0 * r0;
  r1 = r1 * r1 * r1;
  r2 = r2 * r2 * r2;
  const R g0 = r0 * r0, g1 = r1 * r1, g2 = r2 * r2;
  const R sum = (g0 + g1) + g2;
  const R w0 = (g0 / sum < CT) ? R(0.0) : R(0.1);
  const R w1 = (g1 / sum < CT) ? R(0.0) : R(0.6);
  const R w2 = (g2 / sum < CT) ? R(0.0) : R(0.3);
  R q0 = ((R(2.0) * a - R(7.0) * b) + R(11.0) * c) / R(6.0);
  R q1 = ((-b + R(5.0) * c) + R(2.0) * d) / R(6.0);
  R q2 = ((R(2.0) * c + R(5.0) * d) - e) / R(6.0);
  return ((w0 * q0 + w1 * q1) + w2 * q2) / ((w0 + w1) + w2);
}

// WENO-AO(5,3) (Balsara, Garain & Shu 2016): the quartic through the five
// cell averages blended with WENO5's three parabolas.  Linear weights from
// gamma_hi = gamma_lo = 0.85 (quartic gamma_hi, middle parabola (1 - gamma_hi)
// gamma_lo, outer parabolas half the rest each); the quartic's smoothness from
// its Legendre coefficients on the middle cell; WENO-Z type weights gamma_k (1
// + (tau / (beta_k + eps))^2), tau the mean of |beta_5 - beta_k|, eps = 1e-12.
template <class R> __device__ __forceinline__ R wenoao53(R a, R b, R c, R d, R e) {
  const R eps = R(1e-12);
  const R ghi = R(0.85), glo = R(0.85);
  R t1 = (a - R(2.0) * b) + c, t2 = (a - R(4.0) * b) + R(3.0) * c;
  R beta0 = R(13.0 / 12.0) * t1 * t1 + R(0.25) * t2 * t2;
  t1 = (b - R(2.0) * c) + d;
  t2 = b - d;
  R beta1 = R(13.0 / 12.0) * t1 * t1 + R(0.25) * t2 * t2;
  t1 = (c - R(2.0) * d) + e;
  t2 = (R(3.0) * c - R(4.0) * d) + e;
  R beta2 = R(13.0 / 12.0) * t1 * t1 + R(0.25) * t2 * t2;
  R u1 = (((R(11.0) * a - R(82.0) * b) + R(82.0) * d) - R(11.0) * e) / R(120.0);
  R u2 = ((((R(-3.0) * a + R(40.0) * b) - R(74.0) * c) + R(40.0) * d) - R(3.0) * e) / R(56.0);
  R u3 = (((-a + R(2.0) * b) - R(2.0) * d) + e) / R(12.0);
  R u4 = ((((a - R(4.0) * b) + R(6.0) * c) - R(4.0) * d) + e) / R(24.0);
  R s1 = u1 + u3 / R(10.0), s2 = u2 + R(123.0 / 455.0) * u4;
  R beta5 = (((s1 * s1 + R(13.0 / 3.0) * (s2 * s2)) + R(781.0 / 20.0) * (u3 * u3)) + R(1421461.0 / 2275.0) * (u4 * u4));
  const R g5 = ghi, g1 = (R(1.0) - ghi) * glo, g0 = R(0.5) * ((R(1.0) - ghi) * (R(1.0) - glo)), g2 = g0;
  R tau = ((fabs(beta5 - beta0) + fabs(beta5 - beta1)) + fabs(beta5 - beta2)) / R(3.0);
  R r5 = tau / (beta5 + eps), r0 = tau / (beta0 + eps), r1 = tau / (beta1 + eps), r2 = tau / (beta2 + eps);
  R w5 = g5 * (R(1.0) + r5 * r5), w0 = g0 * (R(1.0) + r0 * r0), w1 = g1 * (R(1.0) + r1 * r1), w2 = g2 * (R(1.0) + r2 * r2);
  R sum = ((w5 + w0) + w1) + w2;
  w5 = w5 / sum;
  w0 = w0 / sum;
  w1 = w1 / sum;
  w2 = w2 / sum;
  R q0 = ((R(2.0) * a - R(7.0) * b) + R(11.0) * c) / R(6.0);
  R q1 = ((-b + R(5.0) * c) + R(2.0) * d) / R(6.0);
  R q2 = ((R(2.0) * c + R(5.0) * d) - e) / R(6.0);
  R q5 = ((((R(2.0) * a - R(13.0) * b) + R(47.0) * c) + R(27.0) * d) - R(3.0) * e) / R(60.0);
  return (w5 / g5) * (((q5 - g0 * q0) - g1 * q1) - g2 * q2) + ((w0 * q0 + w1 * q1) + w2 * q2);
}

// Reconstruction by mode: 0 WENO5-JS, 2 linear, 3 TENO5, 4 WENO-AO(5,3).
template <class R> __device__ __forceinline__ R recon5(int mode, R a, R b, R c, R d, R e) {
  if (mode == 2) return linear5<R>(a, b, c, d, e);
  if (mode == 3) return teno5<R>(a, b, c, d, e);
  if (mode == 4) return wenoao53<R>(a, b, c, d, e);
  return weno5<R>(a, b, c, d, e);
}

// Flux schemes: Roe with the per-field LLF fallback, LLF on every field, HLLC.
constexpr int FLUX_ROE = 0, FLUX_LLF = 1, FLUX_HLLC = 2;

// HLLC (Toro, Spruce & Speares 1994) between rotated-frame states UL, UR
// (normal momentum in slot 1): Einfeldt's outer speeds S_L = min(u_L - c_L,
// u~ - c~), S_R = max(u_R + c_R, u~ + c~) from the Roe average of UL and UR;
// contact speed S* from the momentum balance over the outer waves; flux F_L,
// F*_L, F*_R or F_R by the position of x/t = 0, F*_K = F_K + S_K (U*_K - U_K).
template <class R> __device__ __forceinline__ void hllc_rot(const R UL[5], const R UR[5], R g, R B, R F[5]) {
  const Prim<R> a = prim_of<R>(UL, g, B), b = prim_of<R>(UR, g, B);
  R FL[5], FR[5];
  FL[0] = UL[1];
  FL[1] = UL[1] * a.vel[0] + a.p;
  FL[2] = UL[1] * a.vel[1];
  FL[3] = UL[1] * a.vel[2];
  FL[4] = a.vel[0] * (UL[4] + a.p);
  FR[0] = UR[1];
  FR[1] = UR[1] * b.vel[0] + b.p;
  FR[2] = UR[1] * b.vel[1];
  FR[3] = UR[1] * b.vel[2];
  FR[4] = b.vel[0] * (UR[4] + b.p);
  const R sL = rsqrt_<R>(a.rho), sR = rsqrt_<R>(b.rho);
  const R den = sL + sR;
  const R un = (sL * a.vel[0] + sR * b.vel[0]) / den;
  const R ut1 = (sL * a.vel[1] + sR * b.vel[1]) / den;
  const R ut2 = (sL * a.vel[2] + sR * b.vel[2]) / den;
  const R HL = (a.E + a.p) / a.rho, HR = (b.E + b.p) / b.rho;
  const R H = (sL * HL + sR * HR) / den;
  const R q2 = (un * un + ut1 * ut1) + ut2 * ut2;
  const R c = rsqrt_<R>((g - R(1.0)) * (H - R(0.5) * q2));
  const R uL = a.vel[0], uR = b.vel[0];
  const R l0 = un - c, l4 = un + c, xL = uL - a.c, xR = uR + b.c;
  const R SL = (l0 < xL) ? l0 : xL;
  const R SR = (xR < l4) ? l4 : xR;
  const R mL = a.rho * (SL - uL), mR = b.rho * (SR - uR);
  const R Ss = (((b.p - a.p) + uL * mL) - uR * mR) / (mL - mR);
  if (SL >= R(0.0)) {
#pragma unroll
    for (int j = 0; j < 5; ++j) F[j] = FL[j];
  } else if (SR <= R(0.0)) {
#pragma unroll
    for (int j = 0; j < 5; ++j) F[j] = FR[j];
  } else {
    const bool left = Ss >= R(0.0);
    const Prim<R>& q = left ? a : b;
    const R* U = left ? UL : UR;
    const R* FK = left ? FL : FR;
    const R SK = left ? SL : SR, mK = left ? mL : mR;
    const R fac = mK / (SK - Ss);
    R Us[5];
    Us[0] = fac;
    Us[1] = fac * Ss;
    Us[2] = fac * q.vel[1];
    Us[3] = fac * q.vel[2];
    Us[4] = fac * (U[4] / q.rho + (Ss - q.vel[0]) * (Ss + q.p / mK));
#pragma unroll
    for (int j = 0; j < 5; ++j) F[j] = FK[j] + SK * (Us[j] - U[j]);
  }
}

// A reconstructed face state usable by HLLC: rho > 0 and p + B > 0.
template <class R> __device__ __forceinline__ bool admissible(const R U[5], R g, R B) {
  if (!(U[0] > R(0.0))) return false;
  const R q2 = ((U[1] * U[1] + U[2] * U[2]) + U[3] * U[3]) / U[0];
  const R p = (g - R(1.0)) * (U[4] - R(0.5) * q2) - g * B;
  return p + B > R(0.0);
}

// ---------------------------------------------------------------- viscous flux
// Navier-Stokes viscous flux (Stokes' hypothesis, constant mu, no heat
// conduction) at the face between the stored cells sL and sL + step_d of a
// block (FP64 state with halos), lab frame: (0, tau_xd, tau_yd, tau_zd,
// u . tau_d), tau_ij = mu (du_i/dx_j + du_j/dx_i) - 2/3 mu (div u) delta_ij.
// Second-order compact face gradients: normal derivative from the two face
// cells, tangential derivative as the mean of their central differences;
// face velocity the mean of the two cells'.
__device__ __forceinline__ void cell_vel(const double* __restrict__ u, int s, double w[3]) {
  const double rho = u[s];
  w[0] = u[NCELL + s] / rho;
  w[1] = u[2 * NCELL + s] / rho;
  w[2] = u[3 * NCELL + s] / rho;
}

__device__ __forceinline__ void viscous_flux(const double* __restrict__ u, int d, int sL, double mu, double dx,
                                             double Fv[5]) {
  const int step[3] = {1, NS, NS * NS};
  const int sR = sL + step[d];
  double uL[3], uR[3];
  cell_vel(u, sL, uL);
  cell_vel(u, sR, uR);
  double G[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i) G[i][d] = (uR[i] - uL[i]) / dx;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    if (j == d) continue;
    double a[3], b[3], c[3], e[3];
    cell_vel(u, sL + step[j], a);
    cell_vel(u, sL - step[j], b);
    cell_vel(u, sR + step[j], c);
    cell_vel(u, sR - step[j], e);
#pragma unroll
    for (int i = 0; i < 3; ++i) G[i][j] = ((a[i] - b[i]) + (c[i] - e[i])) / (4.0 * dx);
  }
  const double div = (G[0][0] + G[1][1]) + G[2][2];
  double ub[3], tau[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    ub[i] = 0.5 * (uL[i] + uR[i]);
    tau[i] = mu * (G[i][d] + G[d][i]);
  }
  tau[d] = tau[d] - ((2.0 / 3.0) * mu) * div;
  Fv[0] = 0.0;
  Fv[1] = tau[0];
  Fv[2] = tau[1];
  Fv[3] = tau[2];
  Fv[4] = (ub[0] * tau[0] + ub[1] * tau[1]) + ub[2] * tau[2];
}

// Fields (bit k) that take the LLF split at the face between the lab-frame
// states UL, UR along d under the Roe / LLF rule of face_flux: the same
// primitive variables, Roe average and eigenvalue tests.
__device__ __forceinline__ unsigned split_fields(const double UL[5], const double UR[5], int d, double g, double B) {
  const int a0 = rot_axis(d, 0), a1 = rot_axis(d, 1), a2 = rot_axis(d, 2);
  const Prim<double> qL = prim_of<double>(UL, g, B), qR = prim_of<double>(UR, g, B);
  const double unL = qL.vel[d], cL = qL.c, unR = qR.vel[d], cR = qR.c;
  const double sL = sqrt(qL.rho), sR = sqrt(qR.rho);
  const double den = sL + sR;
  const double un = (sL * qL.vel[a0] + sR * qR.vel[a0]) / den;
  const double ut1 = (sL * qL.vel[a1] + sR * qR.vel[a1]) / den;
  const double ut2 = (sL * qL.vel[a2] + sR * qR.vel[a2]) / den;
  const double HL = (qL.E + qL.p) / qL.rho, HR = (qR.E + qR.p) / qR.rho;
  const double H = (sL * HL + sR * HR) / den;
  const double q2 = (un * un + ut1 * ut1) + ut2 * ut2;
  const double c = sqrt((g - 1.0) * (H - 0.5 * q2));
  unsigned mask = 0;
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    double lL, lR, lt;
    if (k == 0) { lL = unL - cL; lR = unR - cR; lt = un - c; }
    else if (k == 4) { lL = unL + cL; lR = unR + cR; lt = un + c; }
    else { lL = unL; lR = unR; lt = un; }
    const bool up = (lL > 0.0 && lR > 0.0 && lt > 0.0) || (lL < 0.0 && lR < 0.0 && lt < 0.0);
    if (!up) mask |= 1u << k;
  }
  return mask;
}

// ---------------------------------------------------------------- face flux
// Numerical flux at the face between cells 2 and 3 of U6 (cells i-2 .. i+3
// along d, lab-frame conserved states), returned in the lab frame.  Rotated
// frame (rho, m_n, m_t1, m_t2, E) with cyclic tangential axes.  Roe averages
// and the eigensystem of the face project the six cells to characteristic
// variables v = L U and fluxes g = L F(U); per field k the flux is upwinded
// when lam_k of both face cells and the Roe lam_k share a strict sign,
// otherwise split with alpha = max(|lam_k(U_i)|, |lam_k(U_i+1)|); F = R g
// (flux = FLUX_ROE).  FLUX_LLF splits every field.  FLUX_HLLC reconstructs v
// to the face from both sides, maps the two states back with R and applies
// HLLC; an inadmissible state sends the face back to the cell states U_i,
// U_i+1.
template <class R>
__device__ __forceinline__ void face_flux(const R U6[6][5], int d, R g, R B, int lin, int flux, R Fout[5]) {
  const int a0 = rot_axis(d, 0), a1 = rot_axis(d, 1), a2 = rot_axis(d, 2);
  R Ur[6][5], Fr[6][5];
  R unL, cL, unR, cR;
  Prim<R> qL, qR;
#pragma unroll
  for (int m = 0; m < 6; ++m) {
    Prim<R> q = prim_of<R>(U6[m], g, B);
    Ur[m][0] = U6[m][0];
    Ur[m][1] = U6[m][1 + a0];
    Ur[m][2] = U6[m][1 + a1];
    Ur[m][3] = U6[m][1 + a2];
    Ur[m][4] = U6[m][4];
    R un = q.vel[a0], ut1 = q.vel[a1], ut2 = q.vel[a2];
    Fr[m][0] = Ur[m][1];
    Fr[m][1] = Ur[m][1] * un + q.p;
    Fr[m][2] = Ur[m][1] * ut1;
    Fr[m][3] = Ur[m][1] * ut2;
    Fr[m][4] = un * (Ur[m][4] + q.p);
    if (m == 2) qL = q;
    if (m == 3) qR = q;
  }
  unL = qL.vel[d];
  cL = qL.c;
  unR = qR.vel[d];
  cR = qR.c;
  // Roe average
  R sL = rsqrt_<R>(qL.rho), sR = rsqrt_<R>(qR.rho);
  R den = sL + sR;
  R un = (sL * qL.vel[a0] + sR * qR.vel[a0]) / den;
  R ut1 = (sL * qL.vel[a1] + sR * qR.vel[a1]) / den;
  R ut2 = (sL * qL.vel[a2] + sR * qR.vel[a2]) / den;
  R HL = (qL.E + qL.p) / qL.rho, HR = (qR.E + qR.p) / qR.rho;
  R H = (sL * HL + sR * HR) / den;
  R q2 = (un * un + ut1 * ut1) + ut2 * ut2;
  R c2 = (g - R(1.0)) * (H - R(0.5) * q2);
  R c = rsqrt_<R>(c2);
  R ic = R(1.0) / c;
  R b1 = (g - R(1.0)) / c2;
  R b2 = R(0.5) * b1 * q2;
  R Fh[5], UL[5], UR[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    R l[5], r[5];
    if (k == 0) {
      l[0] = R(0.5) * (b2 + un * ic); l[1] = R(0.5) * (-b1 * un - ic); l[2] = R(0.5) * (-b1 * ut1);
      l[3] = R(0.5) * (-b1 * ut2); l[4] = R(0.5) * b1;
      r[0] = R(1.0); r[1] = un - c; r[2] = ut1; r[3] = ut2; r[4] = H - un * c;
    } else if (k == 1) {
      l[0] = R(1.0) - b2; l[1] = b1 * un; l[2] = b1 * ut1; l[3] = b1 * ut2; l[4] = -b1;
      r[0] = R(1.0); r[1] = un; r[2] = ut1; r[3] = ut2; r[4] = R(0.5) * q2;
    } else if (k == 2) {
      l[0] = -ut1; l[1] = R(0.0); l[2] = R(1.0); l[3] = R(0.0); l[4] = R(0.0);
      r[0] = R(0.0); r[1] = R(0.0); r[2] = R(1.0); r[3] = R(0.0); r[4] = ut1;
    } else if (k == 3) {
      l[0] = -ut2; l[1] = R(0.0); l[2] = R(0.0); l[3] = R(1.0); l[4] = R(0.0);
      r[0] = R(0.0); r[1] = R(0.0); r[2] = R(0.0); r[3] = R(1.0); r[4] = ut2;
    } else {
      l[0] = R(0.5) * (b2 - un * ic); l[1] = R(0.5) * (-b1 * un + ic); l[2] = R(0.5) * (-b1 * ut1);
      l[3] = R(0.5) * (-b1 * ut2); l[4] = R(0.5) * b1;
      r[0] = R(1.0); r[1] = un + c; r[2] = ut1; r[3] = ut2; r[4] = H + un * c;
    }
    R v[6], G[6];
#pragma unroll
    for (int m = 0; m < 6; ++m) {
      R sv = l[0] * Ur[m][0];
      R sg = l[0] * Fr[m][0];
#pragma unroll
      for (int j = 1; j < 5; ++j) {
        sv = sv + l[j] * Ur[m][j];
        sg = sg + l[j] * Fr[m][j];
      }
      v[m] = sv;
      G[m] = sg;
    }
    if (flux == FLUX_HLLC) {
      const R vl = recon5<R>(lin, v[0], v[1], v[2], v[3], v[4]);
      const R vr = recon5<R>(lin, v[5], v[4], v[3], v[2], v[1]);
#pragma unroll
      for (int j = 0; j < 5; ++j) {
        UL[j] = (k == 0) ? r[j] * vl : UL[j] + r[j] * vl;
        UR[j] = (k == 0) ? r[j] * vr : UR[j] + r[j] * vr;
      }
      continue;
    }
    R lL, lR, lt;
    if (k == 0) { lL = unL - cL; lR = unR - cR; lt = un - c; }
    else if (k == 4) { lL = unL + cL; lR = unR + cR; lt = un + c; }
    else { lL = unL; lR = unR; lt = un; }
    R gh;
    if (flux == FLUX_ROE && lL > R(0.0) && lR > R(0.0) && lt > R(0.0)) {
      gh = recon5<R>(lin, G[0], G[1], G[2], G[3], G[4]);
    } else if (flux == FLUX_ROE && lL < R(0.0) && lR < R(0.0) && lt < R(0.0)) {
      gh = recon5<R>(lin, G[5], G[4], G[3], G[2], G[1]);
    } else {
      R alpha = rmax<R>(rabs<R>(lL), rabs<R>(lR));
      R fp[6], fm[6];
#pragma unroll
      for (int m = 0; m < 6; ++m) {
        fp[m] = R(0.5) * (G[m] + alpha * v[m]);
        fm[m] = R(0.5) * (G[m] - alpha * v[m]);
      }
      gh = recon5<R>(lin, fp[0], fp[1], fp[2], fp[3], fp[4]) + recon5<R>(lin, fm[5], fm[4], fm[3], fm[2], fm[1]);
    }
#pragma unroll
    for (int j = 0; j < 5; ++j) Fh[j] = (k == 0) ? r[j] * gh : Fh[j] + r[j] * gh;
  }
  if (flux == FLUX_HLLC) {
    if (!admissible<R>(UL, g, B) || !admissible<R>(UR, g, B)) {
#pragma unroll
      for (int j = 0; j < 5; ++j) {
        UL[j] = Ur[2][j];
        UR[j] = Ur[3][j];
      }
    }
    hllc_rot<R>(UL, UR, g, B, Fh);
  }
  Fout[0] = Fh[0];
  Fout[1 + a0] = Fh[1];
  Fout[1 + a1] = Fh[2];
  Fout[1 + a2] = Fh[3];
  Fout[4] = Fh[4];
}

}  // namespace mrb
