// Plain FP64 CPU oracle of the block-based multiresolution (MR) Euler method of
// Hoppe, Adami & Adams, "A modular massively parallel computing environment for
// three-dimensional multiresolution simulations of compressible flows"
// (arXiv:2012.04385).
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call
// this file: only the test suite, the smoke check and the CPU-baseline leg of the
// benchmark use it.  It shares no code, header, table or constant generator with
// the CUDA library; the two are written independently from the paper.
//
// Build rules: C++17, scalar double, -ffp-contract=off (no fused multiply-add, so
// every formula rounds in the order written), OpenMP only over independent blocks.
// Every reduction runs in a fixed order, so results do not depend on the thread
// count.
//
// Evaluation order.  Every formula below is evaluated left to right exactly as
// written; the order is part of the oracle's definition (the paper fixes none).
//
// Pins (tests/test_oracle_*.py): free-stream preservation, conservation on
// periodic domains, the exact Sod solution, 5th-order convergence on an advected
// density wave, L.R = I and the Roe property of the eigensystem, WENO5/linear
// special cases, WENO5-JS against its definition, A(P(u)) = u and quartic reproduction of P, the Morton
// neighbour example of Fig. (NeighborLookup) and brute force in all 26
// directions, tag invariants, the Roe/LLF per-field switch in closed form on a
// transonic step, TENO5 cutoff and smooth-data cases, WENO-AO(5,3)
// against its definition (polynomial fits, exact integrals), HLLC exact on
// isolated shocks and stationary contacts, the LLF step flux in closed form,
// the Sod solution for each flux scheme, second order in time of TVD-RK2,
// the CFL time step in closed form, symmetry walls as the mirror image of a
// doubled periodic box, the level thresholds on perturbed cells, each
// refined octant and the halo fill at jumps exact on a quartic, batched
// instances bit-identical to each run alone, conservation across two-level
// jumps, the gravity source term, the projection by brute force, the viscous
// terms on a linear velocity field and the shear-wave decay, the right-hand
// side commuting with rotations and mirrors of the axes.
// The detail norm is a reading (the paper names only the l-infinity norm
// over the block with its halo); a single perturbed cell on a uniform state
// pins its parts (the leaf's value as the scale, rho and E, the halo).

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

// Block geometry (Sec. 3 and Sec. 5: 16^3 internal cells, four halo cells per side).
constexpr int NB = 16;
constexpr int HW = 4;
constexpr int NS = NB + 2 * HW;              // 24 stored cells per edge
constexpr int NCELL = NS * NS * NS;          // 13824
constexpr int NINT = NB * NB * NB;           // 4096
constexpr int NV = 5;                        // rho, rho u, rho v, rho w, E
constexpr int NFACE = NB * NB;               // 256 faces per block side
constexpr int NSHADOW = 7;                   // shadow levels of the 64-bit id (Sec. 3)
constexpr uint64_t MASK56 = (1ull << 56) - 1;

constexpr int BC_ZERO_GRADIENT = 0, BC_PERIODIC = 1, BC_SYMMETRY = 2;
constexpr int RECON_WENO = 0, RECON_LINEAR = 2, RECON_TENO = 3, RECON_WENOAO = 4;
constexpr int FLUX_ROE = 0, FLUX_LLF = 1, FLUX_HLLC = 2;
constexpr int8_t TAG_KEEP = 0, TAG_REFINE = 1, TAG_COARSEN = -1;

inline int sidx(int i, int j, int k) { return ((k + HW) * NS + (j + HW)) * NS + (i + HW); }
inline int iidx(int i, int j, int k) { return (k * NB + j) * NB + i; }
inline int floordiv2(int i) { return (i >= 0) ? i / 2 : -((-i + 1) / 2); }

}  // namespace

extern "C" {

// Run configuration.  Mirrors the physical set-up of the paper's runs (Sec. 5);
// laid out int32 first, then double, so that a ctypes Structure can build it.
struct orc_config {
  int32_t n_instances;
  int32_t base_blocks[3];
  int32_t lmax[256];
  int32_t bc[6];          // x-, x+, y-, y+, z-, z+
  int32_t recon;          // 0 = WENO5-JS, 2 = linear 5th-order upwind everywhere, 3 = TENO5, 4 = WENO-AO(5,3)
  int32_t n_threads;      // 0 = OpenMP default
  int32_t rk_stages;      // 3 = TVD-RK3 (default when 0), 2 = TVD-RK2
  int32_t flux;           // 0 = Roe with per-field LLF fallback, 1 = LLF on every field, 2 = HLLC
  double domain_lo[3];
  double dx0;             // level-0 cell size
  double gamma, B, cfl;
  double gravity[3];
  double eps;             // threshold at l_max (Eq. UserEpsilon already applied)
  double mu;              // dynamic viscosity of the Navier-Stokes terms; 0 = Euler
  int32_t lts;            // 1 = local time stepping per level (all instances with the same l_max)
};

}  // extern "C"

namespace {

struct Node {
  uint64_t key = 0;
  int inst = 0, level = 0;
  int64_t X[3] = {0, 0, 0};   // block coordinates on its level
  bool leaf = true;
  std::vector<double> u;      // [5][24^3] conserved state incl. halo
  std::vector<double> un;     // [5][16^3] u^n of the current RK step
  std::vector<double> L;      // [5][16^3] right-hand side
  std::vector<double> face;   // [6][5][16][16] boundary-face fluxes
  std::vector<double> fmac;   // [6][5][16][16] boundary-face fluxes integrated over a macro time step (LTS)
  void alloc() {
    u.assign((size_t)NV * NCELL, 0.0);
    un.assign((size_t)NV * NINT, 0.0);
    L.assign((size_t)NV * NINT, 0.0);
    face.assign((size_t)6 * NV * NFACE, 0.0);
    fmac.assign((size_t)6 * NV * NFACE, 0.0);
  }
};

struct Ctx {
  orc_config c;
  std::map<uint64_t, Node> nodes;   // ascending key = (instance, level, Morton)
};

// ---------------------------------------------------------------- Morton ids
// Sec. 3, Eq. (MortonBits)/(AlpacaBits): 3 bits per level (bit 0 = x, bit 1 = y,
// bit 2 = z), the finest level in the lowest group, a headbit above the top
// group, seven shadow levels carrying the level-0 block coordinates.  In batched
// runs the instance number sits in bits 56..63.
uint64_t make_key(int inst, int level, const int64_t X[3]) {
  int ng = NSHADOW + level;
  uint64_t m = 0;
  for (int b = 0; b < ng; ++b)
    for (int d = 0; d < 3; ++d) m |= (uint64_t)((X[d] >> b) & 1) << (3 * b + d);
  return ((uint64_t)inst << 56) | (1ull << (3 * ng)) | m;
}

int key_level(uint64_t key) {
  uint64_t m = key & MASK56;
  int h = 63 - __builtin_clzll(m);
  return h / 3 - NSHADOW;
}

// Alg. (NeighborLookup): the same-level neighbour one step along axis d.  The
// headbit is removed, every third bit starting at d is processed from the right
// with  bit <- bit XNOR f  and  f <- bit OR f  (positive direction) or
// f <- (NOT bit) OR f  (negative direction), and the headbit is put back.  A
// carry out of the top group, or a result on a shadow position beyond the base
// grid, is the domain boundary; periodic axes wrap within the base grid.
bool axis_step(const orc_config& c, uint64_t key, int d, int sign, uint64_t* out) {
  uint64_t inst = key >> 56;
  uint64_t m = key & MASK56;
  int level = key_level(key);
  int nbits = 3 * (NSHADOW + level);
  uint64_t head = 1ull << nbits;
  uint64_t id = m ^ head;
  int f = 0;
  for (int i = d; i < nbits; i += 3) {
    int bit = (int)((id >> i) & 1);
    int nbit = !(bit ^ f);
    id = (id & ~(1ull << i)) | ((uint64_t)nbit << i);
    f = (sign > 0) ? (nbit | f) : ((!nbit) | f);
  }
  int64_t x = 0;
  for (int b = 0; b < NSHADOW + level; ++b) x |= (int64_t)((id >> (3 * b + d)) & 1) << b;
  int64_t nl = (int64_t)c.base_blocks[d] << level;
  if (f == 0 || x >= nl) {
    if (c.bc[2 * d] != BC_PERIODIC) return false;
    x = (sign > 0) ? 0 : nl - 1;
    for (int b = 0; b < NSHADOW + level; ++b) {
      int i = 3 * b + d;
      id = (id & ~(1ull << i)) | ((uint64_t)((x >> b) & 1) << i);
    }
  }
  *out = (inst << 56) | head | id;
  return true;
}

// Diagonal neighbours by concatenating the axis steps (Sec. 3).
bool neighbour(const orc_config& c, uint64_t key, int sx, int sy, int sz, uint64_t* out) {
  int s[3] = {sx, sy, sz};
  uint64_t k = key;
  for (int d = 0; d < 3; ++d) {
    if (s[d] == 0) continue;
    if (!axis_step(c, k, d, s[d], &k)) return false;
  }
  *out = k;
  return true;
}

// Elementary functions of the face-flux chain (the counting type at the end of
// this file has its own).
inline double osqrt(double x) { return std::sqrt(x); }
inline double oabs(double x) { return std::fabs(x); }
inline double omax(double a, double b) { return std::max(a, b); }
inline double omin(double a, double b) { return std::min(a, b); }

// ------------------------------------------------------------ EOS and fluxes
// Eq. (Euler) with the stiffened-gas EOS, Eq. (StiffenedGas):
// p = (gamma-1) rho e - gamma B,  E = rho e + 1/2 rho |v|^2,  c^2 = gamma (p+B)/rho.
// The face-flux chain below (EOS, fluxes, eigensystem, reconstructions,
// HLLC, face flux) is written once for a scalar type T: the oracle runs it
// on double; the operation count of the roofline runs the same code on a
// counting number type (end of this file).
template <class T> struct PrimT { T rho, vel[3], p, c, E; };
using Prim = PrimT<double>;

template <class T> PrimT<T> prim_of(const T U[5], double g, double B) {
  PrimT<T> q;
  q.rho = U[0];
  q.vel[0] = U[1] / q.rho;
  q.vel[1] = U[2] / q.rho;
  q.vel[2] = U[3] / q.rho;
  T q2 = (q.vel[0] * q.vel[0] + q.vel[1] * q.vel[1]) + q.vel[2] * q.vel[2];
  q.p = (g - 1.0) * (U[4] - 0.5 * q.rho * q2) - g * B;
  q.c = osqrt(g * (q.p + B) / q.rho);
  q.E = U[4];
  return q;
}

// Rotated frame for direction d: (rho, m_n, m_t1, m_t2, E) with the tangential
// axes in cyclic order, so that one set of x-direction formulas serves all three.
inline int rot_axis(int d, int j) { return (d + j) % 3; }  // j = 0 normal, 1, 2 tangential

template <class T> void rotate(const T U[5], int d, T R[5]) {
  R[0] = U[0];
  R[1] = U[1 + rot_axis(d, 0)];
  R[2] = U[1 + rot_axis(d, 1)];
  R[3] = U[1 + rot_axis(d, 2)];
  R[4] = U[4];
}

template <class T> void unrotate(const T R[5], int d, T U[5]) {
  U[0] = R[0];
  U[1 + rot_axis(d, 0)] = R[1];
  U[1 + rot_axis(d, 1)] = R[2];
  U[1 + rot_axis(d, 2)] = R[3];
  U[4] = R[4];
}

// Physical flux along d in the rotated frame: (m_n, m_n u_n + p, m_n u_t1, m_n u_t2, u_n (E + p)).
template <class T> void flux_rot(const T Ur[5], const PrimT<T>& q, int d, T F[5]) {
  T un = q.vel[rot_axis(d, 0)];
  T ut1 = q.vel[rot_axis(d, 1)];
  T ut2 = q.vel[rot_axis(d, 2)];
  F[0] = Ur[1];
  F[1] = Ur[1] * un + q.p;
  F[2] = Ur[1] * ut1;
  F[3] = Ur[1] * ut2;
  F[4] = un * (Ur[4] + q.p);
}

// Roe average at a face and its eigensystem in the rotated frame (Roe 1981,
// named in Sec. 2.2).  Rows of Lm are left eigenvectors, columns of Rm right
// eigenvectors, lam the eigenvalues (u-c, u, u, u, u+c).
template <class T> struct EigenT { T Lm[5][5], Rm[5][5], lam[5]; };
using Eigen = EigenT<double>;

template <class T> EigenT<T> roe_eigen(const PrimT<T>& a, const PrimT<T>& b, int d, double g) {
  T sL = osqrt(a.rho), sR = osqrt(b.rho);
  T den = sL + sR;
  T un = (sL * a.vel[rot_axis(d, 0)] + sR * b.vel[rot_axis(d, 0)]) / den;
  T ut1 = (sL * a.vel[rot_axis(d, 1)] + sR * b.vel[rot_axis(d, 1)]) / den;
  T ut2 = (sL * a.vel[rot_axis(d, 2)] + sR * b.vel[rot_axis(d, 2)]) / den;
  T HL = (a.E + a.p) / a.rho, HR = (b.E + b.p) / b.rho;
  T H = (sL * HL + sR * HR) / den;
  T q2 = (un * un + ut1 * ut1) + ut2 * ut2;
  T c2 = (g - 1.0) * (H - 0.5 * q2);
  T c = osqrt(c2);
  T ic = 1.0 / c;
  T b1 = (g - 1.0) / c2;
  T b2 = 0.5 * b1 * q2;
  EigenT<T> e;
  T l0[5] = {0.5 * (b2 + un * ic), 0.5 * (-b1 * un - ic), 0.5 * (-b1 * ut1), 0.5 * (-b1 * ut2), 0.5 * b1};
  T l1[5] = {1.0 - b2, b1 * un, b1 * ut1, b1 * ut2, -b1};
  T l2[5] = {-ut1, 0.0, 1.0, 0.0, 0.0};
  T l3[5] = {-ut2, 0.0, 0.0, 1.0, 0.0};
  T l4[5] = {0.5 * (b2 - un * ic), 0.5 * (-b1 * un + ic), 0.5 * (-b1 * ut1), 0.5 * (-b1 * ut2), 0.5 * b1};
  T r0[5] = {1.0, un - c, ut1, ut2, H - un * c};
  T r1[5] = {1.0, un, ut1, ut2, 0.5 * q2};
  T r2[5] = {0.0, 0.0, 1.0, 0.0, ut1};
  T r3[5] = {0.0, 0.0, 0.0, 1.0, ut2};
  T r4[5] = {1.0, un + c, ut1, ut2, H + un * c};
  const T* ls[5] = {l0, l1, l2, l3, l4};
  const T* rs[5] = {r0, r1, r2, r3, r4};
  for (int k = 0; k < 5; ++k)
    for (int j = 0; j < 5; ++j) {
      e.Lm[k][j] = ls[k][j];
      e.Rm[j][k] = rs[k][j];
    }
  e.lam[0] = un - c;
  e.lam[1] = un;
  e.lam[2] = un;
  e.lam[3] = un;
  e.lam[4] = un + c;
  return e;
}

// WENO5-JS (Jiang & Shu 1996, cited in Sec. 2.2) reconstructing the value at
// the right face of the middle cell of (a, b, c, d, e); epsilon = 1e-6, linear
// weights (0.1, 0.6, 0.3).
template <class T> T weno5(T a, T b, T c, T d, T e) {
  const double eps = 1e-6;
  T t1 = (a - 2.0 * b) + c, t2 = (a - 4.0 * b) + 3.0 * c;
  T beta0 = (13.0 / 12.0) * t1 * t1 + 0.25 * t2 * t2;
  t1 = (b - 2.0 * c) + d;
  t2 = b - d;
  T beta1 = (13.0 / 12.0) * t1 * t1 + 0.25 * t2 * t2;
  t1 = (c - 2.0 * d) + e;
  t2 = (3.0 * c - 4.0 * d) + e;
  T beta2 = (13.0 / 12.0) * t1 * t1 + 0.25 * t2 * t2;
  T a0 = 0.1 / ((eps + beta0) * (eps + beta0));
  T a1 = 0.6 / ((eps + beta1) * (eps + beta1));
  T a2 = 0.3 / ((eps + beta2) * (eps + beta2));
  T sum = (a0 + a1) + a2;
  T q0 = ((2.0 * a - 7.0 * b) + 11.0 * c) / 6.0;
  T q1 = ((-b + 5.0 * c) + 2.0 * d) / 6.0;
  T q2 = ((2.0 * c + 5.0 * d) - e) / 6.0;
  return ((a0 * q0 + a1 * q1) + a2 * q2) / sum;
}

// The same three candidate stencils combined with the linear weights: the
// 5th-order upwind reconstruction.
template <class T> T linear5(T a, T b, T c, T d, T e) {
  T q0 = ((2.0 * a - 7.0 * b) + 11.0 * c) / 6.0;
  T q1 = ((-b + 5.0 * c) + 2.0 * d) / 6.0;
  T q2 = ((2.0 * c + 5.0 * d) - e) / 6.0;
  return (0.1 * q0 + 0.6 * q1) + 0.3 * q2;
}

// TENO5 (Fu, Hu & Adams 2016, one of the reconstructions the paper's modular
// framework offers, Sec. 2.2): the WENO5 candidate stencils and smoothness
// indicators; each stencil is kept or dropped by a sharp cutoff on its
// relative smoothness chi_k = gamma_k / sum gamma, gamma_k = (C + tau5 /
// (beta_k + eps))^q with tau5 = |beta0 - beta2|, C = 1, q = 6, eps = 1e-40,
// cutoff C_T = 1e-5; the kept stencils are combined with the linear weights,
// renormalised.
template <class T> T teno5(T a, T b, T c, T d, T e) {
  const double eps = 1e-40, CT = 1e-5;
  T t1 = (a - 2.0 * b) + c, t2 = (a - 4.0 * b) + 3.0 * c;
  T beta0 = (13.0 / 12.0) * t1 * t1 + 0.25 * t2 * t2;
  t1 = (b - 2.0 * c) + d;
  t2 = b - d;
  T beta1 = (13.0 / 12.0) * t1 * t1 + 0.25 * t2 * t2;
  t1 = (c - 2.0 * d) + e;
  t2 = (3.0 * c - 4.0 * d) + e;
  T beta2 = (13.0 / 12.0) * t1 * t1 + 0.25 * t2 * t2;
  const T tau = oabs(beta0 - beta2);
  T r0 = 1.0 + tau / (beta0 + eps), r1 = 1.0 + tau / (beta1 + eps), r2 = 1.0 + tau / (beta2 + eps);
  r0 = r0 * r0 * r0;
  r1 = r1 * r1 * r1;
  r2 = r2 * r2 * r2;
  const T g0 = r0 * r0, g1 = r1 * r1, g2 = r2 * r2;
  const T sum = (g0 + g1) + g2;
  const double w0 = (g0 / sum < CT) ? 0.0 : 0.1;
  const double w1 = (g1 / sum < CT) ? 0.0 : 0.6;
  const double w2 = (g2 / sum < CT) ? 0.0 : 0.3;
  T q0 = ((2.0 * a - 7.0 * b) + 11.0 * c) / 6.0;
  T q1 = ((-b + 5.0 * c) + 2.0 * d) / 6.0;
  T q2 = ((2.0 * c + 5.0 * d) - e) / 6.0;
  return ((w0 * q0 + w1 * q1) + w2 * q2) / ((w0 + w1) + w2);
}

// WENO-AO(5,3) (Balsara, Garain & Shu 2016, one of the stencils Sec. 2.2
// lists): the quartic through all five cell averages is blended with the three
// parabolas of WENO5.  Smoothness of the parabolas as in WENO5-JS; of the
// quartic, the sum over derivative orders 1..4 of the integral of the squared
// derivative over the middle cell, written with the Legendre coefficients of
// the quartic on that cell.  Linear weights from gamma_hi = gamma_lo = 0.85:
// quartic gamma_hi, middle parabola (1 - gamma_hi) gamma_lo, outer parabolas
// (1 - gamma_hi)(1 - gamma_lo)/2 each.  Nonlinear weights of WENO-Z type,
// gamma_k (1 + (tau / (beta_k + eps))^2), tau the mean of |beta_5 - beta_k|,
// eps = 1e-12, normalised.  Value at the right face of the middle cell:
// (w_5 / gamma_5)(q_5 - sum gamma_k q_k) + sum w_k q_k over the parabolas k.
template <class T> T wenoao53(T a, T b, T c, T d, T e) {
  const double eps = 1e-12;
  const double ghi = 0.85, glo = 0.85;
  T t1 = (a - 2.0 * b) + c, t2 = (a - 4.0 * b) + 3.0 * c;
  T beta0 = (13.0 / 12.0) * t1 * t1 + 0.25 * t2 * t2;
  t1 = (b - 2.0 * c) + d;
  t2 = b - d;
  T beta1 = (13.0 / 12.0) * t1 * t1 + 0.25 * t2 * t2;
  t1 = (c - 2.0 * d) + e;
  t2 = (3.0 * c - 4.0 * d) + e;
  T beta2 = (13.0 / 12.0) * t1 * t1 + 0.25 * t2 * t2;
  // Legendre coefficients of the quartic on the middle cell (a..e = u_{i-2..i+2})
  T u1 = (((11.0 * a - 82.0 * b) + 82.0 * d) - 11.0 * e) / 120.0;
  T u2 = ((((-3.0 * a + 40.0 * b) - 74.0 * c) + 40.0 * d) - 3.0 * e) / 56.0;
  T u3 = (((-a + 2.0 * b) - 2.0 * d) + e) / 12.0;
  T u4 = ((((a - 4.0 * b) + 6.0 * c) - 4.0 * d) + e) / 24.0;
  T s1 = u1 + u3 / 10.0, s2 = u2 + (123.0 / 455.0) * u4;
  T beta5 = (((s1 * s1 + (13.0 / 3.0) * (s2 * s2)) + (781.0 / 20.0) * (u3 * u3)) + (1421461.0 / 2275.0) * (u4 * u4));
  const double g5 = ghi, g1 = (1.0 - ghi) * glo, g0 = 0.5 * ((1.0 - ghi) * (1.0 - glo)), g2 = g0;
  T tau = ((oabs(beta5 - beta0) + oabs(beta5 - beta1)) + oabs(beta5 - beta2)) / 3.0;
  T r5 = tau / (beta5 + eps), r0 = tau / (beta0 + eps), r1 = tau / (beta1 + eps), r2 = tau / (beta2 + eps);
  T w5 = g5 * (1.0 + r5 * r5), w0 = g0 * (1.0 + r0 * r0), w1 = g1 * (1.0 + r1 * r1), w2 = g2 * (1.0 + r2 * r2);
  T sum = ((w5 + w0) + w1) + w2;
  w5 = w5 / sum;
  w0 = w0 / sum;
  w1 = w1 / sum;
  w2 = w2 / sum;
  T q0 = ((2.0 * a - 7.0 * b) + 11.0 * c) / 6.0;
  T q1 = ((-b + 5.0 * c) + 2.0 * d) / 6.0;
  T q2 = ((2.0 * c + 5.0 * d) - e) / 6.0;
  T q5 = ((((2.0 * a - 13.0 * b) + 47.0 * c) + 27.0 * d) - 3.0 * e) / 60.0;
  return (w5 / g5) * (((q5 - g0 * q0) - g1 * q1) - g2 * q2) + ((w0 * q0 + w1 * q1) + w2 * q2);
}

template <class T> inline T recon5(int mode, T a, T b, T c, T d, T e) {
  if (mode == RECON_LINEAR) return linear5(a, b, c, d, e);
  if (mode == RECON_TENO) return teno5(a, b, c, d, e);
  if (mode == RECON_WENOAO) return wenoao53(a, b, c, d, e);
  return weno5(a, b, c, d, e);
}

// HLLC approximate Riemann solver (Toro, Spruce & Speares 1994; Sec. 2.2 lists
// it beside Roe and LLF) on rotated-frame states UL, UR (normal momentum in
// slot 1).  Outer signal speeds after Einfeldt: S_L = min(u_L - c_L, u~ - c~),
// S_R = max(u_R + c_R, u~ + c~), ~ the Roe average of UL and UR.  Contact speed
// S* from the momentum balance over both outer waves.  The flux is F_L, F*_L,
// F*_R or F_R by where x/t = 0 falls among S_L <= S* <= S_R, with
// F*_K = F_K + S_K (U*_K - U_K) and U*_K = rho_K (S_K - u_K) / (S_K - S*) times
// (1, S*, v_K, w_K, E_K / rho_K + (S* - u_K)(S* + p_K / (rho_K (S_K - u_K)))).
template <class T> void hllc_rot(const T UL[5], const T UR[5], double g, double B, T F[5]) {
  PrimT<T> a = prim_of(UL, g, B), b = prim_of(UR, g, B);
  T FL[5], FR[5];
  flux_rot(UL, a, 0, FL);
  flux_rot(UR, b, 0, FR);
  EigenT<T> e = roe_eigen(a, b, 0, g);
  T uL = a.vel[0], uR = b.vel[0];
  T SL = omin(uL - a.c, e.lam[0]);
  T SR = omax(uR + b.c, e.lam[4]);
  T mL = a.rho * (SL - uL), mR = b.rho * (SR - uR);
  T Ss = (((b.p - a.p) + uL * mL) - uR * mR) / (mL - mR);
  if (SL >= 0.0) {
    for (int j = 0; j < 5; ++j) F[j] = FL[j];
  } else if (SR <= 0.0) {
    for (int j = 0; j < 5; ++j) F[j] = FR[j];
  } else {
    const bool left = Ss >= 0.0;
    const PrimT<T>& q = left ? a : b;
    const T* U = left ? UL : UR;
    const T* FK = left ? FL : FR;
    T SK = left ? SL : SR, mK = left ? mL : mR;
    T fac = mK / (SK - Ss);
    T Us[5];
    Us[0] = fac;
    Us[1] = fac * Ss;
    Us[2] = fac * q.vel[1];
    Us[3] = fac * q.vel[2];
    Us[4] = fac * (U[4] / q.rho + (Ss - q.vel[0]) * (Ss + q.p / mK));
    for (int j = 0; j < 5; ++j) F[j] = FK[j] + SK * (Us[j] - U[j]);
  }
}

// Reconstructed face state admissible for HLLC: positive density and p + B > 0.
template <class T> bool admissible(const T U[5], double g, double B) {
  if (!(U[0] > 0.0)) return false;
  T q2 = ((U[1] * U[1] + U[2] * U[2]) + U[3] * U[3]) / U[0];
  T p = (g - 1.0) * (U[4] - 0.5 * q2) - g * B;
  return p + B > 0.0;
}

// Numerical flux at the face between cells 2 and 3 of a six-cell stencil
// (cells i-2 .. i+3), along direction d, returned in the lab frame.
// Characteristic-wise reconstruction: v = L U, g = L F(U) with the Roe
// matrices of the face.  flux = FLUX_ROE: per field k, Roe upwinding when the
// cell eigenvalues on both sides and the Roe eigenvalue share a strict sign,
// else the local Lax-Friedrichs split with alpha = max(|lam_k(U_i)|,
// |lam_k(U_{i+1})|) from the two cells sharing the face (Sec. 2.2); F = R g_hat.
// flux = FLUX_LLF: that split on every field.  flux = FLUX_HLLC: the
// characteristic variables are reconstructed to the face from the left
// (cells i-2..i+2) and from the right (cells i+3..i-1), mapped back with R to
// the states U_L, U_R, and HLLC gives the flux; where either state is not
// admissible the face falls back to the cell states U_i, U_{i+1}.
template <class T>
void face_flux(const T U6[6][5], int d, double g, double B, int mode, int flux, T Fout[5]) {
  PrimT<T> q[6];
  T Ur[6][5], Fr[6][5];
  for (int m = 0; m < 6; ++m) {
    q[m] = prim_of(U6[m], g, B);
    rotate(U6[m], d, Ur[m]);
    flux_rot(Ur[m], q[m], d, Fr[m]);
  }
  EigenT<T> e = roe_eigen(q[2], q[3], d, g);
  T v[5][6], gc[5][6];
  for (int k = 0; k < 5; ++k)
    for (int m = 0; m < 6; ++m) {
      T sv = e.Lm[k][0] * Ur[m][0];
      T sg = e.Lm[k][0] * Fr[m][0];
      for (int j = 1; j < 5; ++j) {
        sv = sv + e.Lm[k][j] * Ur[m][j];
        sg = sg + e.Lm[k][j] * Fr[m][j];
      }
      v[k][m] = sv;
      gc[k][m] = sg;
    }
  if (flux == FLUX_HLLC) {
    T vL[5], vR[5], UL[5], UR[5], Fh[5];
    for (int k = 0; k < 5; ++k) {
      vL[k] = recon5(mode, v[k][0], v[k][1], v[k][2], v[k][3], v[k][4]);
      vR[k] = recon5(mode, v[k][5], v[k][4], v[k][3], v[k][2], v[k][1]);
    }
    for (int j = 0; j < 5; ++j) {
      T sl = e.Rm[j][0] * vL[0], sr = e.Rm[j][0] * vR[0];
      for (int k = 1; k < 5; ++k) {
        sl = sl + e.Rm[j][k] * vL[k];
        sr = sr + e.Rm[j][k] * vR[k];
      }
      UL[j] = sl;
      UR[j] = sr;
    }
    if (!admissible(UL, g, B) || !admissible(UR, g, B)) {
      for (int j = 0; j < 5; ++j) {
        UL[j] = Ur[2][j];
        UR[j] = Ur[3][j];
      }
    }
    hllc_rot(UL, UR, g, B, Fh);
    unrotate(Fh, d, Fout);
    return;
  }
  T unL = q[2].vel[d], unR = q[3].vel[d];
  T lamL[5] = {unL - q[2].c, unL, unL, unL, unL + q[2].c};
  T lamR[5] = {unR - q[3].c, unR, unR, unR, unR + q[3].c};
  T gh[5];
  for (int k = 0; k < 5; ++k) {
    T lL = lamL[k], lR = lamR[k], lt = e.lam[k];
    const T* G = gc[k];
    if (flux == FLUX_ROE && lL > 0.0 && lR > 0.0 && lt > 0.0) {
      gh[k] = recon5(mode, G[0], G[1], G[2], G[3], G[4]);
    } else if (flux == FLUX_ROE && lL < 0.0 && lR < 0.0 && lt < 0.0) {
      gh[k] = recon5(mode, G[5], G[4], G[3], G[2], G[1]);
    } else {
      T alpha = omax(oabs(lL), oabs(lR));
      T fp[6], fm[6];
      for (int m = 0; m < 6; ++m) {
        fp[m] = 0.5 * (G[m] + alpha * v[k][m]);
        fm[m] = 0.5 * (G[m] - alpha * v[k][m]);
      }
      gh[k] = recon5(mode, fp[0], fp[1], fp[2], fp[3], fp[4]) + recon5(mode, fm[5], fm[4], fm[3], fm[2], fm[1]);
    }
  }
  T Fr_hat[5];
  for (int j = 0; j < 5; ++j) {
    T s = e.Rm[j][0] * gh[0];
    for (int k = 1; k < 5; ++k) s = s + e.Rm[j][k] * gh[k];
    Fr_hat[j] = s;
  }
  unrotate(Fr_hat, d, Fout);
}

// ------------------------------------------------------------ selector features
// Learned reconstruction selector (not in the paper; a reading of the
// selector the benchmark adds).  Features of the face between cells 2 and 3
// of U6: for the characteristic fields k = 0 (u-c), 1 (entropy), 4 (u+c),
// with g_m = L_k F(U_m), v_m = L_k U_m over the six stencil cells m = 0..5
// (i-2 .. i+3) and alpha_k = max(|lam_k(U_i)|, |lam_k(U_{i+1})|) (the LLF
// speed of the field), the five consecutive variations
// d = s (|g_{m+1} - g_m| + alpha_k |v_{m+1} - v_m|), s the sign of the flux
// difference (of the variable difference where the flux difference is zero),
// compressed as sign(d) log10(1 + 1e6 |d|) / 8 (absolute units, like WENO's
// epsilon).  The selector decides for these three fields; the shear fields
// keep WENO5.  Label: 1 when, for field 0, 1 or 4 and any reconstruction the
// face performs (one for Roe upwinding, two for the LLF split),
// |WENO5 - linear5| exceeds both tau_lab times the largest |input| of that
// reconstruction and the absolute floor 1e-6 (below which a difference is
// rounding noise of O(1) fluxes in FP32).
inline bool selected_field(int k) { return k == 0 || k == 1 || k == 4; }

double compress_diff(double d) {
  double a = std::log10(1.0 + 1e6 * std::fabs(d)) / 8.0;
  return d < 0.0 ? -a : a;
}

// aux (nullable, 5 values): [0] the largest (|WENO5 - linear5| - threshold)
// over the label's checks (the label is 1 when it is positive), [1] the largest
// |input| of those checks, [2..4] per selected field the largest |g_m| +
// alpha_k |v_m| over the six cells (the size of the values the field's
// variations are differences of).
void face_features(const double U6[6][5], int d, double g, double B, double tau_lab, double feats[15], int* label,
                   double* aux = nullptr) {
  Prim q[6];
  double Ur[6][5], Fr[6][5];
  for (int m = 0; m < 6; ++m) {
    q[m] = prim_of(U6[m], g, B);
    rotate(U6[m], d, Ur[m]);
    flux_rot(Ur[m], q[m], d, Fr[m]);
  }
  Eigen e = roe_eigen(q[2], q[3], d, g);
  const int ks[3] = {0, 1, 4};
  for (int t = 0; t < 3; ++t) {
    int k = ks[t];
    double gk[6], vk[6];
    for (int m = 0; m < 6; ++m) {
      double sg = e.Lm[k][0] * Fr[m][0], sv = e.Lm[k][0] * Ur[m][0];
      for (int j = 1; j < 5; ++j) {
        sg = sg + e.Lm[k][j] * Fr[m][j];
        sv = sv + e.Lm[k][j] * Ur[m][j];
      }
      gk[m] = sg;
      vk[m] = sv;
    }
    double unL0 = q[2].vel[d], unR0 = q[3].vel[d];
    double lL = (k == 0) ? unL0 - q[2].c : (k == 4 ? unL0 + q[2].c : unL0);
    double lR = (k == 0) ? unR0 - q[3].c : (k == 4 ? unR0 + q[3].c : unR0);
    double alpha = std::max(std::fabs(lL), std::fabs(lR));
    for (int m = 0; m < 5; ++m) {
      double dg = gk[m + 1] - gk[m], dv = vk[m + 1] - vk[m];
      double sgn = (dg != 0.0) ? (dg < 0.0 ? -1.0 : 1.0) : (dv < 0.0 ? -1.0 : 1.0);
      feats[5 * t + m] = compress_diff(sgn * (std::fabs(dg) + alpha * std::fabs(dv)));
    }
    if (aux) {
      double S = 0.0;
      for (int m = 0; m < 6; ++m) S = std::max(S, std::fabs(gk[m]) + alpha * std::fabs(vk[m]));
      aux[2 + t] = S;
    }
  }
  double unL = q[2].vel[d], unR = q[3].vel[d];
  double lamL[5] = {unL - q[2].c, unL, unL, unL, unL + q[2].c};
  double lamR[5] = {unR - q[3].c, unR, unR, unR, unR + q[3].c};
  int lab = 0;
  double margin = -INFINITY, scale = 0.0;
  auto check = [&](const double f[5]) {
    double sc = 0.0;
    for (int m = 0; m < 5; ++m) sc = std::max(sc, std::fabs(f[m]));
    double dw = std::fabs(weno5(f[0], f[1], f[2], f[3], f[4]) - linear5(f[0], f[1], f[2], f[3], f[4]));
    if (dw > std::max(tau_lab * sc, 1e-6)) lab = 1;
    margin = std::max(margin, dw - std::max(tau_lab * sc, 1e-6));
    scale = std::max(scale, sc);
  };
  for (int k = 0; k < 5; ++k) {
    if (!selected_field(k)) continue;
    double G[6], V[6];
    for (int m = 0; m < 6; ++m) {
      double sv = e.Lm[k][0] * Ur[m][0], sg = e.Lm[k][0] * Fr[m][0];
      for (int j = 1; j < 5; ++j) {
        sv = sv + e.Lm[k][j] * Ur[m][j];
        sg = sg + e.Lm[k][j] * Fr[m][j];
      }
      V[m] = sv;
      G[m] = sg;
    }
    double lL = lamL[k], lR = lamR[k], lt = e.lam[k];
    if (lL > 0.0 && lR > 0.0 && lt > 0.0) {
      double f[5] = {G[0], G[1], G[2], G[3], G[4]};
      check(f);
    } else if (lL < 0.0 && lR < 0.0 && lt < 0.0) {
      double f[5] = {G[5], G[4], G[3], G[2], G[1]};
      check(f);
    } else {
      double alpha = std::max(std::fabs(lL), std::fabs(lR));
      double fp[5], fm[5];
      for (int m = 0; m < 5; ++m) fp[m] = 0.5 * (G[m] + alpha * V[m]);
      for (int m = 0; m < 5; ++m) fm[m] = 0.5 * (G[5 - m] - alpha * V[5 - m]);
      check(fp);
      check(fm);
    }
  }
  *label = lab;
  if (aux) {
    aux[0] = margin;
    aux[1] = scale;
  }
}

// ------------------------------------------------------------ MR operators
// Prediction, Eq. (Prediction) with the Q-terms of the appendix.  c0 = -22/128,
// c1 = 3/128, c_pq = c_p c_q, c_rpq = c_r c_p c_q, where index 0 belongs to an
// offset of one parent cell and index 1 to an offset of two.  Q_z is read with
// u_{i,j,k+2} (the printed u_{i+2,j,k+2} breaks the symmetry with Q_x and Q_y).
// The lower child half along an axis takes the sign +1, the upper -1.
struct Stencil {
  const double* P;
  int i, j, k;
  double at(int a, int b, int c) const { return P[sidx(i + a, j + b, k + c)]; }
};

const double C0 = -22.0 / 128.0, C1 = 3.0 / 128.0;
inline double cidx(int off) { return off == 1 ? C0 : C1; }

// c_pq [ (u(+p,+q) + u(-p,-q)) - (u(-p,+q) + u(+p,-q)) ] on the axis pair (A, B)
double mix2(const Stencil& s, int A, int Bx, int p, int q) {
  auto u = [&](int sp, int sq) {
    int o[3] = {0, 0, 0};
    o[A] = sp * p;
    o[Bx] = sq * q;
    return s.at(o[0], o[1], o[2]);
  };
  return (u(1, 1) + u(-1, -1)) - (u(-1, 1) + u(1, -1));
}

// sum over the four sign triples of positive parity of u(s) - u(-s)
double mix3(const Stencil& s, int p, int q, int r) {
  const int sg[4][3] = {{1, 1, 1}, {1, -1, -1}, {-1, -1, 1}, {-1, 1, -1}};
  double acc = 0.0;
  for (int t = 0; t < 4; ++t) {
    double term = s.at(sg[t][0] * p, sg[t][1] * q, sg[t][2] * r) - s.at(-sg[t][0] * p, -sg[t][1] * q, -sg[t][2] * r);
    acc = (t == 0) ? term : acc + term;
  }
  return acc;
}

struct QTerms { double u, Qx, Qy, Qz, Qxy, Qxz, Qyz, Qxyz; };

QTerms qterms(const double* P, int i, int j, int k) {
  Stencil s{P, i, j, k};
  QTerms t;
  t.u = s.at(0, 0, 0);
  t.Qx = C0 * (s.at(1, 0, 0) - s.at(-1, 0, 0)) + C1 * (s.at(2, 0, 0) - s.at(-2, 0, 0));
  t.Qy = C0 * (s.at(0, 1, 0) - s.at(0, -1, 0)) + C1 * (s.at(0, 2, 0) - s.at(0, -2, 0));
  t.Qz = C0 * (s.at(0, 0, 1) - s.at(0, 0, -1)) + C1 * (s.at(0, 0, 2) - s.at(0, 0, -2));
  const int pq[4][2] = {{1, 1}, {2, 2}, {1, 2}, {2, 1}};   // c00, c11, c01, c10
  double qxy = 0, qxz = 0, qyz = 0;
  for (int t2 = 0; t2 < 4; ++t2) {
    int p = pq[t2][0], q = pq[t2][1];
    double cc = cidx(p) * cidx(q);
    double a = cc * mix2(s, 0, 1, p, q), b = cc * mix2(s, 0, 2, p, q), c = cc * mix2(s, 1, 2, p, q);
    qxy = (t2 == 0) ? a : qxy + a;
    qxz = (t2 == 0) ? b : qxz + b;
    qyz = (t2 == 0) ? c : qyz + c;
  }
  t.Qxy = qxy;
  t.Qxz = qxz;
  t.Qyz = qyz;
  // c000, c111, c001, c110, c011, c100, c010, c101 (offsets x, y, z)
  const int pqr[8][3] = {{1, 1, 1}, {2, 2, 2}, {1, 1, 2}, {2, 2, 1}, {1, 2, 2}, {2, 1, 1}, {1, 2, 1}, {2, 1, 2}};
  double qxyz = 0;
  for (int t3 = 0; t3 < 8; ++t3) {
    int p = pqr[t3][0], q = pqr[t3][1], r = pqr[t3][2];
    double cc = cidx(p) * cidx(q) * cidx(r);
    double a = cc * mix3(s, p, q, r);
    qxyz = (t3 == 0) ? a : qxyz + a;
  }
  t.Qxyz = qxyz;
  return t;
}

inline double predict_from(const QTerms& t, double sx, double sy, double sz) {
  return t.u + sx * t.Qx + sy * t.Qy + sz * t.Qz + (sx * sy) * t.Qxy + (sx * sz) * t.Qxz + (sy * sz) * t.Qyz +
         (sx * sy * sz) * t.Qxyz;
}

// Value of fine cell (i, j, k) (stored index of child `ch`, i.e. in [-4, 20)^3)
// predicted from the parent's stored array P of one variable.
double predict_cell(const double* P, int ch, int i, int j, int k) {
  int c[3] = {ch & 1, (ch >> 1) & 1, (ch >> 2) & 1};
  int f[3] = {i, j, k}, p[3];
  double s[3];
  for (int d = 0; d < 3; ++d) {
    int h = floordiv2(f[d]);
    p[d] = 8 * c[d] + h;
    s[d] = (f[d] - 2 * h == 0) ? 1.0 : -1.0;
  }
  QTerms t = qterms(P, p[0], p[1], p[2]);
  return predict_from(t, s[0], s[1], s[2]);
}

// ------------------------------------------------------------ context helpers
double dx_of(const Ctx& C, int level) { return std::ldexp(C.c.dx0, -level); }

bool is_outside_region(const Ctx& C, const Node& n, int sx, int sy, int sz) {
  int s[3] = {sx, sy, sz};
  for (int d = 0; d < 3; ++d) {
    if (s[d] == 0) continue;
    int64_t nl = (int64_t)C.c.base_blocks[d] << n.level;
    bool edge = (s[d] < 0) ? (n.X[d] == 0) : (n.X[d] == nl - 1);
    if (edge && C.c.bc[2 * d + (s[d] > 0 ? 1 : 0)] != BC_PERIODIC) return true;
  }
  return false;
}

std::vector<Node*> nodes_at(Ctx& C, int level, bool leaves_only) {
  std::vector<Node*> v;
  for (auto& kv : C.nodes)
    if ((level < 0 || kv.second.level == level) && (!leaves_only || kv.second.leaf)) v.push_back(&kv.second);
  return v;
}

int max_level(const Ctx& C) {
  int m = 0;
  for (auto& kv : C.nodes) m = std::max(m, kv.second.level);
  return m;
}

Node* find(Ctx& C, uint64_t key) {
  auto it = C.nodes.find(key);
  return it == C.nodes.end() ? nullptr : &it->second;
}

Node* parent_of(Ctx& C, const Node& n) {
  if (n.level == 0) return nullptr;
  uint64_t inst = n.key >> 56;
  uint64_t pk = ((n.key & MASK56) >> 3) | (inst << 56);
  return find(C, pk);
}

int child_index(const Node& n) { return (int)(n.key & 7); }

// ------------------------------------------------------------ halo fill
// Sec. 3 (Fig. MrCommunicationMesh) and Alg. (ComputeLoop): a halo region facing
// a same-level node (brother or cousin, leaf or not) is a copy of its internal
// cells; a region facing no same-level node is predicted from the block's own
// parent; a region beyond the domain boundary takes the boundary condition.
// Levels are processed coarse to fine because prediction reads the parent's halo.
void apply_bc(const Ctx& C, Node& n) {
  for (int d = 0; d < 3; ++d) {
    for (int side = 0; side < 2; ++side) {
      int bc = C.c.bc[2 * d + side];
      if (bc == BC_PERIODIC) continue;
      int64_t nl = (int64_t)C.c.base_blocks[d] << n.level;
      if (side == 0 && n.X[d] != 0) continue;
      if (side == 1 && n.X[d] != nl - 1) continue;
      for (int k = -HW; k < NB + HW; ++k)
        for (int j = -HW; j < NB + HW; ++j)
          for (int i = -HW; i < NB + HW; ++i) {
            int c[3] = {i, j, k};
            int a = c[d];
            bool ghost = (side == 0) ? (a < 0) : (a >= NB);
            if (!ghost) continue;
            int src[3] = {i, j, k};
            if (bc == BC_ZERO_GRADIENT) src[d] = (side == 0) ? 0 : NB - 1;
            else src[d] = (side == 0) ? (-1 - a) : (2 * NB - 1 - a);
            for (int v = 0; v < NV; ++v) {
              double val = n.u[(size_t)v * NCELL + sidx(src[0], src[1], src[2])];
              if (bc == BC_SYMMETRY && v == 1 + d) val = -val;
              n.u[(size_t)v * NCELL + sidx(i, j, k)] = val;
            }
          }
    }
  }
}

void fill_node(Ctx& C, Node& n) {
  // resolve the 26 regions
  int kind[27];          // 0 outside, 1 copy, 2 predict
  const Node* src[27];
  for (int sz = -1; sz <= 1; ++sz)
    for (int sy = -1; sy <= 1; ++sy)
      for (int sx = -1; sx <= 1; ++sx) {
        int r = (sz + 1) * 9 + (sy + 1) * 3 + (sx + 1);
        src[r] = nullptr;
        kind[r] = 0;
        if (r == 13) continue;
        if (is_outside_region(C, n, sx, sy, sz)) continue;
        uint64_t nk;
        bool ok = neighbour(C.c, n.key, sx, sy, sz, &nk);
        if (!ok) continue;
        Node* nb = find(C, nk);
        if (nb) {
          kind[r] = 1;
          src[r] = nb;
        } else {
          kind[r] = 2;
        }
      }
  Node* par = parent_of(C, n);
  int ch = child_index(n);
  for (int k = -HW; k < NB + HW; ++k)
    for (int j = -HW; j < NB + HW; ++j)
      for (int i = -HW; i < NB + HW; ++i) {
        int sx = i < 0 ? -1 : (i >= NB ? 1 : 0);
        int sy = j < 0 ? -1 : (j >= NB ? 1 : 0);
        int sz = k < 0 ? -1 : (k >= NB ? 1 : 0);
        int r = (sz + 1) * 9 + (sy + 1) * 3 + (sx + 1);
        if (r == 13 || kind[r] == 0) continue;
        for (int v = 0; v < NV; ++v) {
          double val;
          if (kind[r] == 1) {
            val = src[r]->u[(size_t)v * NCELL + sidx(i - NB * sx, j - NB * sy, k - NB * sz)];
          } else {
            val = predict_cell(&par->u[(size_t)v * NCELL], ch, i, j, k);
          }
          n.u[(size_t)v * NCELL + sidx(i, j, k)] = val;
        }
      }
  apply_bc(C, n);
}

void fill_halos(Ctx& C) {
  int lm = max_level(C);
  for (int l = 0; l <= lm; ++l) {
    std::vector<Node*> v = nodes_at(C, l, false);
#pragma omp parallel for schedule(dynamic)
    for (long t = 0; t < (long)v.size(); ++t) fill_node(C, *v[t]);
  }
}

// ------------------------------------------------------------ right-hand side
// Sec. 2.2: dimension-by-dimension face fluxes; L = -sum_d (F_{+1/2} - F_{-1/2})/dx
// evaluated as ((Fx_lo - Fx_hi) + (Fy_lo - Fy_hi) + (Fz_lo - Fz_hi)) / dx, plus the
// gravity source S = (0, rho g, m . g) of Eq. (Euler) when gravity is set.
// Viscous flux of the Navier-Stokes equations (Sec. 2.1 names them beside
// Eq. Euler; Stokes' hypothesis, constant dynamic viscosity mu, no heat
// conduction) at the face between the stored cells cL and cL + e_d of node n,
// lab frame: (0, tau_xd, tau_yd, tau_zd, u . tau_d) with
// tau_ij = mu (du_i/dx_j + du_j/dx_i) - 2/3 mu (div u) delta_ij.  Second-order
// compact face gradients: the normal derivative from the two face cells, a
// tangential derivative as the mean of the two face cells' central
// differences; the face velocity is the mean of the two face cells'.
void viscous_flux(const Node& n, int d, const int cL[3], double mu, double dx, double Fv[5]) {
  auto vel = [&](const int c[3], double w[3]) {
    int s = sidx(c[0], c[1], c[2]);
    double rho = n.u[s];
    w[0] = n.u[NCELL + s] / rho;
    w[1] = n.u[2 * NCELL + s] / rho;
    w[2] = n.u[3 * NCELL + s] / rho;
  };
  int cR[3] = {cL[0], cL[1], cL[2]};
  cR[d] += 1;
  double uL[3], uR[3];
  vel(cL, uL);
  vel(cR, uR);
  double G[3][3];   // G[i][j] = du_i / dx_j at the face
  for (int i = 0; i < 3; ++i) G[i][d] = (uR[i] - uL[i]) / dx;
  for (int j = 0; j < 3; ++j) {
    if (j == d) continue;
    int lp[3] = {cL[0], cL[1], cL[2]}, lm[3] = {cL[0], cL[1], cL[2]};
    int rp[3] = {cR[0], cR[1], cR[2]}, rm[3] = {cR[0], cR[1], cR[2]};
    lp[j] += 1;
    lm[j] -= 1;
    rp[j] += 1;
    rm[j] -= 1;
    double a[3], b[3], c[3], e[3];
    vel(lp, a);
    vel(lm, b);
    vel(rp, c);
    vel(rm, e);
    for (int i = 0; i < 3; ++i) G[i][j] = ((a[i] - b[i]) + (c[i] - e[i])) / (4.0 * dx);
  }
  double div = (G[0][0] + G[1][1]) + G[2][2];
  double ub[3], tau[3];
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

void leaf_rhs(const Ctx& C, Node& n) {
  double g = C.c.gamma, B = C.c.B;
  double dx = dx_of(C, n.level);
  // flux[d][v][face along d][t] for every face of the block (17 per pencil)
  std::vector<double> F((size_t)3 * NV * (NB + 1) * NFACE);
  auto fidx = [&](int d, int v, int f, int a, int b) {
    return ((((size_t)d * NV + v) * (NB + 1) + f) * NB + b) * NB + a;
  };
  for (int d = 0; d < 3; ++d) {
    for (int b = 0; b < NB; ++b)
      for (int a = 0; a < NB; ++a)
        for (int f = 0; f <= NB; ++f) {
          double U6[6][5];
          for (int m = 0; m < 6; ++m) {
            int along = f - 3 + m;
            int c[3];
            c[d] = along;
            c[(d == 0) ? 1 : 0] = a;
            c[(d == 2) ? 1 : 2] = b;
            for (int v = 0; v < NV; ++v) U6[m][v] = n.u[(size_t)v * NCELL + sidx(c[0], c[1], c[2])];
          }
          double Fo[5];
          face_flux(U6, d, g, B, C.c.recon, C.c.flux, Fo);
          if (C.c.mu > 0.0) {
            // Navier-Stokes: the face flux is F(U) - F_v(U, grad u)
            int cl[3];
            cl[d] = f - 1;
            cl[(d == 0) ? 1 : 0] = a;
            cl[(d == 2) ? 1 : 2] = b;
            double Fv[5];
            viscous_flux(n, d, cl, C.c.mu, dx, Fv);
            for (int v = 0; v < NV; ++v) Fo[v] = Fo[v] - Fv[v];
          }
          for (int v = 0; v < NV; ++v) F[fidx(d, v, f, a, b)] = Fo[v];
        }
  }
  // tangential index pairs: d=0 -> (y, z), d=1 -> (x, z), d=2 -> (x, y)
  for (int k = 0; k < NB; ++k)
    for (int j = 0; j < NB; ++j)
      for (int i = 0; i < NB; ++i)
        for (int v = 0; v < NV; ++v) {
          double acc = F[fidx(0, v, i, j, k)] - F[fidx(0, v, i + 1, j, k)];
          acc = acc + (F[fidx(1, v, j, i, k)] - F[fidx(1, v, j + 1, i, k)]);
          acc = acc + (F[fidx(2, v, k, i, j)] - F[fidx(2, v, k + 1, i, j)]);
          double Lv = acc / dx;
          n.L[(size_t)v * NINT + iidx(i, j, k)] = Lv;
        }
  double gx = C.c.gravity[0], gy = C.c.gravity[1], gz = C.c.gravity[2];
  if (gx != 0.0 || gy != 0.0 || gz != 0.0) {
    for (int k = 0; k < NB; ++k)
      for (int j = 0; j < NB; ++j)
        for (int i = 0; i < NB; ++i) {
          int s = sidx(i, j, k), t = iidx(i, j, k);
          double rho = n.u[s], mx = n.u[NCELL + s], my = n.u[2 * NCELL + s], mz = n.u[3 * NCELL + s];
          n.L[(size_t)1 * NINT + t] = n.L[(size_t)1 * NINT + t] + rho * gx;
          n.L[(size_t)2 * NINT + t] = n.L[(size_t)2 * NINT + t] + rho * gy;
          n.L[(size_t)3 * NINT + t] = n.L[(size_t)3 * NINT + t] + rho * gz;
          n.L[(size_t)4 * NINT + t] = n.L[(size_t)4 * NINT + t] + ((mx * gx + my * gy) + mz * gz);
        }
  }
  // boundary-face fluxes for the jump correction: side 2d at face 0, 2d+1 at face 16
  for (int d = 0; d < 3; ++d)
    for (int v = 0; v < NV; ++v)
      for (int b = 0; b < NB; ++b)
        for (int a = 0; a < NB; ++a) {
          n.face[(((size_t)(2 * d) * NV + v) * NB + b) * NB + a] = F[fidx(d, v, 0, a, b)];
          n.face[(((size_t)(2 * d + 1) * NV + v) * NB + b) * NB + a] = F[fidx(d, v, NB, a, b)];
        }
}

void compute_L_all(Ctx& C) {
  std::vector<Node*> v = nodes_at(C, -1, true);
#pragma omp parallel for schedule(dynamic)
  for (long t = 0; t < (long)v.size(); ++t) leaf_rhs(C, *v[t]);
}

// Face fluxes of internal nodes: the mean of the four child faces covering each
// parent face cell, bottom-up (the face buffers that keep jumps conservative,
// Sec. 4 and Alg. (ComputeLoop) averaging of F).  Tangential axes (t1, t2):
// x-faces (y, z), y-faces (x, z), z-faces (x, y).
void average_faces(Ctx& C) {
  int lm = max_level(C);
  for (int l = lm - 1; l >= 0; --l) {
    std::vector<Node*> v = nodes_at(C, l, false);
#pragma omp parallel for schedule(dynamic)
    for (long t = 0; t < (long)v.size(); ++t) {
      Node& P = *v[t];
      if (P.leaf) continue;
      uint64_t inst = P.key >> 56;
      for (int s = 0; s < 6; ++s) {
        int d = s / 2, hi = s & 1;
        int t1 = (d == 0) ? 1 : 0, t2 = (d == 2) ? 1 : 2;
        for (int bb = 0; bb < NB; ++bb)
          for (int aa = 0; aa < NB; ++aa) {
            int ct1 = aa / 8, ct2 = bb / 8;
            int cb[3];
            cb[d] = hi;
            cb[t1] = ct1;
            cb[t2] = ct2;
            int ch = cb[0] | (cb[1] << 1) | (cb[2] << 2);
            uint64_t ck = (((P.key & MASK56) << 3) | (uint64_t)ch) | (inst << 56);
            const Node* c = find(C, ck);
            int fa = 2 * (aa - 8 * ct1), fb = 2 * (bb - 8 * ct2);
            for (int v2 = 0; v2 < NV; ++v2) {
              auto f = [&](int x, int y) { return c->face[(((size_t)s * NV + v2) * NB + fb + y) * NB + fa + x]; };
              double val = 0.25 * ((f(0, 0) + f(1, 0)) + (f(0, 1) + f(1, 1)));
              P.face[(((size_t)s * NV + v2) * NB + bb) * NB + aa] = val;
            }
          }
      }
    }
  }
}

// Jump correction (Sec. 4 and Alg. (ComputeLoop)): a leaf face that touches a
// finer region replaces its own flux by the averaged fine flux.  Applied to the
// stage result, as the paper adjusts coarse cell values after integration:
// u += b_s (dt dL), dL = (F_coarse - F_fine)/dx on an upper face and
// (F_fine - F_coarse)/dx on a lower face; sides in the order x-, x+, y-, y+, z-, z+.
// With target_L the same correction is added to L instead (L += dL).
void jump_correct(Ctx& C, bool target_L, double bs, const double* dt) {
  std::vector<Node*> v = nodes_at(C, -1, true);
#pragma omp parallel for schedule(dynamic)
  for (long t = 0; t < (long)v.size(); ++t) {
    Node& n = *v[t];
    double dx = dx_of(C, n.level);
    for (int s = 0; s < 6; ++s) {
      int d = s / 2, hi = s & 1;
      uint64_t nk;
      if (!axis_step(C.c, n.key, d, hi ? 1 : -1, &nk)) continue;
      const Node* nb = find(C, nk);
      if (!nb || nb->leaf) continue;
      int so = s ^ 1;
      int t1 = (d == 0) ? 1 : 0, t2 = (d == 2) ? 1 : 2;
      for (int bb = 0; bb < NB; ++bb)
        for (int aa = 0; aa < NB; ++aa) {
          int c[3];
          c[d] = hi ? NB - 1 : 0;
          c[t1] = aa;
          c[t2] = bb;
          for (int v2 = 0; v2 < NV; ++v2) {
            double Fc = n.face[(((size_t)s * NV + v2) * NB + bb) * NB + aa];
            double Ff = nb->face[(((size_t)so * NV + v2) * NB + bb) * NB + aa];
            double dL = hi ? (Fc - Ff) / dx : (Ff - Fc) / dx;
            if (target_L) {
              double& Lr = n.L[(size_t)v2 * NINT + iidx(c[0], c[1], c[2])];
              Lr = Lr + dL;
            } else {
              double& ur = n.u[(size_t)v2 * NCELL + sidx(c[0], c[1], c[2])];
              ur = ur + bs * (dt[n.inst] * dL);
            }
          }
        }
    }
  }
}

// ------------------------------------------------------------ time integration
// TVD-RK3 in Shu-Osher form: u1 = un + dt L(un); u2 = 3/4 un + 1/4 (u1 + dt L(u1));
// u3 = 1/3 un + 2/3 (u2 + dt L(u2)); evaluated as t = u + dt L, out = a un + b t.
// TVD-RK2 (the paper's standard second-order Runge-Kutta, Sec. 5, in the same
// form): u1 = un + dt L(un); u2 = 1/2 un + 1/2 (u1 + dt L(u1)).
const double RK_A3[3] = {0.0, 0.75, 1.0 / 3.0};
const double RK_B3[3] = {1.0, 0.25, 2.0 / 3.0};
const double RK_A2[2] = {0.0, 0.5};
const double RK_B2[2] = {1.0, 0.5};

inline int rk_stages(const Ctx& C) { return C.c.rk_stages == 2 ? 2 : 3; }
inline double rk_a(const Ctx& C, int s) { return rk_stages(C) == 2 ? RK_A2[s] : RK_A3[s]; }
inline double rk_b(const Ctx& C, int s) { return rk_stages(C) == 2 ? RK_B2[s] : RK_B3[s]; }

void rk_update_nodes(Ctx& C, const std::vector<Node*>& v, int s, const double* dt) {
#pragma omp parallel for schedule(dynamic)
  for (long t = 0; t < (long)v.size(); ++t) {
    Node& n = *v[t];
    double h = dt[n.inst];
    for (int var = 0; var < NV; ++var)
      for (int k = 0; k < NB; ++k)
        for (int j = 0; j < NB; ++j)
          for (int i = 0; i < NB; ++i) {
            size_t si = (size_t)var * NCELL + sidx(i, j, k);
            size_t ii = (size_t)var * NINT + iidx(i, j, k);
            if (s == 0) n.un[ii] = n.u[si];
            double tt = n.u[si] + h * n.L[ii];
            n.u[si] = (s == 0) ? tt : (rk_a(C, s) * n.un[ii] + rk_b(C, s) * tt);
          }
  }
}

void rk_update(Ctx& C, int s, const double* dt) { rk_update_nodes(C, nodes_at(C, -1, true), s, dt); }

// Averaging, Eq. (Averaging): a parent cell is the mean of its eight children,
// summed pairwise in Morton order ((c0+c1)+(c2+c3))+((c4+c5)+(c6+c7)), levels
// from fine to coarse.
void average_children(Ctx& C, Node& P) {
  uint64_t inst = P.key >> 56;
  const Node* ch[8];
  for (int c = 0; c < 8; ++c) ch[c] = find(C, (((P.key & MASK56) << 3) | (uint64_t)c) | (inst << 56));
  for (int K = 0; K < NB; ++K)
    for (int J = 0; J < NB; ++J)
      for (int I = 0; I < NB; ++I) {
        int o = (I / 8) | ((J / 8) << 1) | ((K / 8) << 2);
        const Node* c = ch[o];
        int fi = 2 * (I - 8 * (I / 8)), fj = 2 * (J - 8 * (J / 8)), fk = 2 * (K - 8 * (K / 8));
        for (int v2 = 0; v2 < NV; ++v2) {
          const double* u = &c->u[(size_t)v2 * NCELL];
          double c0 = u[sidx(fi, fj, fk)], c1 = u[sidx(fi + 1, fj, fk)];
          double c2 = u[sidx(fi, fj + 1, fk)], c3 = u[sidx(fi + 1, fj + 1, fk)];
          double c4 = u[sidx(fi, fj, fk + 1)], c5 = u[sidx(fi + 1, fj, fk + 1)];
          double c6 = u[sidx(fi, fj + 1, fk + 1)], c7 = u[sidx(fi + 1, fj + 1, fk + 1)];
          P.u[(size_t)v2 * NCELL + sidx(I, J, K)] = 0.125 * (((c0 + c1) + (c2 + c3)) + ((c4 + c5) + (c6 + c7)));
        }
      }
}

void project(Ctx& C) {
  int lm = max_level(C);
  for (int l = lm - 1; l >= 0; --l) {
    std::vector<Node*> v = nodes_at(C, l, false);
#pragma omp parallel for schedule(dynamic)
    for (long t = 0; t < (long)v.size(); ++t) {
      Node& P = *v[t];
      if (P.leaf) continue;
      average_children(C, P);
    }
  }
}

// Eq. (Cfl): dt = CFL dx_lmax / ( max|u|+c + max|v|+c + max|w|+c ), each maximum
// over all leaf internal cells of the instance, summed in x, y, z order.
// Eq. (Cfl), extended for the viscous terms by the explicit diffusion limit
// of the second-order Laplacian in 3D: dt_v = k dx^2 / (6 max(mu / rho)); the
// step is the smaller of the two.
void cfl_dt(Ctx& C, double* dt) {
  int ni = C.c.n_instances;
  std::vector<double> sm((size_t)ni * 3, 0.0), ir((size_t)ni, 0.0);
  for (auto& kv : C.nodes) {
    Node& n = kv.second;
    if (!n.leaf) continue;
    for (int k = 0; k < NB; ++k)
      for (int j = 0; j < NB; ++j)
        for (int i = 0; i < NB; ++i) {
          double U[5];
          for (int v = 0; v < NV; ++v) U[v] = n.u[(size_t)v * NCELL + sidx(i, j, k)];
          Prim q = prim_of(U, C.c.gamma, C.c.B);
          for (int d = 0; d < 3; ++d) sm[(size_t)n.inst * 3 + d] = std::max(sm[(size_t)n.inst * 3 + d], std::fabs(q.vel[d]) + q.c);
          ir[n.inst] = std::max(ir[n.inst], 1.0 / q.rho);
        }
  }
  for (int i = 0; i < ni; ++i) {
    double dxl = dx_of(C, C.c.lmax[i]);
    dt[i] = C.c.cfl * dxl / ((sm[(size_t)i * 3] + sm[(size_t)i * 3 + 1]) + sm[(size_t)i * 3 + 2]);
    if (C.c.mu > 0.0) dt[i] = std::min(dt[i], (C.c.cfl * (dxl * dxl)) / ((6.0 * C.c.mu) * ir[i]));
  }
}

// ------------------------------------------------------------ MR analysis
// Eq. (DetailFunction): d = u_B - P(u_parent) over the block including its halo
// (Sec. 3; ghost cells beyond a non-periodic domain boundary are not cells of
// the domain and are left out).  Block norm (l-infinity, relative to the fine
// value, over rho and E): delta_B = max |d_v| / |u_v|.  Eq. (LevelWiseEpsilon)
// with D = 3: eps_l = 2^{-3 (lmax - l)} eps.
double block_delta(Ctx& C, Node& n) {
  Node* P = parent_of(C, n);
  int ch = child_index(n);
  double delta = 0.0;
  const int vars[2] = {0, 4};
  for (int k = -HW; k < NB + HW; ++k)
    for (int j = -HW; j < NB + HW; ++j)
      for (int i = -HW; i < NB + HW; ++i) {
        int sx = i < 0 ? -1 : (i >= NB ? 1 : 0);
        int sy = j < 0 ? -1 : (j >= NB ? 1 : 0);
        int sz = k < 0 ? -1 : (k >= NB ? 1 : 0);
        bool ghost = false;
        int s[3] = {sx, sy, sz};
        for (int d = 0; d < 3; ++d) {
          if (s[d] == 0) continue;
          int64_t nl = (int64_t)C.c.base_blocks[d] << n.level;
          bool edge = (s[d] < 0) ? (n.X[d] == 0) : (n.X[d] == nl - 1);
          if (edge && C.c.bc[2 * d + (s[d] > 0 ? 1 : 0)] != BC_PERIODIC) ghost = true;
        }
        if (ghost) continue;
        for (int vi = 0; vi < 2; ++vi) {
          int v = vars[vi];
          double uf = n.u[(size_t)v * NCELL + sidx(i, j, k)];
          double pr = predict_cell(&P->u[(size_t)v * NCELL], ch, i, j, k);
          double r = std::fabs(uf - pr) / std::fabs(uf);
          delta = std::max(delta, r);
        }
      }
  return delta;
}

// Tags of the leaves (Eq. Thresholding with Eq. LevelWiseEpsilon, D = 3):
// REFINE a leaf on level l below l_max whose detail exceeds
// eps_l = 2^{-3 (lmax - l)} eps; COARSEN a complete group of eight leaf
// siblings at level >= 2 (no node on level 1 is ever coarsened, Sec. 4) whose
// details are all below eps_l; equality keeps the block.  In the analysis between time steps (allow_refine) a
// group is kept while its parent's own detail exceeds the parent's threshold:
// the parent would be refined again at once (its children, just predicted
// from it, have no details), so coarsening them would make the tree
// alternate between two states from step to step.
void predict_and_tag(Ctx& C, int allow_refine, int8_t* tags, double* deltas) {
  std::vector<Node*> leaves = nodes_at(C, -1, true);
  std::vector<double> dl(leaves.size(), 0.0);
#pragma omp parallel for schedule(dynamic)
  for (long t = 0; t < (long)leaves.size(); ++t)
    if (leaves[t]->level >= 1) dl[t] = block_delta(C, *leaves[t]);
  std::map<uint64_t, size_t> pos;
  for (size_t t = 0; t < leaves.size(); ++t) pos[leaves[t]->key] = t;
  // details of the parents of complete leaf groups at level >= 2
  std::map<uint64_t, double> dpar;
  if (allow_refine) {
    std::vector<Node*> par;
    for (Node* n : leaves)
      if (n->level >= 2 && (n->key & 7ull) == 0) par.push_back(parent_of(C, *n));
    std::vector<double> dp(par.size(), 0.0);
#pragma omp parallel for schedule(dynamic)
    for (long t = 0; t < (long)par.size(); ++t) dp[t] = block_delta(C, *par[t]);
    for (size_t t = 0; t < par.size(); ++t) dpar[par[t]->key] = dp[t];
  }
  for (size_t t = 0; t < leaves.size(); ++t) {
    Node& n = *leaves[t];
    int8_t tag = TAG_KEEP;
    if (n.level >= 1) {
      int lmx = C.c.lmax[n.inst];
      double el = std::ldexp(C.c.eps, -3 * (lmx - n.level));
      if (allow_refine && dl[t] > el && n.level < lmx) {
        tag = TAG_REFINE;
      } else if (n.level >= 2) {
        bool all = true;
        uint64_t inst = n.key >> 56;
        uint64_t pk = (n.key & MASK56) >> 3;
        for (int c = 0; c < 8 && all; ++c) {
          uint64_t sk = ((pk << 3) | (uint64_t)c) | (inst << 56);
          auto it = pos.find(sk);
          if (it == pos.end()) { all = false; break; }
          if (!(dl[it->second] < el)) all = false;
        }
        if (all && allow_refine) {
          double ep = std::ldexp(C.c.eps, -3 * (lmx - (n.level - 1)));
          if (dpar[pk | (inst << 56)] > ep) all = false;
        }
        if (all) tag = TAG_COARSEN;
      }
    }
    tags[t] = tag;
    if (deltas) deltas[t] = dl[t];
  }
}

Node make_child(const Node& P, int ch) {
  Node c;
  c.inst = P.inst;
  c.level = P.level + 1;
  for (int d = 0; d < 3; ++d) c.X[d] = 2 * P.X[d] + ((ch >> d) & 1);
  c.key = make_key(c.inst, c.level, c.X);
  c.leaf = true;
  c.alloc();
  for (int v = 0; v < NV; ++v)
    for (int k = -HW; k < NB + HW; ++k)
      for (int j = -HW; j < NB + HW; ++j)
        for (int i = -HW; i < NB + HW; ++i)
          c.u[(size_t)v * NCELL + sidx(i, j, k)] = predict_cell(&P.u[(size_t)v * NCELL], ch, i, j, k);
  return c;
}

// Refinement creates the eight children from the prediction of the parent over
// their whole stored range; coarsening removes a complete sibling group (the
// parent already holds their average).  Refinements are applied before
// coarsenings, each in ascending key order.
int64_t remesh(Ctx& C, const int8_t* tags) {
  std::vector<Node*> leaves = nodes_at(C, -1, true);
  std::vector<uint64_t> ref, coarse_parents;
  std::map<uint64_t, int> ccount;
  for (size_t t = 0; t < leaves.size(); ++t) {
    Node& n = *leaves[t];
    if (tags[t] == TAG_REFINE && n.level < C.c.lmax[n.inst]) ref.push_back(n.key);
    if (tags[t] == TAG_COARSEN && n.level >= 2) {
      uint64_t inst = n.key >> 56;
      uint64_t pk = ((n.key & MASK56) >> 3) | (inst << 56);
      ccount[pk] += 1;
    }
  }
  for (auto& kv : ccount)
    if (kv.second == 8) coarse_parents.push_back(kv.first);
  std::vector<Node> made(ref.size() * 8);
#pragma omp parallel for schedule(dynamic)
  for (long t = 0; t < (long)made.size(); ++t) made[t] = make_child(*find(C, ref[t / 8]), (int)(t % 8));
  for (size_t t = 0; t < made.size(); ++t) C.nodes.emplace(made[t].key, std::move(made[t]));
  for (uint64_t k : ref) find(C, k)->leaf = false;
  for (uint64_t pk : coarse_parents) {
    uint64_t inst = pk >> 56;
    for (int ch = 0; ch < 8; ++ch) C.nodes.erase((((pk & MASK56) << 3) | (uint64_t)ch) | (inst << 56));
    find(C, pk)->leaf = true;
  }
  int64_t nl = 0;
  for (auto& kv : C.nodes) nl += kv.second.leaf ? 1 : 0;
  return nl;
}

// Census of the Roe / LLF switch (used to count the algorithm's work): for
// every face of every leaf (17 x 16 x 16 per direction), which characteristic
// fields take the LLF split under the per-field rule of face_flux.
// counts[k] = faces where field k is split, counts[5] = faces.
void flux_census(Ctx& C, uint64_t* counts) {
  for (int k = 0; k < 6; ++k) counts[k] = 0;
  double g = C.c.gamma, B = C.c.B;
  for (auto& kv : C.nodes) {
    const Node& n = kv.second;
    if (!n.leaf) continue;
    for (int d = 0; d < 3; ++d)
      for (int b = 0; b < NB; ++b)
        for (int a = 0; a < NB; ++a)
          for (int f = 0; f <= NB; ++f) {
            double U[2][5];
            for (int m = 0; m < 2; ++m) {
              int c[3];
              c[d] = f - 1 + m;
              c[(d == 0) ? 1 : 0] = a;
              c[(d == 2) ? 1 : 2] = b;
              for (int v = 0; v < NV; ++v) U[m][v] = n.u[(size_t)v * NCELL + sidx(c[0], c[1], c[2])];
            }
            Prim qL = prim_of(U[0], g, B), qR = prim_of(U[1], g, B);
            Eigen e = roe_eigen(qL, qR, d, g);
            double unL = qL.vel[d], unR = qR.vel[d];
            double lamL[5] = {unL - qL.c, unL, unL, unL, unL + qL.c};
            double lamR[5] = {unR - qR.c, unR, unR, unR, unR + qR.c};
            for (int k = 0; k < 5; ++k) {
              double lL = lamL[k], lR = lamR[k], lt = e.lam[k];
              bool up = (lL > 0.0 && lR > 0.0 && lt > 0.0) || (lL < 0.0 && lR < 0.0 && lt < 0.0);
              if (!up) counts[k] += 1;
            }
            counts[5] += 1;
          }
  }
}

// Conservation sums: per instance, sum over leaves (key order) of the cell sum
// (storage order) times dx^3.
void sums(Ctx& C, double* out) {
  int ni = C.c.n_instances;
  for (int i = 0; i < ni * NV; ++i) out[i] = 0.0;
  for (auto& kv : C.nodes) {
    Node& n = kv.second;
    if (!n.leaf) continue;
    double dx = dx_of(C, n.level);
    double vol = dx * dx * dx;
    for (int v = 0; v < NV; ++v) {
      double s = 0.0;
      for (int k = 0; k < NB; ++k)
        for (int j = 0; j < NB; ++j)
          for (int i = 0; i < NB; ++i) s = s + n.u[(size_t)v * NCELL + sidx(i, j, k)];
      out[(size_t)n.inst * NV + v] = out[(size_t)n.inst * NV + v] + s * vol;
    }
  }
}

void stage(Ctx& C, int s, const double* dt) {
  fill_halos(C);
  compute_L_all(C);
  average_faces(C);
  rk_update(C, s, dt);
  jump_correct(C, false, rk_b(C, s), dt);
  project(C);
}

// ------------------------------------------------------------ local time stepping
// Reading of Eq. (LtsTimestep) with Alg. (ComputeLoop) and Alg. (Integration)
// (the paper gives their order but not the data each step acts on; the choices
// below are this reading's):
//  * a macro time step starts with Delta t_L from Eq. (Cfl) (L = l_max, the
//    same for every instance), fixed for the macro step; level l advances in
//    steps of Delta t_l = 2^(L - l) Delta t_L (Eq. LtsTimestep);
//  * micro steps r = 0 .. 2^L - 1: every level whose step starts at r (r a
//    multiple of 2^(L - l)) and that holds nodes takes one full Runge-Kutta
//    step, coarse levels first;
//  * a level's step advances all its nodes, leaves and internal nodes alike
//    (an internal node carries that level's approximation of the finer region
//    it covers, which its neighbours' stencils and its children's predicted
//    halos read); each stage fills the halos of all nodes (levels coarse to
//    fine: a region without a same-level neighbour is predicted from the
//    parent), with the nodes of coarser levels -- whose current step spans the
//    stage's time -- interpolated linearly in time between the start (u^n) and
//    the end of that step; it then computes the right-hand side of the
//    level's nodes, updates them with Delta t_l and adds each leaf's
//    boundary-face fluxes, weighted by the stage's share of the step
//    (TVD-RK3: 1/6, 1/6, 2/3; TVD-RK2: 1/2, 1/2) times Delta t_l, to its
//    integrated fluxes;
//  * after a micro step every level whose step ends there is synchronised:
//    the internal nodes of that level and finer ones are replaced by the
//    average of their children (Eq. Averaging), finest first;
//  * at the end of the macro step the integrated fluxes of internal nodes are
//    averaged from their children (bottom-up) and every leaf face that
//    touches a refined neighbour exchanges its own integrated flux for the
//    finer side's (Alg. ComputeLoop's adjustment of coarse cell values with
//    the averaged fine fluxes), so the macro step is conservative; then the
//    averaging once more.
// With l_max = 0 this is global stepping.
const double RK_W3[3] = {1.0 / 6.0, 1.0 / 6.0, 2.0 / 3.0};
const double RK_W2[2] = {0.5, 0.5};
inline double rk_w(const Ctx& C, int s) { return rk_stages(C) == 2 ? RK_W2[s] : RK_W3[s]; }
// Stage times as fractions of the step (TVD-RK3: 0, 1, 1/2; TVD-RK2: 0, 1).
const double RK_C3[3] = {0.0, 1.0, 0.5};
const double RK_C2[2] = {0.0, 1.0};
inline double rk_c(const Ctx& C, int s) { return rk_stages(C) == 2 ? RK_C2[s] : RK_C3[s]; }

// Averaging of the internal nodes of levels lo .. l_max - 1 (finest first).
void project_from(Ctx& C, int lo) {
  int lm = max_level(C);
  for (int l = lm - 1; l >= lo; --l) {
    std::vector<Node*> v = nodes_at(C, l, false);
#pragma omp parallel for schedule(dynamic)
    for (long t = 0; t < (long)v.size(); ++t) {
      Node& P = *v[t];
      if (P.leaf) continue;
      average_children(C, P);
    }
  }
}

// A stage of level `level` at micro step r.
void lts_level_stage(Ctx& C, int level, int r, int L, int s, const double* dtl) {
  std::vector<Node*> coarse;
  std::vector<double> theta;
  for (int m = 0; m < level; ++m)
    for (Node* n : nodes_at(C, m, false)) {
      const int span = 1 << (L - m);
      const int r0 = r - r % span;
      coarse.push_back(n);
      theta.push_back(((double)(r - r0) + rk_c(C, s) * (double)(1 << (L - level))) / (double)span);
    }
  std::vector<std::vector<double>> keep(coarse.size());
#pragma omp parallel for schedule(dynamic)
  for (long t = 0; t < (long)coarse.size(); ++t) {
    Node& n = *coarse[t];
    const double th = theta[t];
    keep[t].resize((size_t)NV * NINT);
    for (int var = 0; var < NV; ++var)
      for (int k = 0; k < NB; ++k)
        for (int j = 0; j < NB; ++j)
          for (int i = 0; i < NB; ++i) {
            const size_t si = (size_t)var * NCELL + sidx(i, j, k), ii = (size_t)var * NINT + iidx(i, j, k);
            keep[t][ii] = n.u[si];
            n.u[si] = (1.0 - th) * n.un[ii] + th * n.u[si];
          }
  }
  fill_halos(C);
  std::vector<Node*> v = nodes_at(C, level, false);
#pragma omp parallel for schedule(dynamic)
  for (long t = 0; t < (long)v.size(); ++t) leaf_rhs(C, *v[t]);
  rk_update_nodes(C, v, s, dtl);
#pragma omp parallel for schedule(dynamic)
  for (long t = 0; t < (long)v.size(); ++t) {
    Node& n = *v[t];
    if (!n.leaf) continue;
    const double w = rk_w(C, s) * dtl[n.inst];
    for (size_t e = 0; e < n.fmac.size(); ++e) n.fmac[e] = n.fmac[e] + w * n.face[e];
  }
#pragma omp parallel for schedule(dynamic)
  for (long t = 0; t < (long)coarse.size(); ++t) {
    Node& n = *coarse[t];
    for (int var = 0; var < NV; ++var)
      for (int k = 0; k < NB; ++k)
        for (int j = 0; j < NB; ++j)
          for (int i = 0; i < NB; ++i)
            n.u[(size_t)var * NCELL + sidx(i, j, k)] = keep[t][(size_t)var * NINT + iidx(i, j, k)];
  }
}

// Integrated face fluxes of internal nodes: the mean of the four child faces
// covering each parent face cell, bottom-up (as average_faces does per stage).
void average_fmac(Ctx& C) {
  int lm = max_level(C);
  for (int l = lm - 1; l >= 0; --l) {
    std::vector<Node*> v = nodes_at(C, l, false);
#pragma omp parallel for schedule(dynamic)
    for (long t = 0; t < (long)v.size(); ++t) {
      Node& P = *v[t];
      if (P.leaf) continue;
      uint64_t inst = P.key >> 56;
      for (int s = 0; s < 6; ++s) {
        int d = s / 2, hi = s & 1;
        int t1 = (d == 0) ? 1 : 0, t2 = (d == 2) ? 1 : 2;
        for (int bb = 0; bb < NB; ++bb)
          for (int aa = 0; aa < NB; ++aa) {
            int ct1 = aa / 8, ct2 = bb / 8;
            int cb[3];
            cb[d] = hi;
            cb[t1] = ct1;
            cb[t2] = ct2;
            int ch = cb[0] | (cb[1] << 1) | (cb[2] << 2);
            uint64_t ck = (((P.key & MASK56) << 3) | (uint64_t)ch) | (inst << 56);
            const Node* c = find(C, ck);
            int fa = 2 * (aa - 8 * ct1), fb = 2 * (bb - 8 * ct2);
            for (int v2 = 0; v2 < NV; ++v2) {
              auto f = [&](int x, int y) { return c->fmac[(((size_t)s * NV + v2) * NB + fb + y) * NB + fa + x]; };
              P.fmac[(((size_t)s * NV + v2) * NB + bb) * NB + aa] = 0.25 * ((f(0, 0) + f(1, 0)) + (f(0, 1) + f(1, 1)));
            }
          }
      }
    }
  }
}

// The end-of-macro-step correction: a leaf face whose same-level neighbour is
// refined takes the finer side's integrated flux, u += (F_c - F_f)/dx on an
// upper face and (F_f - F_c)/dx on a lower one, sides x-, x+, y-, y+, z-, z+.
void lts_reflux(Ctx& C) {
  std::vector<Node*> v = nodes_at(C, -1, true);
#pragma omp parallel for schedule(dynamic)
  for (long t = 0; t < (long)v.size(); ++t) {
    Node& n = *v[t];
    double dx = dx_of(C, n.level);
    for (int s = 0; s < 6; ++s) {
      int d = s / 2, hi = s & 1;
      uint64_t nk;
      if (!axis_step(C.c, n.key, d, hi ? 1 : -1, &nk)) continue;
      const Node* nb = find(C, nk);
      if (!nb || nb->leaf) continue;
      int so = s ^ 1;
      int t1 = (d == 0) ? 1 : 0, t2 = (d == 2) ? 1 : 2;
      for (int bb = 0; bb < NB; ++bb)
        for (int aa = 0; aa < NB; ++aa) {
          int c[3];
          c[d] = hi ? NB - 1 : 0;
          c[t1] = aa;
          c[t2] = bb;
          for (int v2 = 0; v2 < NV; ++v2) {
            double Fc = n.fmac[(((size_t)s * NV + v2) * NB + bb) * NB + aa];
            double Ff = nb->fmac[(((size_t)so * NV + v2) * NB + bb) * NB + aa];
            double dU = hi ? (Fc - Ff) / dx : (Ff - Fc) / dx;
            double& ur = n.u[(size_t)v2 * NCELL + sidx(c[0], c[1], c[2])];
            ur = ur + dU;
          }
        }
    }
  }
}

void lts_macro_step(Ctx& C, double* dt) {
  cfl_dt(C, dt);
  const int L = C.c.lmax[0];
  for (auto& kv : C.nodes) std::fill(kv.second.fmac.begin(), kv.second.fmac.end(), 0.0);
  std::vector<double> dtl((size_t)C.c.n_instances);
  for (int r = 0; r < (1 << L); ++r) {
    for (int l = 0; l <= L; ++l) {
      if (r % (1 << (L - l)) != 0) continue;
      if (nodes_at(C, l, false).empty()) continue;
      for (int i = 0; i < C.c.n_instances; ++i) dtl[i] = std::ldexp(dt[i], L - l);
      for (int s = 0; s < rk_stages(C); ++s) lts_level_stage(C, l, r, L, s, dtl.data());
    }
    // levels whose step ends with this micro step: synchronise them
    int lo = L;
    for (int l = L; l >= 0; --l)
      if ((r + 1) % (1 << (L - l)) == 0) lo = l;
    project_from(C, lo);
  }
  average_fmac(C);
  lts_reflux(C);
  project(C);
}

bool any_mr(const Ctx& C) {
  for (int i = 0; i < C.c.n_instances; ++i)
    if (C.c.lmax[i] > 0) return true;
  return false;
}

// ------------------------------------------------------------ operation count
// Measurement only (the roofline's algorithmic FLOPs), never part of a result.
// Sym is a counting number type: it carries the double value (so every branch
// of the face-flux chain is taken as for that value) and a node of an
// expression graph.  Nodes are hash-consed on (operation, operands), so an
// expression the chain evaluates twice from the same operands is one node
// (what common-subexpression elimination keeps once: the primitive variables
// and physical flux of a cell shared by the faces of a row).  Values built only
// from literals and from the run constants gamma and B fold to constants; a
// multiplication by a literal 0 or +-1 and an addition of a literal 0 are no
// operation (the zero and unit entries of the eigenvectors).  The count is
// the number of add, subtract, multiply, divide and square-root nodes
// reachable from the outputs and from the operands of every comparison (the
// branch decisions: the eigenvalue signs of the Roe/LLF switch, the TENO5
// cutoff, HLLC's admissibility and wave pattern), so values the chain computes
// but never uses (the v = L U projections of fields that are upwinded) are not
// counted.  Negation, absolute value, max/min and comparisons count as no
// operation.
enum SymOp : int32_t { S_IN, S_CONST, S_ADD, S_SUB, S_MUL, S_DIV, S_SQRT, S_NEG, S_ABS, S_MAX, S_MIN };

struct SymGraph {
  struct Rec { int32_t op, a, b; };
  std::vector<Rec> nodes;
  std::map<std::tuple<int32_t, int32_t, int32_t, uint64_t>, int32_t> index;
  int32_t make(int32_t op, int32_t a, int32_t b, uint64_t extra = 0) {
    if ((op == S_ADD || op == S_MUL) && a > b) std::swap(a, b);
    auto key = std::make_tuple(op, a, b, extra);
    auto it = index.find(key);
    if (it != index.end()) return it->second;
    nodes.push_back({op, a, b});
    const int32_t id = (int32_t)nodes.size() - 1;
    index.emplace(key, id);
    return id;
  }
};
SymGraph* g_sym = nullptr;

struct Sym {
  double v;
  int32_t id;   // -1: a constant
  Sym() : v(0.0), id(-1) {}
  Sym(double x) : v(x), id(-1) {}
  static Sym input(double x, uint64_t serial) {
    Sym s(x);
    s.id = g_sym->make(S_IN, -1, -1, serial);
    return s;
  }
  int32_t node() const {
    if (id >= 0) return id;
    uint64_t bits;
    std::memcpy(&bits, &v, 8);
    return g_sym->make(S_CONST, -1, -1, bits);
  }
};

inline Sym sym_node(double v, int32_t op, const Sym& a, const Sym& b) {
  Sym r(v);
  r.id = g_sym->make(op, a.node(), b.node());
  return r;
}
inline Sym operator-(const Sym& a) {
  if (a.id < 0) return Sym(-a.v);
  Sym r(-a.v);
  r.id = g_sym->make(S_NEG, a.id, -1);
  return r;
}
inline Sym operator+(const Sym& a, const Sym& b) {
  if (a.id < 0 && b.id < 0) return Sym(a.v + b.v);
  if (a.id < 0 && a.v == 0.0) return b;
  if (b.id < 0 && b.v == 0.0) return a;
  return sym_node(a.v + b.v, S_ADD, a, b);
}
inline Sym operator-(const Sym& a, const Sym& b) {
  if (a.id < 0 && b.id < 0) return Sym(a.v - b.v);
  if (b.id < 0 && b.v == 0.0) return a;
  if (a.id < 0 && a.v == 0.0) return -b;
  return sym_node(a.v - b.v, S_SUB, a, b);
}
inline Sym operator*(const Sym& a, const Sym& b) {
  if (a.id < 0 && b.id < 0) return Sym(a.v * b.v);
  if ((a.id < 0 && a.v == 0.0) || (b.id < 0 && b.v == 0.0)) return Sym(0.0);
  if (a.id < 0 && a.v == 1.0) return b;
  if (b.id < 0 && b.v == 1.0) return a;
  if (a.id < 0 && a.v == -1.0) return -b;
  if (b.id < 0 && b.v == -1.0) return -a;
  return sym_node(a.v * b.v, S_MUL, a, b);
}
inline Sym operator/(const Sym& a, const Sym& b) {
  if (a.id < 0 && b.id < 0) return Sym(a.v / b.v);
  if (b.id < 0 && b.v == 1.0) return a;
  return sym_node(a.v / b.v, S_DIV, a, b);
}
inline Sym osqrt(const Sym& a) {
  if (a.id < 0) return Sym(std::sqrt(a.v));
  Sym r(std::sqrt(a.v));
  r.id = g_sym->make(S_SQRT, a.id, -1);
  return r;
}
inline Sym oabs(const Sym& a) {
  if (a.id < 0) return Sym(std::fabs(a.v));
  Sym r(std::fabs(a.v));
  r.id = g_sym->make(S_ABS, a.id, -1);
  return r;
}
inline Sym omax(const Sym& a, const Sym& b) {
  if (a.id < 0 && b.id < 0) return Sym(std::max(a.v, b.v));
  return sym_node(std::max(a.v, b.v), S_MAX, a, b);
}
inline Sym omin(const Sym& a, const Sym& b) {
  if (a.id < 0 && b.id < 0) return Sym(std::min(a.v, b.v));
  return sym_node(std::min(a.v, b.v), S_MIN, a, b);
}
// A comparison decides a branch, so the values it compares are needed: their
// nodes become roots of the count like the outputs.
std::vector<int32_t>* g_sym_roots = nullptr;
inline void sym_decides(const Sym& a, const Sym& b) {
  if (a.id >= 0) g_sym_roots->push_back(a.id);
  if (b.id >= 0) g_sym_roots->push_back(b.id);
}
inline bool operator<(const Sym& a, const Sym& b) { sym_decides(a, b); return a.v < b.v; }
inline bool operator>(const Sym& a, const Sym& b) { sym_decides(a, b); return a.v > b.v; }
inline bool operator<=(const Sym& a, const Sym& b) { sym_decides(a, b); return a.v <= b.v; }
inline bool operator>=(const Sym& a, const Sym& b) { sym_decides(a, b); return a.v >= b.v; }

// Operations reachable from the outputs, by kind: [0] FLOPs (the sum of the
// next four), [1] add and subtract, [2] multiply, [3] divide, [4] square root.
void sym_count(const std::vector<int32_t>& outputs, int64_t counts[5]) {
  std::vector<char> seen(g_sym->nodes.size(), 0);
  std::vector<int32_t> stack(outputs.begin(), outputs.end());
  for (int i = 0; i < 5; ++i) counts[i] = 0;
  while (!stack.empty()) {
    const int32_t n = stack.back();
    stack.pop_back();
    if (n < 0 || seen[n]) continue;
    seen[n] = 1;
    const SymGraph::Rec r = g_sym->nodes[n];
    if (r.op == S_ADD || r.op == S_SUB) counts[1]++;
    if (r.op == S_MUL) counts[2]++;
    if (r.op == S_DIV) counts[3]++;
    if (r.op == S_SQRT) counts[4]++;
    stack.push_back(r.a);
    stack.push_back(r.b);
  }
  counts[0] = counts[1] + counts[2] + counts[3] + counts[4];
}

// One row of a block along direction d: the 17 faces between cells -1..16
// (stencil cells -3..18, i.e. Urow[m] for cell m - 3, conserved variables in
// the lab frame), each by face_flux exactly as leaf_rhs evaluates it.
void count_row(const double* Urow, int d, double g, double B, int mode, int flux, int64_t counts[5]) {
  SymGraph graph;
  std::vector<int32_t> roots;
  g_sym = &graph;
  g_sym_roots = &roots;
  Sym U[NB + 6][5];
  for (int m = 0; m < NB + 6; ++m)
    for (int v = 0; v < NV; ++v) U[m][v] = Sym::input(Urow[m * NV + v], (uint64_t)(m * NV + v));
  std::vector<int32_t> out;
  for (int f = 0; f <= NB; ++f) {
    Sym U6[6][5], Fo[5];
    for (int m = 0; m < 6; ++m)
      for (int v = 0; v < NV; ++v) U6[m][v] = U[f + m][v];
    face_flux(U6, d, g, B, mode, flux, Fo);
    for (int v = 0; v < NV; ++v) out.push_back(Fo[v].node());
  }
  out.insert(out.end(), roots.begin(), roots.end());
  sym_count(out, counts);
  g_sym = nullptr;
  g_sym_roots = nullptr;
}

// One reconstruction of the given mode on five inputs.
void count_recon(int mode, int64_t counts[5]) {
  SymGraph graph;
  std::vector<int32_t> roots;
  g_sym = &graph;
  g_sym_roots = &roots;
  Sym a[5];
  for (int m = 0; m < 5; ++m) a[m] = Sym::input(1.0 + 0.1 * m * m, (uint64_t)m);
  Sym r = recon5(mode, a[0], a[1], a[2], a[3], a[4]);
  roots.push_back(r.node());
  sym_count(roots, counts);
  g_sym = nullptr;
  g_sym_roots = nullptr;
}

}  // namespace

// =============================================================== C interface
extern "C" {

void* orc_create(const orc_config* cfg) {
  Ctx* C = new Ctx();
  C->c = *cfg;
#ifdef _OPENMP
  if (cfg->n_threads > 0) omp_set_num_threads(cfg->n_threads);
#endif
  for (int inst = 0; inst < cfg->n_instances; ++inst)
    for (int64_t z = 0; z < cfg->base_blocks[2]; ++z)
      for (int64_t y = 0; y < cfg->base_blocks[1]; ++y)
        for (int64_t x = 0; x < cfg->base_blocks[0]; ++x) {
          Node n;
          n.inst = inst;
          n.level = 0;
          n.X[0] = x;
          n.X[1] = y;
          n.X[2] = z;
          n.key = make_key(inst, 0, n.X);
          n.leaf = true;
          n.alloc();
          C->nodes.emplace(n.key, std::move(n));
        }
  return C;
}

void orc_destroy(void* h) { delete (Ctx*)h; }

int64_t orc_list(void* h, int32_t level, int32_t leaves_only, uint64_t* keys, int64_t cap) {
  Ctx& C = *(Ctx*)h;
  int64_t n = 0;
  for (auto& kv : C.nodes) {
    const Node& nd = kv.second;
    if (level >= 0 && nd.level != level) continue;
    if (leaves_only && !nd.leaf) continue;
    if (keys && n < cap) keys[n] = nd.key;
    ++n;
  }
  return n;
}

// Block geometry in the same order as orc_list: geo[n][4] = (level, X, Y, Z),
// block coordinates on that level.
int64_t orc_list_geometry(void* h, int32_t level, int32_t leaves_only, int64_t* geo, int64_t cap) {
  Ctx& C = *(Ctx*)h;
  int64_t n = 0;
  for (auto& kv : C.nodes) {
    const Node& nd = kv.second;
    if (level >= 0 && nd.level != level) continue;
    if (leaves_only && !nd.leaf) continue;
    if (geo && n < cap) {
      geo[4 * n] = nd.level;
      geo[4 * n + 1] = nd.X[0];
      geo[4 * n + 2] = nd.X[1];
      geo[4 * n + 3] = nd.X[2];
    }
    ++n;
  }
  return n;
}

// prim: [n][5][16][16][16] primitive (rho, u, v, w, p) of the internal cells.
int orc_set_state(void* h, const uint64_t* keys, int64_t n, const double* prim) {
  Ctx& C = *(Ctx*)h;
  double g = C.c.gamma, B = C.c.B;
  for (int64_t b = 0; b < n; ++b) {
    Node* nd = find(C, keys[b]);
    if (!nd) return -1;
    const double* P = prim + (size_t)b * NV * NINT;
    for (int k = 0; k < NB; ++k)
      for (int j = 0; j < NB; ++j)
        for (int i = 0; i < NB; ++i) {
          int t = iidx(i, j, k), s = sidx(i, j, k);
          double rho = P[t], u = P[NINT + t], v = P[2 * NINT + t], w = P[3 * NINT + t], p = P[4 * NINT + t];
          double q2 = (u * u + v * v) + w * w;
          nd->u[s] = rho;
          nd->u[NCELL + s] = rho * u;
          nd->u[2 * NCELL + s] = rho * v;
          nd->u[3 * NCELL + s] = rho * w;
          nd->u[4 * NCELL + s] = (p + g * B) / (g - 1.0) + 0.5 * rho * q2;
        }
  }
  return 0;
}

// Conserved state written directly (internal cells), [n][5][16^3].
int orc_set_cons(void* h, const uint64_t* keys, int64_t n, const double* cons) {
  Ctx& C = *(Ctx*)h;
  for (int64_t b = 0; b < n; ++b) {
    Node* nd = find(C, keys[b]);
    if (!nd) return -1;
    for (int v = 0; v < NV; ++v)
      for (int k = 0; k < NB; ++k)
        for (int j = 0; j < NB; ++j)
          for (int i = 0; i < NB; ++i)
            nd->u[(size_t)v * NCELL + sidx(i, j, k)] = cons[((size_t)b * NV + v) * NINT + iidx(i, j, k)];
  }
  return 0;
}

// cons: [n][5][16^3] (with_halo = 0) or [n][5][24^3] (with_halo = 1).
int orc_get_state(void* h, const uint64_t* keys, int64_t n, double* cons, int32_t with_halo) {
  Ctx& C = *(Ctx*)h;
  for (int64_t b = 0; b < n; ++b) {
    Node* nd = find(C, keys[b]);
    if (!nd) return -1;
    if (with_halo) {
      std::memcpy(cons + (size_t)b * NV * NCELL, nd->u.data(), sizeof(double) * NV * NCELL);
    } else {
      for (int v = 0; v < NV; ++v)
        for (int k = 0; k < NB; ++k)
          for (int j = 0; j < NB; ++j)
            for (int i = 0; i < NB; ++i)
              cons[((size_t)b * NV + v) * NINT + iidx(i, j, k)] = nd->u[(size_t)v * NCELL + sidx(i, j, k)];
    }
  }
  return 0;
}

void orc_fill_halos(void* h) { fill_halos(*(Ctx*)h); }

// L of every leaf (leaf order) including the jump correction: [nleaves][5][16^3].
void orc_compute_rhs(void* h, double* L) {
  Ctx& C = *(Ctx*)h;
  compute_L_all(C);
  average_faces(C);
  jump_correct(C, true, 1.0, nullptr);
  if (L) {
    size_t b = 0;
    for (auto& kv : C.nodes) {
      if (!kv.second.leaf) continue;
      std::memcpy(L + b * NV * NINT, kv.second.L.data(), sizeof(double) * NV * NINT);
      ++b;
    }
  }
}

// One Runge-Kutta stage on the leaves: L, update, jump correction (halos must be filled).
void orc_rk_stage(void* h, int32_t s, const double* dt) {
  Ctx& C = *(Ctx*)h;
  compute_L_all(C);
  average_faces(C);
  rk_update(C, s, dt);
  jump_correct(C, false, rk_b(C, s), dt);
}

void orc_project(void* h) { project(*(Ctx*)h); }
void orc_cfl_dt(void* h, double* dt) { cfl_dt(*(Ctx*)h, dt); }
void orc_predict_and_tag(void* h, int32_t allow_refine, int8_t* tags, double* deltas) {
  predict_and_tag(*(Ctx*)h, allow_refine, tags, deltas);
}
int64_t orc_remesh(void* h, const int8_t* tags) { return remesh(*(Ctx*)h, tags); }
void orc_sums(void* h, double* out) { sums(*(Ctx*)h, out); }
void orc_flux_census(void* h, uint64_t* counts) { flux_census(*(Ctx*)h, counts); }

// nsteps full steps: CFL, the Runge-Kutta stages, then (with MR) analysis and remesh.
// dt_hist (nullable) receives [nsteps][n_instances].
void orc_step(void* h, int32_t nsteps, double* dt_hist) {
  Ctx& C = *(Ctx*)h;
  std::vector<double> dt((size_t)C.c.n_instances);
  for (int st = 0; st < nsteps; ++st) {
    if (C.c.lts) {
      lts_macro_step(C, dt.data());
    } else {
      cfl_dt(C, dt.data());
      for (int s = 0; s < rk_stages(C); ++s) stage(C, s, dt.data());
    }
    if (dt_hist) std::memcpy(dt_hist + (size_t)st * C.c.n_instances, dt.data(), sizeof(double) * C.c.n_instances);
    if (any_mr(C)) {
      fill_halos(C);
      std::vector<int8_t> tags((size_t)orc_list(h, -1, 1, nullptr, 0));
      predict_and_tag(C, 1, tags.data(), nullptr);
      remesh(C, tags.data());
    }
  }
}

// One LTS macro step without the MR analysis (dt: [n_instances] out, Delta t_L).
void orc_lts_macro_step(void* h, double* dt) { lts_macro_step(*(Ctx*)h, dt); }

// Same-level neighbour by Alg. (NeighborLookup): returns 1 and the id, or 0 at
// a non-periodic domain boundary.
int32_t orc_neighbor(const orc_config* cfg, uint64_t key, int32_t sx, int32_t sy, int32_t sz, uint64_t* out) {
  return neighbour(*cfg, key, sx, sy, sz, out) ? 1 : 0;
}

uint64_t orc_make_key(int32_t inst, int32_t level, int64_t x, int64_t y, int64_t z) {
  int64_t X[3] = {x, y, z};
  return make_key(inst, level, X);
}

int32_t orc_key_level(uint64_t key) { return key_level(key); }

// ---- pure functions exported for the pins
double orc_weno5(const double* f) { return weno5(f[0], f[1], f[2], f[3], f[4]); }
double orc_linear5(const double* f) { return linear5(f[0], f[1], f[2], f[3], f[4]); }
double orc_teno5(const double* f) { return teno5(f[0], f[1], f[2], f[3], f[4]); }
double orc_wenoao53(const double* f) { return wenoao53(f[0], f[1], f[2], f[3], f[4]); }

void orc_flux(const double* U, int32_t d, double g, double B, double* F) {
  Prim q = prim_of(U, g, B);
  double Ur[5], Fr[5];
  rotate(U, d, Ur);
  flux_rot(Ur, q, d, Fr);
  unrotate(Fr, d, F);
}

// Rotated-frame eigensystem of the Roe average between UL and UR (lab-frame
// conserved states) along d; Lm, Rm row-major 5x5.
void orc_roe_eigen(const double* UL, const double* UR, int32_t d, double g, double B, double* Lm, double* Rm,
                   double* lam) {
  Prim a = prim_of(UL, g, B), b = prim_of(UR, g, B);
  Eigen e = roe_eigen(a, b, d, g);
  for (int i = 0; i < 5; ++i) {
    lam[i] = e.lam[i];
    for (int j = 0; j < 5; ++j) {
      Lm[i * 5 + j] = e.Lm[i][j];
      Rm[i * 5 + j] = e.Rm[i][j];
    }
  }
}

void orc_face_flux(const double* U6, int32_t d, double g, double B, int32_t mode, int32_t flux, double* F) {
  double U[6][5];
  for (int m = 0; m < 6; ++m)
    for (int v = 0; v < 5; ++v) U[m][v] = U6[m * 5 + v];
  face_flux(U, d, g, B, mode, flux, F);
}

// HLLC flux between two lab-frame states along d (lab frame out).
void orc_hllc(const double* UL, const double* UR, int32_t d, double g, double B, double* F) {
  double a[5], b[5], Fr[5];
  rotate(UL, d, a);
  rotate(UR, d, b);
  hllc_rot(a, b, g, B, Fr);
  unrotate(Fr, d, F);
}

// Selector features [15] and label of one face (six lab-frame cells [6][5]).
void orc_face_features(const double* U6, int32_t d, double g, double B, double tau_lab, double* feats,
                       int32_t* label, double* aux) {
  double U[6][5];
  for (int m = 0; m < 6; ++m)
    for (int v = 0; v < 5; ++v) U[m][v] = U6[m * 5 + v];
  int lab = 0;
  face_features(U, d, g, B, tau_lab, feats, &lab, aux);
  *label = lab;
}

// Child `ch` (bit 0 x, bit 1 y, bit 2 z) predicted over its whole stored range
// from a parent's stored array (one variable, 24^3).
void orc_predict_block(const double* parent, int32_t ch, double* child) {
  for (int k = -HW; k < NB + HW; ++k)
    for (int j = -HW; j < NB + HW; ++j)
      for (int i = -HW; i < NB + HW; ++i) child[sidx(i, j, k)] = predict_cell(parent, ch, i, j, k);
}

// Parent internal cells (16^3) from the eight children's stored arrays (8 x 24^3).
void orc_average_block(const double* children, double* parent) {
  for (int K = 0; K < NB; ++K)
    for (int J = 0; J < NB; ++J)
      for (int I = 0; I < NB; ++I) {
        int o = (I / 8) | ((J / 8) << 1) | ((K / 8) << 2);
        const double* u = children + (size_t)o * NCELL;
        int fi = 2 * (I - 8 * (I / 8)), fj = 2 * (J - 8 * (J / 8)), fk = 2 * (K - 8 * (K / 8));
        double c0 = u[sidx(fi, fj, fk)], c1 = u[sidx(fi + 1, fj, fk)];
        double c2 = u[sidx(fi, fj + 1, fk)], c3 = u[sidx(fi + 1, fj + 1, fk)];
        double c4 = u[sidx(fi, fj, fk + 1)], c5 = u[sidx(fi + 1, fj, fk + 1)];
        double c6 = u[sidx(fi, fj + 1, fk + 1)], c7 = u[sidx(fi + 1, fj + 1, fk + 1)];
        parent[iidx(I, J, K)] = 0.125 * (((c0 + c1) + (c2 + c3)) + ((c4 + c5) + (c6 + c7)));
      }
}

// Operation counts of the face flux (measurement of the roofline's algorithmic
// FLOPs; see count_row): counts[5] = FLOPs, add/sub, mul, div, sqrt.
void orc_count_row_flops(const double* Urow, int32_t d, double g, double B, int32_t mode, int32_t flux,
                         int64_t* counts) {
  count_row(Urow, d, g, B, mode, flux, counts);
}
void orc_count_recon_flops(int32_t mode, int64_t* counts) { count_recon(mode, counts); }

int32_t orc_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

}  // extern "C"
