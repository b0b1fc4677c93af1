// Fused right-hand side + Runge-Kutta stage kernel of the FP64 path (Sec. 2.2
// and Alg. ComputeLoop of arXiv:2012.04385, with the Shu-Osher TVD-RK3 or
// TVD-RK2 stages); every reconstruction, flux scheme and the viscous terms
// are run-time choices here.
//
// One CTA works on one z-slab (16 x 16 x TZ internal cells) of one leaf block
// at a time, looping over (leaf, slab) items.  For each direction it computes
// every face flux of the slab (17 faces per pencil; threads walk the faces
// linearly so neighbouring threads read neighbouring cells), keeps them in
// shared memory, and each thread accumulates the flux differences of the
// cells of its (i, j) column.  The stage update then reads u^(s) and u^n and
// writes u^(s+1) into the other stage buffer.  Boundary-face fluxes go to the
// block's face buffers for the jump correction.
#pragma once

#include "kernels.cuh"

namespace mrb {

constexpr int RHS_TZ = 4;
constexpr int RHS_NSLAB = NB / RHS_TZ;
constexpr int RHS_FMAX = NB * NB * (RHS_TZ + 1);   // >= 17 * 16 * RHS_TZ
constexpr int RHS_THREADS = 256;


// Faces of one direction D of the slab starting at z0: fluxes into Fs, boundary
// faces into the face buffers, then the flux differences into acc.
template <class R, int D>
__device__ __forceinline__ void rhs_dir(const double* __restrict__ u, double* __restrict__ fb, R* Fs, int z0, R g,
                                        R B, int lin, int flux, double mu, double dx,
                                        double (&acc)[RHS_TZ][NV]) {
  const int ti = threadIdx.x & 15, tj = threadIdx.x >> 4;
  constexpr int nf = (D == 2) ? NB * NB * (RHS_TZ + 1) : (NB + 1) * NB * RHS_TZ;
  constexpr int stride = (D == 0) ? 1 : (D == 1 ? NS : NS * NS);
  for (int f = threadIdx.x; f < nf; f += blockDim.x) {
    int ci, cj, ck, fa;
    if (D == 0) {
      fa = f % 17;
      int r = f / 17;
      cj = r % 16;
      ck = z0 + r / 16;
      ci = fa - 3;
    } else if (D == 1) {
      ci = f % 16;
      int r = f / 16;
      fa = r % 17;
      ck = z0 + r / 17;
      cj = fa - 3;
    } else {
      ci = f % 16;
      int r = f / 16;
      cj = r % 16;
      fa = r / 16;
      ck = z0 + fa - 3;
    }
    const int base = sidx(ci, cj, ck);
    R U6[6][5];
#pragma unroll
    for (int m = 0; m < 6; ++m)
#pragma unroll
      for (int v = 0; v < 5; ++v) U6[m][v] = R(u[v * NCELL + base + m * stride]);
    R F[5];
    face_flux<R>(U6, D, g, B, lin, flux, F);
    if (mu > 0.0) {
      // Navier-Stokes: F(U) - F_v at the face between stencil cells 2 and 3
      double Fv[5];
      viscous_flux(u, D, base + 2 * stride, mu, dx, Fv);
#pragma unroll
      for (int v = 0; v < 5; ++v) F[v] = R(double(F[v]) - Fv[v]);
    }
#pragma unroll
    for (int v = 0; v < 5; ++v) Fs[v * RHS_FMAX + f] = F[v];
    const int gface = (D == 2) ? z0 + fa : fa;
    if (gface == 0 || gface == NB) {
      const int side = 2 * D + (gface == NB ? 1 : 0);
      int ta, tb;
      if (D == 0) { ta = cj; tb = ck; }
      else if (D == 1) { ta = ci; tb = ck; }
      else { ta = ci; tb = cj; }
#pragma unroll
      for (int v = 0; v < 5; ++v) fb[((side * NV + v) * NB + tb) * NB + ta] = double(F[v]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int kz = 0; kz < RHS_TZ; ++kz) {
    int lo, hi;
    if (D == 0) { lo = (kz * 16 + tj) * 17 + ti; hi = lo + 1; }
    else if (D == 1) { lo = (kz * 17 + tj) * 16 + ti; hi = lo + 16; }
    else { lo = (kz * 16 + tj) * 16 + ti; hi = lo + 256; }
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      double diff = double(Fs[v * RHS_FMAX + lo]) - double(Fs[v * RHS_FMAX + hi]);
      acc[kz][v] = (D == 0) ? diff : acc[kz][v] + diff;
    }
  }
  __syncthreads();
}

template <class R>
__global__ void __launch_bounds__(RHS_THREADS) k_rhs_rk(Topo t, Phys p, Pool pool, int cur, int stage,
                                                       const double* __restrict__ dt, double* __restrict__ rhs_out,
                                                       int level) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* Fs = reinterpret_cast<R*>(smem_raw);
  const int nitems = stage_nodes(t, level) * RHS_NSLAB;
  const double* __restrict__ src = pool.bufp(cur);
  double* __restrict__ dst = pool.bufp(cur ^ 1);
  const R g = R(p.gamma), B = R(p.B);
  const int lin = p.recon;   // reconstruction mode: 0 WENO5, 2 linear, 3 TENO5, 4 WENO-AO(5,3)
  const int flux = p.flux;   // FLUX_ROE, FLUX_LLF or FLUX_HLLC
  const int ti = threadIdx.x & 15, tj = threadIdx.x >> 4;
  const ItemRange IR = item_range(nitems, p.blocked);
  for (int w = IR.first; w < IR.end; w += IR.step) {
    const int li = w / RHS_NSLAB, z0 = (w % RHS_NSLAB) * RHS_TZ;
    const int node = stage_node(t, level, li);
    const int slot = t.slot[node];
    const double* __restrict__ u = src + (size_t)slot * SLOT_U;
    double* __restrict__ fb = pool.face + (size_t)slot * SLOT_F;
    double acc[RHS_TZ][NV];
    const double dxn = ldexp(p.dx0, -t.level[node]);
    rhs_dir<R, 0>(u, fb, Fs, z0, g, B, lin, flux, p.mu, dxn, acc);
    rhs_dir<R, 1>(u, fb, Fs, z0, g, B, lin, flux, p.mu, dxn, acc);
    rhs_dir<R, 2>(u, fb, Fs, z0, g, B, lin, flux, p.mu, dxn, acc);
    const int inst = t.inst[node];
    const double dx = ldexp(p.dx0, -t.level[node]);
    const double h = dt ? node_dt(t, p, dt, node, level) : 0.0;
    (void)inst;
#pragma unroll
    for (int kz = 0; kz < RHS_TZ; ++kz) {
      const int k = z0 + kz;
      const int s = sidx(ti, tj, k), ii = iidx(ti, tj, k);
      double L[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) L[v] = acc[kz][v] / dx;
      if (p.has_grav) {
        double rho = u[s], mx = u[NCELL + s], my = u[2 * NCELL + s], mz = u[3 * NCELL + s];
        L[1] = L[1] + rho * p.grav[0];
        L[2] = L[2] + rho * p.grav[1];
        L[3] = L[3] + rho * p.grav[2];
        L[4] = L[4] + ((mx * p.grav[0] + my * p.grav[1]) + mz * p.grav[2]);
      }
      if (rhs_out) {
#pragma unroll
        for (int v = 0; v < 5; ++v) rhs_out[((size_t)li * NV + v) * NINT + ii] = L[v];
      } else {
        double* __restrict__ unb = pool.un + (size_t)slot * SLOT_N;
        double* __restrict__ o = dst + (size_t)slot * SLOT_U;
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          const double us = u[v * NCELL + s];
          double un;
          if (stage == 0) {
            un = us;
            unb[v * NINT + ii] = us;
          } else {
            un = unb[v * NINT + ii];
          }
          const double tt = us + h * L[v];
          o[v * NCELL + s] = (stage == 0) ? tt : (kRkA[rk_row(p)][stage] * un + kRkB[rk_row(p)][stage] * tt);
        }
      }
    }
  }
}

template <class R>
void launch_rhs_rk_impl(const Topo& t, const Phys& p, const Pool& pool, int cur, int stage, const double* dt,
                        double* rhs_out, cudaStream_t st, int level) {
  const size_t smem = sizeof(R) * NV * RHS_FMAX;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_rhs_rk<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = true;
  }
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rhs_rk<R>, RHS_THREADS, smem);
  if (per_sm < 1) per_sm = 1;
  const int grid = sm_count() * per_sm * (g_tune.stage_waves < 1 ? 1 : g_tune.stage_waves);
  k_rhs_rk<R><<<grid, RHS_THREADS, smem, st>>>(t, p, pool, cur, stage, dt, rhs_out, level);
  ++g_kernel_launches;
}

}  // namespace mrb
