// FP64 kernels of the block-based MR Euler hot path (arXiv:2012.04385): halo
// fill, fused RHS + TVD-RK3 stage, face-flux averaging and jump correction,
// averaging (projection), CFL reduction, MR details and tags, refinement
// prediction, neighbour table, conservation sums, state import/export.
//
// Built with -fmad=false: every double is the correctly rounded result of the
// operation order written here.
#include "mr.cuh"
#include "rhs.cuh"

namespace mrb {

long long g_kernel_launches = 0;

Tune g_tune = {1, 8, 4, 8};

int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

// ---------------------------------------------------------------- state in/out
__global__ void k_set_state(Topo t, Phys p, Pool pool, int cur, const int32_t* __restrict__ nodes, int n,
                            const double* __restrict__ prim) {
  const double g = p.gamma, B = p.B;
  const size_t total = (size_t)n * NINT;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int b = (int)(e / NINT), c = (int)(e % NINT);
    const int i = c % 16, j = (c / 16) % 16, k = c / 256;
    const double* P = prim + (size_t)b * NV * NINT;
    double rho = P[c], u = P[NINT + c], v = P[2 * NINT + c], w = P[3 * NINT + c], pr = P[4 * NINT + c];
    double q2 = (u * u + v * v) + w * w;
    double* U = pool.bufp(cur) + (size_t)t.slot[nodes[b]] * SLOT_U;
    const int s = sidx(i, j, k);
    U[s] = rho;
    U[NCELL + s] = rho * u;
    U[2 * NCELL + s] = rho * v;
    U[3 * NCELL + s] = rho * w;
    U[4 * NCELL + s] = (pr + g * B) / (g - 1.0) + 0.5 * rho * q2;
  }
}

void launch_set_state(const Topo& t, const Phys& p, const Pool& pool, int cur, const int32_t* nodes, int n,
                      const double* prim, cudaStream_t st) {
  if (n <= 0) return;
  k_set_state<<<sm_count() * 4, 256, 0, st>>>(t, p, pool, cur, nodes, n, prim);
  ++g_kernel_launches;
}

__global__ void k_set_cons(Topo t, Pool pool, int cur, const int32_t* __restrict__ nodes, int n,
                           const double* __restrict__ cons) {
  const size_t total = (size_t)n * NV * NINT;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int b = (int)(e / ((size_t)NV * NINT));
    const int r = (int)(e % ((size_t)NV * NINT));
    const int v = r / NINT, c = r % NINT;
    double* U = pool.bufp(cur) + (size_t)t.slot[nodes[b]] * SLOT_U + (size_t)v * NCELL;
    U[sidx(c % 16, (c / 16) % 16, c / 256)] = cons[e];
  }
}

void launch_set_cons(const Topo& t, const Pool& pool, int cur, const int32_t* nodes, int n, const double* cons,
                     cudaStream_t st) {
  if (n <= 0) return;
  k_set_cons<<<sm_count() * 4, 256, 0, st>>>(t, pool, cur, nodes, n, cons);
  ++g_kernel_launches;
}

__global__ void k_get_state(Topo t, Pool pool, int cur, const int32_t* __restrict__ nodes, int n,
                            double* __restrict__ out, int with_halo) {
  const int per = with_halo ? NCELL : NINT;
  const size_t total = (size_t)n * NV * per;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int b = (int)(e / ((size_t)NV * per));
    const int r = (int)(e % ((size_t)NV * per));
    const int v = r / per, c = r % per;
    const double* U = pool.bufp(cur) + (size_t)t.slot[nodes[b]] * SLOT_U + (size_t)v * NCELL;
    int s;
    if (with_halo) s = c;
    else s = sidx(c % 16, (c / 16) % 16, c / 256);
    out[e] = U[s];
  }
}

void launch_get_state(const Topo& t, const Pool& pool, int cur, const int32_t* nodes, int n, double* out,
                      int with_halo, cudaStream_t st) {
  if (n <= 0) return;
  k_get_state<<<sm_count() * 4, 256, 0, st>>>(t, pool, cur, nodes, n, out, with_halo);
  ++g_kernel_launches;
}

// ---------------------------------------------------------------- halo fill (mr.cuh)
void launch_fill_level(const Topo& t, const Phys& p, const Pool& pool, int cur, int level, cudaStream_t st,
                       int mode) {
  if (p.precision == 1) {
    launch_fill_level_f32(t, p, pool, cur, level, st, mode);
    return;
  }
  // the FP64 stage kernel reads every halo region: no stage-partial fill
  const NodeSet ns{level, nullptr, 0};
  const int m = (mode == FILL_STAGE) ? FILL_FULL : mode;
  k_fill_regions_t<double><<<sm_count() * g_tune.fill_copy, 256, 0, st>>>(t, pool, cur, ns, m);
  k_fill_predict_t<double><<<sm_count() * g_tune.fill_pred, 256, 0, st>>>(t, pool, cur, ns, m);
  k_fill_bc<<<sm_count() * 4, 256, 0, st>>>(t, p, pool, cur, ns, m);
  g_kernel_launches += 3;
}

void launch_fill_list(const Topo& t, const Phys& p, const Pool& pool, int cur, const int32_t* list, int n,
                      cudaStream_t st) {
  if (n <= 0) return;
  if (p.precision == 1) {
    launch_fill_list_f32(t, p, pool, cur, list, n, st);
    return;
  }
  const NodeSet ns{0, list, n};
  k_fill_regions_t<double><<<sm_count() * 8, 256, 0, st>>>(t, pool, cur, ns, FILL_FULL);
  k_fill_predict_t<double><<<sm_count() * 4, 256, 0, st>>>(t, pool, cur, ns, FILL_FULL);
  k_fill_bc<<<sm_count() * 4, 256, 0, st>>>(t, p, pool, cur, ns, FILL_FULL);
  g_kernel_launches += 3;
}

// ---------------------------------------------------------------- RHS + RK (FP64)
void launch_rhs_rk_f64(const Topo& t, const Phys& p, const Pool& pool, int cur, int stage, const double* dt,
                       double* rhs_out, cudaStream_t st, int level) {
  launch_rhs_rk_impl<double>(t, p, pool, cur, stage, dt, rhs_out, st, level);
}

// ---------------------------------------------------------------- face fluxes of internal nodes
// parent face cell = mean of the 2 x 2 covering child face cells, levels fine to coarse
__global__ void k_face_avg_level(Topo t, double* __restrict__ faces, int level) {
  const int beg = t.cnt[CNT_LVL + level], end = t.cnt[CNT_LVL + level + 1];
  for (int w = beg + blockIdx.x; w < end; w += gridDim.x) {
    const int node = t.lvl_nodes[w];
    const int c0 = t.child0[node];
    if (c0 < 0) continue;
    double* F = faces + (size_t)t.slot[node] * SLOT_F;
    for (int e = threadIdx.x; e < 6 * NFACE; e += blockDim.x) {
      const int s = e / NFACE, aa = e % 16, bb = (e / 16) % 16;
      const int d = s / 2, hi = s & 1;
      const int t1 = (d == 0) ? 1 : 0, t2 = (d == 2) ? 1 : 2;
      const int ct1 = aa / 8, ct2 = bb / 8;
      int cb[3];
      cb[d] = hi;
      cb[t1] = ct1;
      cb[t2] = ct2;
      const int ch = cb[0] | (cb[1] << 1) | (cb[2] << 2);
      const double* C = faces + (size_t)t.slot[c0 + ch] * SLOT_F;
      const int fa = 2 * (aa - 8 * ct1), fbb = 2 * (bb - 8 * ct2);
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const double* cf = C + (s * NV + v) * NFACE;
        double f00 = cf[fbb * NB + fa], f10 = cf[fbb * NB + fa + 1];
        double f01 = cf[(fbb + 1) * NB + fa], f11 = cf[(fbb + 1) * NB + fa + 1];
        F[(s * NV + v) * NFACE + bb * NB + aa] = 0.25 * ((f00 + f10) + (f01 + f11));
      }
    }
  }
}

void launch_face_avg_level(const Topo& t, const Pool& pool, int level, cudaStream_t st, int integrated) {
  k_face_avg_level<<<sm_count() * 4, 256, 0, st>>>(t, integrated ? pool.fmac : pool.face, level);
  ++g_kernel_launches;
}

// ---------------------------------------------------------------- local time stepping
// (Eq. LtsTimestep; the reading: a level's step advances all its nodes, the
// halo fill of each stage sees coarser levels interpolated in time, levels are
// averaged from their children when their step ends, and the boundary-face
// fluxes integrated over the macro step are exchanged at its end.)

// Nodes of levels 0 .. below-1: their internal cells become (1 - theta) u^n +
// theta u, the end state u kept in the other stage buffer (restore = 0), or are
// put back from there (restore = 1).
__global__ void k_lts_interp(Topo t, Pool pool, int cur, int below, LevelTheta th, int restore) {
  const int end = t.cnt[CNT_LVL + below];
  for (int w = t.cnt[CNT_LVL + 0] + blockIdx.x; w < end; w += gridDim.x) {
    const int node = t.lvl_nodes[w];
    const size_t slot = (size_t)t.slot[node];
    double* U = pool.bufp(cur) + slot * SLOT_U;
    double* K = pool.bufp(cur ^ 1) + slot * SLOT_U;
    const double* N = pool.un + slot * SLOT_N;
    const double q = th.th[t.level[node]];
    for (int e = threadIdx.x; e < NV * NINT; e += blockDim.x) {
      const int v = e / NINT, ii = e % NINT;
      const int s = v * NCELL + sidx(ii % 16, (ii / 16) % 16, ii / 256);
      if (restore) {
        U[s] = K[s];
      } else {
        const double u = U[s];
        K[s] = u;
        U[s] = (1.0 - q) * N[e] + q * u;
      }
    }
  }
}

void launch_lts_interp(const Topo& t, const Pool& pool, int cur, int below, const LevelTheta& th, int restore,
                       cudaStream_t st) {
  if (below <= 0) return;
  k_lts_interp<<<sm_count() * 4, 256, 0, st>>>(t, pool, cur, below, th, restore);
  ++g_kernel_launches;
}

// Internal cells (and FP32 records) of the nodes of `level`: cur^1 -> cur.
__global__ void k_lts_copyback(Topo t, Pool pool, int cur, int level) {
  const int beg = t.cnt[CNT_LVL + level], end = t.cnt[CNT_LVL + level + 1];
  for (int w = beg + blockIdx.x; w < end; w += gridDim.x) {
    const size_t slot = (size_t)t.slot[t.lvl_nodes[w]];
    double* U = pool.bufp(cur) + slot * SLOT_U;
    const double* O = pool.bufp(cur ^ 1) + slot * SLOT_U;
    for (int e = threadIdx.x; e < NV * NINT; e += blockDim.x) {
      const int v = e / NINT, ii = e % NINT;
      const int s = v * NCELL + sidx(ii % 16, (ii / 16) % 16, ii / 256);
      U[s] = O[s];
    }
    if (pool.shp(0)) {
      float* R = pool.shp(cur) + slot * SLOT_SH;
      const float* Q = pool.shp(cur ^ 1) + slot * SLOT_SH;
      for (int e = threadIdx.x; e < SLOT_SH; e += blockDim.x) R[e] = Q[e];
    }
  }
}

void launch_lts_copyback(const Topo& t, const Pool& pool, int cur, int level, cudaStream_t st) {
  k_lts_copyback<<<sm_count() * 4, 256, 0, st>>>(t, pool, cur, level);
  ++g_kernel_launches;
}

// Integrated boundary-face fluxes of leaves: zero all (zero = 1) or, for the
// leaves of `level`, add (w_stage x dt 2^(lmax - level)) x the stage's face fluxes.
__global__ void k_lts_fmac(Topo t, Phys p, Pool pool, int level, int stage, const double* __restrict__ dt, int zero) {
  const int beg = zero ? 0 : t.cnt[CNT_LVL + level];
  const int end = zero ? t.cnt[CNT_NLEAVES] : t.cnt[CNT_LVL + level + 1];
  for (int w = beg + blockIdx.x; w < end; w += gridDim.x) {
    const int node = zero ? t.leaves[w] : t.lvl_nodes[w];
    if (t.child0[node] >= 0) continue;
    const size_t slot = (size_t)t.slot[node];
    double* M = pool.fmac + slot * SLOT_F;
    if (zero) {
      for (int e = threadIdx.x; e < SLOT_F; e += blockDim.x) M[e] = 0.0;
      continue;
    }
    const double* F = pool.face + slot * SLOT_F;
    const double wgt = kRkW[rk_row(p)][stage] * ldexp(dt[t.inst[node]], p.lmax[t.inst[node]] - level);
    for (int e = threadIdx.x; e < SLOT_F; e += blockDim.x) M[e] = M[e] + wgt * F[e];
  }
}

void launch_lts_fmac(const Topo& t, const Phys& p, const Pool& pool, int level, int stage, const double* dt,
                     int zero, cudaStream_t st) {
  k_lts_fmac<<<sm_count() * 4, 256, 0, st>>>(t, p, pool, level, stage, dt, zero);
  ++g_kernel_launches;
}

// u += (F_c - F_f)/dx on an upper face, (F_f - F_c)/dx on a lower one, with the
// integrated fluxes of the leaf and of its refined same-level neighbour.
__global__ void k_lts_reflux(Topo t, Phys p, Pool pool, int cur) {
  const int nitems = t.cnt[CNT_JUMP];
  for (int w = blockIdx.x; w < nitems; w += gridDim.x) {
    const int li = t.jump[w] >> 6, mask = t.jump[w] & 63;
    const int node = t.leaves[li];
    const double* Fc_all = pool.fmac + (size_t)t.slot[node] * SLOT_F;
    const double dx = ldexp(p.dx0, -t.level[node]);
    double* U = pool.bufp(cur) + (size_t)t.slot[node] * SLOT_U;
#pragma unroll 1
    for (int s = 0; s < 6; ++s) {
      const int d = s / 2, hi = s & 1;
      int sv[3] = {0, 0, 0};
      sv[d] = hi ? 1 : -1;
      const int r = (sv[2] + 1) * 9 + (sv[1] + 1) * 3 + (sv[0] + 1);
      if (!((mask >> s) & 1)) continue;
      const int nb = t.nbr[(size_t)node * 27 + r];
      const double* Ff_all = pool.fmac + (size_t)t.slot[nb] * SLOT_F;
      const int so = s ^ 1;
      const int t1 = (d == 0) ? 1 : 0, t2 = (d == 2) ? 1 : 2;
      for (int e = threadIdx.x; e < NFACE; e += blockDim.x) {
        const int aa = e % 16, bb = e / 16;
        int c[3];
        c[d] = hi ? NB - 1 : 0;
        c[t1] = aa;
        c[t2] = bb;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          const double Fc = Fc_all[(s * NV + v) * NFACE + e];
          const double Ff = Ff_all[(so * NV + v) * NFACE + e];
          const double dU = hi ? (Fc - Ff) / dx : (Ff - Fc) / dx;
          double& ur = U[v * NCELL + sidx(c[0], c[1], c[2])];
          ur = ur + dU;
        }
      }
      __syncthreads();
    }
  }
}

void launch_lts_reflux(const Topo& t, const Phys& p, const Pool& pool, int cur, cudaStream_t st) {
  k_lts_reflux<<<sm_count() * 4, 256, 0, st>>>(t, p, pool, cur);
  ++g_kernel_launches;
}

// ---------------------------------------------------------------- jump correction
// A leaf face whose same-level neighbour is refined takes the averaged fine
// flux: dL = (F_c - F_f)/dx on an upper face, (F_f - F_c)/dx on a lower one,
// applied to the stage result as u += b_s (dt dL) (or added to L in the
// inspection form), sides x-, x+, y-, y+, z-, z+ in order.
__global__ void k_jump(Topo t, Phys p, Pool pool, int target, int stage, const double* __restrict__ dt,
                       double* __restrict__ rhs_out) {
  const int nitems = t.cnt[CNT_JUMP];
  for (int w = blockIdx.x; w < nitems; w += gridDim.x) {
    const int li = t.jump[w] >> 6, mask = t.jump[w] & 63;
    const int node = t.leaves[li];
    const double* Fc_all = pool.face + (size_t)t.slot[node] * SLOT_F;
    const double dx = ldexp(p.dx0, -t.level[node]);
    const double h = dt ? dt[t.inst[node]] : 0.0;
    const double bs = kRkB[rk_row(p)][stage];
    double* U = pool.bufp(target) + (size_t)t.slot[node] * SLOT_U;
#pragma unroll 1
    for (int s = 0; s < 6; ++s) {
      const int d = s / 2, hi = s & 1;
      int sv[3] = {0, 0, 0};
      sv[d] = hi ? 1 : -1;
      const int r = (sv[2] + 1) * 9 + (sv[1] + 1) * 3 + (sv[0] + 1);
      if (!((mask >> s) & 1)) continue;      // the side's neighbour is not refined
      const int nb = t.nbr[(size_t)node * 27 + r];
      const double* Ff_all = pool.face + (size_t)t.slot[nb] * SLOT_F;
      const int so = s ^ 1;
      const int t1 = (d == 0) ? 1 : 0, t2 = (d == 2) ? 1 : 2;
      for (int e = threadIdx.x; e < NFACE; e += blockDim.x) {
        const int aa = e % 16, bb = e / 16;
        int c[3];
        c[d] = hi ? NB - 1 : 0;
        c[t1] = aa;
        c[t2] = bb;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          const double Fc = Fc_all[(s * NV + v) * NFACE + e];
          const double Ff = Ff_all[(so * NV + v) * NFACE + e];
          const double dL = hi ? (Fc - Ff) / dx : (Ff - Fc) / dx;
          if (rhs_out) {
            double& Lr = rhs_out[((size_t)li * NV + v) * NINT + iidx(c[0], c[1], c[2])];
            Lr = Lr + dL;
          } else {
            double& ur = U[v * NCELL + sidx(c[0], c[1], c[2])];
            ur = ur + bs * (h * dL);
            // the mixed-precision path's FP32 stage increment follows the correction
            if (pool.dl) pool.dl[(size_t)t.slot[node] * SLOT_N + v * NINT + iidx(c[0], c[1], c[2])] += (float)(bs * (h * dL));
          }
        }
      }
      __syncthreads();
    }
  }
}

void launch_jump(const Topo& t, const Phys& p, const Pool& pool, int target, int stage, const double* dt,
                 double* rhs_out, cudaStream_t st) {
  k_jump<<<sm_count() * 4, 256, 0, st>>>(t, p, pool, target, stage, dt, rhs_out);
  ++g_kernel_launches;
}

// ---------------------------------------------------------------- averaging (mr.cuh)
void launch_project_level(const Topo& t, const Pool& pool, int buf, int level, cudaStream_t st) {
  k_project_octants<<<sm_count() * g_tune.project, 256, 0, st>>>(t, pool, buf, level);
  ++g_kernel_launches;
}

// ---------------------------------------------------------------- CFL
// Block-wide maxima of N values per thread (sh: [N][8] for 256 threads); the
// result is valid in the first warp.
template <int N>
__device__ __forceinline__ void block_max(double v[N], double* sh) {
  for (int q = 0; q < N; ++q)
    for (int o = 16; o > 0; o >>= 1) v[q] = fmax(v[q], __shfl_xor_sync(0xffffffffu, v[q], o));
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0)
    for (int q = 0; q < N; ++q) sh[q * 8 + wid] = v[q];
  __syncthreads();
  if (threadIdx.x < 32) {
    for (int q = 0; q < N; ++q) {
      double x = (lane < 8) ? sh[q * 8 + lane] : 0.0;
      for (int o = 4; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(0xffffffffu, x, o));
      v[q] = x;
    }
  }
  __syncthreads();
}

__global__ void __launch_bounds__(256) k_cfl(Topo t, Phys p, Pool pool, int cur,
                                             unsigned long long* __restrict__ smax, int* __restrict__ status) {
  __shared__ double sh[32];
  const int nleaves = t.cnt[CNT_NLEAVES];
  for (int li = blockIdx.x; li < nleaves; li += gridDim.x) {
    const int node = t.leaves[li];
    const double* U = pool.bufp(cur) + (size_t)t.slot[node] * SLOT_U;
    double m[4] = {0.0, 0.0, 0.0, 0.0};   // max |u_d| + c per direction, max 1/rho
    bool bad = false;
    for (int e = threadIdx.x; e < NINT; e += blockDim.x) {
      const int s = sidx(e % 16, (e / 16) % 16, e / 256);
      double Uc[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) Uc[v] = U[v * NCELL + s];
      Prim<double> q = prim_of<double>(Uc, p.gamma, p.B);
      if (!(q.rho > 0.0) || !(q.p + p.B > 0.0)) bad = true;
#pragma unroll
      for (int d = 0; d < 3; ++d) m[d] = fmax(m[d], fabs(q.vel[d]) + q.c);
      if (p.mu > 0.0) m[3] = fmax(m[3], 1.0 / q.rho);
    }
    if (bad) atomicExch(status, (int)ST_NONPHYS);
    block_max<4>(m, sh);
    if (threadIdx.x == 0) {
      const int inst = t.inst[node];
      for (int d = 0; d < 4; ++d) atomicMax(&smax[inst * 4 + d], (unsigned long long)__double_as_longlong(m[d]));
    }
  }
}

__global__ void k_cfl_finish(Phys p, const unsigned long long* __restrict__ smax, double* __restrict__ dt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= p.n_inst) return;
  const double s0 = __longlong_as_double((long long)smax[i * 4]);
  const double s1 = __longlong_as_double((long long)smax[i * 4 + 1]);
  const double s2 = __longlong_as_double((long long)smax[i * 4 + 2]);
  const double dxl = ldexp(p.dx0, -p.lmax[i]);
  double h = p.cfl * dxl / ((s0 + s1) + s2);
  if (p.mu > 0.0) {
    // explicit diffusion limit of the viscous terms: k dx^2 / (6 max(mu / rho))
    const double mr = __longlong_as_double((long long)smax[i * 4 + 3]);
    const double hv = (p.cfl * (dxl * dxl)) / ((6.0 * p.mu) * mr);
    h = (hv < h) ? hv : h;
  }
  dt[i] = h;
}

void launch_cfl(const Topo& t, const Phys& p, const Pool& pool, int cur, unsigned long long* smax, double* dt,
                int* status, cudaStream_t st) {
  cudaMemsetAsync(smax, 0, sizeof(unsigned long long) * 4 * p.n_inst, st);
  if (p.precision == 1) launch_cfl_speeds_f32(t, p, pool, cur, smax, status, st);
  else {
    k_cfl<<<sm_count() * 4, 256, 0, st>>>(t, p, pool, cur, smax, status);
    ++g_kernel_launches;
  }
  k_cfl_finish<<<(p.n_inst + 127) / 128, 128, 0, st>>>(p, smax, dt);
  ++g_kernel_launches;
}

// ---------------------------------------------------------------- MR details (mr.cuh) and tags
__global__ void k_tags(Topo t, Phys p, const double* __restrict__ delta_node, int allow_refine,
                       int8_t* __restrict__ tags, double* __restrict__ delta_leaf) {
  const int nleaves = t.cnt[CNT_NLEAVES];
  for (int li = blockIdx.x * blockDim.x + threadIdx.x; li < nleaves; li += gridDim.x * blockDim.x) {
    const int node = t.leaves[li];
    const int lvl = t.level[node];
    const double dl = (lvl >= 1) ? delta_node[node] : 0.0;
    int8_t tag = 0;
    if (lvl >= 1) {
      const int lmx = p.lmax[t.inst[node]];
      const double el = ldexp(p.eps, -3 * (lmx - lvl));
      if (allow_refine && dl > el && lvl < lmx) {
        tag = 1;
      } else if (lvl >= 2) {
        const int c0 = t.child0[t.parent[node]];
        bool all = true;
        for (int c = 0; c < 8; ++c) {
          const int sn = c0 + c;
          if (t.child0[sn] >= 0 || !(delta_node[sn] < el)) {
            all = false;
            break;
          }
        }
        // between time steps a group stays while its parent's own detail asks
        // for it (the parent would be refined again at once)
        if (all && allow_refine && delta_node[t.parent[node]] > ldexp(p.eps, -3 * (lmx - (lvl - 1)))) all = false;
        if (all) tag = -1;
      }
    }
    tags[li] = tag;
    if (delta_leaf) delta_leaf[li] = dl;
  }
}

void launch_delta_tags(const Topo& t, const Phys& p, const Pool& pool, int cur, double* delta_node,
                       int allow_refine, int8_t* tags, double* delta_leaf, int n_leaves_cap, cudaStream_t st) {
  if (p.precision == 1) launch_delta_f32(t, p, pool, cur, delta_node, allow_refine, st);
  else {
    k_delta_t<double><<<sm_count() * 4, 256, 0, st>>>(t, p, pool, cur, delta_node, allow_refine);
    ++g_kernel_launches;
  }
  k_tags<<<(n_leaves_cap + 255) / 256, 256, 0, st>>>(t, p, delta_node, allow_refine, tags, delta_leaf);
  ++g_kernel_launches;
}

// ---------------------------------------------------------------- Roe / LLF census
// counts[k] += faces (of every leaf, 17 x 16 x 16 per direction) where field k
// takes the LLF split; counts[5] += faces.  Per-thread counts, warp sums, one
// atomic per warp and counter.
__global__ void __launch_bounds__(256) k_flux_census(Topo t, Phys p, Pool pool, int cur,
                                                     unsigned long long* __restrict__ counts) {
  const long long nfaces = (long long)t.cnt[CNT_NLEAVES] * 3 * 17 * NFACE;
  unsigned c[6] = {0, 0, 0, 0, 0, 0};
  for (long long it = (long long)blockIdx.x * blockDim.x + threadIdx.x; it < nfaces;
       it += (long long)gridDim.x * blockDim.x) {
    const int li = (int)(it / (3 * 17 * NFACE));
    const int r = (int)(it % (3 * 17 * NFACE));
    const int d = r / (17 * NFACE), f = (r % (17 * NFACE)) / NFACE, ab = r % NFACE;
    const int a = ab % NB, b = ab / NB;
    int cl[3];
    cl[d] = f - 1;
    cl[(d == 0) ? 1 : 0] = a;
    cl[(d == 2) ? 1 : 2] = b;
    const int step[3] = {1, NS, NS * NS};
    const int sL = sidx(cl[0], cl[1], cl[2]), sR = sL + step[d];
    const double* U = pool.bufp(cur) + (size_t)t.slot[t.leaves[li]] * SLOT_U;
    double UL[5], UR[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      UL[v] = U[v * NCELL + sL];
      UR[v] = U[v * NCELL + sR];
    }
    const unsigned m = split_fields(UL, UR, d, p.gamma, p.B);
#pragma unroll
    for (int k = 0; k < 5; ++k) c[k] += (m >> k) & 1u;
    c[5] += 1;
  }
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    unsigned x = c[k];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0 && x) atomicAdd(&counts[k], (unsigned long long)x);
  }
}

void launch_flux_census(const Topo& t, const Phys& p, const Pool& pool, int cur, unsigned long long* counts,
                        cudaStream_t st) {
  cudaMemsetAsync(counts, 0, 6 * sizeof(unsigned long long), st);
  k_flux_census<<<sm_count() * 8, 256, 0, st>>>(t, p, pool, cur, counts);
  ++g_kernel_launches;
}

// ---------------------------------------------------------------- refinement (mr.cuh)
void launch_refine_fill(const Topo& t, const Phys& p, const Pool& pool, int cur, const int32_t* pairs, int n,
                        cudaStream_t st) {
  if (n <= 0) return;
  if (p.precision == 1) k_refine_fill_t<float><<<sm_count() * 8, 256, 0, st>>>(t, pool, cur, pairs, n);
  else k_refine_fill_t<double><<<sm_count() * 8, 256, 0, st>>>(t, pool, cur, pairs, n);
  ++g_kernel_launches;
}

// ---------------------------------------------------------------- neighbour table
// Same-level neighbour of every node in the 26 directions from block
// coordinates: outside a non-periodic boundary -> -2; otherwise the id of the
// (wrapped) neighbour position is looked up by binary search in the sorted ids
// (-1 when no node of that level exists there).
__device__ __forceinline__ uint64_t make_key_dev(int inst, int level, const int X[3]) {
  const int ng = 7 + level;
  uint64_t m = 0;
  for (int b = 0; b < ng; ++b)
    for (int d = 0; d < 3; ++d) m |= (uint64_t)((X[d] >> b) & 1) << (3 * b + d);
  return ((uint64_t)inst << 56) | (1ull << (3 * ng)) | m;
}

__global__ void k_nbr(Topo t, Phys p, int32_t* __restrict__ nbr_out) {
  const int nn = t.cnt[CNT_NNODES];
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nn * 27; e += gridDim.x * blockDim.x) {
    const int node = e / 27, r = e % 27;
    if (r == 13) {
      nbr_out[e] = node;
      continue;
    }
    const int s[3] = {r % 3 - 1, (r / 3) % 3 - 1, r / 9 - 1};
    const int lvl = t.level[node];
    int X[3];
    bool outside = false;
    for (int d = 0; d < 3; ++d) {
      const int nl = p.nb[d] << lvl;
      int x = t.X[(size_t)node * 3 + d] + s[d];
      if (x < 0 || x >= nl) {
        if (p.bc[2 * d] == 1) x = (x + nl) % nl;
        else outside = true;
      }
      X[d] = x;
    }
    if (outside) {
      nbr_out[e] = -2;
      continue;
    }
    const uint64_t key = make_key_dev(t.inst[node], lvl, X);
    int lo = 0, hi = nn - 1, found = -1;
    while (lo <= hi) {
      const int mid = (lo + hi) >> 1;
      const uint64_t km = t.keys[mid];
      if (km == key) { found = mid; break; }
      if (km < key) lo = mid + 1;
      else hi = mid - 1;
    }
    nbr_out[e] = found;
  }
}

__global__ void k_jump_list(Topo t, int32_t* __restrict__ jump, int32_t* __restrict__ cnt) {
  const int nleaves = t.cnt[CNT_NLEAVES];
  for (int li = blockIdx.x * blockDim.x + threadIdx.x; li < nleaves; li += gridDim.x * blockDim.x) {
    const int node = t.leaves[li];
    int mask = 0;
#pragma unroll
    for (int s = 0; s < 6; ++s) {
      const int d = s / 2, hi = s & 1;
      const int r = 13 + (hi ? 1 : -1) * (d == 0 ? 1 : (d == 1 ? 3 : 9));
      const int nb = t.nbr[(size_t)node * 27 + r];
      if (nb >= 0 && t.child0[nb] >= 0) mask |= 1 << s;
    }
    if (mask) jump[atomicAdd(&cnt[CNT_JUMP], 1)] = 64 * li + mask;
  }
}

void launch_jump_list(const Topo& t, int32_t* jump, int32_t* cnt, int n_leaves_cap, cudaStream_t st) {
  k_jump_list<<<(n_leaves_cap + 255) / 256 + 1, 256, 0, st>>>(t, jump, cnt);
  ++g_kernel_launches;
}

void launch_nbr(const Topo& t, const Phys& p, int32_t* nbr_out, int nnodes_cap, cudaStream_t st) {
  const int n = nnodes_cap * 27;
  k_nbr<<<(n + 255) / 256, 256, 0, st>>>(t, p, nbr_out);
  ++g_kernel_launches;
}

// ---------------------------------------------------------------- conservation sums
__global__ void __launch_bounds__(256) k_sums_partial(Topo t, Phys p, Pool pool, int cur, double* __restrict__ partial) {
  __shared__ double sh[5][8];
  const int nleaves = t.cnt[CNT_NLEAVES];
  for (int li = blockIdx.x; li < nleaves; li += gridDim.x) {
    const int node = t.leaves[li];
    const double* U = pool.bufp(cur) + (size_t)t.slot[node] * SLOT_U;
    double s[5] = {0, 0, 0, 0, 0};
    for (int e = threadIdx.x; e < NINT; e += blockDim.x) {
      const int c = sidx(e % 16, (e / 16) % 16, e / 256);
#pragma unroll
      for (int v = 0; v < 5; ++v) s[v] += U[v * NCELL + c];
    }
#pragma unroll
    for (int v = 0; v < 5; ++v)
      for (int o = 16; o > 0; o >>= 1) s[v] += __shfl_xor_sync(0xffffffffu, s[v], o);
    if ((threadIdx.x & 31) == 0)
      for (int v = 0; v < 5; ++v) sh[v][threadIdx.x >> 5] = s[v];
    __syncthreads();
    if (threadIdx.x < 5) {
      double x = 0.0;
      for (int q = 0; q < 8; ++q) x += sh[threadIdx.x][q];
      const double dx = ldexp(p.dx0, -t.level[node]);
      partial[(size_t)li * 5 + threadIdx.x] = x * (dx * dx * dx);
    }
    __syncthreads();
  }
}

__global__ void k_sums_finish(Topo t, Phys p, const double* __restrict__ partial, double* __restrict__ out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= p.n_inst * 5) return;
  const int inst = e / 5, v = e % 5;
  const int nleaves = t.cnt[CNT_NLEAVES];
  double acc = 0.0;
  for (int li = 0; li < nleaves; ++li)
    if (t.inst[t.leaves[li]] == inst) acc += partial[(size_t)li * 5 + v];
  out[e] = acc;
}

void launch_sums(const Topo& t, const Phys& p, const Pool& pool, int cur, double* partial, double* out,
                 int nleaves_cap, cudaStream_t st) {
  (void)nleaves_cap;
  k_sums_partial<<<sm_count() * 4, 256, 0, st>>>(t, p, pool, cur, partial);
  ++g_kernel_launches;
  k_sums_finish<<<(p.n_inst * 5 + 127) / 128, 128, 0, st>>>(t, p, partial, out);
  ++g_kernel_launches;
}

}  // namespace mrb
