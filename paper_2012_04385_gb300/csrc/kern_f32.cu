// Mixed-precision stage kernel (MRB_FP32_ACC64): reconstruction, fluxes and
// flux differences in FP32 from the FP64 state; the TVD-RK3 update of the FP64
// state in FP64.  Built with FMA contraction and the fast FP32 reciprocal and
// square-root approximations.
#include "mr.cuh"
#include "stage_f32.cuh"

namespace mrb {

void launch_rhs_rk_f32(const Topo& t, const Phys& p, const Pool& pool, int cur, int stage, const double* dt,
                       double* rhs_out, cudaStream_t st, int level) {
  if (p.mu > 0.0) launch_stage_f32<32>(t, p, pool, cur, stage, dt, rhs_out, st, level);   // WENO5, Roe, viscous
  else if (p.flux == 1) launch_rhs_rk_f32_llf(t, p, pool, cur, stage, dt, rhs_out, st, level);
  else if (p.flux == 2) launch_rhs_rk_f32_hllc(t, p, pool, cur, stage, dt, rhs_out, st, level);
  else if (p.recon == 2) launch_stage_f32<2>(t, p, pool, cur, stage, dt, rhs_out, st, level);
  else if (p.recon == 3) launch_stage_f32<4>(t, p, pool, cur, stage, dt, rhs_out, st, level);
  else if (p.recon == 4) launch_stage_f32<5>(t, p, pool, cur, stage, dt, rhs_out, st, level);
  else if (p.recon == 1 && p.mlp) {
    // the selector is evaluated on the stage-0 state; stages 1 and 2 use its decisions
    if (stage == 0 || rhs_out) launch_stage_f32<1>(t, p, pool, cur, stage, dt, rhs_out, st, level);
    else launch_stage_f32<3>(t, p, pool, cur, stage, dt, rhs_out, st, level);
  } else launch_stage_f32<0>(t, p, pool, cur, stage, dt, rhs_out, st, level);
}

void launch_fill_level_f32(const Topo& t, const Phys& p, const Pool& pool, int cur, int level, cudaStream_t st,
                           int mode) {
  const NodeSet ns{level, nullptr, 0};
  k_fill_regions_t<float><<<sm_count() * g_tune.fill_copy, 256, 0, st>>>(t, pool, cur, ns, mode);
  k_fill_predict_t<float><<<sm_count() * g_tune.fill_pred, 256, 0, st>>>(t, pool, cur, ns, mode);
  k_fill_bc<<<sm_count() * 4, 256, 0, st>>>(t, p, pool, cur, ns, mode);
  g_kernel_launches += 3;
}

void launch_fill_list_f32(const Topo& t, const Phys& p, const Pool& pool, int cur, const int32_t* list, int n,
                          cudaStream_t st) {
  const NodeSet ns{0, list, n};
  k_fill_regions_t<float><<<sm_count() * 8, 256, 0, st>>>(t, pool, cur, ns, FILL_FULL);
  k_fill_predict_t<float><<<sm_count() * 4, 256, 0, st>>>(t, pool, cur, ns, FILL_FULL);
  k_fill_bc<<<sm_count() * 4, 256, 0, st>>>(t, p, pool, cur, ns, FILL_FULL);
  g_kernel_launches += 3;
}

// FP32 records of stage buffer b: one CTA per item, the records of the item's
// internal cells recomputed from the FP64 values (make_record, the same
// arithmetic as the stage kernel's own conversion).
__global__ void __launch_bounds__(256) k_shadow(Topo t, Phys p, Pool pool, int b, int mode,
                                                const int32_t* __restrict__ list, int n, int stride) {
  const float g = (float)p.gamma, B = (float)p.B, gm1 = (float)(p.gamma - 1.0);
  const int nitems = (mode == SH_INTERNAL) ? t.cnt[CNT_NNODES] : (mode == SH_JUMP ? t.cnt[CNT_JUMP] : n);
  for (int w = blockIdx.x; w < nitems; w += gridDim.x) {
    int node, mask = 0;
    if (mode == SH_INTERNAL) {
      node = w;
      if (t.child0[node] < 0) continue;           // leaves keep the stage kernel's records
    } else if (mode == SH_JUMP) {
      node = t.leaves[t.jump[w] >> 6];
      mask = t.jump[w] & 63;
    } else {
      node = list[(size_t)w * stride];
    }
    const double* U = pool.bufp(b) + (size_t)t.slot[node] * SLOT_U;
    float* R = pool.shp(b) + (size_t)t.slot[node] * SLOT_SH;
    if (mode == SH_JUMP) {
      // the plane of cells next to each side whose neighbour is refined
      for (int sd = 0; sd < 6; ++sd) {
        if (!((mask >> sd) & 1)) continue;
        const int d = sd / 2, hi = sd & 1;
        const int t1 = (d == 0) ? 1 : 0, t2 = (d == 2) ? 1 : 2;
        for (int e = threadIdx.x; e < NFACE; e += blockDim.x) {
          int c[3];
          c[d] = hi ? NB - 1 : 0;
          c[t1] = e % 16;
          c[t2] = e / 16;
          const int s = sidx(c[0], c[1], c[2]), ii = iidx(c[0], c[1], c[2]);
          float rec[6];
          make_record(U[s], U[NCELL + s], U[2 * NCELL + s], U[3 * NCELL + s], U[4 * NCELL + s], g, B, gm1, rec);
#pragma unroll
          for (int f = 0; f < 6; ++f) R[f * NINT + ii] = rec[f];
        }
      }
    } else {
      for (int e = threadIdx.x; e < NINT; e += blockDim.x) {
        const int s = sidx(e % 16, (e / 16) % 16, e / 256);
        float rec[6];
        make_record(U[s], U[NCELL + s], U[2 * NCELL + s], U[3 * NCELL + s], U[4 * NCELL + s], g, B, gm1, rec);
#pragma unroll
        for (int f = 0; f < 6; ++f) R[f * NINT + e] = rec[f];
      }
    }
  }
}

void launch_shadow(const Topo& t, const Phys& p, const Pool& pool, int b, int mode, const int32_t* list, int n,
                   int stride, cudaStream_t st) {
  if (!pool.shp(0)) return;
  k_shadow<<<sm_count() * 4, 256, 0, st>>>(t, p, pool, b, mode, list, n, stride);
  ++g_kernel_launches;
}

// Records of the listed nodes' internal cells (kept, or converted afresh).
__global__ void __launch_bounds__(256) k_get_records(Topo t, Phys p, Pool pool, int cur,
                                                     const int32_t* __restrict__ nodes, int n, float* __restrict__ out,
                                                     int fresh) {
  const float g = (float)p.gamma, B = (float)p.B, gm1 = (float)(p.gamma - 1.0);
  for (int b = blockIdx.x; b < n; b += gridDim.x) {
    const int slot = t.slot[nodes[b]];
    const double* U = pool.bufp(cur) + (size_t)slot * SLOT_U;
    const float* R = pool.shp(cur) + (size_t)slot * SLOT_SH;
    float* o = out + (size_t)b * SLOT_SH;
    for (int e = threadIdx.x; e < NINT; e += blockDim.x) {
      if (fresh) {
        const int s = sidx(e % 16, (e / 16) % 16, e / 256);
        float rec[6];
        make_record(U[s], U[NCELL + s], U[2 * NCELL + s], U[3 * NCELL + s], U[4 * NCELL + s], g, B, gm1, rec);
#pragma unroll
        for (int f = 0; f < 6; ++f) o[f * NINT + e] = rec[f];
      } else {
#pragma unroll
        for (int f = 0; f < 6; ++f) o[f * NINT + e] = R[f * NINT + e];
      }
    }
  }
}

void launch_get_records(const Topo& t, const Phys& p, const Pool& pool, int cur, const int32_t* nodes, int n,
                        float* out, int fresh, cudaStream_t st) {
  if (n <= 0) return;
  k_get_records<<<sm_count() * 4, 256, 0, st>>>(t, p, pool, cur, nodes, n, out, fresh);
  ++g_kernel_launches;
}

void launch_delta_f32(const Topo& t, const Phys& p, const Pool& pool, int cur, double* delta_node, int all_nodes,
                      cudaStream_t st) {
  k_delta_t<float><<<sm_count() * 4, 256, 0, st>>>(t, p, pool, cur, delta_node, all_nodes);
  ++g_kernel_launches;
}

// Per-instance maxima of |u_d| + c (and of 1/rho, for the viscous limit) over
// the leaves' internal cells: speeds in FP32, maxima (exact) and the time step
// of Eq. (Cfl) in FP64.
__global__ void __launch_bounds__(256) k_cfl_f32(Topo t, Phys p, Pool pool, int cur,
                                                 unsigned long long* __restrict__ smax, int* __restrict__ status) {
  __shared__ float sh[4][8];
  const int nleaves = t.cnt[CNT_NLEAVES];
  const float g = (float)p.gamma, B = (float)p.B, gm1 = (float)(p.gamma - 1.0);
  for (int li = blockIdx.x; li < nleaves; li += gridDim.x) {
    const int node = t.leaves[li];
    const double* U = pool.bufp(cur) + (size_t)t.slot[node] * SLOT_U;
    float m0 = 0.f, m1 = 0.f, m2 = 0.f, m3 = 0.f;   // max |u_d| + c, max 1/rho
    bool bad = false;
    for (int e = threadIdx.x; e < NINT; e += blockDim.x) {
      const int s = sidx(e % 16, (e / 16) % 16, e / 256);
      const float r = d2f_fast(U[s]), ir = frcp(r);
      const float vx = d2f_fast(U[NCELL + s]) * ir, vy = d2f_fast(U[2 * NCELL + s]) * ir;
      const float vz = d2f_fast(U[3 * NCELL + s]) * ir;
      const float q2 = fmaf(vx, vx, fmaf(vy, vy, vz * vz));
      const float pr = fmaf(gm1, fmaf(-0.5f * r, q2, d2f_fast(U[4 * NCELL + s])), -g * B);
      if (!(r > 0.f) || !(pr + B > 0.f)) bad = true;
      const float c = sqrtf(g * (pr + B) * ir);
      m0 = fmaxf(m0, fabsf(vx) + c);
      m1 = fmaxf(m1, fabsf(vy) + c);
      m2 = fmaxf(m2, fabsf(vz) + c);
      m3 = fmaxf(m3, ir);
    }
    if (bad) atomicExch(status, (int)ST_NONPHYS);
    for (int o = 16; o > 0; o >>= 1) {
      m0 = fmaxf(m0, __shfl_xor_sync(0xffffffffu, m0, o));
      m1 = fmaxf(m1, __shfl_xor_sync(0xffffffffu, m1, o));
      m2 = fmaxf(m2, __shfl_xor_sync(0xffffffffu, m2, o));
      m3 = fmaxf(m3, __shfl_xor_sync(0xffffffffu, m3, o));
    }
    if ((threadIdx.x & 31) == 0) {
      sh[0][threadIdx.x >> 5] = m0;
      sh[1][threadIdx.x >> 5] = m1;
      sh[2][threadIdx.x >> 5] = m2;
      sh[3][threadIdx.x >> 5] = m3;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
      float x = sh[threadIdx.x][0];
      for (int q = 1; q < 8; ++q) x = fmaxf(x, sh[threadIdx.x][q]);
      atomicMax(&smax[t.inst[node] * 4 + threadIdx.x], (unsigned long long)__double_as_longlong(f2d_fast(x)));
    }
    __syncthreads();
  }
}

void launch_cfl_speeds_f32(const Topo& t, const Phys& p, const Pool& pool, int cur, unsigned long long* smax,
                           int* status, cudaStream_t st) {
  k_cfl_f32<<<sm_count() * 4, 256, 0, st>>>(t, p, pool, cur, smax, status);
  ++g_kernel_launches;
}

}  // namespace mrb
