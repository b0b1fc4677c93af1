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

// Details of the mixed-precision path with rho and E in packed FP32 pairs:
// the parent box staged once as (rho, E) pairs, the Q-terms of Eq.
// Prediction and the eight predictions of each parent cell computed two
// variables per instruction.  delta = max over both variables of
// |u - P(u_parent)| / |u|, as k_delta_t.
struct SAcc2 {
  const float2* s;
  int i0, j0, k0;
  __device__ __forceinline__ float2 operator()(int i, int j, int k) const {
    return s[(k - k0) * 256 + (j - j0) * 16 + (i - i0)];
  }
};

__device__ __forceinline__ float2 mix2p(const SAcc2& P, int i, int j, int k, int Ax, int Bx, int p, int q) {
  const int a1 = Ax == 0 ? p : 0, b1 = Ax == 1 ? p : 0, c1 = Ax == 2 ? p : 0;
  const int a2 = Bx == 0 ? q : 0, b2 = Bx == 1 ? q : 0, c2 = Bx == 2 ? q : 0;
  return f2sub(f2add(P(i + a1 + a2, j + b1 + b2, k + c1 + c2), P(i - a1 - a2, j - b1 - b2, k - c1 - c2)),
               f2add(P(i - a1 + a2, j - b1 + b2, k - c1 + c2), P(i + a1 - a2, j + b1 - b2, k + c1 - c2)));
}

__device__ __forceinline__ float2 mix3p(const SAcc2& P, int i, int j, int k, int p, int q, int r) {
  const int sg[4][3] = {{1, 1, 1}, {1, -1, -1}, {-1, -1, 1}, {-1, 1, -1}};
  float2 acc = make_float2(0.f, 0.f);
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const float2 term = f2sub(P(i + sg[t][0] * p, j + sg[t][1] * q, k + sg[t][2] * r),
                              P(i - sg[t][0] * p, j - sg[t][1] * q, k - sg[t][2] * r));
    acc = (t == 0) ? term : f2add(acc, term);
  }
  return acc;
}

__global__ void __launch_bounds__(256) k_delta_p(Topo t, Phys p, Pool pool, int cur, double* __restrict__ delta_node,
                                                 int all_nodes) {
  __shared__ double sh[8];
  __shared__ float2 box[4096];      // (rho, E) of the parent's cells 8 cb - 4 .. 8 cb + 11 per axis
  const int nitems = all_nodes ? t.cnt[CNT_NNODES] : t.cnt[CNT_NLEAVES];
  const double* B = pool.bufp(cur);
  const float C0 = -22.f / 128.f, C1 = 3.f / 128.f;
  for (int li = blockIdx.x; li < nitems; li += gridDim.x) {
    const int node = all_nodes ? li : t.leaves[li];
    const int lvl = t.level[node];
    if (lvl == 0) {
      if (threadIdx.x == 0) delta_node[node] = 0.0;
      continue;
    }
    const int par = t.parent[node];
    const double* U = B + (size_t)t.slot[node] * SLOT_U;
    const double* P = B + (size_t)t.slot[par] * SLOT_U;
    const int ch = (int)(t.keys[node] & 7ull);
    const int cb0 = ch & 1, cb1 = (ch >> 1) & 1, cb2 = (ch >> 2) & 1;
    bool gl[3], gh[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int nl = p.nb[d] << lvl;
      const int Xd = t.X[(size_t)node * 3 + d];
      gl[d] = (Xd == 0) && (p.bc[2 * d] != 1);
      gh[d] = (Xd == nl - 1) && (p.bc[2 * d + 1] != 1);
    }
    const int bx0 = 8 * cb0 - 4, by0 = 8 * cb1 - 4, bz0 = 8 * cb2 - 4;
    for (int e = threadIdx.x; e < 4096; e += blockDim.x) {
      const int s = sidx(bx0 + e % 16, by0 + (e / 16) % 16, bz0 + e / 256);
      box[e] = make_float2(d2f_fast(P[s]), d2f_fast(P[4 * NCELL + s]));
    }
    __syncthreads();
    const SAcc2 A{box, bx0, by0, bz0};
    float m = 0.f;
    for (int q = threadIdx.x; q < 1728; q += blockDim.x) {
      const int rx = q % 12 - 2, ry = (q / 12) % 12 - 2, rz = q / 144 - 2;
      const bool ghost = (rx < 0 && gl[0]) || (rx >= 8 && gh[0]) || (ry < 0 && gl[1]) || (ry >= 8 && gh[1]) ||
                         (rz < 0 && gl[2]) || (rz >= 8 && gh[2]);
      if (ghost) continue;
      const int i = 8 * cb0 + rx, j = 8 * cb1 + ry, k = 8 * cb2 + rz;
      const float2 u = A(i, j, k);
      const float2 Qx = f2fma(f2s(C0), f2sub(A(i + 1, j, k), A(i - 1, j, k)), f2mul(f2s(C1), f2sub(A(i + 2, j, k), A(i - 2, j, k))));
      const float2 Qy = f2fma(f2s(C0), f2sub(A(i, j + 1, k), A(i, j - 1, k)), f2mul(f2s(C1), f2sub(A(i, j + 2, k), A(i, j - 2, k))));
      const float2 Qz = f2fma(f2s(C0), f2sub(A(i, j, k + 1), A(i, j, k - 1)), f2mul(f2s(C1), f2sub(A(i, j, k + 2), A(i, j, k - 2))));
      const int pq[4][2] = {{1, 1}, {2, 2}, {1, 2}, {2, 1}};
      float2 Qxy = make_float2(0.f, 0.f), Qxz = Qxy, Qyz = Qxy;
#pragma unroll
      for (int t2 = 0; t2 < 4; ++t2) {
        const int pp = pq[t2][0], qq = pq[t2][1];
        const float cc = (pp == 1 ? C0 : C1) * (qq == 1 ? C0 : C1);
        const float2 a = f2mul(f2s(cc), mix2p(A, i, j, k, 0, 1, pp, qq));
        const float2 b = f2mul(f2s(cc), mix2p(A, i, j, k, 0, 2, pp, qq));
        const float2 c = f2mul(f2s(cc), mix2p(A, i, j, k, 1, 2, pp, qq));
        Qxy = (t2 == 0) ? a : f2add(Qxy, a);
        Qxz = (t2 == 0) ? b : f2add(Qxz, b);
        Qyz = (t2 == 0) ? c : f2add(Qyz, c);
      }
      const int pqr[8][3] = {{1, 1, 1}, {2, 2, 2}, {1, 1, 2}, {2, 2, 1}, {1, 2, 2}, {2, 1, 1}, {1, 2, 1}, {2, 1, 2}};
      float2 Qxyz = make_float2(0.f, 0.f);
#pragma unroll
      for (int t3 = 0; t3 < 8; ++t3) {
        const int pp = pqr[t3][0], qq = pqr[t3][1], rr = pqr[t3][2];
        const float cc = (pp == 1 ? C0 : C1) * (qq == 1 ? C0 : C1) * (rr == 1 ? C0 : C1);
        const float2 a = f2mul(f2s(cc), mix3p(A, i, j, k, pp, qq, rr));
        Qxyz = (t3 == 0) ? a : f2add(Qxyz, a);
      }
#pragma unroll
      for (int sub = 0; sub < 8; ++sub) {
        const int a = sub & 1, b = (sub >> 1) & 1, c = (sub >> 2) & 1;
        // the lower child takes +Q: signs of the seven terms of the prediction
        float2 pr = a ? f2sub(u, Qx) : f2add(u, Qx);
        pr = b ? f2sub(pr, Qy) : f2add(pr, Qy);
        pr = c ? f2sub(pr, Qz) : f2add(pr, Qz);
        pr = (a ^ b) ? f2sub(pr, Qxy) : f2add(pr, Qxy);
        pr = (a ^ c) ? f2sub(pr, Qxz) : f2add(pr, Qxz);
        pr = (b ^ c) ? f2sub(pr, Qyz) : f2add(pr, Qyz);
        pr = (a ^ b ^ c) ? f2sub(pr, Qxyz) : f2add(pr, Qxyz);
        const int s = sidx(2 * rx + a, 2 * ry + b, 2 * rz + c);
        const float2 uf = make_float2(d2f_fast(U[s]), d2f_fast(U[4 * NCELL + s]));
        const float2 dd = f2sub(uf, pr);
        const float r0 = fabsf(dd.x / uf.x), r1 = fabsf(dd.y / uf.y);
        m = fmaxf(m, fmaxf(r0, r1));
      }
    }
    double md = f2d_fast(m);
    for (int o = 16; o > 0; o >>= 1) md = fmax(md, __shfl_xor_sync(0xffffffffu, md, o));
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = md;
    __syncthreads();
    if (threadIdx.x == 0) {
      double x = sh[0];
      for (int q = 1; q < (int)(blockDim.x >> 5); ++q) x = fmax(x, sh[q]);
      delta_node[node] = x;
    }
    __syncthreads();
  }
}

void launch_delta_f32(const Topo& t, const Phys& p, const Pool& pool, int cur, double* delta_node, int all_nodes,
                      cudaStream_t st) {
  k_delta_p<<<sm_count() * 4, 256, 0, st>>>(t, p, pool, cur, delta_node, all_nodes);
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
