// Multiresolution kernels templated on the arithmetic type R: halo fill
// (copy / prediction / boundary condition) and the MR details of the leaves.
// R = double reproduces the FP64 operation order exactly (built with
// -fmad=false); R = float serves the mixed-precision path, where halo values
// are stencil inputs and the details a refinement heuristic.
//
// Prediction (Eq. Prediction with the appendix Q-terms) is evaluated once per
// parent cell: the eight fine cells of a parent cell share its Q-terms and
// differ only in the signs (+ for the lower half along an axis, - for the
// upper).  A halo of four fine cells is two parent cells deep, so the eight
// fine cells of a parent cell always lie in the same halo region.
#pragma once

#include "convert.cuh"
#include "kernels.cuh"

namespace mrb {

template <class R> struct QT {
  R u, Qx, Qy, Qz, Qxy, Qxz, Qyz, Qxyz;
};

template <class R> __device__ __forceinline__ R to_r(double x) { return R(x); }
template <> __device__ __forceinline__ float to_r<float>(double x) { return d2f_fast(x); }
template <class R> __device__ __forceinline__ double from_r(R x) { return double(x); }
template <> __device__ __forceinline__ double from_r<float>(float x) { return f2d_fast(x); }

template <class R> __device__ __forceinline__ R pld(const double* P, int i, int j, int k) {
  return to_r<R>(P[sidx(i, j, k)]);
}

template <class R> __device__ __forceinline__ R qc(int off) { return off == 1 ? R(-22.0 / 128.0) : R(3.0 / 128.0); }

template <class R>
__device__ __forceinline__ R mix2t(const double* P, int i, int j, int k, int A, int Bx, int p, int q) {
  int o1[3] = {0, 0, 0}, o2[3] = {0, 0, 0}, o3[3] = {0, 0, 0}, o4[3] = {0, 0, 0};
  o1[A] = p; o1[Bx] = q;
  o2[A] = -p; o2[Bx] = -q;
  o3[A] = -p; o3[Bx] = q;
  o4[A] = p; o4[Bx] = -q;
  return (pld<R>(P, i + o1[0], j + o1[1], k + o1[2]) + pld<R>(P, i + o2[0], j + o2[1], k + o2[2])) -
         (pld<R>(P, i + o3[0], j + o3[1], k + o3[2]) + pld<R>(P, i + o4[0], j + o4[1], k + o4[2]));
}

template <class R> __device__ __forceinline__ R mix3t(const double* P, int i, int j, int k, int p, int q, int r) {
  const int sg[4][3] = {{1, 1, 1}, {1, -1, -1}, {-1, -1, 1}, {-1, 1, -1}};
  R acc = R(0);
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    R term = pld<R>(P, i + sg[t][0] * p, j + sg[t][1] * q, k + sg[t][2] * r) -
             pld<R>(P, i - sg[t][0] * p, j - sg[t][1] * q, k - sg[t][2] * r);
    acc = (t == 0) ? term : acc + term;
  }
  return acc;
}

template <class R> __device__ __forceinline__ QT<R> qterms_t(const double* P, int i, int j, int k) {
  const R C0 = R(-22.0 / 128.0), C1 = R(3.0 / 128.0);
  QT<R> t;
  t.u = pld<R>(P, i, j, k);
  t.Qx = C0 * (pld<R>(P, i + 1, j, k) - pld<R>(P, i - 1, j, k)) + C1 * (pld<R>(P, i + 2, j, k) - pld<R>(P, i - 2, j, k));
  t.Qy = C0 * (pld<R>(P, i, j + 1, k) - pld<R>(P, i, j - 1, k)) + C1 * (pld<R>(P, i, j + 2, k) - pld<R>(P, i, j - 2, k));
  t.Qz = C0 * (pld<R>(P, i, j, k + 1) - pld<R>(P, i, j, k - 1)) + C1 * (pld<R>(P, i, j, k + 2) - pld<R>(P, i, j, k - 2));
  const int pq[4][2] = {{1, 1}, {2, 2}, {1, 2}, {2, 1}};
  R qxy = R(0), qxz = R(0), qyz = R(0);
#pragma unroll
  for (int t2 = 0; t2 < 4; ++t2) {
    const int p = pq[t2][0], q = pq[t2][1];
    const R cc = qc<R>(p) * qc<R>(q);
    const R a = cc * mix2t<R>(P, i, j, k, 0, 1, p, q);
    const R b = cc * mix2t<R>(P, i, j, k, 0, 2, p, q);
    const R c = cc * mix2t<R>(P, i, j, k, 1, 2, p, q);
    qxy = (t2 == 0) ? a : qxy + a;
    qxz = (t2 == 0) ? b : qxz + b;
    qyz = (t2 == 0) ? c : qyz + c;
  }
  t.Qxy = qxy;
  t.Qxz = qxz;
  t.Qyz = qyz;
  const int pqr[8][3] = {{1, 1, 1}, {2, 2, 2}, {1, 1, 2}, {2, 2, 1}, {1, 2, 2}, {2, 1, 1}, {1, 2, 1}, {2, 1, 2}};
  R qxyz = R(0);
#pragma unroll
  for (int t3 = 0; t3 < 8; ++t3) {
    const int p = pqr[t3][0], q = pqr[t3][1], r = pqr[t3][2];
    const R cc = qc<R>(p) * qc<R>(q) * qc<R>(r);
    const R a = cc * mix3t<R>(P, i, j, k, p, q, r);
    qxyz = (t3 == 0) ? a : qxyz + a;
  }
  t.Qxyz = qxyz;
  return t;
}

template <class R> __device__ __forceinline__ R predict_t(const QT<R>& t, R sx, R sy, R sz) {
  return t.u + sx * t.Qx + sy * t.Qy + sz * t.Qz + (sx * sy) * t.Qxy + (sx * sz) * t.Qxz + (sy * sz) * t.Qyz +
         (sx * sy * sz) * t.Qxyz;
}

__device__ __forceinline__ int sgn_region(int rel) { return rel < 0 ? -1 : (rel >= 8 ? 1 : 0); }

// ---------------------------------------------------------------- halo fill
// One CTA per node of `level`: copy regions from same-level neighbours,
// predicted regions from the parent (per parent cell), then the boundary
// passes x-, x+, y-, y+, z-, z+ on the node's own cells.
template <class R>
__global__ void __launch_bounds__(256) k_fill_level_t(Topo t, Phys p, Pool pool, int cur, int level) {
  const int beg = t.cnt[CNT_LVL + level], end = t.cnt[CNT_LVL + level + 1];
  double* buf = pool.buf[cur];
  __shared__ int kind[27];
  __shared__ int src_slot[27];
  __shared__ int any_pred;
  for (int w = beg + blockIdx.x; w < end; w += gridDim.x) {
    const int node = t.lvl_nodes[w];
    double* u = buf + (size_t)t.slot[node] * SLOT_U;
    const int par = t.parent[node];
    const double* P = (par >= 0) ? buf + (size_t)t.slot[par] * SLOT_U : nullptr;
    const int ch = (int)(t.keys[node] & 7ull);
    __syncthreads();
    if (threadIdx.x == 0) any_pred = 0;
    __syncthreads();
    if (threadIdx.x < 27) {
      const int nb = t.nbr[(size_t)node * 27 + threadIdx.x];
      const int kd = (threadIdx.x == 13) ? 0 : ((nb >= 0) ? 1 : ((nb == -1 && P != nullptr) ? 2 : 0));
      kind[threadIdx.x] = kd;
      src_slot[threadIdx.x] = (nb >= 0) ? t.slot[nb] : -1;
      if (kd == 2) atomicOr(&any_pred, 1);
    }
    __syncthreads();
    // copies
    for (int idx = threadIdx.x; idx < NCELL; idx += blockDim.x) {
      const int i = idx % NS - HW, j = (idx / NS) % NS - HW, k = idx / (NS * NS) - HW;
      const int sx = i < 0 ? -1 : (i >= NB ? 1 : 0), sy = j < 0 ? -1 : (j >= NB ? 1 : 0),
                sz = k < 0 ? -1 : (k >= NB ? 1 : 0);
      const int r = (sz + 1) * 9 + (sy + 1) * 3 + (sx + 1);
      if (kind[r] != 1) continue;
      const double* s = buf + (size_t)src_slot[r] * SLOT_U;
      const int off = idx - NB * (sx + NS * sy + NS * NS * sz);
#pragma unroll
      for (int v = 0; v < NV; ++v) u[v * NCELL + idx] = s[v * NCELL + off];
    }
    // predictions, one parent cell (eight fine cells) per step
    if (any_pred) {
      const int cb[3] = {ch & 1, (ch >> 1) & 1, (ch >> 2) & 1};
      for (int e = threadIdx.x; e < 12 * 12 * 12 * NV; e += blockDim.x) {
        const int v = e / 1728, q = e % 1728;
        const int rx = q % 12 - 2, ry = (q / 12) % 12 - 2, rz = q / 144 - 2;   // parent cell relative to the child
        const int r = (sgn_region(rz) + 1) * 9 + (sgn_region(ry) + 1) * 3 + (sgn_region(rx) + 1);
        if (kind[r] != 2) continue;
        const QT<R> qt = qterms_t<R>(P + v * NCELL, 8 * cb[0] + rx, 8 * cb[1] + ry, 8 * cb[2] + rz);
#pragma unroll
        for (int sub = 0; sub < 8; ++sub) {
          const int a = sub & 1, b = (sub >> 1) & 1, c = (sub >> 2) & 1;
          const R val = predict_t<R>(qt, a ? R(-1) : R(1), b ? R(-1) : R(1), c ? R(-1) : R(1));
          u[v * NCELL + sidx(2 * rx + a, 2 * ry + b, 2 * rz + c)] = from_r<R>(val);
        }
      }
    }
    __syncthreads();
#pragma unroll 1
    for (int d = 0; d < 3; ++d) {
#pragma unroll 1
      for (int side = 0; side < 2; ++side) {
        const int bc = p.bc[2 * d + side];
        if (bc == 1) continue;
        const int nl = p.nb[d] << level;
        const int Xd = t.X[(size_t)node * 3 + d];
        if (side == 0 && Xd != 0) continue;
        if (side == 1 && Xd != nl - 1) continue;
        // ghost slab: 4 cells deep along d, the full stored extent across
        for (int e = threadIdx.x; e < HW * NS * NS; e += blockDim.x) {
          const int g0 = e % HW, a1 = (e / HW) % NS - HW, a2 = e / (HW * NS) - HW;
          const int a = (side == 0) ? (-1 - g0) : (NB + g0);
          int c[3], sc[3];
          c[d] = a;
          c[(d + 1) % 3] = a1;
          c[(d + 2) % 3] = a2;
          sc[0] = c[0];
          sc[1] = c[1];
          sc[2] = c[2];
          if (bc == 0) sc[d] = (side == 0) ? 0 : NB - 1;
          else sc[d] = (side == 0) ? (-1 - a) : (2 * NB - 1 - a);
          const int di = sidx(c[0], c[1], c[2]), si = sidx(sc[0], sc[1], sc[2]);
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            double val = u[v * NCELL + si];
            if (bc == 2 && v == 1 + d) val = -val;
            u[v * NCELL + di] = val;
          }
        }
        __syncthreads();
      }
    }
  }
}

// ---------------------------------------------------------------- details
// delta of a leaf at level >= 1: max over its stored cells that are not ghost
// cells and over rho, E of |u - P(u_parent)| / |u|.
template <class R>
__global__ void __launch_bounds__(256) k_delta_t(Topo t, Phys p, Pool pool, int cur, double* __restrict__ delta_node) {
  __shared__ double sh[8];
  const int nleaves = t.cnt[CNT_NLEAVES];
  const double* B = pool.buf[cur];
  for (int li = blockIdx.x; li < nleaves; li += gridDim.x) {
    const int node = t.leaves[li];
    const int lvl = t.level[node];
    if (lvl == 0) {
      if (threadIdx.x == 0) delta_node[node] = 0.0;
      continue;
    }
    const int par = t.parent[node];
    const double* U = B + (size_t)t.slot[node] * SLOT_U;
    const double* P = B + (size_t)t.slot[par] * SLOT_U;
    const int ch = (int)(t.keys[node] & 7ull);
    const int cb[3] = {ch & 1, (ch >> 1) & 1, (ch >> 2) & 1};
    bool gl[3], gh[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int nl = p.nb[d] << lvl;
      const int Xd = t.X[(size_t)node * 3 + d];
      gl[d] = (Xd == 0) && (p.bc[2 * d] != 1);
      gh[d] = (Xd == nl - 1) && (p.bc[2 * d + 1] != 1);
    }
    R m = R(0);
    for (int e = threadIdx.x; e < 2 * 1728; e += blockDim.x) {
      const int vi = e / 1728, q = e % 1728;
      const int v = vi == 0 ? 0 : 4;
      const int rx = q % 12 - 2, ry = (q / 12) % 12 - 2, rz = q / 144 - 2;
      // all eight fine cells of this parent cell share the ghost status
      const bool ghost = (rx < 0 && gl[0]) || (rx >= 8 && gh[0]) || (ry < 0 && gl[1]) || (ry >= 8 && gh[1]) ||
                         (rz < 0 && gl[2]) || (rz >= 8 && gh[2]);
      if (ghost) continue;
      const QT<R> qt = qterms_t<R>(P + v * NCELL, 8 * cb[0] + rx, 8 * cb[1] + ry, 8 * cb[2] + rz);
#pragma unroll
      for (int sub = 0; sub < 8; ++sub) {
        const int a = sub & 1, b = (sub >> 1) & 1, c = (sub >> 2) & 1;
        const R pr = predict_t<R>(qt, a ? R(-1) : R(1), b ? R(-1) : R(1), c ? R(-1) : R(1));
        const R uf = to_r<R>(U[v * NCELL + sidx(2 * rx + a, 2 * ry + b, 2 * rz + c)]);
        const R r = (uf - pr) / uf;
        m = (r < R(0) ? -r : r) > m ? (r < R(0) ? -r : r) : m;
      }
    }
    double md = from_r<R>(m);
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

}  // namespace mrb
