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

// ---------------------------------------------------------------- halo fill by region
// Sec. 3 (Fig. MrCommunicationMesh): a halo region facing a same-level node
// is a copy of its internal cells, one facing no same-level node is predicted
// from the node's parent (one parent cell, eight fine cells, per step).  One
// work item per (node, halo region) on a persistent grid; k_fill_bc then
// applies the boundary conditions.  With leaf_faces_only, leaves get only
// their predicted face regions (the mixed-precision stage kernel reads face
// neighbours' cells directly); internal nodes, whose halos feed their
// children's predictions, are filled completely.
__device__ __forceinline__ int region_extent(int s) { return s == 0 ? NB : HW; }
__device__ __forceinline__ int region_start(int s) { return s < 0 ? -HW : (s == 0 ? 0 : NB); }

template <class R>
__global__ void __launch_bounds__(256) k_fill_regions_t(Topo t, Pool pool, int cur, int level, int leaf_faces_only) {
  const int beg = t.cnt[CNT_LVL + level], end = t.cnt[CNT_LVL + level + 1];
  double* buf = pool.buf[cur];
  const int nitems = (end - beg) * 26;
  for (int w = blockIdx.x; w < nitems; w += gridDim.x) {
    const int node = t.lvl_nodes[beg + w / 26];
    const int r = w % 26 < 13 ? w % 26 : w % 26 + 1;      // skip the centre
    const int sx = r % 3 - 1, sy = (r / 3) % 3 - 1, sz = r / 9 - 1;
    const bool face = (sx != 0) + (sy != 0) + (sz != 0) == 1;
    const bool partial = leaf_faces_only && t.child0[node] < 0;
    if (partial && !face) continue;
    const int nb = t.nbr[(size_t)node * 27 + r];
    const int par = t.parent[node];
    double* u = buf + (size_t)t.slot[node] * SLOT_U;
    if (nb >= 0) {
      if (partial) continue;                              // read directly by the stage kernel
      const double* src = buf + (size_t)t.slot[nb] * SLOT_U;
      const int ex = region_extent(sx), ey = region_extent(sy), ez = region_extent(sz);
      const int x0 = region_start(sx), y0 = region_start(sy), z0 = region_start(sz);
      const int n = ex * ey * ez;
      for (int e = threadIdx.x; e < n * NV; e += blockDim.x) {
        const int v = e / n, c = e % n;
        const int i = x0 + c % ex, j = y0 + (c / ex) % ey, k = z0 + c / (ex * ey);
        u[v * NCELL + sidx(i, j, k)] = src[v * NCELL + sidx(i - NB * sx, j - NB * sy, k - NB * sz)];
      }
    } else if (nb == -1 && par >= 0) {
      const double* P = buf + (size_t)t.slot[par] * SLOT_U;
      const int ch = (int)(t.keys[node] & 7ull);
      const int cb[3] = {ch & 1, (ch >> 1) & 1, (ch >> 2) & 1};
      // parent cells covering the region, relative to the child's origin
      const int px = sx < 0 ? 2 : (sx == 0 ? 8 : 2), py = sy < 0 ? 2 : (sy == 0 ? 8 : 2), pz = sz < 0 ? 2 : (sz == 0 ? 8 : 2);
      const int qx0 = sx < 0 ? -2 : (sx == 0 ? 0 : 8), qy0 = sy < 0 ? -2 : (sy == 0 ? 0 : 8), qz0 = sz < 0 ? -2 : (sz == 0 ? 0 : 8);
      const int n = px * py * pz;
      for (int e = threadIdx.x; e < n * NV; e += blockDim.x) {
        const int v = e / n, c = e % n;
        const int rx = qx0 + c % px, ry = qy0 + (c / px) % py, rz = qz0 + c / (px * py);
        const QT<R> qt = qterms_t<R>(P + v * NCELL, 8 * cb[0] + rx, 8 * cb[1] + ry, 8 * cb[2] + rz);
#pragma unroll
        for (int sub = 0; sub < 8; ++sub) {
          const int a = sub & 1, b = (sub >> 1) & 1, cc = (sub >> 2) & 1;
          const R val = predict_t<R>(qt, a ? R(-1) : R(1), b ? R(-1) : R(1), cc ? R(-1) : R(1));
          u[v * NCELL + sidx(2 * rx + a, 2 * ry + b, 2 * rz + cc)] = from_r<R>(val);
        }
      }
    }
  }
}

// Boundary passes x-, x+, y-, y+, z-, z+ of the nodes of `level` on the
// domain boundary (after their copies and predictions).
static __global__ void __launch_bounds__(256) k_fill_bc(Topo t, Phys p, Pool pool, int cur, int level) {
  const int beg = t.cnt[CNT_LVL + level], end = t.cnt[CNT_LVL + level + 1];
  double* buf = pool.buf[cur];
  for (int w = beg + blockIdx.x; w < end; w += gridDim.x) {
    const int node = t.lvl_nodes[w];
    bool any = false;
    for (int d = 0; d < 3; ++d) {
      const int nl = p.nb[d] << level, Xd = t.X[(size_t)node * 3 + d];
      any = any || (Xd == 0 && p.bc[2 * d] != 1) || (Xd == nl - 1 && p.bc[2 * d + 1] != 1);
    }
    if (!any) continue;
    double* u = buf + (size_t)t.slot[node] * SLOT_U;
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
        for (int e = threadIdx.x; e < HW * NS * NS; e += blockDim.x) {
          const int g0 = e % HW, a1 = (e / HW) % NS - HW, a2 = e / (HW * NS) - HW;
          const int a = (side == 0) ? (-1 - g0) : (NB + g0);
          const int sa = (bc == 0) ? ((side == 0) ? 0 : NB - 1) : ((side == 0) ? (-1 - a) : (2 * NB - 1 - a));
          int di, si;
          if (d == 0) { di = sidx(a, a1, a2); si = sidx(sa, a1, a2); }
          else if (d == 1) { di = sidx(a2, a, a1); si = sidx(a2, sa, a1); }
          else { di = sidx(a1, a2, a); si = sidx(a1, a2, sa); }
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

namespace mrb {

// New child: every stored cell predicted from the parent (Eq. Prediction).
// R = double evaluates the prediction in FP64; R = float evaluates the Q-term
// corrections in FP32 and adds them to the FP64 parent value, so that the
// children's mean stays the parent value up to FP64 rounding (the eight
// corrections of a parent cell are sign-symmetric and cancel exactly).
template <class R>
__global__ void __launch_bounds__(256) k_refine_fill_t(Topo t, Pool pool, int cur, const int32_t* __restrict__ pairs,
                                                      int n) {
  double* B = pool.buf[cur];
  const int nitems = n * 8;
  for (int w = blockIdx.x; w < nitems; w += gridDim.x) {
    const int child = pairs[2 * (w / 8)], par = pairs[2 * (w / 8) + 1];
    const int zq = w % 8;                                      // 8 chunks of the 12 x 12 x 12 parent cells
    double* U = B + (size_t)t.slot[child] * SLOT_U;
    const double* P = B + (size_t)t.slot[par] * SLOT_U;
    const int ch = (int)(t.keys[child] & 7ull);
    const int cb[3] = {ch & 1, (ch >> 1) & 1, (ch >> 2) & 1};
    for (int e = threadIdx.x; e < 216 * NV; e += blockDim.x) {
      const int v = e / 216, r = e % 216 + zq * 216;
      const int pi = 8 * cb[0] - 2 + r % 12, pj = 8 * cb[1] - 2 + (r / 12) % 12, pk = 8 * cb[2] - 2 + r / 144;
      const QT<R> q = qterms_t<R>(P + v * NCELL, pi, pj, pk);
      const double base = P[v * NCELL + sidx(pi, pj, pk)];
#pragma unroll
      for (int sub = 0; sub < 8; ++sub) {
        const int a = sub & 1, b = (sub >> 1) & 1, c = (sub >> 2) & 1;
        const int fi = 2 * (pi - 8 * cb[0]) + a, fj = 2 * (pj - 8 * cb[1]) + b, fk = 2 * (pk - 8 * cb[2]) + c;
        double val;
        if (sizeof(R) == sizeof(double)) {
          val = from_r<R>(predict_t<R>(q, a ? R(-1) : R(1), b ? R(-1) : R(1), c ? R(-1) : R(1)));
        } else {
          QT<R> q0 = q;
          q0.u = R(0);
          val = base + from_r<R>(predict_t<R>(q0, a ? R(-1) : R(1), b ? R(-1) : R(1), c ? R(-1) : R(1)));
        }
        U[v * NCELL + sidx(fi, fj, fk)] = val;
      }
    }
  }
}

// Averaging, Eq. (Averaging), levels fine to coarse; one work item per
// (internal node, octant): the octant's 512 parent cells come from one child.
static __global__ void __launch_bounds__(256) k_project_octants(Topo t, Pool pool, int buf, int level) {
  const int beg = t.cnt[CNT_LVL + level], end = t.cnt[CNT_LVL + level + 1];
  double* B = pool.buf[buf];
  const int nitems = (end - beg) * 8;
  for (int w = blockIdx.x; w < nitems; w += gridDim.x) {
    const int node = t.lvl_nodes[beg + w / 8];
    const int c0 = t.child0[node];
    if (c0 < 0) continue;
    const int o = w % 8;
    double* Pp = B + (size_t)t.slot[node] * SLOT_U;
    const double* C = B + (size_t)t.slot[c0 + o] * SLOT_U;
    const int ox = 8 * (o & 1), oy = 8 * ((o >> 1) & 1), oz = 8 * ((o >> 2) & 1);
    for (int e = threadIdx.x; e < 512 * NV; e += blockDim.x) {
      const int v = e / 512, c = e % 512;
      const int I = c % 8, J = (c / 8) % 8, K = c / 64;
      const int fi = 2 * I, fj = 2 * J, fk = 2 * K;
      const double* u = C + v * NCELL;
      const double c0v = u[sidx(fi, fj, fk)], c1v = u[sidx(fi + 1, fj, fk)];
      const double c2v = u[sidx(fi, fj + 1, fk)], c3v = u[sidx(fi + 1, fj + 1, fk)];
      const double c4v = u[sidx(fi, fj, fk + 1)], c5v = u[sidx(fi + 1, fj, fk + 1)];
      const double c6v = u[sidx(fi, fj + 1, fk + 1)], c7v = u[sidx(fi + 1, fj + 1, fk + 1)];
      Pp[v * NCELL + sidx(ox + I, oy + J, oz + K)] = 0.125 * (((c0v + c1v) + (c2v + c3v)) + ((c4v + c5v) + (c6v + c7v)));
    }
  }
}

}  // namespace mrb
