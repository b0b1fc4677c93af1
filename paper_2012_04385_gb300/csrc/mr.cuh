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

// Parent values for the Q-terms: the stored FP64 array, converted to R on
// load, or a box of R values staged in shared memory (origin i0, j0, k0 in
// stored coordinates, row length nx, plane size nxy).  Both give the same R
// value for a cell, so the Q-terms do not depend on where they are read.
template <class R> struct GAcc {
  const double* P;
  __device__ __forceinline__ R operator()(int i, int j, int k) const { return to_r<R>(P[sidx(i, j, k)]); }
};
template <class R> struct SAcc {
  const R* s;
  int i0, j0, k0, nx, nxy;
  __device__ __forceinline__ R operator()(int i, int j, int k) const {
    return s[(k - k0) * nxy + (j - j0) * nx + (i - i0)];
  }
};

template <class R> __device__ __forceinline__ R qc(int off) { return off == 1 ? R(-22.0 / 128.0) : R(3.0 / 128.0); }

template <class R, class A>
__device__ __forceinline__ R mix2t(const A& P, int i, int j, int k, int Ax, int Bx, int p, int q) {
  int o1[3] = {0, 0, 0}, o2[3] = {0, 0, 0}, o3[3] = {0, 0, 0}, o4[3] = {0, 0, 0};
  o1[Ax] = p; o1[Bx] = q;
  o2[Ax] = -p; o2[Bx] = -q;
  o3[Ax] = -p; o3[Bx] = q;
  o4[Ax] = p; o4[Bx] = -q;
  return (P(i + o1[0], j + o1[1], k + o1[2]) + P(i + o2[0], j + o2[1], k + o2[2])) -
         (P(i + o3[0], j + o3[1], k + o3[2]) + P(i + o4[0], j + o4[1], k + o4[2]));
}

template <class R, class A> __device__ __forceinline__ R mix3t(const A& P, int i, int j, int k, int p, int q, int r) {
  const int sg[4][3] = {{1, 1, 1}, {1, -1, -1}, {-1, -1, 1}, {-1, 1, -1}};
  R acc = R(0);
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    R term = P(i + sg[t][0] * p, j + sg[t][1] * q, k + sg[t][2] * r) - P(i - sg[t][0] * p, j - sg[t][1] * q, k - sg[t][2] * r);
    acc = (t == 0) ? term : acc + term;
  }
  return acc;
}

// Q-terms of parent cell (i, j, k) (Eq. Prediction with the appendix
// coefficients c0 = -22/128, c1 = 3/128).
template <class R, class A> __device__ __forceinline__ QT<R> qterms_t(const A& P, int i, int j, int k) {
  const R C0 = R(-22.0 / 128.0), C1 = R(3.0 / 128.0);
  QT<R> t;
  t.u = P(i, j, k);
  t.Qx = C0 * (P(i + 1, j, k) - P(i - 1, j, k)) + C1 * (P(i + 2, j, k) - P(i - 2, j, k));
  t.Qy = C0 * (P(i, j + 1, k) - P(i, j - 1, k)) + C1 * (P(i, j + 2, k) - P(i, j - 2, k));
  t.Qz = C0 * (P(i, j, k + 1) - P(i, j, k - 1)) + C1 * (P(i, j, k + 2) - P(i, j, k - 2));
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

// Stage the parent values of the box [i0, i0+nx) x [j0, j0+ny) x [k0, k0+nz)
// (stored coordinates) of variable v into shared memory as R; all threads.
template <class R>
__device__ __forceinline__ void stage_box(R* __restrict__ s, const double* __restrict__ P, int i0, int j0, int k0,
                                          int nx, int ny, int nz) {
  const int n = nx * ny * nz;
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    const int i = e % nx, j = (e / nx) % ny, k = e / (nx * ny);
    s[e] = to_r<R>(P[sidx(i0 + i, j0 + j, k0 + k)]);
  }
}

template <class R> __device__ __forceinline__ R predict_t(const QT<R>& t, R sx, R sy, R sz) {
  return t.u + sx * t.Qx + sy * t.Qy + sz * t.Qz + (sx * sy) * t.Qxy + (sx * sz) * t.Qxz + (sy * sz) * t.Qyz +
         (sx * sy * sz) * t.Qxyz;
}


// ---------------------------------------------------------------- halo fill by region
// Sec. 3 (Fig. MrCommunicationMesh): a halo region facing a same-level node
// is a copy of its internal cells, one facing no same-level node is predicted
// from the node's parent (one parent cell, eight fine cells, per step).  One
// warp per (node, halo region) on a persistent grid; k_fill_bc then applies
// the boundary conditions.  The nodes are those of one level, or a list.
// Internal nodes, whose halos feed their children's predictions, are always
// filled completely; leaves according to the fill mode (FILL_* in kernels.cuh).

struct NodeSet {
  int level;                // nodes of this level, when list is null
  const int32_t* list;      // else these nodes
  int n;
};

__device__ __forceinline__ void nodeset_range(const Topo& t, const NodeSet& ns, int& beg, int& cnt) {
  if (ns.list) {
    beg = 0;
    cnt = ns.n;
  } else {
    beg = t.cnt[CNT_LVL + ns.level];
    cnt = t.cnt[CNT_LVL + ns.level + 1] - beg;
  }
}
__device__ __forceinline__ int nodeset_node(const Topo& t, const NodeSet& ns, int beg, int i) {
  return ns.list ? ns.list[i] : t.lvl_nodes[beg + i];
}

// Variable q of the fill: all five, or rho (q = 0) and E (q = 1) only.
__device__ __forceinline__ int fill_var(bool detail_only, int q) { return detail_only ? 4 * q : q; }

__device__ __forceinline__ int region_start(int s) { return s < 0 ? -HW : (s == 0 ? 0 : NB); }

__device__ __forceinline__ int region_log2(int s) { return s == 0 ? 4 : 2; }   // extents 16 or 4

// One warp per (node, halo region).  Extents are powers of two, so the element
// index splits with shifts; copies move 16-byte pairs of doubles (every
// region row starts on a 32-byte boundary of the 24^3 array).
template <class R>
__global__ void __launch_bounds__(256) k_fill_regions_t(Topo t, Pool pool, int cur, NodeSet ns, int mode) {
  int beg, cnt;
  nodeset_range(t, ns, beg, cnt);
  double* buf = pool.bufp(cur);
  const int nitems = cnt * 26;
  const int lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  for (int w = blockIdx.x * wpb + (threadIdx.x >> 5); w < nitems; w += gridDim.x * wpb) {
    const int node = nodeset_node(t, ns, beg, w / 26);
    const int r = w % 26 < 13 ? w % 26 : w % 26 + 1;      // skip the centre
    const int sx = r % 3 - 1, sy = (r / 3) % 3 - 1, sz = r / 9 - 1;
    const bool face = (sx != 0) + (sy != 0) + (sz != 0) == 1;
    const bool leaf = t.child0[node] < 0;
    const bool partial = mode == FILL_STAGE && leaf;
    const bool detail_only = mode == FILL_DETAIL && leaf;
    const int nvar = detail_only ? 2 : NV;
    if (partial && !face) continue;
    const int nb = t.nbr[(size_t)node * 27 + r];
    double* u = buf + (size_t)t.slot[node] * SLOT_U;
    if (nb >= 0) {
      if (partial) continue;                              // read directly by the stage kernel
      const double* src = buf + (size_t)t.slot[nb] * SLOT_U;
      const int lx = region_log2(sx) - 1, ly = region_log2(sy), lz = region_log2(sz);   // x in pairs
      const int x0 = region_start(sx), y0 = region_start(sy), z0 = region_start(sz);
      const int lxy = lx + ly, ln = lxy + lz;
      const int soff = -NB * (sx + NS * (sy + NS * sz));
      const int ne = nvar << ln;               // a multiple of 32
      // four 16-byte loads in flight per lane before their stores
      for (int e0 = lane; e0 < ne; e0 += 128) {
        double2 val[4];
        int dst[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int e = e0 + 32 * q;
          const int v = fill_var(detail_only, e >> ln), c = e & ((1 << ln) - 1);
          const int i = x0 + 2 * (c & ((1 << lx) - 1)), j = y0 + ((c >> lx) & ((1 << ly) - 1)), k = z0 + (c >> lxy);
          dst[q] = v * NCELL + sidx(i, j, k);
          if (e < ne) val[q] = *reinterpret_cast<const double2*>(src + dst[q] + soff);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (e0 + 32 * q < ne) *reinterpret_cast<double2*>(u + dst[q]) = val[q];
      }
    }
  }
}

// Predicted halo regions (no same-level node on that side, the node has a
// parent): one CTA per node, one region after the other; the parent cells
// of the region and their +-2 stencil (6 or 12 per axis) are staged in shared
// memory as R for the variables filled, then every thread evaluates the
// Q-terms of parent cells and writes their eight fine cells.
template <class R>
__global__ void __launch_bounds__(256) k_fill_predict_t(Topo t, Pool pool, int cur, NodeSet ns, int mode) {
  __shared__ R box[NV * 864];
  __shared__ unsigned rmask;
  int beg, cnt;
  nodeset_range(t, ns, beg, cnt);
  double* buf = pool.bufp(cur);
  for (int w = blockIdx.x; w < cnt; w += gridDim.x) {
    const int node = nodeset_node(t, ns, beg, w);
    const int par = t.parent[node];
    if (par < 0) continue;                                   // level 0: no prediction
    const bool leaf = t.child0[node] < 0;
    const bool partial = mode == FILL_STAGE && leaf;
    const bool detail_only = mode == FILL_DETAIL && leaf;
    const int nvar = detail_only ? 2 : NV;
    if (threadIdx.x < 32) {
      bool want = false;
      const int r = threadIdx.x;
      if (r < 27 && r != 13) {
        const int sx = r % 3 - 1, sy = (r / 3) % 3 - 1, sz = r / 9 - 1;
        const bool face = (sx != 0) + (sy != 0) + (sz != 0) == 1;
        want = t.nbr[(size_t)node * 27 + r] == -1 && (!partial || face);
      }
      const unsigned m = __ballot_sync(0xffffffffu, want);
      if (threadIdx.x == 0) rmask = m;
    }
    __syncthreads();
    unsigned m = rmask;
    __syncthreads();
    if (!m) continue;
    double* u = buf + (size_t)t.slot[node] * SLOT_U;
    const double* P = buf + (size_t)t.slot[par] * SLOT_U;
    const int ch = (int)(t.keys[node] & 7ull);
    const int cb[3] = {ch & 1, (ch >> 1) & 1, (ch >> 2) & 1};
    while (m) {
      const int r = __ffs(m) - 1;
      m &= m - 1;
      const int sx = r % 3 - 1, sy = (r / 3) % 3 - 1, sz = r / 9 - 1;
      // parent cells of the region relative to the child's origin: [q0, q0 + n)
      const int lx = sx == 0 ? 3 : 1, ly = sy == 0 ? 3 : 1, lz = sz == 0 ? 3 : 1;
      const int qx0 = sx < 0 ? -2 : (sx == 0 ? 0 : 8), qy0 = sy < 0 ? -2 : (sy == 0 ? 0 : 8), qz0 = sz < 0 ? -2 : (sz == 0 ? 0 : 8);
      // staged box: those parent cells +-2, in the parent's stored coordinates
      const int bx0 = 8 * cb[0] + qx0 - 2, by0 = 8 * cb[1] + qy0 - 2, bz0 = 8 * cb[2] + qz0 - 2;
      const int nx = (1 << lx) + 4, ny = (1 << ly) + 4, nz = (1 << lz) + 4;
      const int nb = nx * ny * nz;
      for (int q = 0; q < nvar; ++q)
        stage_box<R>(box + q * nb, P + fill_var(detail_only, q) * NCELL, bx0, by0, bz0, nx, ny, nz);
      __syncthreads();
      const int lxy = lx + ly, ln = lxy + lz;
      for (int e = threadIdx.x; e < (nvar << ln); e += blockDim.x) {
        const int q = e >> ln, c = e & ((1 << ln) - 1);
        const int v = fill_var(detail_only, q);
        const int rx = qx0 + (c & ((1 << lx) - 1)), ry = qy0 + ((c >> lx) & ((1 << ly) - 1)), rz = qz0 + (c >> lxy);
        const SAcc<R> A{box + q * nb, bx0, by0, bz0, nx, nx * ny};
        const QT<R> qt = qterms_t<R>(A, 8 * cb[0] + rx, 8 * cb[1] + ry, 8 * cb[2] + rz);
#pragma unroll
        for (int sub = 0; sub < 8; ++sub) {
          const int a = sub & 1, b = (sub >> 1) & 1, cc = (sub >> 2) & 1;
          const R val = predict_t<R>(qt, a ? R(-1) : R(1), b ? R(-1) : R(1), cc ? R(-1) : R(1));
          u[v * NCELL + sidx(2 * rx + a, 2 * ry + b, 2 * rz + cc)] = from_r<R>(val);
        }
      }
      __syncthreads();
    }
  }
}

// Boundary conditions of the nodes of `level` on the domain boundary (after
// their copies and predictions).  The oracle applies the x, y and z passes in
// turn; their composition maps each ghost cell to one source cell, every
// coordinate beyond a non-periodic side being mapped back into the block
// (zero gradient: the nearest internal cell; any other condition: the mirror
// cell, with the normal momentum negated under symmetry).  So one warp per
// (node, side) item fills the side's 4 x 24 x 24 slab from source cells that this
// kernel never writes; cells in two slabs get the same value twice.  Work
// items are (node, side, chunk of 256 slab cells), one warp each.
__device__ __forceinline__ int bc_map(int x, int blo, int bhi, int& flip, int bit) {
  if (x < 0 && blo >= 0) {
    flip ^= (blo == 2) ? bit : 0;
    return blo == 0 ? 0 : -1 - x;
  }
  if (x >= NB && bhi >= 0) {
    flip ^= (bhi == 2) ? bit : 0;
    return bhi == 0 ? NB - 1 : 2 * NB - 1 - x;
  }
  return x;
}

static __global__ void __launch_bounds__(256) k_fill_bc(Topo t, Phys p, Pool pool, int cur, NodeSet ns, int mode) {
  // sides: the level's boundary items, or every side of the listed nodes
  int beg, cnt;
  if (ns.list) {
    beg = 0;
    cnt = 6 * ns.n;
  } else {
    beg = t.cnt[CNT_BC + ns.level];
    cnt = t.cnt[CNT_BC + ns.level + 1] - beg;
  }
  double* buf = pool.bufp(cur);
  constexpr int NCHUNK = 9;                  // 2304 slab cells = 9 chunks of 256
  const int nitems = cnt * NCHUNK;
  const int lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  for (int w = blockIdx.x * wpb + (threadIdx.x >> 5); w < nitems; w += gridDim.x * wpb) {
    int node, side;
    if (ns.list) {
      node = ns.list[w / (6 * NCHUNK)];
      side = (w / NCHUNK) % 6;
    } else {
      const int it = t.bc_items[beg + w / NCHUNK];
      node = it >> 3;
      side = it & 7;
    }
    const int d = side >> 1, chunk = w % NCHUNK;
    const int level = t.level[node];
    const bool detail_only = mode == FILL_DETAIL && t.child0[node] < 0;
    int blo[3], bhi[3];   // condition of each boundary side of this node, -1 if none (or periodic)
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const int nl = p.nb[q] << level, Xq = t.X[(size_t)node * 3 + q];
      blo[q] = (Xq == 0 && p.bc[2 * q] != 1) ? p.bc[2 * q] : -1;
      bhi[q] = (Xq == nl - 1 && p.bc[2 * q + 1] != 1) ? p.bc[2 * q + 1] : -1;
    }
    const int bself = (side & 1) ? (d == 0 ? bhi[0] : (d == 1 ? bhi[1] : bhi[2]))
                                 : (d == 0 ? blo[0] : (d == 1 ? blo[1] : blo[2]));
    if (bself < 0) continue;
    double* u = buf + (size_t)t.slot[node] * SLOT_U;
    constexpr int n = HW * NS * NS;           // 2304 = 72 x 32
    for (int e0 = chunk * 256 + lane; e0 < (chunk + 1) * 256; e0 += 4 * 32) {
      double val[4][NV];
      int di[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int e = e0 + 32 * q;
        const int g0 = e % HW, a1 = (e / HW) % NS - HW, a2 = e / (HW * NS) - HW;
        const int a = (side & 1) ? NB + g0 : -1 - g0;
        const int x = (d == 0) ? a : (d == 1 ? a2 : a1);
        const int y = (d == 0) ? a1 : (d == 1 ? a : a2);
        const int z = (d == 0) ? a2 : (d == 1 ? a1 : a);
        int flip = 0;
        const int sx = bc_map(x, blo[0], bhi[0], flip, 1);
        const int sy = bc_map(y, blo[1], bhi[1], flip, 2);
        const int sz = bc_map(z, blo[2], bhi[2], flip, 4);
        di[q] = sidx(x, y, z);
        const int si = sidx(sx, sy, sz);
        if (e < n) {
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            if (detail_only && v >= 1 && v <= 3) continue;
            const double s = u[v * NCELL + si];
            val[q][v] = (v >= 1 && v <= 3 && ((flip >> (v - 1)) & 1)) ? -s : s;
          }
        }
      }
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (e0 + 32 * q < n) {
#pragma unroll
          for (int v = 0; v < NV; ++v)
            if (!(detail_only && v >= 1 && v <= 3)) u[v * NCELL + di[q]] = val[q][v];
        }
    }
  }
}

// ---------------------------------------------------------------- details
// delta of a node at level >= 1: max over its stored cells that are not ghost
// cells and over rho, E of |u - P(u_parent)| / |u|.  Every leaf, and with
// `all_nodes` every node (the tags then also read the details of the parents
// of leaf groups).
template <class R>
__global__ void __launch_bounds__(256) k_delta_t(Topo t, Phys p, Pool pool, int cur, double* __restrict__ delta_node,
                                                 int all_nodes) {
  __shared__ double sh[8];
  __shared__ R box[4096];           // the parent's cells 8 cb - 4 .. 8 cb + 11 per axis, one variable
  const int nitems = all_nodes ? t.cnt[CNT_NNODES] : t.cnt[CNT_NLEAVES];
  const double* B = pool.bufp(cur);
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
    const int cb[3] = {ch & 1, (ch >> 1) & 1, (ch >> 2) & 1};
    bool gl[3], gh[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int nl = p.nb[d] << lvl;
      const int Xd = t.X[(size_t)node * 3 + d];
      gl[d] = (Xd == 0) && (p.bc[2 * d] != 1);
      gh[d] = (Xd == nl - 1) && (p.bc[2 * d + 1] != 1);
    }
    const int bx0 = 8 * cb[0] - 4, by0 = 8 * cb[1] - 4, bz0 = 8 * cb[2] - 4;
    R m = R(0);
    for (int vi = 0; vi < 2; ++vi) {
      const int v = vi == 0 ? 0 : 4;
      stage_box<R>(box, P + v * NCELL, bx0, by0, bz0, 16, 16, 16);
      __syncthreads();
      const SAcc<R> A{box, bx0, by0, bz0, 16, 256};
      for (int q = threadIdx.x; q < 1728; q += blockDim.x) {
        const int rx = q % 12 - 2, ry = (q / 12) % 12 - 2, rz = q / 144 - 2;
        // all eight fine cells of this parent cell share the ghost status
        const bool ghost = (rx < 0 && gl[0]) || (rx >= 8 && gh[0]) || (ry < 0 && gl[1]) || (ry >= 8 && gh[1]) ||
                           (rz < 0 && gl[2]) || (rz >= 8 && gh[2]);
        if (ghost) continue;
        const QT<R> qt = qterms_t<R>(A, 8 * cb[0] + rx, 8 * cb[1] + ry, 8 * cb[2] + rz);
#pragma unroll
        for (int sub = 0; sub < 8; ++sub) {
          const int a = sub & 1, b = (sub >> 1) & 1, c = (sub >> 2) & 1;
          const R pr = predict_t<R>(qt, a ? R(-1) : R(1), b ? R(-1) : R(1), c ? R(-1) : R(1));
          const R uf = to_r<R>(U[v * NCELL + sidx(2 * rx + a, 2 * ry + b, 2 * rz + c)]);
          const R r = (uf - pr) / uf;
          m = (r < R(0) ? -r : r) > m ? (r < R(0) ? -r : r) : m;
        }
      }
      __syncthreads();
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
  __shared__ R box[4096];           // the parent's cells 8 cb - 4 .. 8 cb + 11 per axis, one variable
  double* B = pool.bufp(cur);
  const int nitems = n * NV;
  for (int w = blockIdx.x; w < nitems; w += gridDim.x) {
    const int child = pairs[2 * (w / NV)], par = pairs[2 * (w / NV) + 1];
    const int v = w % NV;
    double* U = B + (size_t)t.slot[child] * SLOT_U + v * NCELL;
    const double* P = B + (size_t)t.slot[par] * SLOT_U + v * NCELL;
    const int ch = (int)(t.keys[child] & 7ull);
    const int cb[3] = {ch & 1, (ch >> 1) & 1, (ch >> 2) & 1};
    const int bx0 = 8 * cb[0] - 4, by0 = 8 * cb[1] - 4, bz0 = 8 * cb[2] - 4;
    stage_box<R>(box, P, bx0, by0, bz0, 16, 16, 16);
    __syncthreads();
    const SAcc<R> A{box, bx0, by0, bz0, 16, 256};
    for (int r = threadIdx.x; r < 1728; r += blockDim.x) {
      const int pi = 8 * cb[0] - 2 + r % 12, pj = 8 * cb[1] - 2 + (r / 12) % 12, pk = 8 * cb[2] - 2 + r / 144;
      const QT<R> q = qterms_t<R>(A, pi, pj, pk);
      const double base = P[sidx(pi, pj, pk)];
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
        U[sidx(fi, fj, fk)] = val;
      }
    }
    __syncthreads();
  }
}

// Averaging, Eq. (Averaging), levels fine to coarse; one work item per
// (internal node, octant): the octant's 512 parent cells come from one child.
static __global__ void __launch_bounds__(256) k_project_octants(Topo t, Pool pool, int buf, int level) {
  const int beg = t.cnt[CNT_LVL + level], end = t.cnt[CNT_LVL + level + 1];
  double* B = pool.bufp(buf);
  const int nitems = (end - beg) * 8;
  for (int w = blockIdx.x; w < nitems; w += gridDim.x) {
    const int node = t.lvl_nodes[beg + w / 8];
    const int c0 = t.child0[node];
    if (c0 < 0) continue;
    const int o = w % 8;
    double* __restrict__ Pp = B + (size_t)t.slot[node] * SLOT_U;
    const double* __restrict__ C = B + (size_t)t.slot[c0 + o] * SLOT_U;
    const int ox = 8 * (o & 1), oy = 8 * ((o >> 1) & 1), oz = 8 * ((o >> 2) & 1);
    // two parent cells per iteration, their eight 16-byte child loads in flight together
    for (int e0 = threadIdx.x; e0 < 512 * NV; e0 += 2 * blockDim.x) {
      double2 a[2][4];
      int dst[2];
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int e = e0 + q * blockDim.x;
        const int v = e / 512, c = e % 512;
        const int I = c % 8, J = (c / 8) % 8, K = c / 64;
        const int fi = 2 * I, fj = 2 * J, fk = 2 * K;
        dst[q] = v * NCELL + sidx(ox + I, oy + J, oz + K);
        // fi is even: each x-pair of children is one aligned 16-byte load
        const double* u = C + v * NCELL;
        if (e < 512 * NV) {
          a[q][0] = *reinterpret_cast<const double2*>(u + sidx(fi, fj, fk));
          a[q][1] = *reinterpret_cast<const double2*>(u + sidx(fi, fj + 1, fk));
          a[q][2] = *reinterpret_cast<const double2*>(u + sidx(fi, fj, fk + 1));
          a[q][3] = *reinterpret_cast<const double2*>(u + sidx(fi, fj + 1, fk + 1));
        }
      }
#pragma unroll
      for (int q = 0; q < 2; ++q)
        if (e0 + q * blockDim.x < 512 * NV)
          Pp[dst[q]] = 0.125 * (((a[q][0].x + a[q][0].y) + (a[q][1].x + a[q][1].y)) +
                                ((a[q][2].x + a[q][2].y) + (a[q][3].x + a[q][3].y)));
    }
  }
}

}  // namespace mrb
