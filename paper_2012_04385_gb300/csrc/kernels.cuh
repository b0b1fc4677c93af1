// Kernels of the block-based MR Euler hot path (arXiv:2012.04385) and their
// launch interface.  Work lists, node arrays and counts live in device memory,
// so every kernel runs a grid-stride loop over a count it reads on the device;
// the same launch stays valid when remeshing changes the tree (which is what
// lets the stage sequence be replayed from a CUDA graph).
#pragma once

#include "physics.cuh"

namespace mrb {

constexpr int MAXL = 11;              // deepest level
constexpr int CNT_NNODES = 0, CNT_NLEAVES = 1, CNT_LVL = 2;   // lvl offsets at CNT_LVL + l, l = 0..MAXL+1
constexpr int CNT_BC = CNT_LVL + MAXL + 2;                     // bc item offsets at CNT_BC + l, l = 0..MAXL+1
constexpr int CNT_JUMP = CNT_BC + MAXL + 2;                    // number of jump items
constexpr int CNT_SIZE = CNT_JUMP + 1;

enum : int { ST_OK = 0, ST_NONPHYS = 6 };

// Halo fill modes, for leaves (internal nodes are always filled completely):
//   FILL_FULL       every region, every variable;
//   FILL_STAGE      only the predicted face regions (the mixed-precision stage
//                   kernel reads same-level face neighbours' cells directly);
//   FILL_DETAIL     every region, rho and E only (the detail norm's inputs).
enum : int { FILL_FULL = 0, FILL_STAGE = 1, FILL_DETAIL = 2 };

// Node arrays, in ascending id order (instance, level, Morton).
struct Topo {
  const uint64_t* keys;
  const int32_t* slot;     // pool slot of the node
  const int32_t* level;
  const int32_t* inst;
  const int32_t* X;        // [n][3] block coordinates on the node's level
  const int32_t* parent;   // node index or -1
  const int32_t* child0;   // first of 8 consecutive children, or -1 for a leaf
  const int32_t* nbr;      // [n][27] same-level neighbour node, -1 none, -2 beyond the boundary
  const int32_t* leaves;   // leaf node indices, ascending id
  const int32_t* lvl_nodes;// node indices grouped by level
  const int32_t* bc_items; // 8 * node + side of every non-periodic domain-boundary side, grouped by level
  const int32_t* jump;     // 64 * leaf index + mask of the sides whose same-level neighbour is refined
  const int32_t* cnt;      // counts, see CNT_*
};

struct Phys {
  double gamma, B, cfl, dx0, eps;
  double mu;               // dynamic viscosity of the Navier-Stokes terms; 0 = Euler
  double inv_dx0;          // 1 / dx0 (1 / dx of level l is its exact 2^l multiple)
  double grav[3];
  int bc[6];
  int nb[3];
  int n_inst;
  int recon;
  int has_grav;
  int precision;           // 0 FP64, 1 FP32 bulk (MRB_FP64 / MRB_FP32_ACC64)
  int rk;                  // Runge-Kutta stages per step: 3 (TVD-RK3) or 2 (TVD-RK2)
  int flux;                // MRB_FLUX_*: Roe with LLF fallback, LLF, HLLC
  float mlp_tau;           // learned selector: linear reconstruction when logit < mlp_tau
  const float* mlp;        // learned selector parameters (device, FP32), or null
  unsigned long long* lin_count;   // [0] faces sent to linear, [1] faces evaluated
  const int32_t* lmax;     // device [n_inst]
  int blocked;             // stage kernels: 1 = a contiguous run of work items per CTA, 0 = strided by the grid
  int lts;                 // local time stepping (Eq. LtsTimestep)
};

// Launch shapes of the scheduling-only tunables (mrb_autotune): every choice
// gives bit-identical results.  Set from the calling context before its
// launches.
struct Tune {
  int stage_waves;         // stage-kernel CTAs = SMs x resident CTAs per SM x stage_waves
  int fill_copy;           // region-copy fill CTAs per SM
  int fill_pred;           // prediction fill CTAs per SM
  int project;             // averaging CTAs per SM
};
extern Tune g_tune;

// This CTA's work items: strided by the grid, or one contiguous run.
struct ItemRange {
  int first, step, end;
};
__device__ __forceinline__ ItemRange item_range(int nitems, int blocked) {
  if (!blocked) return ItemRange{(int)blockIdx.x, (int)gridDim.x, nitems};
  const int per = (nitems + (int)gridDim.x - 1) / (int)gridDim.x;
  const int a = (int)blockIdx.x * per;
  return ItemRange{a, 1, a + per < nitems ? a + per : nitems};
}

// Shu-Osher coefficients of stage s: out = a u^n + b (u + dt L); row 0 TVD-RK3,
// row 1 TVD-RK2.
__device__ __constant__ static const double kRkA[2][3] = {{0.0, 0.75, 1.0 / 3.0}, {0.0, 0.5, 0.0}};
__device__ __constant__ static const double kRkB[2][3] = {{1.0, 0.25, 2.0 / 3.0}, {1.0, 0.5, 0.0}};
__device__ __forceinline__ int rk_row(const Phys& p) { return p.rk == 2 ? 1 : 0; }
// Weights of the stage right-hand sides in the step (u^(n+1) = u^n + dt sum_s
// w_s L(u^(s))): TVD-RK3 1/6, 1/6, 2/3; TVD-RK2 1/2, 1/2.
__device__ __constant__ static const double kRkW[2][3] = {{1.0 / 6.0, 1.0 / 6.0, 2.0 / 3.0}, {0.5, 0.5, 0.0}};

// Work items of a stage launch: every leaf (level < 0) or every node of one
// level (local time stepping); the node of item k and the item count.
__device__ __forceinline__ int stage_nodes(const Topo& t, int level) {
  return level < 0 ? t.cnt[CNT_NLEAVES] : t.cnt[CNT_LVL + level + 1] - t.cnt[CNT_LVL + level];
}
__device__ __forceinline__ int stage_node(const Topo& t, int level, int k) {
  return level < 0 ? t.leaves[k] : t.lvl_nodes[t.cnt[CNT_LVL + level] + k];
}
// The time step of a node: dt of its instance, times 2^(lmax - level) under
// local time stepping.
__device__ __forceinline__ double node_dt(const Topo& t, const Phys& p, const double* dt, int node, int level) {
  const int inst = t.inst[node];
  return level < 0 ? dt[inst] : ldexp(dt[inst], p.lmax[inst] - level);
}

struct Pool {
  double* buf[2];          // stage buffers, [slot][5][24^3]
  double* un;              // u^n, [slot][5][16^3]
  double* face;            // face fluxes, [slot][6][5][16][16]
  uint32_t* sel;           // learned selector decisions of the current step, [slot][SLOT_SEL]
  // FP32 primitive records (rho, vx, vy, vz, p, E) of the internal cells of
  // buf[b], [slot][6][16^3]; kept by the mixed-precision path only (null
  // otherwise), rewritten by every kernel that writes internal cells
  float* sh[2];
  // boundary-face fluxes integrated over a macro time step (local time
  // stepping only), [slot][6][5][16][16]
  double* fmac;
  // FP32 increments u^(s) - u^n of the stage (mixed-precision path only, null
  // otherwise), [slot][5][16^3]
  float* dl;
  // The arrays of stage buffer b, chosen by selection: indexing the arrays
  // above with a run-time b would make the compiler copy the whole kernel
  // parameter into local memory and read the pointers back from there.
  __host__ __device__ __forceinline__ double* bufp(int b) const { return b ? buf[1] : buf[0]; }
  __host__ __device__ __forceinline__ float* shp(int b) const { return b ? sh[1] : sh[0]; }
};

__device__ __forceinline__ double ldexp_(double x, int e) { return ldexp(x, e); }

// ---------------------------------------------------------------- launches
// (defined in kern_f64.cu / kern_f32.cu; all asynchronous on `st`)
void launch_set_state(const Topo& t, const Phys& p, const Pool& pool, int cur, const int32_t* nodes, int n,
                      const double* prim, cudaStream_t st);
void launch_set_cons(const Topo& t, const Pool& pool, int cur, const int32_t* nodes, int n, const double* cons,
                     cudaStream_t st);
void launch_get_state(const Topo& t, const Pool& pool, int cur, const int32_t* nodes, int n, double* out,
                      int with_halo, cudaStream_t st);
void launch_fill_level(const Topo& t, const Phys& p, const Pool& pool, int cur, int level, cudaStream_t st,
                       int mode = 0);
// every halo region of the listed nodes (device list of n node indices), all variables
void launch_fill_list(const Topo& t, const Phys& p, const Pool& pool, int cur, const int32_t* list, int n,
                      cudaStream_t st);
// level < 0: every leaf with dt; level >= 0 (local time stepping): every node
// of that level, leaves and internal nodes, with dt 2^(lmax - level)
void launch_rhs_rk_f64(const Topo& t, const Phys& p, const Pool& pool, int cur, int stage, const double* dt,
                       double* rhs_out, cudaStream_t st, int level = -1);
void launch_rhs_rk_f32(const Topo& t, const Phys& p, const Pool& pool, int cur, int stage, const double* dt,
                       double* rhs_out, cudaStream_t st, int level = -1);
// FP32 stage kernels of the flux variants (separate translation units):
// LLF on every field, and HLLC, each with every non-learned reconstruction.
void launch_rhs_rk_f32_llf(const Topo& t, const Phys& p, const Pool& pool, int cur, int stage, const double* dt,
                           double* rhs_out, cudaStream_t st, int level = -1);
void launch_rhs_rk_f32_hllc(const Topo& t, const Phys& p, const Pool& pool, int cur, int stage, const double* dt,
                            double* rhs_out, cudaStream_t st, int level = -1);
// internal nodes' face fluxes of `level` from their children (faces = pool.face,
// or the macro step's integrated fluxes pool.fmac with integrated = 1)
void launch_face_avg_level(const Topo& t, const Pool& pool, int level, cudaStream_t st, int integrated = 0);
// ---- local time stepping
// Interpolation in time of the nodes of levels < below (factor theta[m] per
// level m; the end state kept in the other stage buffer), or its undoing.
struct LevelTheta {
  double th[MAXL + 1];
};
void launch_lts_interp(const Topo& t, const Pool& pool, int cur, int below, const LevelTheta& th, int restore,
                       cudaStream_t st);
// Internal cells (and FP32 records) of the nodes of `level`: buffer cur^1 -> cur.
void launch_lts_copyback(const Topo& t, const Pool& pool, int cur, int level, cudaStream_t st);
// Integrated fluxes: zero those of every leaf, or add weight x face fluxes to
// those of the leaves of `level` (weight = kRkW[stage] x dt 2^(lmax - level)).
void launch_lts_fmac(const Topo& t, const Phys& p, const Pool& pool, int level, int stage, const double* dt,
                     int zero, cudaStream_t st);
// End of the macro step: leaf faces next to refined neighbours take the finer
// side's integrated flux.
void launch_lts_reflux(const Topo& t, const Phys& p, const Pool& pool, int cur, cudaStream_t st);
void launch_jump(const Topo& t, const Phys& p, const Pool& pool, int target, int stage, const double* dt,
                 double* rhs_out, cudaStream_t st);
void launch_project_level(const Topo& t, const Pool& pool, int buf, int level, cudaStream_t st);
void launch_cfl(const Topo& t, const Phys& p, const Pool& pool, int cur, unsigned long long* smax, double* dt,
                int* status, cudaStream_t st);
void launch_delta_tags(const Topo& t, const Phys& p, const Pool& pool, int cur, double* delta_node,
                       int allow_refine, int8_t* tags, double* delta_leaf, int n_leaves_cap, cudaStream_t st);
void launch_refine_fill(const Topo& t, const Phys& p, const Pool& pool, int cur, const int32_t* pairs, int n,
                        cudaStream_t st);
// Leaves with resolution jumps (a same-level face neighbour that is refined):
// jump[] = 64 * leaf index + side mask, counted into cnt[CNT_JUMP] (item
// order unspecified; every item is independent).
void launch_jump_list(const Topo& t, int32_t* jump, int32_t* cnt, int n_leaves_cap, cudaStream_t st);
void launch_nbr(const Topo& t, const Phys& p, int32_t* nbr_out, int nnodes_cap, cudaStream_t st);
void launch_sums(const Topo& t, const Phys& p, const Pool& pool, int cur, double* partial, double* out,
                 int nleaves_cap, cudaStream_t st);
// mixed-precision variants (kern_f32.cu)
void launch_fill_level_f32(const Topo& t, const Phys& p, const Pool& pool, int cur, int level, cudaStream_t st,
                           int mode);
void launch_fill_list_f32(const Topo& t, const Phys& p, const Pool& pool, int cur, const int32_t* list, int n,
                          cudaStream_t st);
// Roe / LLF census of every leaf face (FP64 decisions on the stage buffer):
// counts[k] faces where field k takes the LLF split, counts[5] faces.
void launch_flux_census(const Topo& t, const Phys& p, const Pool& pool, int cur, unsigned long long* counts,
                        cudaStream_t st);
void launch_delta_f32(const Topo& t, const Phys& p, const Pool& pool, int cur, double* delta_node, int all_nodes,
                      cudaStream_t st);
void launch_cfl_speeds_f32(const Topo& t, const Phys& p, const Pool& pool, int cur, unsigned long long* smax,
                           int* status, cudaStream_t st);
// FP32 records of stage buffer b from its FP64 internal cells (mixed-precision
// path): SH_INTERNAL every internal node (after averaging), SH_JUMP the
// boundary planes that the jump correction changed, SH_LIST the nodes of a
// device list of n entries (every `stride`-th entry is a node index).
enum : int { SH_INTERNAL = 0, SH_JUMP = 1, SH_LIST = 2 };
void launch_shadow(const Topo& t, const Phys& p, const Pool& pool, int b, int mode, const int32_t* list, int n,
                   int stride, cudaStream_t st);
// Records of the listed nodes (kept, or converted afresh from the FP64 state).
void launch_get_records(const Topo& t, const Phys& p, const Pool& pool, int cur, const int32_t* nodes, int n,
                        float* out, int fresh, cudaStream_t st);
void launch_face_samples(const Topo& t, const Phys& p, const Pool& pool, int cur, float tau_lab, int64_t stride,
                         float* feats, uint8_t* labels, int64_t* where, int64_t cap, cudaStream_t st);
int sm_count();
// kernel launches issued by this process (host-side counter, bumped by every launch_* wrapper)
extern long long g_kernel_launches;

}  // namespace mrb
