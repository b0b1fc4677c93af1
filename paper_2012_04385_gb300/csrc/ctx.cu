// Host control of libmrb: the C ABI of include/mrb.h, the light-weight topology
// (ids, levels, parents, children, work lists; Sec. 3 of arXiv:2012.04385
// separates it from the heavy block data), the pool slot allocator, remeshing,
// and the CUDA-graph replay of the stage sequence.
//
// The topology is authoritative on the host and mirrored into fixed-capacity
// device arrays after every change; all kernels read it (and its counts) from
// device memory, so the captured stage graph stays valid across remeshes.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <exception>
#include <string>
#include <vector>

#include "kernels.cuh"
#include "mrb.h"

using namespace mrb;

namespace {

constexpr uint64_t MASK56 = (1ull << 56) - 1;

struct HNode {
  uint64_t key;
  int32_t slot, level, inst;
  int32_t X[3];
};

uint64_t make_key(int inst, int level, const int32_t X[3]) {
  const int ng = 7 + level;
  uint64_t m = 0;
  for (int b = 0; b < ng; ++b)
    for (int d = 0; d < 3; ++d) m |= (uint64_t)((X[d] >> b) & 1) << (3 * b + d);
  return ((uint64_t)inst << 56) | (1ull << (3 * ng)) | m;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Err : std::exception {
  int code;
  std::string msg;
  Err(int c, std::string m) : code(c), msg(std::move(m)) {}
};

#define CK(call)                                                                                     \
  do {                                                                                               \
    cudaError_t e_ = (call);                                                                         \
    if (e_ != cudaSuccess) throw Err(MRB_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

}  // namespace

struct mrb_ctx {
  mrb_config cfg{};
  cudaStream_t st = nullptr;
  char* pool = nullptr;
  size_t pool_bytes = 0;
  int64_t nslots = 0;
  Pool P{};
  Phys phys{};
  int cur = 0;
  int max_lmax = 0;

  std::vector<HNode> nodes;          // sorted by key
  std::vector<int32_t> free_slots;   // stack, back = next
  std::vector<int32_t> h_parent, h_child0, h_leaves, h_lvl_nodes, h_bc_items, h_cnt;

  uint64_t* d_keys = nullptr;
  int32_t *d_slot = nullptr, *d_level = nullptr, *d_inst = nullptr, *d_X = nullptr, *d_parent = nullptr,
          *d_child0 = nullptr, *d_nbr = nullptr, *d_leaves = nullptr, *d_lvl_nodes = nullptr, *d_bc_items = nullptr, *d_jump = nullptr, *d_cnt = nullptr,
          *d_lmax = nullptr, *d_list = nullptr;
  double *d_dt = nullptr, *d_delta_node = nullptr, *d_partial = nullptr;
  unsigned long long* d_census = nullptr;   // mrb_flux_census counters (allocated on first use)
  unsigned long long* d_smax = nullptr;
  int8_t* d_tags = nullptr;
  int* d_status = nullptr;
  unsigned long long* d_lin = nullptr;
  std::vector<void*> allocs;

  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  cudaStream_t cap_st = nullptr;     // private stream for capture (the caller's may be the legacy stream)
  bool graph_dirty = true;
  bool detail_filled = false;        // leaves' halos hold rho and E only (fill before the details)
  char* h_stage = nullptr;           // pinned staging of the topology uploads
  int32_t* h_list = nullptr;         // pinned staging of work lists
  cudaEvent_t stage_ev = nullptr, list_ev = nullptr;
  long long graph_kernels[2] = {0, 0};
  int capturing = -1;                // graph parity being captured, or -1
  cudaEvent_t gev[2][3][2] = {};     // events around the stage kernel inside each graph
  bool prof = false;
  double prof_ms = 0.0;
  long long prof_rhs = 0, prof_base = 0;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pend;   // direct launches awaiting their timing
  Tune tune{1, 8, 4, 8};             // launch shapes of this context (mrb_set_tune / mrb_autotune)
  std::string err;

  Topo topo() const {
    Topo t;
    t.keys = d_keys;
    t.slot = d_slot;
    t.level = d_level;
    t.inst = d_inst;
    t.X = d_X;
    t.parent = d_parent;
    t.child0 = d_child0;
    t.nbr = d_nbr;
    t.leaves = d_leaves;
    t.lvl_nodes = d_lvl_nodes;
    t.bc_items = d_bc_items;
    t.jump = d_jump;
    t.cnt = d_cnt;
    return t;
  }

  template <class T> T* dalloc(size_t n) {
    void* p = nullptr;
    if (cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T)) != cudaSuccess) throw Err(MRB_ENOMEM, "cudaMalloc failed");
    allocs.push_back(p);
    return (T*)p;
  }

  int64_t find(uint64_t key) const {
    auto it = std::lower_bound(nodes.begin(), nodes.end(), key, [](const HNode& a, uint64_t k) { return a.key < k; });
    if (it == nodes.end() || it->key != key) return -1;
    return it - nodes.begin();
  }

  int n_leaves() const { return (int)h_leaves.size(); }

  // derived arrays + upload + neighbour table
  void rebuild() {
    const int n = (int)nodes.size();
    h_parent.assign(n, -1);
    h_child0.assign(n, -1);
    h_leaves.clear();
    // Parents by a merge: ids are sorted (instance, then level through the
    // headbit, then Morton order), and along each (instance, level) run the
    // parent ids (id >> 3) do not decrease.  The first child of a parent in
    // id order is its child 0 (siblings come in complete groups of eight).
    {
      int64_t q = 0;
      int run_inst = -1, run_level = -1;
      for (int i = 0; i < n; ++i) {
        const HNode& a = nodes[i];
        if (a.level == 0) continue;
        const uint64_t pk = ((a.key & MASK56) >> 3) | ((a.key >> 56) << 56);
        if (a.inst != run_inst || a.level != run_level) {
          q = std::lower_bound(nodes.begin(), nodes.end(), pk,
                               [](const HNode& b, uint64_t k) { return b.key < k; }) - nodes.begin();
          run_inst = a.inst;
          run_level = a.level;
        }
        while (q < n && nodes[q].key < pk) ++q;
        if (q < n && nodes[q].key == pk) {
          h_parent[i] = (int32_t)q;
          if (h_child0[q] < 0) h_child0[q] = i;
        }
      }
    }
    for (int i = 0; i < n; ++i)
      if (h_child0[i] < 0) h_leaves.push_back(i);
    h_cnt.assign(CNT_SIZE, 0);
    h_cnt[CNT_NNODES] = n;
    h_cnt[CNT_NLEAVES] = (int)h_leaves.size();
    h_lvl_nodes.clear();
    for (int l = 0; l <= MAXL; ++l) {
      h_cnt[CNT_LVL + l] = (int)h_lvl_nodes.size();
      for (int i = 0; i < n; ++i)
        if (nodes[i].level == l) h_lvl_nodes.push_back(i);
    }
    h_cnt[CNT_LVL + MAXL + 1] = (int)h_lvl_nodes.size();
    // boundary-condition work: the non-periodic domain-boundary sides of each node
    h_bc_items.clear();
    for (int l = 0; l <= MAXL; ++l) {
      h_cnt[CNT_BC + l] = (int)h_bc_items.size();
      for (int q = h_cnt[CNT_LVL + l]; q < h_cnt[CNT_LVL + l + 1]; ++q) {
        const int i = h_lvl_nodes[q];
        for (int d = 0; d < 3; ++d) {
          const int nl = cfg.base_blocks[d] << l;
          if (nodes[i].X[d] == 0 && cfg.bc[2 * d] != MRB_BC_PERIODIC) h_bc_items.push_back(8 * i + 2 * d);
          if (nodes[i].X[d] == nl - 1 && cfg.bc[2 * d + 1] != MRB_BC_PERIODIC) h_bc_items.push_back(8 * i + 2 * d + 1);
        }
      }
    }
    h_cnt[CNT_BC + MAXL + 1] = (int)h_bc_items.size();
    h_cnt[CNT_JUMP] = 0;     // counted on the device after the neighbour table
    // one pinned staging area for every array (asynchronous copies); the
    // previous rebuild's copies have long finished when it is rewritten
    if (stage_ev) CK(cudaEventSynchronize(stage_ev));
    char* q = h_stage;
    auto put = [&](void* dev, const void* src, size_t bytes) {
      if (bytes == 0) return;
      std::memcpy(q, src, bytes);
      CK(cudaMemcpyAsync(dev, q, bytes, cudaMemcpyHostToDevice, st));
      q += (bytes + 15) & ~(size_t)15;
    };
    {
      uint64_t* k = reinterpret_cast<uint64_t*>(q);
      for (int i = 0; i < n; ++i) k[i] = nodes[i].key;
      CK(cudaMemcpyAsync(d_keys, k, sizeof(uint64_t) * n, cudaMemcpyHostToDevice, st));
      q += (sizeof(uint64_t) * n + 15) & ~(size_t)15;
      int32_t* a = reinterpret_cast<int32_t*>(q);
      for (int i = 0; i < n; ++i) {
        a[i] = nodes[i].slot;
        a[n + i] = nodes[i].level;
        a[2 * n + i] = nodes[i].inst;
        for (int d = 0; d < 3; ++d) a[3 * n + 3 * i + d] = nodes[i].X[d];
      }
      CK(cudaMemcpyAsync(d_slot, a, sizeof(int32_t) * n, cudaMemcpyHostToDevice, st));
      CK(cudaMemcpyAsync(d_level, a + n, sizeof(int32_t) * n, cudaMemcpyHostToDevice, st));
      CK(cudaMemcpyAsync(d_inst, a + 2 * n, sizeof(int32_t) * n, cudaMemcpyHostToDevice, st));
      CK(cudaMemcpyAsync(d_X, a + 3 * n, sizeof(int32_t) * 3 * n, cudaMemcpyHostToDevice, st));
      q += (sizeof(int32_t) * 6 * n + 15) & ~(size_t)15;
    }
    put(d_parent, h_parent.data(), sizeof(int32_t) * n);
    put(d_child0, h_child0.data(), sizeof(int32_t) * n);
    put(d_leaves, h_leaves.data(), sizeof(int32_t) * h_leaves.size());
    put(d_lvl_nodes, h_lvl_nodes.data(), sizeof(int32_t) * h_lvl_nodes.size());
    put(d_bc_items, h_bc_items.data(), sizeof(int32_t) * h_bc_items.size());
    put(d_cnt, h_cnt.data(), sizeof(int32_t) * CNT_SIZE);
    launch_nbr(topo(), phys, d_nbr, n, st);
    launch_jump_list(topo(), d_jump, d_cnt, (int)h_leaves.size(), st);
    CK(cudaGetLastError());
    CK(cudaEventRecord(stage_ev, st));
  }

  void check_launch() { CK(cudaGetLastError()); }

  std::vector<int32_t> nodes_of(const uint64_t* keys, int64_t n) const {
    std::vector<int32_t> out((size_t)n);
    for (int64_t b = 0; b < n; ++b) {
      int64_t i = find(keys[b]);
      if (i < 0) throw Err(MRB_EINVAL, "unknown block id");
      out[b] = (int32_t)i;
    }
    return out;
  }

  void upload_list(const std::vector<int32_t>& v) {
    if ((int64_t)v.size() > 2 * nslots) throw Err(MRB_ECAPACITY, "list longer than the pool");
    // pinned staging; wait until the device has read the previous list
    if (list_ev) CK(cudaEventSynchronize(list_ev));
    if (!v.empty()) std::memcpy(h_list, v.data(), sizeof(int32_t) * v.size());
    CK(cudaMemcpyAsync(d_list, h_list, sizeof(int32_t) * v.size(), cudaMemcpyHostToDevice, st));
  }
  // after the kernels that read d_list have been launched
  void list_used() { CK(cudaEventRecord(list_ev, st)); }

  // ---- the steps
  void fill_halos(int mode = FILL_FULL) {
    for (int l = 0; l <= max_lmax; ++l) launch_fill_level(topo(), phys, P, cur, l, st, mode);
  }
  void stage(int s, const double* dt) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (capturing >= 0) {
      e0 = gev[capturing][s][0];
      e1 = gev[capturing][s][1];
    } else if (prof) {
      CK(cudaEventCreate(&e0));
      CK(cudaEventCreate(&e1));
      pend.push_back({e0, e1});
    }
    // inside a capture an event record is a graph node only when marked external
    const unsigned flags = (capturing >= 0) ? cudaEventRecordExternal : cudaEventRecordDefault;
    if (e0) CK(cudaEventRecordWithFlags(e0, st, flags));
    if (cfg.precision == MRB_FP32_ACC64) launch_rhs_rk_f32(topo(), phys, P, cur, s, dt, nullptr, st);
    else launch_rhs_rk_f64(topo(), phys, P, cur, s, dt, nullptr, st);
    if (e1) CK(cudaEventRecordWithFlags(e1, st, flags));
    for (int l = max_lmax - 1; l >= 0; --l) launch_face_avg_level(topo(), P, l, st);
    launch_jump(topo(), phys, P, cur ^ 1, s, dt, nullptr, st);
    launch_shadow(topo(), phys, P, cur ^ 1, SH_JUMP, nullptr, 0, 0, st);
    cur ^= 1;
  }
  void project() {
    for (int l = max_lmax - 1; l >= 0; --l) launch_project_level(topo(), P, cur, l, st);
    launch_shadow(topo(), phys, P, cur, SH_INTERNAL, nullptr, 0, 0, st);
  }
  void step_stages() {
    launch_cfl(topo(), phys, P, cur, d_smax, d_dt, d_status, st);
    // the mixed-precision stage kernel reads face neighbours directly, so the
    // stage fill of leaves is limited to predicted and boundary face regions;
    // the viscous gradients read edge halo cells, which need the full fill
    const int mode = (cfg.precision == MRB_FP32_ACC64 && !(cfg.mu > 0.0)) ? FILL_STAGE : FILL_FULL;
    for (int s = 0; s < phys.rk; ++s) {
      fill_halos(mode);
      stage(s, d_dt);
      project();
    }
  }

  // Local time stepping, one macro step (Eq. LtsTimestep; the reading is the
  // oracle's: coarse levels first, every node of a stepping level advances,
  // coarser levels interpolated in time for the halo fills, levels averaged
  // from their children when their step ends, integrated boundary-face fluxes
  // exchanged at the end).  Direct launches; the stage kernels write the other
  // stage buffer, copied back after each stage, so `cur` does not change.
  void step_lts() {
    launch_cfl(topo(), phys, P, cur, d_smax, d_dt, d_status, st);
    launch_lts_fmac(topo(), phys, P, 0, 0, d_dt, 1, st);
    const int L = max_lmax;
    const int fmode = (cfg.precision == MRB_FP32_ACC64 && !(cfg.mu > 0.0)) ? FILL_STAGE : FILL_FULL;
    const double cst[2][3] = {{0.0, 1.0, 0.5}, {0.0, 1.0, 0.0}};   // stage times, TVD-RK3 / TVD-RK2
    const int row = (phys.rk == 2) ? 1 : 0;
    for (int r = 0; r < (1 << L); ++r) {
      for (int l = 0; l <= L; ++l) {
        if (r % (1 << (L - l)) != 0) continue;
        if (h_cnt[CNT_LVL + l + 1] - h_cnt[CNT_LVL + l] == 0) continue;
        for (int s = 0; s < phys.rk; ++s) {
          LevelTheta th{};
          for (int m = 0; m < l; ++m) {
            const int span = 1 << (L - m);
            const int r0 = r - r % span;
            th.th[m] = ((double)(r - r0) + cst[row][s] * (double)(1 << (L - l))) / (double)span;
          }
          launch_lts_interp(topo(), P, cur, l, th, 0, st);
          // the stepping level's halos, and those of the coarser levels its
          // predictions read; finer levels are filled when they step
          for (int ll = 0; ll <= l; ++ll) launch_fill_level(topo(), phys, P, cur, ll, st, fmode);
          if (cfg.precision == MRB_FP32_ACC64) launch_rhs_rk_f32(topo(), phys, P, cur, s, d_dt, nullptr, st, l);
          else launch_rhs_rk_f64(topo(), phys, P, cur, s, d_dt, nullptr, st, l);
          launch_lts_copyback(topo(), P, cur, l, st);
          launch_lts_fmac(topo(), phys, P, l, s, d_dt, 0, st);
          launch_lts_interp(topo(), P, cur, l, th, 1, st);
        }
      }
      // levels whose step ends with this micro step: averaged from their children
      int lo = L;
      for (int l = L; l >= 0; --l)
        if ((r + 1) % (1 << (L - l)) == 0) lo = l;
      for (int l = max_lmax - 1; l >= lo; --l) launch_project_level(topo(), P, cur, l, st);
      launch_shadow(topo(), phys, P, cur, SH_INTERNAL, nullptr, 0, 0, st);
    }
    for (int l = max_lmax - 1; l >= 0; --l) launch_face_avg_level(topo(), P, l, st, 1);
    launch_lts_reflux(topo(), phys, P, cur, st);
    launch_shadow(topo(), phys, P, cur, SH_JUMP, nullptr, 0, 0, st);
    project();
  }

  void capture_graphs() {
    for (int g = 0; g < 2; ++g) {
      if (graph[g]) cudaGraphExecDestroy(graph[g]);
      graph[g] = nullptr;
    }
    if (!cap_st) CK(cudaStreamCreateWithFlags(&cap_st, cudaStreamNonBlocking));
    for (int g = 0; g < 2; ++g)
      for (int s = 0; s < 3; ++s)
        for (int q = 0; q < 2; ++q)
          if (!gev[g][s][q]) CK(cudaEventCreate(&gev[g][s][q]));
    const int save = cur;
    cudaStream_t user = st;
    st = cap_st;
    for (int g = 0; g < 2; ++g) {
      cur = g;
      cudaGraph_t gr;
      const long long before = g_kernel_launches;
      cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        capturing = g;
        step_stages();
        capturing = -1;
        e = cudaStreamEndCapture(st, &gr);
      }
      graph_kernels[g] = g_kernel_launches - before;
      g_kernel_launches = before;
      if (e == cudaSuccess) {
        e = cudaGraphInstantiate(&graph[g], gr, 0);
        cudaGraphDestroy(gr);
      }
      if (e != cudaSuccess) {
        st = user;
        cur = save;
        throw Err(MRB_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
      }
    }
    st = user;
    cur = save;
    graph_dirty = false;
  }

  int64_t remesh(const int8_t* tags_dev) {
    const int nl = n_leaves();
    const bool detail_fill = detail_filled;
    detail_filled = false;
    std::vector<int8_t> tags((size_t)nl);
    if (nl) CK(cudaMemcpyAsync(tags.data(), tags_dev, nl, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    std::vector<int> refine;
    std::vector<uint64_t> coarse_parents;
    std::vector<std::pair<uint64_t, int>> ccount;
    for (int li = 0; li < nl; ++li) {
      const HNode& a = nodes[h_leaves[li]];
      if (tags[li] == MRB_TAG_REFINE && a.level < cfg.lmax[a.inst]) refine.push_back(h_leaves[li]);
      if (tags[li] == MRB_TAG_COARSEN && a.level >= 2) {
        const uint64_t pk = ((a.key & MASK56) >> 3) | ((a.key >> 56) << 56);
        if (!ccount.empty() && ccount.back().first == pk) ccount.back().second++;
        else ccount.push_back({pk, 1});
      }
    }
    for (auto& c : ccount)
      if (c.second == 8) coarse_parents.push_back(c.first);
    if ((int64_t)refine.size() * 8 > (int64_t)free_slots.size() + 8 * (int64_t)coarse_parents.size())
      throw Err(MRB_ECAPACITY, "block pool exhausted by refinement");
    if (refine.empty() && coarse_parents.empty()) return nl;
    if (detail_fill && !refine.empty()) {
      // the halos of leaves were filled for the details only (rho, E): complete
      // those of the blocks about to be refined, whose children are predicted
      // over their whole stored range
      upload_list(refine);
      launch_fill_list(topo(), phys, P, cur, d_list, (int)refine.size(), st);
      list_used();
      check_launch();
    }

    // coarsening frees slots first (ascending key order), refinement then takes them
    std::vector<char> removed(nodes.size(), 0);
    for (uint64_t pk : coarse_parents) {
      const int64_t pi = find(pk);
      const int c0 = h_child0[pi];
      for (int c = 0; c < 8; ++c) removed[c0 + c] = 1;
    }
    std::vector<int32_t> freed;
    for (size_t i = 0; i < nodes.size(); ++i)
      if (removed[i]) freed.push_back(nodes[i].slot);
    for (auto it = freed.rbegin(); it != freed.rend(); ++it) free_slots.push_back(*it);
    std::vector<HNode> next;
    next.reserve(nodes.size() + 8 * refine.size());
    for (size_t i = 0; i < nodes.size(); ++i)
      if (!removed[i]) next.push_back(nodes[i]);
    std::vector<std::pair<uint64_t, uint64_t>> newpairs;  // (child key, parent key)
    for (int pi : refine) {
      const HNode p = nodes[pi];
      for (int ch = 0; ch < 8; ++ch) {
        HNode c;
        c.inst = p.inst;
        c.level = p.level + 1;
        for (int d = 0; d < 3; ++d) c.X[d] = 2 * p.X[d] + ((ch >> d) & 1);
        c.key = make_key(c.inst, c.level, c.X);
        c.slot = free_slots.back();
        free_slots.pop_back();
        next.push_back(c);
        newpairs.push_back({c.key, p.key});
      }
    }
    std::sort(next.begin(), next.end(), [](const HNode& a, const HNode& b) { return a.key < b.key; });
    nodes.swap(next);
    rebuild();
    if (!newpairs.empty()) {
      std::vector<int32_t> pairs;
      pairs.reserve(2 * newpairs.size());
      for (auto& pr : newpairs) {
        pairs.push_back((int32_t)find(pr.first));
        pairs.push_back((int32_t)find(pr.second));
      }
      upload_list(pairs);
      launch_refine_fill(topo(), phys, P, cur, d_list, (int)newpairs.size(), st);
      launch_shadow(topo(), phys, P, cur, SH_LIST, d_list, (int)newpairs.size(), 2, st);
      list_used();
      check_launch();
    }
    return n_leaves();
  }

  void destroy() {
    for (int g = 0; g < 2; ++g)
      if (graph[g]) cudaGraphExecDestroy(graph[g]);
    if (cap_st) cudaStreamDestroy(cap_st);
    for (int g = 0; g < 2; ++g)
      for (int s = 0; s < 3; ++s)
        for (int q = 0; q < 2; ++q)
          if (gev[g][s][q]) cudaEventDestroy(gev[g][s][q]);
    for (auto& pr : pend) {
      cudaEventDestroy(pr.first);
      cudaEventDestroy(pr.second);
    }
    for (void* p : allocs) cudaFree(p);
    allocs.clear();
    if (stage_ev) cudaEventSynchronize(stage_ev);
    if (list_ev) cudaEventSynchronize(list_ev);
    if (stage_ev) cudaEventDestroy(stage_ev);
    if (list_ev) cudaEventDestroy(list_ev);
    if (h_stage) cudaFreeHost(h_stage);
    if (h_list) cudaFreeHost(h_list);
    stage_ev = list_ev = nullptr;
    h_stage = nullptr;
    h_list = nullptr;
  }
};

namespace {

thread_local std::string g_last_error;

int fail(mrb_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  g_last_error = msg;
  return code;
}

template <class F> int guarded(mrb_ctx* c, F&& f) {
  if (!c) return fail(nullptr, MRB_EINVAL, "null context");
  g_tune = c->tune;       // this context's launch shapes for the launches below
  try {
    f();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(c, MRB_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
    return MRB_OK;
  } catch (const Err& e) {
    return fail(c, e.code, e.msg);
  } catch (const std::exception& e) {
    return fail(c, MRB_ENOMEM, e.what());
  } catch (...) {
    return fail(c, MRB_EINVAL, "unknown error");
  }
}

int check_config(const mrb_config* cfg) {
  if (!cfg) return MRB_EINVAL;
  if (cfg->n_instances < 1 || cfg->n_instances > MRB_MAX_INSTANCES) return MRB_EINVAL;
  for (int d = 0; d < 3; ++d)
    if (cfg->base_blocks[d] < 1 || cfg->base_blocks[d] > 128) return MRB_EINVAL;
  for (int i = 0; i < cfg->n_instances; ++i)
    if (cfg->lmax[i] < 0 || cfg->lmax[i] > MRB_MAX_LEVEL) return MRB_EINVAL;
  for (int d = 0; d < 3; ++d)
    if ((cfg->bc[2 * d] == MRB_BC_PERIODIC) != (cfg->bc[2 * d + 1] == MRB_BC_PERIODIC)) return MRB_EINVAL;
  for (int s = 0; s < 6; ++s)
    if (cfg->bc[s] < 0 || cfg->bc[s] > 2) return MRB_EINVAL;
  if (cfg->precision != MRB_FP64 && cfg->precision != MRB_FP32_ACC64) return MRB_EINVAL;
  if (cfg->recon < 0 || cfg->recon > 4) return MRB_EINVAL;
  if (cfg->flux < 0 || cfg->flux > 2) return MRB_EINVAL;
  if (cfg->recon == MRB_RECON_LEARNED && cfg->flux != MRB_FLUX_ROE) return MRB_EINVAL;
  if (!(cfg->mu >= 0.0) || !std::isfinite(cfg->mu)) return MRB_EINVAL;
  // the mixed-precision viscous kernel exists for WENO5-JS with the Roe flux
  if (cfg->mu > 0.0 && cfg->precision == MRB_FP32_ACC64 &&
      (cfg->recon != MRB_RECON_WENO5 || cfg->flux != MRB_FLUX_ROE))
    return MRB_EINVAL;
  if (cfg->rk_stages != 0 && cfg->rk_stages != 2 && cfg->rk_stages != 3) return MRB_EINVAL;
  if (cfg->lts != 0 && cfg->lts != 1) return MRB_EINVAL;
  if (cfg->lts)
    for (int i = 1; i < cfg->n_instances; ++i)
      if (cfg->lmax[i] != cfg->lmax[0]) return MRB_EINVAL;   // one micro-step schedule for all instances
  if (!(cfg->dx0 > 0) || !(cfg->gamma > 1.0) || !(cfg->cfl > 0)) return MRB_EINVAL;
  return MRB_OK;
}

constexpr size_t slot_doubles() { return 2 * (size_t)SLOT_U + SLOT_N + SLOT_F + SLOT_SEL / 2; }

}  // namespace

extern "C" {

size_t mrb_pool_bytes(const mrb_config* cfg, int64_t n_slots) {
  if (check_config(cfg) != MRB_OK || n_slots <= 0) return 0;
  const size_t n = (size_t)n_slots;
  // the mixed-precision path also keeps FP32 records of both stage buffers' internal cells
  const size_t sh = (cfg->precision == MRB_FP32_ACC64) ? align256(n * SLOT_SH * 4) * 2 + align256(n * SLOT_N * 4) : 0;
  // local time stepping also keeps the boundary-face fluxes integrated over a macro step
  const size_t fm = cfg->lts ? align256(n * SLOT_F * 8) : 0;
  return align256(n * SLOT_U * 8) * 2 + align256(n * SLOT_N * 8) + align256(n * SLOT_F * 8) + align256(n * SLOT_SEL * 4) +
         sh + fm;
}

int mrb_init_blocks(const mrb_config* cfg, void* pool, size_t pool_bytes, mrb_ctx** out) {
  if (!out) return fail(nullptr, MRB_EINVAL, "null output");
  *out = nullptr;
  int rc = check_config(cfg);
  if (rc != MRB_OK) return fail(nullptr, rc, "invalid configuration");
  if (!pool || ((uintptr_t)pool & 255)) return fail(nullptr, MRB_EINVAL, "pool must be non-null and 256-byte aligned");
  mrb_ctx* c = new mrb_ctx();
  c->cfg = *cfg;
  c->st = (cudaStream_t)cfg->stream;
  c->pool = (char*)pool;
  c->pool_bytes = pool_bytes;
  // largest slot count that fits
  int64_t lo = 0, hi = (int64_t)(pool_bytes / (slot_doubles() * 8)) + 1;
  while (lo < hi) {
    int64_t mid = (lo + hi + 1) / 2;
    if (mrb_pool_bytes(cfg, mid) <= pool_bytes) lo = mid;
    else hi = mid - 1;
  }
  c->nslots = lo;
  int64_t n0 = (int64_t)cfg->n_instances * cfg->base_blocks[0] * cfg->base_blocks[1] * cfg->base_blocks[2];
  if (c->nslots < n0) {
    delete c;
    return fail(nullptr, MRB_ECAPACITY, "pool smaller than the level-0 blocks");
  }
  rc = guarded(c, [&] {
    const size_t n = (size_t)c->nslots;
    char* q = c->pool;
    c->P.buf[0] = (double*)q;
    q += align256(n * SLOT_U * 8);
    c->P.buf[1] = (double*)q;
    q += align256(n * SLOT_U * 8);
    c->P.un = (double*)q;
    q += align256(n * SLOT_N * 8);
    c->P.face = (double*)q;
    q += align256(n * SLOT_F * 8);
    c->P.sel = (uint32_t*)q;
    q += align256(n * SLOT_SEL * 4);
    c->P.sh[0] = c->P.sh[1] = nullptr;
    if (cfg->precision == MRB_FP32_ACC64) {
      c->P.sh[0] = (float*)q;
      q += align256(n * SLOT_SH * 4);
      c->P.sh[1] = (float*)q;
      q += align256(n * SLOT_SH * 4);
      c->P.dl = (float*)q;
      q += align256(n * SLOT_N * 4);
    }
    c->P.fmac = nullptr;
    if (cfg->lts) c->P.fmac = (double*)q;
    Phys& p = c->phys;
    p.gamma = cfg->gamma;
    p.B = cfg->B;
    p.cfl = cfg->cfl;
    p.dx0 = cfg->dx0;
    p.inv_dx0 = 1.0 / cfg->dx0;
    p.eps = cfg->eps;
    p.mu = cfg->mu;
    for (int d = 0; d < 3; ++d) {
      p.grav[d] = cfg->gravity[d];
      p.nb[d] = cfg->base_blocks[d];
    }
    p.has_grav = (cfg->gravity[0] != 0.0 || cfg->gravity[1] != 0.0 || cfg->gravity[2] != 0.0) ? 1 : 0;
    for (int s = 0; s < 6; ++s) p.bc[s] = cfg->bc[s];
    p.n_inst = cfg->n_instances;
    p.recon = cfg->recon;
    p.precision = cfg->precision;
    p.rk = (cfg->rk_stages == 2) ? 2 : 3;
    p.flux = cfg->flux;
    p.mlp = (const float*)cfg->mlp_weights;
    p.mlp_tau = (float)cfg->mlp_tau;
    p.blocked = 0;
    p.lts = cfg->lts ? 1 : 0;
    c->max_lmax = 0;
    for (int i = 0; i < cfg->n_instances; ++i) c->max_lmax = std::max(c->max_lmax, (int)cfg->lmax[i]);
    c->d_keys = c->dalloc<uint64_t>(n);
    c->d_slot = c->dalloc<int32_t>(n);
    c->d_level = c->dalloc<int32_t>(n);
    c->d_inst = c->dalloc<int32_t>(n);
    c->d_X = c->dalloc<int32_t>(3 * n);
    c->d_parent = c->dalloc<int32_t>(n);
    c->d_child0 = c->dalloc<int32_t>(n);
    c->d_nbr = c->dalloc<int32_t>(27 * n);
    c->d_leaves = c->dalloc<int32_t>(n);
    c->d_lvl_nodes = c->dalloc<int32_t>(n);
    c->d_bc_items = c->dalloc<int32_t>(6 * n);
    c->d_jump = c->dalloc<int32_t>(n);
    c->d_cnt = c->dalloc<int32_t>(CNT_SIZE);
    c->d_lmax = c->dalloc<int32_t>(cfg->n_instances);
    c->d_list = c->dalloc<int32_t>(2 * n);
    c->d_dt = c->dalloc<double>(cfg->n_instances);
    c->d_smax = c->dalloc<unsigned long long>(4 * (size_t)cfg->n_instances);
    c->d_delta_node = c->dalloc<double>(n);
    c->d_partial = c->dalloc<double>(5 * n);
    c->d_tags = c->dalloc<int8_t>(n);
    c->d_status = c->dalloc<int>(1);
    c->d_lin = c->dalloc<unsigned long long>(2);
    // pinned staging of the topology uploads (keys, six int arrays of n, parent,
    // child0, leaves, level lists, boundary items of 6 n, counts) and of work lists
    if (cudaMallocHost((void**)&c->h_stage, 80 * n + 4 * CNT_SIZE + 256) != cudaSuccess ||
        cudaMallocHost((void**)&c->h_list, sizeof(int32_t) * 2 * n) != cudaSuccess)
      throw Err(MRB_ENOMEM, "pinned host staging");
    CK(cudaEventCreateWithFlags(&c->stage_ev, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&c->list_ev, cudaEventDisableTiming));
    p.lin_count = c->d_lin;
    p.lmax = c->d_lmax;
    CK(cudaMemsetAsync(c->d_lin, 0, 2 * sizeof(unsigned long long), c->st));
    CK(cudaMemcpyAsync(c->d_lmax, cfg->lmax, sizeof(int32_t) * cfg->n_instances, cudaMemcpyHostToDevice, c->st));
    CK(cudaMemsetAsync(c->d_status, 0, sizeof(int), c->st));
    CK(cudaMemsetAsync(c->d_cnt, 0, sizeof(int32_t) * CNT_SIZE, c->st));
    c->free_slots.clear();
    for (int64_t s = c->nslots - 1; s >= 0; --s) c->free_slots.push_back((int32_t)s);
    for (int inst = 0; inst < cfg->n_instances; ++inst)
      for (int z = 0; z < cfg->base_blocks[2]; ++z)
        for (int y = 0; y < cfg->base_blocks[1]; ++y)
          for (int x = 0; x < cfg->base_blocks[0]; ++x) {
            HNode a;
            a.inst = inst;
            a.level = 0;
            a.X[0] = x;
            a.X[1] = y;
            a.X[2] = z;
            a.key = make_key(inst, 0, a.X);
            a.slot = 0;
            c->nodes.push_back(a);
          }
    std::sort(c->nodes.begin(), c->nodes.end(), [](const HNode& a, const HNode& b) { return a.key < b.key; });
    for (auto& a : c->nodes) {
      a.slot = c->free_slots.back();
      c->free_slots.pop_back();
    }
    c->rebuild();
  });
  if (rc != MRB_OK) {
    c->destroy();
    delete c;
    return rc;
  }
  *out = c;
  return MRB_OK;
}

int mrb_n_blocks(mrb_ctx* c, int32_t level, int32_t leaves_only, int64_t* n) {
  return guarded(c, [&] {
    if (!n) throw Err(MRB_EINVAL, "null count");
    int64_t k = 0;
    for (size_t i = 0; i < c->nodes.size(); ++i) {
      if (level >= 0 && c->nodes[i].level != level) continue;
      if (leaves_only && c->h_child0[i] >= 0) continue;
      ++k;
    }
    *n = k;
  });
}

int mrb_list_blocks(mrb_ctx* c, int32_t level, int32_t leaves_only, uint64_t* keys_host, int64_t* geo_host,
                    int64_t cap, int64_t* n) {
  return guarded(c, [&] {
    int64_t k = 0;
    for (size_t i = 0; i < c->nodes.size(); ++i) {
      const HNode& a = c->nodes[i];
      if (level >= 0 && a.level != level) continue;
      if (leaves_only && c->h_child0[i] >= 0) continue;
      if (k < cap) {
        if (keys_host) keys_host[k] = a.key;
        if (geo_host) {
          geo_host[4 * k] = a.level;
          geo_host[4 * k + 1] = a.X[0];
          geo_host[4 * k + 2] = a.X[1];
          geo_host[4 * k + 3] = a.X[2];
        }
      }
      ++k;
    }
    if (n) *n = k;
    if (k > cap && (keys_host || geo_host)) throw Err(MRB_ECAPACITY, "list buffer too small");
  });
}

int mrb_set_state(mrb_ctx* c, const uint64_t* keys_host, int64_t n, const double* prim_dev) {
  return guarded(c, [&] {
    if (n < 0 || (n > 0 && (!keys_host || !prim_dev))) throw Err(MRB_EINVAL, "bad arguments");
    std::vector<int32_t> v = c->nodes_of(keys_host, n);
    c->upload_list(v);
    launch_set_state(c->topo(), c->phys, c->P, c->cur, c->d_list, (int)n, prim_dev, c->st);
    launch_shadow(c->topo(), c->phys, c->P, c->cur, SH_LIST, c->d_list, (int)n, 1, c->st);
    c->list_used();
  });
}

int mrb_set_cons(mrb_ctx* c, const uint64_t* keys_host, int64_t n, const double* cons_dev) {
  return guarded(c, [&] {
    if (n < 0 || (n > 0 && (!keys_host || !cons_dev))) throw Err(MRB_EINVAL, "bad arguments");
    std::vector<int32_t> v = c->nodes_of(keys_host, n);
    c->upload_list(v);
    launch_set_cons(c->topo(), c->P, c->cur, c->d_list, (int)n, cons_dev, c->st);
    launch_shadow(c->topo(), c->phys, c->P, c->cur, SH_LIST, c->d_list, (int)n, 1, c->st);
    c->list_used();
  });
}

int mrb_get_state(mrb_ctx* c, const uint64_t* keys_host, int64_t n, double* cons_dev, int32_t with_halo) {
  return guarded(c, [&] {
    if (n < 0 || (n > 0 && (!keys_host || !cons_dev))) throw Err(MRB_EINVAL, "bad arguments");
    std::vector<int32_t> v = c->nodes_of(keys_host, n);
    c->upload_list(v);
    launch_get_state(c->topo(), c->P, c->cur, c->d_list, (int)n, cons_dev, with_halo ? 1 : 0, c->st);
    c->list_used();
  });
}

int mrb_get_records(mrb_ctx* c, const uint64_t* keys_host, int64_t n, float* records_dev, int32_t fresh) {
  return guarded(c, [&] {
    if (!c->P.sh[0]) throw Err(MRB_EINVAL, "no FP32 records in an FP64 context");
    if (n < 0 || (n > 0 && (!keys_host || !records_dev))) throw Err(MRB_EINVAL, "bad arguments");
    std::vector<int32_t> v = c->nodes_of(keys_host, n);
    c->upload_list(v);
    launch_get_records(c->topo(), c->phys, c->P, c->cur, c->d_list, (int)n, records_dev, fresh ? 1 : 0, c->st);
    c->list_used();
  });
}

int mrb_fill_halos(mrb_ctx* c) {
  return guarded(c, [&] { c->fill_halos(); });
}

int mrb_compute_rhs(mrb_ctx* c, double* rhs_dev) {
  return guarded(c, [&] {
    if (!rhs_dev) throw Err(MRB_EINVAL, "null rhs");
    if (c->cfg.precision == MRB_FP32_ACC64) launch_rhs_rk_f32(c->topo(), c->phys, c->P, c->cur, 0, nullptr, rhs_dev, c->st);
    else launch_rhs_rk_f64(c->topo(), c->phys, c->P, c->cur, 0, nullptr, rhs_dev, c->st);
    for (int l = c->max_lmax - 1; l >= 0; --l) launch_face_avg_level(c->topo(), c->P, l, c->st);
    launch_jump(c->topo(), c->phys, c->P, c->cur, 0, nullptr, rhs_dev, c->st);
  });
}

int mrb_rk_stage(mrb_ctx* c, int32_t stage, const double* dt_dev) {
  return guarded(c, [&] {
    if (stage < 0 || stage >= c->phys.rk || !dt_dev) throw Err(MRB_EINVAL, "bad stage or dt");
    c->stage(stage, dt_dev);
  });
}

int mrb_cfl_dt(mrb_ctx* c, double* dt_dev) {
  return guarded(c, [&] {
    if (!dt_dev) throw Err(MRB_EINVAL, "null dt");
    launch_cfl(c->topo(), c->phys, c->P, c->cur, c->d_smax, dt_dev, c->d_status, c->st);
  });
}

int mrb_mr_project(mrb_ctx* c) {
  return guarded(c, [&] { c->project(); });
}

int mrb_mr_predict_and_tag(mrb_ctx* c, int32_t allow_refine, int8_t* tags_dev, double* delta_dev) {
  return guarded(c, [&] {
    if (!tags_dev) throw Err(MRB_EINVAL, "null tags");
    launch_delta_tags(c->topo(), c->phys, c->P, c->cur, c->d_delta_node, allow_refine ? 1 : 0, tags_dev, delta_dev,
                      c->n_leaves(), c->st);
  });
}

int mrb_remesh(mrb_ctx* c, const int8_t* tags_dev, int64_t* n_leaves) {
  int rc = guarded(c, [&] {
    if (!tags_dev && c->n_leaves() > 0) throw Err(MRB_EINVAL, "null tags");
    int64_t nl = c->remesh(tags_dev);
    if (n_leaves) *n_leaves = nl;
    CK(cudaStreamSynchronize(c->st));
  });
  if (rc != MRB_OK) return rc;
  int st = 0;
  cudaMemcpy(&st, c->d_status, sizeof(int), cudaMemcpyDeviceToHost);
  return st ? fail(c, st, "device status set") : MRB_OK;
}

// Refinement of chosen leaves (Alg. Initialization's "refine all blocks of
// level m-1", and restoring a saved tree): full halo fill, REFINE tags for the
// selected leaves, remesh (children predicted from their parent).
namespace {
int refine_where(mrb_ctx* c, const std::vector<int8_t>& tags, int64_t* n_leaves) {
  int rc = guarded(c, [&] {
    c->fill_halos();
    c->detail_filled = false;
    if (!tags.empty()) CK(cudaMemcpyAsync(c->d_tags, tags.data(), tags.size(), cudaMemcpyHostToDevice, c->st));
    int64_t nl = c->remesh(c->d_tags);
    if (n_leaves) *n_leaves = nl;
    CK(cudaStreamSynchronize(c->st));
  });
  return rc;
}
}  // namespace

int mrb_refine_level(mrb_ctx* c, int32_t level, int64_t* n_leaves) {
  if (!c) return fail(nullptr, MRB_EINVAL, "null context");
  if (level < 0 || level > MRB_MAX_LEVEL) return fail(c, MRB_EINVAL, "bad level");
  std::vector<int8_t> tags((size_t)c->n_leaves());
  for (int li = 0; li < c->n_leaves(); ++li)
    tags[li] = (c->nodes[c->h_leaves[li]].level == level) ? (int8_t)MRB_TAG_REFINE : (int8_t)MRB_TAG_KEEP;
  return refine_where(c, tags, n_leaves);
}

int mrb_refine_keys(mrb_ctx* c, const uint64_t* keys_host, int64_t n, int64_t* n_leaves) {
  if (!c) return fail(nullptr, MRB_EINVAL, "null context");
  if (n < 0 || (n > 0 && !keys_host)) return fail(c, MRB_EINVAL, "bad arguments");
  std::vector<int8_t> tags((size_t)c->n_leaves(), (int8_t)MRB_TAG_KEEP);
  for (int64_t b = 0; b < n; ++b) {
    const int64_t i = c->find(keys_host[b]);
    const auto it = (i < 0) ? c->h_leaves.end() : std::lower_bound(c->h_leaves.begin(), c->h_leaves.end(), (int32_t)i);
    if (it == c->h_leaves.end() || *it != i) return fail(c, MRB_EINVAL, "not the id of a leaf");
    tags[it - c->h_leaves.begin()] = (int8_t)MRB_TAG_REFINE;
  }
  return refine_where(c, tags, n_leaves);
}

int mrb_step(mrb_ctx* c, int32_t nsteps, double* dt_hist_dev) {
  return guarded(c, [&] {
    bool mr = c->max_lmax > 0;
    for (int s = 0; s < nsteps; ++s) {
      const int g = c->cur;
      if (c->phys.lts) {
        c->step_lts();
      } else {
        if (c->graph_dirty) c->capture_graphs();
        CK(cudaGraphLaunch(c->graph[g], c->st));
        g_kernel_launches += c->graph_kernels[g];
        if (c->phys.rk & 1) c->cur ^= 1;   // every stage flips the stage buffer
      }
      if (dt_hist_dev)
        CK(cudaMemcpyAsync(dt_hist_dev + (size_t)s * c->cfg.n_instances, c->d_dt, sizeof(double) * c->cfg.n_instances,
                           cudaMemcpyDeviceToDevice, c->st));
      if (mr) {
        c->fill_halos(FILL_DETAIL);
        c->detail_filled = true;
        launch_delta_tags(c->topo(), c->phys, c->P, c->cur, c->d_delta_node, 1, c->d_tags, nullptr, c->n_leaves(),
                          c->st);
        c->remesh(c->d_tags);
      }
      if (c->prof && !c->phys.lts) {   // (the macro steps of local time stepping are not profiled per stage)
        CK(cudaStreamSynchronize(c->st));
        for (int q = 0; q < c->phys.rk; ++q) {
          float ms = 0.f;
          CK(cudaEventElapsedTime(&ms, c->gev[g][q][0], c->gev[g][q][1]));
          c->prof_ms += ms;
          c->prof_rhs += 1;
        }
      }
    }
  });
}

int mrb_face_samples(mrb_ctx* c, float tau_lab, int64_t stride, float* feats_dev, uint8_t* labels_dev,
                     int64_t* where_dev, int64_t cap, int64_t* n_out) {
  return guarded(c, [&] {
    if (stride < 1 || cap < 0 || (cap > 0 && (!feats_dev || !labels_dev))) throw Err(MRB_EINVAL, "bad arguments");
    const int64_t faces = (int64_t)c->n_leaves() * 3 * 17 * 256;
    const int64_t n = std::min<int64_t>(cap, (faces + stride - 1) / stride);
    if (n > 0) launch_face_samples(c->topo(), c->phys, c->P, c->cur, tau_lab, stride, feats_dev, labels_dev, where_dev, n,
                                   c->st);
    if (n_out) *n_out = n;
  });
}

int mrb_learned_stats(mrb_ctx* c, int64_t* linear_faces, int64_t* evaluated_faces, int32_t reset) {
  return guarded(c, [&] {
    unsigned long long h[2] = {0, 0};
    CK(cudaStreamSynchronize(c->st));
    CK(cudaMemcpy(h, c->d_lin, sizeof(h), cudaMemcpyDeviceToHost));
    if (linear_faces) *linear_faces = (int64_t)h[0];
    if (evaluated_faces) *evaluated_faces = (int64_t)h[1];
    if (reset) CK(cudaMemset(c->d_lin, 0, sizeof(h)));
  });
}

int mrb_profile(mrb_ctx* c, int32_t enable) {
  return guarded(c, [&] {
    CK(cudaStreamSynchronize(c->st));
    for (auto& pr : c->pend) {
      cudaEventDestroy(pr.first);
      cudaEventDestroy(pr.second);
    }
    c->pend.clear();
    c->prof = enable != 0;
    c->prof_ms = 0.0;
    c->prof_rhs = 0;
    c->prof_base = g_kernel_launches;
  });
}

int mrb_profile_read(mrb_ctx* c, double* ms, int64_t* n_rhs, int64_t* n_kernels) {
  return guarded(c, [&] {
    CK(cudaStreamSynchronize(c->st));
    for (auto& pr : c->pend) {
      float t = 0.f;
      CK(cudaEventElapsedTime(&t, pr.first, pr.second));
      c->prof_ms += t;
      c->prof_rhs += 1;
      cudaEventDestroy(pr.first);
      cudaEventDestroy(pr.second);
    }
    c->pend.clear();
    if (ms) *ms = c->prof_ms;
    if (n_rhs) *n_rhs = c->prof_rhs;
    if (n_kernels) *n_kernels = g_kernel_launches - c->prof_base;
  });
}

int mrb_sums(mrb_ctx* c, double* sums_dev) {
  return guarded(c, [&] {
    if (!sums_dev) throw Err(MRB_EINVAL, "null sums");
    launch_sums(c->topo(), c->phys, c->P, c->cur, c->d_partial, sums_dev, c->n_leaves(), c->st);
  });
}

int mrb_flux_census(mrb_ctx* c, uint64_t* counts_host) {
  return guarded(c, [&] {
    if (!counts_host) throw Err(MRB_EINVAL, "null counts");
    if (!c->d_census) c->d_census = c->dalloc<unsigned long long>(6);
    launch_flux_census(c->topo(), c->phys, c->P, c->cur, c->d_census, c->st);
    CK(cudaMemcpyAsync(counts_host, c->d_census, 6 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
  });
}

int mrb_neighbors(mrb_ctx* c, const uint64_t* keys_host, int64_t n, uint64_t* nbr_host) {
  return guarded(c, [&] {
    std::vector<int32_t> idx = c->nodes_of(keys_host, n);
    std::vector<int32_t> all((size_t)c->nodes.size() * 27);
    CK(cudaStreamSynchronize(c->st));
    CK(cudaMemcpy(all.data(), c->d_nbr, sizeof(int32_t) * all.size(), cudaMemcpyDeviceToHost));
    for (int64_t b = 0; b < n; ++b)
      for (int r = 0; r < 27; ++r) {
        const int32_t v = all[(size_t)idx[b] * 27 + r];
        nbr_host[b * 27 + r] = (v >= 0) ? c->nodes[v].key : (v == -1 ? 0ull : 1ull);
      }
  });
}

int mrb_get_tune(mrb_ctx* c, int32_t* params) {
  return guarded(c, [&] {
    if (!params) throw Err(MRB_EINVAL, "null params");
    params[0] = c->tune.stage_waves;
    params[1] = c->phys.blocked;
    params[2] = c->tune.fill_copy;
    params[3] = c->tune.fill_pred;
    params[4] = c->tune.project;
  });
}

namespace {
bool tune_ok(const int32_t* q) {
  return q[0] >= 1 && q[0] <= 8 && (q[1] == 0 || q[1] == 1) && q[2] >= 1 && q[2] <= 32 && q[3] >= 1 && q[3] <= 32 &&
         q[4] >= 1 && q[4] <= 32;
}
void apply_tune(mrb_ctx* c, const int32_t* q) {
  c->tune = Tune{q[0], q[2], q[3], q[4]};
  c->phys.blocked = q[1];
  g_tune = c->tune;
  c->graph_dirty = true;     // the replayed graphs hold launch shapes and kernel arguments
}
}  // namespace

int mrb_set_tune(mrb_ctx* c, const int32_t* params) {
  return guarded(c, [&] {
    if (!params || !tune_ok(params)) throw Err(MRB_EINVAL, "launch shape out of range");
    apply_tune(c, params);
  });
}

// Scheduling-only search: each candidate is timed with CUDA events on the
// context's stream over `reps` repetitions of work that leaves the
// simulation state unchanged -- stage 0 (and, with the learned selector, a
// stage 1 after it) from the current stage buffer, whose writes go to the
// other stage buffer and the per-step scratch (u^n, face fluxes, decisions,
// FP32 records of the other buffer); the halo fill of the current buffer;
// the averaging (the same averages again).  Coordinate search: stage waves
// and item order, then fill shapes, then averaging shape.
int mrb_autotune(mrb_ctx* c, int32_t reps, double* times) {
  return guarded(c, [&] {
    if (reps < 1) throw Err(MRB_EINVAL, "reps < 1");
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    const int fmode = (c->cfg.precision == MRB_FP32_ACC64 && !(c->cfg.mu > 0.0)) ? FILL_STAGE : FILL_FULL;
    launch_cfl(c->topo(), c->phys, c->P, c->cur, c->d_smax, c->d_dt, c->d_status, c->st);
    auto run = [&](int what) {
      if (what == 0) {
        if (c->cfg.precision == MRB_FP32_ACC64) {
          launch_rhs_rk_f32(c->topo(), c->phys, c->P, c->cur, 0, c->d_dt, nullptr, c->st);
          if (c->cfg.recon == MRB_RECON_LEARNED && c->cfg.mlp_weights)
            launch_rhs_rk_f32(c->topo(), c->phys, c->P, c->cur, 1, c->d_dt, nullptr, c->st);
        } else {
          launch_rhs_rk_f64(c->topo(), c->phys, c->P, c->cur, 0, c->d_dt, nullptr, c->st);
        }
      } else if (what == 1) {
        c->fill_halos(fmode);
      } else {
        c->project();
      }
    };
    auto time_of = [&](int what, const int32_t* q) {
      apply_tune(c, q);
      run(what);   // warm-up
      CK(cudaEventRecord(e0, c->st));
      for (int r = 0; r < reps; ++r) run(what);
      CK(cudaEventRecord(e1, c->st));
      CK(cudaEventSynchronize(e1));
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, e0, e1));
      return (double)ms / reps;
    };
    int32_t best[5] = {c->tune.stage_waves, c->phys.blocked, c->tune.fill_copy, c->tune.fill_pred, c->tune.project};
    const int32_t def[5] = {1, 0, 8, 4, 8};
    double t_def[3], t_best[3];
    for (int what = 0; what < 3; ++what) t_def[what] = time_of(what, def);
    std::copy(def, def + 5, best);
    t_best[0] = t_def[0];
    for (int w : {1, 2, 4})
      for (int b : {0, 1}) {
        int32_t q[5] = {w, b, best[2], best[3], best[4]};
        const double tt = time_of(0, q);
        if (tt < t_best[0]) { t_best[0] = tt; best[0] = w; best[1] = b; }
      }
    t_best[1] = t_def[1];
    for (int fc : {4, 8, 16})
      for (int fp : {2, 4, 8}) {
        int32_t q[5] = {best[0], best[1], fc, fp, best[4]};
        const double tt = time_of(1, q);
        if (tt < t_best[1]) { t_best[1] = tt; best[2] = fc; best[3] = fp; }
      }
    t_best[2] = t_def[2];
    for (int pr : {4, 8, 16}) {
      int32_t q[5] = {best[0], best[1], best[2], best[3], pr};
      const double tt = time_of(2, q);
      if (tt < t_best[2]) { t_best[2] = tt; best[4] = pr; }
    }
    apply_tune(c, best);
    CK(cudaMemsetAsync(c->d_lin, 0, 2 * sizeof(unsigned long long), c->st));   // the timed launches' selector counts
    CK(cudaStreamSynchronize(c->st));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (times)
      for (int what = 0; what < 3; ++what) {
        times[2 * what] = t_def[what];
        times[2 * what + 1] = t_best[what];
      }
  });
}

int mrb_status(mrb_ctx* c) {
  if (!c) return MRB_EINVAL;
  int st = 0;
  if (cudaStreamSynchronize(c->st) != cudaSuccess) return fail(c, MRB_ECUDA, "stream synchronisation failed");
  if (cudaMemcpy(&st, c->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail(c, MRB_ECUDA, "status read failed");
  return st;
}

int mrb_sync(mrb_ctx* c) {
  if (!c) return MRB_EINVAL;
  cudaError_t e = cudaStreamSynchronize(c->st);
  if (e != cudaSuccess) return fail(c, MRB_ECUDA, cudaGetErrorString(e));
  int st = mrb_status(c);
  if (st) return fail(c, st, "device status set");
  return MRB_OK;
}

int mrb_clear_status(mrb_ctx* c) {
  return guarded(c, [&] {
    CK(cudaStreamSynchronize(c->st));
    CK(cudaMemset(c->d_status, 0, sizeof(int)));
  });
}

int mrb_destroy(mrb_ctx* c) {
  if (!c) return MRB_EINVAL;
  cudaStreamSynchronize(c->st);
  c->destroy();
  delete c;
  return MRB_OK;
}

const char* mrb_last_error(mrb_ctx* c) {
  if (c) return c->err.c_str();
  return g_last_error.c_str();
}

}  // extern "C"
