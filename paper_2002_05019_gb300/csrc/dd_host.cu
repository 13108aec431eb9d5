// Host side of the GB300 direct domain-decomposition solver: the C ABI of
// include/dd.h, input validation, the symbolic analysis of the arrowhead
// system, device memory, and the launch schedule of factor and solve.
//
// Symbolic analysis (Section II: the block structure of the auxiliary factor
// comes from a symbolic factorization over the clique graph of its blocks):
//   * each domain's unknowns are ordered interior first, interface last, so
//     that the rows of B_i only meet the last n_Gamma columns of L_i;
//   * every domain is a clique over the duals it touches; a dual coupling a set
//     of domains is eliminated at the lowest common ancestor of those domains in
//     the binary domain tree (a nested-dissection order of the dual unknowns:
//     separators after their subtrees);
//   * the front of a tree node holds its separator duals followed by the
//     ancestor duals reached through its subtree's cliques; that structure is
//     the block fill of the auxiliary factor.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <numeric>
#include <vector>

#include "../../include/dd.h"
#include "../../include/dd_diag.h"
#include "dd_internal.h"

namespace {

constexpr int T = DD_TILE;
constexpr int kSolveBlock = 64;   // right-hand sides per direct-solve pass
constexpr int kAheadMaxFronts = 1024;  // look-ahead is possible on levels with at most this many fronts
constexpr int kNormBlocks = 16;   // reduction blocks per column for the refinement norms

inline int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// Front tree of one sparse domain (dd_domain_assembly): local fronts 0..nf-1,
// children before parents; gid maps them to the handle's fronts (root -> the
// domain id).  nf == 0: the domain is one dense front.
struct SparseDomain {
  int nf = 0, root = -1;
  int64_t vec_off = 0;                 // the domain's first row in the stacked primal vector
  std::vector<int32_t> parent, ne, rows, a_front, gid;
  std::vector<int64_t> rows_ptr;
};

struct StepRange {
  int k;
  int64_t diag_off, trsm_off, upd_off, tc_off;
  int n_diag, n_trsm, n_upd, n_tc;
  int n_upd_next, n_tc_next;   // the first tasks of each list update only the next panel column (j = k + 1)
  int64_t grp_off;             // tensor-core task groups: next-column groups then the rest
  int n_grp_next, n_grp_rest;
};

// mixed form, tensor cores: the trailing update of panels k and k + 1 in one
// pass (K = 128) over the columns j >= k + 2; "near" tasks are the columns
// k + 2 and k + 3 (the next pair's panels), "far" tasks the rest
struct PairRange {
  int k;
  int64_t tc2_off;
  int n_near, n_far;
  int64_t grp_off;
  int n_grp_near, n_grp_far;
};

// four-panel updates of steps k .. k + 3 (k = 0, 4, 8, ...): near = columns
// k + 2, k + 3 with panels k, k + 1; far = columns >= k + 4 with all four
struct QuadRange {
  int k;
  int64_t tc_off;
  int n_near, n_far;          // far = columns >= k + 4: first n_far4 of them columns k + 4 .. k + 7
  int n_far4;
  int64_t grp_off;
  int n_grp_near, n_grp_far, n_grp_far4;
};

struct Level {
  std::vector<int32_t> ids;       // fronts in this level
  int64_t ids_off = 0;            // offset into d_level_ids
  std::vector<StepRange> steps;   // factor schedule
  std::vector<PairRange> pairs;   // two-panel updates of steps (0, 1), (2, 3), ... (tensor-core path)
  std::vector<QuadRange> quads;   // four-panel updates of steps (0..3), (4..7), ... (tensor-core path)
  bool ahead = false;             // one-step look-ahead on a second stream
  int max_child_nu = 0;
  int max_ld = 0;                 // largest separator front (pull assembly grid)
  int64_t fwd_off = 0, bwd_off = 0;   // solve tasks (forward by row tile, backward by column tile)
  int n_fwd = 0, n_bwd = 0;
  int upd_split = 0;   // separator levels: CTAs per backward task of the split update-row product
  int n_aux = 0;       // separator fronts of the auxiliary matrix here (the others eliminate domain unknowns)
};

struct DeviceArena {
  std::vector<void*> ptrs;
  size_t bytes = 0;
  template <typename X>
  cudaError_t alloc(X** p, size_t count) {
    *p = nullptr;
    if (count == 0) return cudaSuccess;
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, count * sizeof(X));
    if (e != cudaSuccess) return e;
    ptrs.push_back(q);
    bytes += count * sizeof(X);
    *p = static_cast<X*>(q);
    return cudaSuccess;
  }
  template <typename X>
  cudaError_t upload(X** p, const std::vector<X>& v, cudaStream_t s) {
    cudaError_t e = alloc(p, v.size());
    if (e != cudaSuccess || v.empty()) return e;
    return cudaMemcpyAsync(*p, v.data(), v.size() * sizeof(X), cudaMemcpyHostToDevice, s);
  }
  void release() {
    for (void* q : ptrs) cudaFree(q);
    ptrs.clear();
    bytes = 0;
  }
};

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

struct dd_handle {
  int device = 0;
  cudaStream_t stream = nullptr;
  int prec = DD_PREC_FP64;
  double refine_tol = 1e-13;
  int max_refine = 0;
  int n_sub = 0, n_dual = 0;
  int n_sparse = 0;        // domains factored as nested-dissection front trees
  int64_t ld_lam = 0;      // rows of the solve's row-id vector: n_dual, + n_loc with sparse domains
  int64_t n_scatter = 0;   // entries of the sparse domains' front initialisation
  int64_t* d_sp_dst = nullptr;
  int32_t* d_sp_src = nullptr;
  int32_t* d_lvl0_sparse = nullptr;   // sparse-domain fronts of tree level 0
  int n_lvl0_sparse = 0;
  int64_t n_loc = 0, nnz_total = 0;
  size_t elem = 16;  // bytes per stored complex

  // symbolic
  std::vector<FrontDev> fronts;
  std::vector<Level> levels;
  std::vector<std::vector<int32_t>> leaf_duals;  // sorted duals of each domain
  std::vector<std::vector<int32_t>> leaf_upd;    // the same duals in the front's B-row order
  std::vector<int64_t> leaf_vec_off;
  std::vector<LeafDev> h_leaves_copy;   // for subset recovery
  std::vector<Task> h_bwd_leaf;         // level-0 backward tasks (front, tile)
  cudaGraphExec_t factor_exec = nullptr; // the captured factorization (no per-launch timing)
  int factor_graph_launches = 0;
  size_t fact_nev = 0;                  // timed event pairs in the graph and the class of each
  std::vector<int> fact_cls;
  void* d_sub = nullptr;                // subset recovery scratch (tasks, leaves, segments, rows)
  size_t sub_cap = 0;
  double max_abs_a = 1.0;
  int64_t rows_total = 0;  // sum of front orders (right-hand-side rows)

  // device
  DeviceArena arena;
  void* pool = nullptr;
  size_t pool_bytes = 0;
  FrontDev* d_fronts = nullptr;
  LeafDev* d_leaves = nullptr;
  int32_t *d_rowptr = nullptr, *d_colind = nullptr;
  double2* d_val = nullptr;
  int32_t *d_iperm = nullptr, *d_perm = nullptr;
  int32_t *d_brow = nullptr, *d_blocal = nullptr;
  int8_t* d_bsign = nullptr;
  int32_t *d_blptr = nullptr, *d_bldual = nullptr;
  int8_t* d_blsign = nullptr;
  int32_t* d_btptr = nullptr;
  int64_t* d_btrow = nullptr;
  int8_t* d_btsign = nullptr;
  int32_t *d_upd = nullptr, *d_sep = nullptr, *d_maps = nullptr;
  int32_t* d_imaps = nullptr;      // separator fronts: row -> child update row (-1: none), per child
  int2* d_ztiles = nullptr;        // (front, tile row) of the fronts zeroed before each factorization
  int64_t n_ztiles = 0;
  int32_t *d_level_ids = nullptr, *d_diag_ids = nullptr;
  Task *d_trsm = nullptr, *d_updt = nullptr;
  Task *d_fwd = nullptr, *d_bwd = nullptr;
  Task* d_tc = nullptr;            // tensor-core update tasks (mixed form)
  Task* d_tc2 = nullptr;           // two-panel tensor-core update tasks
  int2* d_grp = nullptr;           // their groups (first task, count): runs of tasks of one row tile
  int* d_counters = nullptr;       // one group counter per tensor-core update launch of a factor
  int n_counters = 0;
  unsigned char* d_ws = nullptr;   // panel operand images (mixed form), four slots
  size_t ws_slot_off[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  float2* d_linv = nullptr;        // mixed form: L_kk^{-1} of every diagonal tile (index tile_off + k)
  uint8_t* d_piv = nullptr;        // restricted Bunch-Kaufman: permutation of every diagonal tile (64 bytes each)
  int pivoting = 0;
  cudaStream_t s2 = nullptr;       // look-ahead: bulk trailing updates run here
  cudaStream_t own_stream = nullptr;  // created when the caller gives no stream
  cudaEvent_t ev_panel = nullptr, ev_rest = nullptr;
  size_t ws_bytes = 0;
  int use_tc = 0;
  bool pair_panels = false;        // two-panel trailing updates (K = 128)
  bool quad_panels = false;        // four-panel trailing updates (K = 256) on levels without look-ahead
  // schedule knobs of the tensor-core path (dd_autotune picks them)
  int ahead_fronts = 32;           // look-ahead on levels with at most this many fronts (0: off)
  int reserve_sms = 16;            // SMs the look-ahead leaves to the panel chain
  int split_sms = 0;               // > 0: the leaf level as two halves on two streams, each update
                                   // leaving this many SMs to the other half's panel chain
  std::vector<Level> halves;       // the leaf level's fronts in two halves of about equal work
  uint64_t tune_key = 0;           // problem key of the schedule cache (front tree, duals, form)
  std::string tune_cache;          // path of the schedule cache ("": none)
  int32_t *d_flag_f = nullptr, *d_flag_b = nullptr;
  int64_t n_tiles = 0;
  int epoch = 0;
  DevStatus* d_status = nullptr;
  DevStatus* d_solve_status = nullptr;
  double* d_partials = nullptr;

  // solve work (grown on demand, freed with the handle)
  int nrhs_cap = 0;
  // captured direct solve (a) and refinement step (b) per right-hand-side count
  struct SolveGraphs {
    cudaGraphExec_t a = nullptr, b = nullptr;
    int la = 0, lb = 0;
  };
  std::map<int, SolveGraphs> solve_graphs;
  void drop_solve_graphs() {
    for (auto& kv : solve_graphs) {
      if (kv.second.a) cudaGraphExecDestroy(kv.second.a);
      if (kv.second.b) cudaGraphExecDestroy(kv.second.b);
    }
    solve_graphs.clear();
  }
  void* rpool = nullptr;
  void* lam_work = nullptr;
  void* upd_part = nullptr;   // update-row partial sums of the backward substitution
  double2 *d_f = nullptr, *d_u = nullptr, *d_r = nullptr, *d_du = nullptr;
  double2 *d_lam = nullptr, *d_dlam = nullptr, *d_g = nullptr;
  std::vector<void*> work_ptrs;

  bool factored = false;
  int time_kernels = 0;
  std::vector<cudaEvent_t> kev;   // event pairs for per-launch timing
  dd_stats stats{};
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  int launches = 0;

  ~dd_handle() {
    if (factor_exec) cudaGraphExecDestroy(factor_exec);
    drop_solve_graphs();
    for (void* q : work_ptrs) cudaFree(q);
    if (d_sub) cudaFree(d_sub);
    arena.release();
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    for (cudaEvent_t e : kev) cudaEventDestroy(e);
    if (ev_panel) cudaEventDestroy(ev_panel);
    if (ev_rest) cudaEventDestroy(ev_rest);
    if (s2) cudaStreamDestroy(s2);
    if (own_stream) cudaStreamDestroy(own_stream);
  }
};

namespace {

int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return DD_OK;
  if (e == cudaErrorMemoryAllocation) return DD_ERR_OOM;
  return DD_ERR_CUDA;
}

#define DD_CUDA(call)                          \
  do {                                         \
    cudaError_t _e = (call);                   \
    if (_e != cudaSuccess) return cuda_status(_e); \
  } while (0)

// ---------------------------------------------------------------------------
// validation
// ---------------------------------------------------------------------------
int validate_subdomain(const dd_subdomain& s, int32_t n_dual, double* max_abs) {
  if (s.n < 1 || !s.rowptr || s.nb < 0) return DD_ERR_INVALID_ARG;
  if (s.rowptr[0] != 0) return DD_ERR_INVALID_ARG;
  const int64_t nnz = s.rowptr[s.n];
  if (nnz < 0 || (nnz > 0 && (!s.colind || !s.val))) return DD_ERR_INVALID_ARG;
  if (s.nb > 0 && (!s.b_dual || !s.b_local || !s.b_sign)) return DD_ERR_INVALID_ARG;
  double amax = 0.0;
  for (int r = 0; r < s.n; ++r) {
    if (s.rowptr[r + 1] < s.rowptr[r]) return DD_ERR_INVALID_ARG;
    bool diag = false;
    for (int32_t q = s.rowptr[r]; q < s.rowptr[r + 1]; ++q) {
      const int32_t c = s.colind[q];
      if (c < 0 || c >= s.n) return DD_ERR_INVALID_ARG;
      if (q > s.rowptr[r] && c <= s.colind[q - 1]) return DD_ERR_INVALID_ARG;
      if (!std::isfinite(s.val[q].re) || !std::isfinite(s.val[q].im)) return DD_ERR_INVALID_ARG;
      amax = std::max(amax, std::hypot(s.val[q].re, s.val[q].im));
      diag |= (c == r);
    }
    if (!diag) return DD_ERR_INVALID_ARG;  // every diagonal entry must be stored
  }
  // symmetry A = A^T (pattern and values, relative 1e-12)
  for (int r = 0; r < s.n; ++r) {
    for (int32_t q = s.rowptr[r]; q < s.rowptr[r + 1]; ++q) {
      const int32_t c = s.colind[q];
      const int32_t* b = s.colind + s.rowptr[c];
      const int32_t* e = s.colind + s.rowptr[c + 1];
      const int32_t* it = std::lower_bound(b, e, r);
      if (it == e || *it != r) return DD_ERR_NOT_SYMMETRIC;
      const dd_c128 v = s.val[q], w = s.val[s.rowptr[c] + (it - b)];
      if (std::hypot(v.re - w.re, v.im - w.im) > 1e-12 * amax) return DD_ERR_NOT_SYMMETRIC;
    }
  }
  for (int q = 0; q < s.nb; ++q) {
    if (s.b_dual[q] < 0 || s.b_dual[q] >= n_dual) return DD_ERR_INVALID_ARG;
    if (s.b_local[q] < 0 || s.b_local[q] >= s.n) return DD_ERR_INVALID_ARG;
    if (s.b_sign[q] != 1 && s.b_sign[q] != -1) return DD_ERR_INVALID_ARG;
  }
  *max_abs = amax;
  return DD_OK;
}

// binary domain tree: parent[] over 2*ns-1 nodes, leaves 0..ns-1
int build_tree(int ns, const dd_options* opt, std::vector<int32_t>& parent) {
  const int nn = 2 * ns - 1;
  parent.assign(nn, -1);
  if (opt && opt->tree_parent) {
    std::vector<int> nchild(nn, 0);
    for (int x = 0; x < nn; ++x) {
      const int p = opt->tree_parent[x];
      if (x == nn - 1) {
        if (p != -1) return DD_ERR_INVALID_ARG;
        continue;
      }
      if (p <= x || p < ns || p >= nn) return DD_ERR_INVALID_ARG;
      nchild[p]++;
      parent[x] = p;
    }
    for (int x = ns; x < nn; ++x)
      if (nchild[x] != 2) return DD_ERR_INVALID_ARG;
    return DD_OK;
  }
  // recursive bisection of the domain centroids (longest extent, median split),
  // or of the index range when no centroids are given; ids in post-order
  int next = ns;
  std::vector<int32_t> ids(ns);
  std::iota(ids.begin(), ids.end(), 0);
  const double* cen = opt ? opt->centroids : nullptr;
  struct Rec {
    static int go(std::vector<int32_t>& v, int lo, int hi, const double* cen, int& next, std::vector<int32_t>& par) {
      if (hi - lo == 1) return v[lo];
      if (cen) {
        double mn[3] = {1e300, 1e300, 1e300}, mx[3] = {-1e300, -1e300, -1e300};
        for (int q = lo; q < hi; ++q)
          for (int a = 0; a < 3; ++a) {
            mn[a] = std::min(mn[a], cen[3 * v[q] + a]);
            mx[a] = std::max(mx[a], cen[3 * v[q] + a]);
          }
        int ax = 0;
        for (int a = 1; a < 3; ++a)
          if (mx[a] - mn[a] > mx[ax] - mn[ax]) ax = a;
        std::stable_sort(v.begin() + lo, v.begin() + hi, [&](int32_t x, int32_t y) {
          return cen[3 * x + ax] < cen[3 * y + ax] || (cen[3 * x + ax] == cen[3 * y + ax] && x < y);
        });
      }
      const int mid = lo + (hi - lo) / 2;
      const int a = go(v, lo, mid, cen, next, par);
      const int b = go(v, mid, hi, cen, next, par);
      const int me = next++;
      par[a] = me;
      par[b] = me;
      return me;
    }
  };
  if (ns > 1) Rec::go(ids, 0, ns, cen, next, parent);
  return DD_OK;
}

void add_flops(dd_handle* h, double ne, double nu, double n_gamma, bool leaf) {
  if (leaf) {
    h->stats.flops_factor += (4.0 / 3.0) * ne * ne * ne + 4.0 * n_gamma * n_gamma * nu + 4.0 * n_gamma * nu * nu;
  } else {
    h->stats.flops_factor += (4.0 / 3.0) * ne * ne * ne + 4.0 * ne * ne * nu + 4.0 * ne * nu * nu;
  }
  h->stats.flops_solve += 8.0 * (ne * ne + 2.0 * ne * nu);
}

int ensure_work(dd_handle* h, int nrhs) {
  if (nrhs <= h->nrhs_cap) return DD_OK;
  h->drop_solve_graphs();   // they refer to the buffers freed here
  for (void* q : h->work_ptrs) cudaFree(q);
  h->work_ptrs.clear();
  h->nrhs_cap = 0;
  auto get = [&](void** p, size_t bytes) -> cudaError_t {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) h->work_ptrs.push_back(*p);
    return e;
  };
  const size_t nr = (size_t)nrhs;
  DD_CUDA(get(&h->rpool, (size_t)h->rows_total * nr * h->elem));
  DD_CUDA(get(&h->lam_work, (size_t)h->ld_lam * nr * h->elem));
  // separator levels of few tiles (their substitution is a chain whose first
  // tile waits for its update-row product): split the update rows of each
  // backward task over enough CTAs to fill the GPU about four times, at least
  // 128 rows per CTA.  Levels of many tiles keep the product inside the
  // substitution, where it overlaps the waits.
  int sms = 1;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
  size_t part_el = 0;
  for (size_t l = 1; l < h->levels.size(); ++l) {
    Level& L = h->levels[l];
    int max_nu = 0;
    for (int32_t f : L.ids) max_nu = std::max(max_nu, h->fronts[f].nu);
    L.upd_split = 0;
    if (max_nu == 0 || L.n_bwd == 0) continue;
    const int by_rows = (max_nu + 127) / 128, by_grid = (4 * sms + L.n_bwd - 1) / L.n_bwd;
    if (L.n_bwd > 2 * sms || by_rows < 2) continue;
    L.upd_split = std::min(by_rows, by_grid);
    part_el = std::max(part_el, (size_t)L.n_bwd * L.upd_split * DD_TILE);
  }
  DD_CUDA(get(&h->upd_part, part_el * nr * h->elem));
  DD_CUDA(get((void**)&h->d_f, (size_t)h->n_loc * nr * 16));
  DD_CUDA(get((void**)&h->d_u, (size_t)h->n_loc * nr * 16));
  DD_CUDA(get((void**)&h->d_r, (size_t)h->n_loc * nr * 16));
  DD_CUDA(get((void**)&h->d_du, (size_t)h->n_loc * nr * 16));
  DD_CUDA(get((void**)&h->d_lam, (size_t)h->n_dual * nr * 16));
  DD_CUDA(get((void**)&h->d_dlam, (size_t)h->n_dual * nr * 16));
  DD_CUDA(get((void**)&h->d_g, (size_t)h->n_dual * nr * 16));
  h->nrhs_cap = nrhs;
  return DD_OK;
}

// one direct solve with the stored factors: (f [n_loc x nrhs], g [n_dual x nrhs] or NULL)
// -> (u, lam) in FP64 (assign)
// subset (optional): backward tasks of the listed leaves and their output
// descriptors (vec_off = row offset in u); other leaves are neither
// back-substituted nor written
struct LeafSubset {
  const Task* bwd = nullptr;
  int n_bwd = 0;
  const LeafDev* leaves = nullptr;
  int n_leaves = 0;
  int64_t ldu = 0;
};

void direct_solve(dd_handle* h, int nrhs, const double2* f, int64_t ldf, const double2* g, double2* u, double2* lam,
                  const LeafSubset* sub = nullptr) {
  cudaStream_t s = h->stream;
  const int p = h->prec == DD_PREC_FP64 ? 0 : 1;
  // ready flags restart from zero every solve, so a captured solve replays unchanged
  cudaMemsetAsync(h->d_flag_f, 0, sizeof(int32_t) * std::max<int64_t>(h->n_tiles, 1), s);
  cudaMemsetAsync(h->d_flag_b, 0, sizeof(int32_t) * std::max<int64_t>(h->n_tiles, 1), s);
  const int ep = 1;
  ddk::launch_rhs_leaf(p, h->rpool, h->d_fronts, h->d_leaves, h->n_sub, h->d_perm, f, ldf, nrhs, s);
  h->launches += 1;
  if (h->n_lvl0_sparse) {   // sparse-domain fronts without children
    ddk::launch_rhs_node(p, h->rpool, h->d_fronts, h->d_lvl0_sparse, h->n_lvl0_sparse, h->d_sep, g, h->n_dual, f,
                         ldf, h->n_dual, nrhs, s);
    h->launches += 1;
  }
  for (size_t l = 0; l < h->levels.size(); ++l) {
    const Level& L = h->levels[l];
    const int32_t* ids = h->d_level_ids + L.ids_off;
    const int n = (int)L.ids.size();
    if (l > 0) {
      ddk::launch_rhs_node(p, h->rpool, h->d_fronts, ids, n, h->d_sep, g, h->n_dual, f, ldf, h->n_dual, nrhs, s);
      ddk::launch_rhs_extend_add(p, h->rpool, h->d_fronts, ids, n, 0, h->d_maps, nrhs, s);
      ddk::launch_rhs_extend_add(p, h->rpool, h->d_fronts, ids, n, 1, h->d_maps, nrhs, s);
      h->launches += 3;
    }
    ddk::launch_forward(p, h->pool, h->rpool, h->d_fronts, h->d_fwd + L.fwd_off, L.n_fwd, nrhs, h->d_flag_f, ep,
                        h->d_solve_status, s, h->d_linv, h->d_piv, h->use_tc);
    h->launches += 1;
  }
  for (size_t l = h->levels.size(); l-- > 0;) {
    const Level& L = h->levels[l];
    const bool leaf_sub = sub && l == 0;
    h->launches += ddk::launch_backward(p, h->pool, h->rpool, h->d_fronts, leaf_sub ? sub->bwd : h->d_bwd + L.bwd_off,
                                        leaf_sub ? sub->n_bwd : L.n_bwd, nrhs, h->d_upd, h->d_sep, h->lam_work,
                                        h->ld_lam, h->d_flag_b, ep, h->d_solve_status, s, h->d_linv, h->d_piv,
                                        l > 0 && L.upd_split > 0 ? h->upd_part : nullptr, L.upd_split,
                                        h->use_tc);
  }
  if (sub)
    ddk::launch_leaf_out(p, h->rpool, h->d_fronts, sub->leaves, sub->n_leaves, h->d_perm, u, sub->ldu, nrhs, 0, s,
                         h->lam_work, h->ld_lam, h->n_dual);
  else
    ddk::launch_leaf_out(p, h->rpool, h->d_fronts, h->d_leaves, h->n_sub, h->d_perm, u, h->n_loc, nrhs, 0, s,
                         h->lam_work, h->ld_lam, h->n_dual);
  ddk::launch_lam_out(p, h->lam_work, h->ld_lam, h->n_dual, nrhs, lam, h->n_dual, 0, s);
  h->launches += 2;
}

__global__ void k_status_init(DevStatus* st) {
  DevStatus z{};
  z.min_abs_d = 0x7FF0000000000000ull;   // +inf
  *st = z;
}

// rows of listed domains: segment q copies rows [seg[3q], seg[3q] + seg[3q+2]) of
// src to rows starting at seg[3q+1] of dst, for every right-hand side
__global__ void k_gather_rows(const double2* src, int64_t lds, double2* dst, int64_t ldd, const int64_t* seg,
                              int nrhs) {
  const int64_t so = seg[3 * blockIdx.x], dof = seg[3 * blockIdx.x + 1], len = seg[3 * blockIdx.x + 2];
  for (int64_t e = threadIdx.x; e < len * nrhs; e += blockDim.x) {
    const int64_t r = e % len, j = e / len;
    dst[dof + r + j * ldd] = src[so + r + j * lds];
  }
}

__global__ void k_axpy(double2* y, const double2* x, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    y[e].x += x[e].x;
    y[e].y += x[e].y;
  }
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

const char* dd_strerror(int code) {
  switch (code) {
    case DD_OK: return "ok";
    case DD_ERR_INVALID_ARG: return "invalid argument";
    case DD_ERR_NOT_SYMMETRIC: return "domain matrix is not symmetric";
    case DD_ERR_SINGULAR_PIVOT: return "zero or non-finite pivot";
    case DD_ERR_OOM: return "out of memory";
    case DD_ERR_CUDA: return "CUDA runtime error";
    case DD_ERR_NOT_FACTORED: return "handle is not factored";
    case DD_ERR_NOT_CONVERGED: return "iterative refinement did not converge";
    case DD_ERR_TIMEOUT: return "device wait timed out";
    case DD_ERR_NO_DEVICE: return "no CUDA device";
    default: return "unknown status";
  }
}

int dd_default_options(dd_options* opt) {
  if (!opt) return DD_ERR_INVALID_ARG;
  std::memset(opt, 0, sizeof(*opt));
  opt->precision = DD_PREC_FP64;
  opt->refine_tol = 1e-13;
  opt->max_refine = 0;
  opt->pivoting = 0;
  opt->update_panels = 2;
  return DD_OK;
}

void dd_free(dd_handle* h) {
  if (!h) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(h->device);
  delete h;
  cudaSetDevice(cur);
}

}  // extern "C"

namespace {
// Front tree of the symbolic analysis, for dd_symbolic (host only)
struct SymbolicOut {
  int32_t max_fronts;
  int32_t* n_front;
  int32_t* parent;
  int32_t* ne;
  int32_t* nu;
  int32_t* dual_front;
  int64_t upd_cap;
  int64_t* upd_ptr;
  int32_t* upd_idx;
};

// dd_setup; with sym, only its host-side validation and symbolic analysis,
// whose front tree is written to sym (no device is touched)
int setup_impl(dd_handle** out, int32_t n_sub, const dd_subdomain* subs, int32_t n_dual, const dd_options* opt_in,
               const SymbolicOut* sym) {
  const auto t_begin = std::chrono::steady_clock::now();
  if (!out) return DD_ERR_INVALID_ARG;
  *out = nullptr;
  if (n_sub < 1 || n_dual < 0 || !subs) return DD_ERR_INVALID_ARG;
  dd_options opt;
  dd_default_options(&opt);
  if (opt_in) opt = *opt_in;
  if (opt.precision != DD_PREC_FP64 && opt.precision != DD_PREC_MIXED) return DD_ERR_INVALID_ARG;
  if (opt.pivoting < 0 || opt.pivoting > 2 || opt.max_refine < 0 || !(opt.refine_tol >= 0))
    return DD_ERR_INVALID_ARG;
  if (opt.update_panels != 1 && opt.update_panels != 2 && opt.update_panels != 4) return DD_ERR_INVALID_ARG;
  if (opt.sparse_min < 0 || opt.sparse_leaf < 0) return DD_ERR_INVALID_ARG;
  if (opt.device < 0) return DD_ERR_INVALID_ARG;

  double amax = 0.0;
  for (int i = 0; i < n_sub; ++i) {
    double a = 0.0;
    const int st = validate_subdomain(subs[i], n_dual, &a);
    if (st != DD_OK) return st;
    amax = std::max(amax, a);
  }

  std::unique_ptr<dd_handle> h(new dd_handle());
  h->device = opt.device;
  h->stream = (cudaStream_t)opt.cuda_stream;
  h->prec = opt.precision;
  h->refine_tol = opt.refine_tol > 0 ? opt.refine_tol : 1e-13;
  h->max_refine = opt.precision == DD_PREC_MIXED ? (opt.max_refine > 0 ? opt.max_refine : 10) : opt.max_refine;
  h->n_sub = n_sub;
  h->n_dual = n_dual;
  h->elem = opt.precision == DD_PREC_FP64 ? 16 : 8;
  h->time_kernels = opt.time_kernels == 2 ? 2 : (opt.time_kernels ? 1 : 0);
  h->use_tc = (opt.precision == DD_PREC_MIXED && !opt.simt_update) ? 1 : 0;
  h->pair_panels = h->use_tc && opt.update_panels >= 2;
  h->quad_panels = h->use_tc && opt.update_panels == 4;
  h->pivoting = opt.pivoting;
  h->max_abs_a = std::max(amax, 1.0);
  cudaStream_t s = h->stream;

  // ---- tree and dual placement ---------------------------------------------
  std::vector<int32_t> parent;
  int st = build_tree(n_sub, &opt, parent);
  if (st != DD_OK) return st;
  const int n_tree = 2 * n_sub - 1;
  // a lone domain with duals gets a root above it
  const bool extra_root = (n_sub == 1 && n_dual > 0);
  const int n_nodes = n_sub - 1 + (extra_root ? 1 : 0);
  const int n_front = n_sub + n_nodes;
  std::vector<int32_t> par(n_front, -1);
  for (int x = 0; x < n_tree; ++x) par[x] = parent[x];
  if (extra_root) par[0] = 1;
  std::vector<int> depth(n_front, 0);
  for (int x = n_front - 1; x >= 0; --x) depth[x] = par[x] < 0 ? 0 : depth[par[x]] + 1;
  auto lca = [&](int a, int b) {
    while (a != b) {
      if (depth[a] >= depth[b]) a = par[a];
      else b = par[b];
    }
    return a;
  };
  std::vector<int32_t> dual_node(n_dual, -1);
  std::vector<int32_t> dual_first(n_dual, -1);
  std::vector<int32_t> dual_count(n_dual, 0);
  for (int i = 0; i < n_sub; ++i)
    for (int q = 0; q < subs[i].nb; ++q) {
      const int d = subs[i].b_dual[q];
      dual_count[d]++;
      dual_node[d] = dual_node[d] < 0 ? i : lca(dual_node[d], i);
    }
  for (int d = 0; d < n_dual; ++d) {
    if (dual_node[d] < 0) return DD_ERR_INVALID_ARG;  // a dual with no B entry makes F singular
    if (dual_node[d] < n_sub) dual_node[d] = par[dual_node[d]];  // touches one domain only
    if (dual_node[d] < 0) return DD_ERR_INVALID_ARG;
  }

  // ---- sparse domains (Section II: sparse direct factorizations of the domains):
  // a domain of at least sparse_min unknowns becomes a tree of fronts, ordered
  // by nested dissection with its interface unknowns last (dd_domain_assembly).
  // The tree's root is front i (its update rows are the domain's duals, as for
  // a dense domain front); the other fronts get ids after the separator fronts.
  // Rows of these fronts carry "row ids": n_dual + the row's index in the
  // stacked primal vector, beside the dual ids of the update rows of the root.
  const int32_t sp_leaf = opt.sparse_leaf > 0 ? opt.sparse_leaf : 256;
  std::vector<SparseDomain> spd(n_sub);
  int n_extra = 0;
  {
    int64_t voff = 0;
    for (int i = 0; i < n_sub; ++i) {
      const dd_subdomain& sd = subs[i];
      SparseDomain& D = spd[i];
      D.vec_off = voff;
      voff += sd.n;
      if (opt.sparse_min <= 0 || sd.n < opt.sparse_min) continue;
      std::vector<int8_t> is_last(sd.n, 0);
      for (int q = 0; q < sd.nb; ++q) is_last[sd.b_local[q]] = 1;
      const int cap = 2 * sd.n + 1;
      D.parent.assign(cap, -1);
      D.ne.assign(cap, 0);
      D.rows_ptr.assign(cap + 1, 0);
      int32_t nf = 0;
      int st2 = dd_domain_assembly(sd.n, sd.rowptr, sd.colind, is_last.data(), sp_leaf, cap, &nf, D.parent.data(),
                                   D.ne.data(), 0, D.rows_ptr.data(), nullptr, nullptr, nullptr, nullptr, nullptr);
      if (st2 != DD_OK) return st2;
      const int64_t nrows = D.rows_ptr[nf];
      const int64_t nnz = sd.rowptr[sd.n];
      D.rows.assign(std::max<int64_t>(nrows, 1), 0);
      std::vector<int32_t> ea(D.rows.size()), arow(std::max<int64_t>(nnz, 1)), acol(arow.size());
      D.a_front.assign(arow.size(), -1);
      st2 = dd_domain_assembly(sd.n, sd.rowptr, sd.colind, is_last.data(), sp_leaf, cap, &nf, D.parent.data(),
                               D.ne.data(), (int64_t)D.rows.size(), D.rows_ptr.data(), D.rows.data(), ea.data(),
                               D.a_front.data(), arow.data(), acol.data());
      if (st2 != DD_OK) return st2;
      D.nf = nf;
      for (int x = 0; x < nf; ++x)
        if (D.parent[x] < 0) {
          if (D.root >= 0) return DD_ERR_INVALID_ARG;   // one tree per domain
          D.root = x;
        }
      // the interface rows must all be eliminated in the root front
      int n_if = 0;
      for (int r = 0; r < sd.n; ++r) n_if += is_last[r];
      if (D.root < 0 || D.ne[D.root] != n_if || D.rows_ptr[D.root + 1] - D.rows_ptr[D.root] != n_if)
        return DD_ERR_INVALID_ARG;
      n_extra += nf - 1;
    }
  }
  const int n_front_dense = n_front;   // domains and separator fronts
  {
    int next = n_front_dense;
    for (int i = 0; i < n_sub; ++i) {
      SparseDomain& D = spd[i];
      D.gid.assign(D.nf, -1);
      for (int x = 0; x < D.nf; ++x) D.gid[x] = x == D.root ? i : next++;
    }
  }
  const int n_front_all = n_front_dense + n_extra;
  h->n_sparse = 0;
  for (int i = 0; i < n_sub; ++i) h->n_sparse += spd[i].nf > 0 ? 1 : 0;
  par.resize(n_front_all, -1);
  for (int i = 0; i < n_sub; ++i)
    for (int x = 0; x < spd[i].nf; ++x)
      if (x != spd[i].root) par[spd[i].gid[x]] = spd[i].gid[spd[i].parent[x]];
  // row id of stacked primal row r (rows of sparse-domain fronts)
  auto vid = [&](int i, int r) -> int32_t { return (int32_t)(n_dual + spd[i].vec_off + r); };
  if (h->n_sparse && (int64_t)n_dual + spd[n_sub - 1].vec_off + subs[n_sub - 1].n > INT32_MAX) return DD_ERR_INVALID_ARG;
  if (h->n_sparse) {   // the scatter initialisation indexes the stacked CSR values with 32-bit ints
    int64_t nnz_all = 0;
    for (int i = 0; i < n_sub; ++i) nnz_all += subs[i].rowptr[subs[i].n];
    if (nnz_all > INT32_MAX) return DD_ERR_INVALID_ARG;
  }

  // ---- leaf structures --------------------------------------------------------
  h->fronts.assign(n_front_all, FrontDev{});
  std::vector<int32_t> h_rowptr, h_colind, h_iperm, h_perm, h_brow, h_blocal, h_blptr, h_bldual;
  std::vector<int8_t> h_bsign, h_blsign;
  std::vector<double2> h_val;
  std::vector<LeafDev> h_leaves(n_sub);
  std::vector<int32_t> h_upd, h_sep, h_maps, h_imaps;
  std::vector<std::vector<int32_t>> sp_sep(n_front_all), sp_upd(n_front_all);   // sparse-domain fronts
  h->leaf_duals.resize(n_sub);
  h->leaf_vec_off.resize(n_sub);
  int64_t vec_off = 0, csr_off = 0;
  int32_t rp_off = 0, b_off = 0;
  for (int i = 0; i < n_sub; ++i) {
    const dd_subdomain& sd = subs[i];
    std::vector<char> is_if(sd.n, 0);
    for (int q = 0; q < sd.nb; ++q) is_if[sd.b_local[q]] = 1;
    std::vector<int32_t> perm;
    perm.reserve(sd.n);
    for (int r = 0; r < sd.n; ++r)
      if (!is_if[r]) perm.push_back(r);
    const int n_int = (int)perm.size();
    for (int r = 0; r < sd.n; ++r)
      if (is_if[r]) perm.push_back(r);
    std::vector<int32_t> iperm(sd.n);
    for (int r = 0; r < sd.n; ++r) iperm[perm[r]] = r;
    std::vector<int32_t> duals(sd.b_dual, sd.b_dual + sd.nb);
    std::sort(duals.begin(), duals.end());
    duals.erase(std::unique(duals.begin(), duals.end()), duals.end());
    h->leaf_duals[i] = duals;

    LeafDev L{};
    L.csr_off = csr_off;
    L.vec_off = vec_off;
    L.rowptr_off = rp_off;
    L.n = sd.n;
    L.perm_off = (int32_t)h_perm.size();
    L.b_off = b_off;
    L.nb = sd.nb;
    L.front = i;
    h_leaves[i] = L;
    h->leaf_vec_off[i] = vec_off;

    FrontDev& F = h->fronts[i];
    F.piv = h->pivoting == 2 ? 1 : 0;   // domain fronts pivot in mode 2 only
    F.kind = 0;
    F.sub = i;
    F.ne = sd.n;
    F.ne_pad = (int32_t)round_up(sd.n, T);
    F.nu = (int32_t)duals.size();
    F.ld = F.ne_pad + (int32_t)round_up(F.nu, T);
    F.n_int = n_int;
    F.upd_off = (int32_t)h_upd.size();
    F.sep_off = 0;
    F.child[0] = F.child[1] = -1;
    h_upd.insert(h_upd.end(), duals.begin(), duals.end());
    const SparseDomain& D = spd[i];
    for (int x = 0; x < D.nf; ++x) {
      // a front of the domain's tree: its own rows, then its update rows (the
      // domain's duals at the root), all given by row ids
      FrontDev& G = h->fronts[D.gid[x]];
      G.piv = h->pivoting == 2 ? 1 : 0;
      G.kind = 2;
      G.sub = i;
      G.ne = D.ne[x];
      G.ne_pad = (int32_t)round_up(G.ne, T);
      G.nu = x == D.root ? (int32_t)duals.size() : (int32_t)(D.rows_ptr[x + 1] - D.rows_ptr[x] - D.ne[x]);
      G.ld = G.ne_pad + (int32_t)round_up(G.nu, T);
      G.n_int = 0;
      G.child[0] = G.child[1] = -1;
      std::vector<int32_t>& own = sp_sep[D.gid[x]];
      for (int64_t q = D.rows_ptr[x]; q < D.rows_ptr[x] + D.ne[x]; ++q) own.push_back(vid(i, D.rows[q]));
      if (x != D.root) {
        std::vector<int32_t>& up = sp_upd[D.gid[x]];
        for (int64_t q = D.rows_ptr[x] + D.ne[x]; q < D.rows_ptr[x + 1]; ++q) up.push_back(vid(i, D.rows[q]));
      }
      add_flops(h.get(), G.ne, G.nu, 0, false);
    }

    const int nnz = sd.rowptr[sd.n];
    h_rowptr.insert(h_rowptr.end(), sd.rowptr, sd.rowptr + sd.n + 1);
    h_colind.insert(h_colind.end(), sd.colind, sd.colind + nnz);
    for (int q = 0; q < nnz; ++q) h_val.push_back(make_double2(sd.val[q].re, sd.val[q].im));
    h_perm.insert(h_perm.end(), perm.begin(), perm.end());
    h_iperm.insert(h_iperm.end(), iperm.begin(), iperm.end());
    for (int q = 0; q < sd.nb; ++q) {
      h_brow.push_back((int32_t)(std::lower_bound(duals.begin(), duals.end(), sd.b_dual[q]) - duals.begin()));
      h_blocal.push_back(sd.b_local[q]);
      h_bsign.push_back(sd.b_sign[q]);
    }
    // B entries sorted by local row (FP64 residual)
    std::vector<int32_t> ord(sd.nb);
    std::iota(ord.begin(), ord.end(), 0);
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return sd.b_local[a] < sd.b_local[b]; });
    std::vector<int32_t> cnt(sd.n + 1, 0);
    for (int q = 0; q < sd.nb; ++q) cnt[sd.b_local[q] + 1]++;
    for (int r = 0; r < sd.n; ++r) cnt[r + 1] += cnt[r];
    h_blptr.insert(h_blptr.end(), cnt.begin(), cnt.end());
    for (int q : ord) {
      h_bldual.push_back(sd.b_dual[q]);
      h_blsign.push_back(sd.b_sign[q]);
    }
    vec_off += sd.n;
    csr_off += nnz;
    rp_off += sd.n + 1;
    b_off += sd.nb;
    const double ng = (double)(sd.n - n_int);
    if (!D.nf) add_flops(h.get(), sd.n, F.nu, ng, true);
  }
  h->n_loc = vec_off;
  h->nnz_total = csr_off;

  // dual -> (stacked row, sign) in fixed order (FP64 residual of B u)
  std::vector<int32_t> h_btptr(n_dual + 1, 0);
  for (int i = 0; i < n_sub; ++i)
    for (int q = 0; q < subs[i].nb; ++q) h_btptr[subs[i].b_dual[q] + 1]++;
  for (int d = 0; d < n_dual; ++d) h_btptr[d + 1] += h_btptr[d];
  std::vector<int64_t> h_btrow(h_btptr[n_dual]);
  std::vector<int8_t> h_btsign(h_btptr[n_dual]);
  {
    std::vector<int32_t> fill(h_btptr.begin(), h_btptr.end() - 1);
    for (int i = 0; i < n_sub; ++i)
      for (int q = 0; q < subs[i].nb; ++q) {
        const int d = subs[i].b_dual[q];
        h_btrow[fill[d]] = h->leaf_vec_off[i] + subs[i].b_local[q];
        h_btsign[fill[d]] = subs[i].b_sign[q];
        fill[d]++;
      }
  }

  // ---- node fronts (post-order: children before parents) ----------------------
  std::vector<std::vector<int32_t>> sep(n_front_all), upd(n_front_all);
  for (int d = 0; d < n_dual; ++d) sep[dual_node[d]].push_back(d);
  for (int i = 0; i < n_sub; ++i) upd[i] = h->leaf_duals[i];
  std::vector<std::vector<int32_t>> children(n_front_all);
  for (int x = 0; x < n_front_all; ++x)
    if (par[x] >= 0) children[par[x]].push_back(x);
  std::vector<int> height(n_front_all, 0);
  // sparse-domain fronts: rows, separator ids and heights (children first)
  for (int i = 0; i < n_sub; ++i) {
    const SparseDomain& D = spd[i];
    for (int x = 0; x < D.nf; ++x) {
      const int g = D.gid[x];
      sep[g] = sp_sep[g];
      if (x != D.root) upd[g] = sp_upd[g];
      if (children[g].size() > 2) return DD_ERR_INVALID_ARG;   // the dissection is binary
      int hgt = 0;
      for (int c : children[g]) hgt = std::max(hgt, height[c] + 1);
      height[g] = hgt;
    }
  }
  for (int v = n_sub; v < n_front; ++v) {
    FrontDev& F = h->fronts[v];
    F.kind = 1;
    F.piv = h->pivoting >= 1 ? 1 : 0;   // auxiliary fronts pivot in modes 1 and 2
    F.sub = -1;
    std::vector<int32_t> all;
    for (int c : children[v]) all.insert(all.end(), upd[c].begin(), upd[c].end());
    std::sort(all.begin(), all.end());
    all.erase(std::unique(all.begin(), all.end()), all.end());
    std::vector<int32_t>& sp = sep[v];  // already sorted (increasing d)
    std::vector<int32_t> up;
    for (int d : all)
      if (dual_node[d] != v) up.push_back(d);
    // every separator dual must be reachable from below
    for (int d : sp)
      if (!std::binary_search(all.begin(), all.end(), d)) return DD_ERR_INVALID_ARG;
    upd[v] = up;
    F.ne = (int32_t)sp.size();
    F.ne_pad = (int32_t)round_up(F.ne, T);
    F.nu = (int32_t)up.size();
    F.ld = F.ne_pad + (int32_t)round_up(F.nu, T);
    F.n_int = 0;
    F.upd_off = (int32_t)h_upd.size();
    h_upd.insert(h_upd.end(), up.begin(), up.end());
    F.sep_off = (int32_t)h_sep.size();
    h_sep.insert(h_sep.end(), sp.begin(), sp.end());
    F.child[0] = F.child[1] = -1;
    int hgt = 0;
    for (size_t slot = 0; slot < children[v].size() && slot < 2; ++slot) {
      const int c = children[v][slot];
      F.child[slot] = c;
      F.map_off[slot] = (int32_t)h_maps.size();
      for (int d : upd[c]) {
        int row;
        if (dual_node[d] == v) row = (int)(std::lower_bound(sp.begin(), sp.end(), d) - sp.begin());
        else row = F.ne_pad + (int)(std::lower_bound(up.begin(), up.end(), d) - up.begin());
        h_maps.push_back(row);
      }
      hgt = std::max(hgt, height[c] + 1);
    }
    height[v] = hgt;
    if (par[v] < 0 && F.nu != 0) return DD_ERR_INVALID_ARG;
    add_flops(h.get(), F.ne, F.nu, 0, false);
    h->stats.max_front = std::max(h->stats.max_front, F.ld);
  }
  for (int g = n_front; g < n_front_all; ++g) h->stats.max_front = std::max(h->stats.max_front, h->fronts[g].ld);
  // sparse-domain fronts: separator ids, children (the extend-add maps follow below)
  for (int i = 0; i < n_sub; ++i)
    for (int g : spd[i].gid) {
      FrontDev& G = h->fronts[g];
      G.sep_off = (int32_t)h_sep.size();
      h_sep.insert(h_sep.end(), sep[g].begin(), sep[g].end());
      for (size_t slot = 0; slot < children[g].size(); ++slot) G.child[slot] = children[g][slot];
    }

  // ---- update-row order: every front's update rows follow its parent's row
  // order, so each extend-add map is increasing and a child's block lands in
  // its parent row by row, in order (coalesced, never transposed) ----------------
  {
    const int64_t n_ids = (int64_t)n_dual + (h->n_sparse ? vec_off : 0);
    std::vector<int32_t> rowpos(std::max<int64_t>(n_ids, 1), -1);
    std::vector<int> order;   // parents before children
    for (int x = 0; x < n_front_all; ++x)
      if (par[x] < 0) order.push_back(x);
    for (size_t q = 0; q < order.size(); ++q)
      for (int c : children[order[q]]) order.push_back(c);
    for (int v : order) {
      if (h->fronts[v].kind == 0) continue;
      const FrontDev& F = h->fronts[v];
      for (size_t r = 0; r < sep[v].size(); ++r) rowpos[sep[v][r]] = (int32_t)r;
      for (size_t r = 0; r < upd[v].size(); ++r) rowpos[upd[v][r]] = F.ne_pad + (int32_t)r;
      for (int c : children[v])
        std::sort(upd[c].begin(), upd[c].end(), [&](int a, int b) { return rowpos[a] < rowpos[b]; });
      for (int d : sep[v]) rowpos[d] = -1;
      for (int d : upd[v]) rowpos[d] = -1;
    }
    h_upd.clear();
    for (int x = 0; x < n_front_all; ++x) {
      h->fronts[x].upd_off = (int32_t)h_upd.size();
      h_upd.insert(h_upd.end(), upd[x].begin(), upd[x].end());
    }
    h_maps.clear();
    for (int v = 0; v < n_front_all; ++v) {
      if (h->fronts[v].kind == 0) continue;
      FrontDev& F = h->fronts[v];
      for (size_t r = 0; r < sep[v].size(); ++r) rowpos[sep[v][r]] = (int32_t)r;
      for (size_t r = 0; r < upd[v].size(); ++r) rowpos[upd[v][r]] = F.ne_pad + (int32_t)r;
      for (int slot = 0; slot < 2; ++slot) {
        const int c = F.child[slot];
        if (c < 0) continue;
        F.map_off[slot] = (int32_t)h_maps.size();
        for (int d : upd[c]) h_maps.push_back(rowpos[d]);
      }
      for (int d : sep[v]) rowpos[d] = -1;
      for (int d : upd[v]) rowpos[d] = -1;
    }
    // inverse maps of the separator fronts (pull assembly): row here -> child
    // update row, -1 where the child has none
    h_imaps.clear();
    for (int v = 0; v < n_front_all; ++v) {
      FrontDev& F = h->fronts[v];
      F.imap_off[0] = F.imap_off[1] = -1;
      if (F.kind != 1) continue;
      for (int slot = 0; slot < 2; ++slot) {
        const int c = F.child[slot];
        if (c < 0) continue;
        F.imap_off[slot] = (int32_t)h_imaps.size();
        h_imaps.insert(h_imaps.end(), (size_t)F.ld, -1);
        for (int a = 0; a < h->fronts[c].nu; ++a) h_imaps[(size_t)F.imap_off[slot] + h_maps[(size_t)F.map_off[slot] + a]] = a;
      }
    }
    // the B rows of each domain front in their new order
    h->leaf_upd.assign(n_sub, {});
    size_t q0 = 0;
    for (int i = 0; i < n_sub; ++i) {
      h->leaf_upd[i] = upd[i];
      for (size_t r = 0; r < upd[i].size(); ++r) rowpos[upd[i][r]] = (int32_t)r;
      for (int q = 0; q < subs[i].nb; ++q) h_brow[q0 + q] = rowpos[subs[i].b_dual[q]];
      q0 += subs[i].nb;
      for (int d : upd[i]) rowpos[d] = -1;
    }
  }

  // ---- offsets, levels, task lists ----------------------------------------------
  int64_t off = 0, roff = 0, toff = 0;
  int64_t bytes_factor = 0;
  for (int x = 0; x < n_front_all; ++x) {
    FrontDev& F = h->fronts[x];
    F.off = off;
    F.roff = roff;
    F.tile_off = (int32_t)toff;
    toff += F.ld / T;
    off += (int64_t)F.ld * F.ld;
    roff += F.ld;
    bytes_factor += ((int64_t)F.ne_pad * (F.ne_pad + 1) / 2 + (int64_t)F.ne_pad * (F.ld - F.ne_pad)) * (int64_t)h->elem;
  }
  h->pool_bytes = (size_t)off * h->elem;
  h->rows_total = roff;
  // lower-triangular tiles zeroed before each factorization: every front but
  // the separator fronts, which the pull assembly writes in full; long tile
  // rows first
  std::vector<int2> h_ztiles;
  for (int x = 0; x < n_front_all; ++x)
    if (h->fronts[x].kind != 1)
      for (int t = 0; t < h->fronts[x].ld / T; ++t) h_ztiles.push_back(make_int2(x, t));
  std::stable_sort(h_ztiles.begin(), h_ztiles.end(), [](const int2& a, const int2& b) { return a.y > b.y; });
  h->n_ztiles = (int64_t)h_ztiles.size();
  h->n_tiles = toff;
  int max_h = 0;
  for (int x = 0; x < n_front_all; ++x) max_h = std::max(max_h, height[x]);
  h->levels.assign(max_h + 1, Level{});
  for (int x = 0; x < n_front_all; ++x)
    if (h->fronts[x].ld > 0 || x < n_sub) {
      h->levels[height[x]].ids.push_back(x);
      if (h->fronts[x].kind == 1) h->levels[height[x]].n_aux++;
    }
  // the leaf level in two halves of about equal work (front work ~ ld^3, each
  // front to the lighter half, largest first) for the split schedule, whose
  // halves run on two streams; their task lists are built with the levels'
  // below and they use the leaf level's image offsets
  h->halves.clear();
  if (h->use_tc && !h->levels.empty() && h->levels[0].ids.size() >= 2) {
    std::vector<int32_t> ord = h->levels[0].ids;
    std::stable_sort(ord.begin(), ord.end(), [&](int32_t a, int32_t b) { return h->fronts[a].ld > h->fronts[b].ld; });
    h->halves.assign(2, Level{});
    double wk[2] = {0.0, 0.0};
    for (int32_t f : ord) {
      const int q = wk[0] <= wk[1] ? 0 : 1;
      const double ld = h->fronts[f].ld;
      h->halves[q].ids.push_back(f);
      if (h->fronts[f].kind == 1) h->halves[q].n_aux++;
      wk[q] += ld * ld * ld;
    }
    for (Level& Hf : h->halves) std::sort(Hf.ids.begin(), Hf.ids.end());
  }
  // mixed form: panel image workspace, reused level after level
  if (h->use_tc) {
    // slots 0 and 1 hold the images of even / odd panels of every level; the
    // look-ahead levels also use slots 2 and 3 (panels k + 2, k + 3 are formed
    // while the two-panel update of k, k + 1 still reads 0 and 1)
    size_t need = 0, need_ahead = 0;
    for (auto& L : h->levels) {
      int64_t w = 0;
      for (int f : L.ids) {
        FrontDev& F = h->fronts[f];
        const int64_t ntr = F.ld / T - 1;  // trailing tiles at the first step
        F.ws_off = w;
        w += ntr * (int64_t)DD_TC_ATILE;
        // a B image (W = L D) only for fronts that pivot; the others' one
        // image of M = L D^(1/2) serves as both operands
        F.ws_boff = F.piv ? w : F.ws_off;
        if (F.piv) w += ntr * (int64_t)DD_TC_BTILE;
      }
      L.ahead = L.ids.size() <= (size_t)kAheadMaxFronts;   // may look ahead (image slots 2, 3)
      need = std::max(need, (size_t)w);
      if (L.ahead) need_ahead = std::max(need_ahead, (size_t)w);
    }
    // four-panel passes hold the images of panels k .. k + 3 at once: slots
    // 0-3 are sized for every level; with look-ahead the far part of a
    // four-panel update still reads them while the next four panels are
    // formed into slots 4-7, sized for the levels that may look ahead
    h->ws_bytes = 4 * need + 4 * need_ahead;
    for (int q = 1; q < 8; ++q) h->ws_slot_off[q] = q <= 4 ? q * need : 4 * need + (q - 4) * need_ahead;
  }
  std::vector<int32_t> h_level_ids, h_diag;
  std::vector<Task> h_trsm, h_updt, h_tc, h_tc2;
  std::vector<int2> h_grp;
  // runs of consecutive tasks with the same (front, row tile), at most
  // kGroupCap long, claimed one at a time by the persistent update kernel (consecutive
  // groups in flight share their column tiles' operand images through L2)
  constexpr int kGroupCap = 8;
  auto add_groups = [&](const std::vector<Task>& tl, int64_t first, int64_t count) -> int {
    int ng = 0;
    for (int64_t q = first; q < first + count;) {
      int64_t e = q + 1;
      while (e < first + count && e - q < kGroupCap && tl[e].f == tl[q].f && tl[e].i == tl[q].i) ++e;
      h_grp.push_back(make_int2((int)q, (int)(e - q)));
      ++ng;
      q = e;
    }
    return ng;
  };
  std::vector<Level*> gen;   // the levels, then the leaf level's halves
  for (auto& L : h->levels) gen.push_back(&L);
  for (auto& L : h->halves) gen.push_back(&L);
  for (size_t gi = 0; gi < gen.size(); ++gi) {
    Level& L = *gen[gi];
    const bool is_half = gi >= h->levels.size();   // the halves repeat the leaf level's work
    L.ids_off = (int64_t)h_level_ids.size();
    h_level_ids.insert(h_level_ids.end(), L.ids.begin(), L.ids.end());
    int max_steps = 0;
    for (int f : L.ids) {
      if (h->fronts[f].kind == 1) L.max_ld = std::max(L.max_ld, h->fronts[f].ld);
      max_steps = std::max(max_steps, h->fronts[f].ne_pad / T);
      for (int slot = 0; slot < 2; ++slot) {
        const int c = h->fronts[f].child[slot];
        if (c >= 0) L.max_child_nu = std::max(L.max_child_nu, h->fronts[c].nu);
      }
    }
    for (int k = 0; k < max_steps; ++k) {
      StepRange R{};
      R.k = k;
      R.diag_off = (int64_t)h_diag.size();
      R.trsm_off = (int64_t)h_trsm.size();
      R.upd_off = (int64_t)h_updt.size();
      R.tc_off = (int64_t)h_tc.size();
      std::vector<Task> upd_next, upd_rest, tc_next, tc_rest;
      double upd_flops = 0.0, trsm_flops = 0.0, diag_flops = 0.0;
      for (int f : L.ids) {
        const FrontDev& F = h->fronts[f];
        const int nte = F.ne_pad / T, nt = F.ld / T;
        if (k >= nte) continue;
        h_diag.push_back(f);
        // rows of B_i vanish on panels made only of interior columns
        auto zero_tile = [&](int i) { return F.kind == 0 && i >= nte && (k + 1) * T <= F.n_int; };
        for (int i = k + 1; i < nt; ++i)
          if (!zero_tile(i)) h_trsm.push_back(Task{f, i, k, 0});
        for (int j = k + 1; j < nt; ++j) {
          if (zero_tile(j)) continue;
          for (int i = j; i < nt; ++i) {
            if (zero_tile(i)) continue;
            if (!h->use_tc) (j == k + 1 ? upd_next : upd_rest).push_back(Task{f, i, j, 0});
          }
        }
        // algorithmic work of this step on the front's exact sizes (no tile
        // padding; 8 real flops per complex multiply-add): the panel's w real
        // columns, the r real rows below it (later eliminated rows, and the
        // update rows unless B vanishes on the panel); the trailing update
        // covers the lower triangle of the r x r block
        {
          const double w = std::min(T, F.ne - k * T);
          const double e = std::max(0, F.ne - (k + 1) * T);
          const double r = e + (zero_tile(nte) ? 0 : F.nu);
          diag_flops += 8.0 * w * (w - 1) * (w + 1) / 6.0;
          trsm_flops += 8.0 * r * w * (w - 1) / 2.0;
          upd_flops += 8.0 * w * r * (r + 1) / 2.0;
        }
        // tensor-core tasks: row tile i x column tiles (j, j + 1); column pairs
        // never straddle the first update-row tile, so both columns of a task
        // share their structurally zero panels
        if (h->use_tc) {
          for (int i = k + 1; i < nt; ++i)
            if (!zero_tile(i) && !zero_tile(k + 1)) tc_next.push_back(Task{f, i, k + 1, 1 | 4});
          const int sb[3] = {k + 2, std::max(nte, k + 2), nt};
          for (int i = k + 2; i < nt; ++i) {
            if (zero_tile(i)) continue;
            for (int sg = 0; sg < 2; ++sg)
              for (int j = sb[sg]; j < sb[sg + 1] && j <= i; j += 2) {
                if (zero_tile(j)) continue;
                const int two = (j + 1 < sb[sg + 1] && j + 1 <= i) ? 2 : 0;
                tc_rest.push_back(Task{f, i, j, 1 | two | 4});
              }
          }
        }
      }
      R.n_upd_next = (int)upd_next.size();
      R.n_tc_next = (int)tc_next.size();
      h_updt.insert(h_updt.end(), upd_next.begin(), upd_next.end());
      h_updt.insert(h_updt.end(), upd_rest.begin(), upd_rest.end());
      h_tc.insert(h_tc.end(), tc_next.begin(), tc_next.end());
      h_tc.insert(h_tc.end(), tc_rest.begin(), tc_rest.end());
      R.n_diag = (int)((int64_t)h_diag.size() - R.diag_off);
      if (!is_half) {
        h->stats.kernel_flops[DD_K_UPDATE] += upd_flops;
        h->stats.kernel_flops[DD_K_TRSM] += trsm_flops;
        h->stats.kernel_flops[DD_K_DIAG] += diag_flops;
      }
      R.n_trsm = (int)((int64_t)h_trsm.size() - R.trsm_off);
      R.n_upd = (int)((int64_t)h_updt.size() - R.upd_off);
      R.n_tc = (int)((int64_t)h_tc.size() - R.tc_off);
      R.grp_off = (int64_t)h_grp.size();
      R.n_grp_next = add_groups(h_tc, R.tc_off, R.n_tc_next);
      R.n_grp_rest = add_groups(h_tc, R.tc_off + R.n_tc_next, R.n_tc - R.n_tc_next);
      L.steps.push_back(R);
    }
    // two-panel updates: column pairs never straddle the first update-row
    // tile, so both columns of a task share their structurally zero panels
    if (h->use_tc)   // built for the tensor-core path whatever update_panels says (dd_autotune)
      for (int k = 0; k + 1 < max_steps; k += 2) {
        PairRange P{};
        P.k = k;
        P.tc2_off = (int64_t)h_tc2.size();
        std::vector<Task> near, far;
        for (int f : L.ids) {
          const FrontDev& F = h->fronts[f];
          const int nte = F.ne_pad / T, nt = F.ld / T;
          if (k >= nte) continue;
          const int np = (k + 1 < nte) ? 2 : 1;
          auto zero = [&](int p, int i) { return F.kind == 0 && i >= nte && (p + 1) * T <= F.n_int; };
          const int sb[3] = {k + 2, std::max(nte, k + 2), nt};
          for (int i = k + 2; i < nt; ++i)
            for (int sg = 0; sg < 2; ++sg)
              for (int j = sb[sg]; j < sb[sg + 1] && j <= i; j += 2) {
                int pm = 0;
                for (int pp = 0; pp < np; ++pp)
                  if (!zero(k + pp, i) && !zero(k + pp, j)) pm |= 4 << pp;
                if (!pm) continue;
                const int two = (j + 1 < sb[sg + 1] && j + 1 <= i) ? 2 : 0;
                (j <= k + 3 ? near : far).push_back(Task{f, i, j, 1 | two | pm});
              }
        }
        P.n_near = (int)near.size();
        P.n_far = (int)far.size();
        h_tc2.insert(h_tc2.end(), near.begin(), near.end());
        h_tc2.insert(h_tc2.end(), far.begin(), far.end());
        P.grp_off = (int64_t)h_grp.size();
        P.n_grp_near = add_groups(h_tc2, P.tc2_off, P.n_near);
        P.n_grp_far = add_groups(h_tc2, P.tc2_off + P.n_near, P.n_far);
        L.pairs.push_back(P);
      }
    // four-panel updates: every column gets each of its panels exactly once
    // (column k + 1: panel k with step k's first update; columns k + 2, k + 3:
    // panels k, k + 1 here (near); column k + 3: panel k + 2 with step k + 2's
    // first update; columns >= k + 4: panels k .. k + 3 here (far))
    if (h->use_tc)
      for (int k = 0; k + 3 < max_steps; k += 4) {
        QuadRange Q{};
        Q.k = k;
        Q.tc_off = (int64_t)h_tc2.size();
        std::vector<Task> near, far;
        for (int f : L.ids) {
          const FrontDev& F = h->fronts[f];
          const int nte = F.ne_pad / T, nt = F.ld / T;
          if (k >= nte) continue;
          const int np = std::min(4, nte - k);
          auto zero = [&](int p, int i) { return F.kind == 0 && i >= nte && (p + 1) * T <= F.n_int; };
          auto mask = [&](int i, int j, int npp) {
            int pm = 0;
            for (int pp = 0; pp < npp; ++pp)
              if (!zero(k + pp, i) && !zero(k + pp, j)) pm |= 4 << pp;
            return pm;
          };
          for (int i = k + 2; i < nt; ++i) {
            // near: columns k + 2 and k + 3, one task when both are on the same side of nte
            const int j0 = k + 2, j1 = k + 3;
            if (j0 <= i && j0 < nt) {
              const bool pair = j1 <= i && j1 < nt && ((j0 < nte) == (j1 < nte));
              const int pm = mask(i, j0, std::min(2, np));
              if (pm) near.push_back(Task{f, i, j0, 1 | (pair ? 2 : 0) | pm});
              if (!pair && j1 <= i && j1 < nt) {
                const int pm1 = mask(i, j1, std::min(2, np));
                if (pm1) near.push_back(Task{f, i, j1, 1 | pm1});
              }
            }
            // far: columns >= k + 4 in pairs that do not straddle nte
            const int sb[3] = {k + 4, std::max(nte, k + 4), nt};
            for (int sg = 0; sg < 2; ++sg)
              for (int j = sb[sg]; j < sb[sg + 1] && j <= i; j += 2) {
                const int pm = mask(i, j, np);
                if (!pm) continue;
                const int two = (j + 1 < sb[sg + 1] && j + 1 <= i) ? 2 : 0;
                far.push_back(Task{f, i, j, 1 | two | pm});
              }
          }
        }
        // far tasks of columns k + 4 .. k + 7 first (the next four panels' columns:
        // the look-ahead schedule applies them on the main stream), the rest after
        std::stable_partition(far.begin(), far.end(), [&](const Task& t) { return t.j <= k + 7; });
        Q.n_near = (int)near.size();
        Q.n_far = (int)far.size();
        Q.n_far4 = (int)std::count_if(far.begin(), far.end(), [&](const Task& t) { return t.j <= k + 7; });
        h_tc2.insert(h_tc2.end(), near.begin(), near.end());
        h_tc2.insert(h_tc2.end(), far.begin(), far.end());
        Q.grp_off = (int64_t)h_grp.size();
        Q.n_grp_near = add_groups(h_tc2, Q.tc_off, Q.n_near);
        Q.n_grp_far4 = add_groups(h_tc2, Q.tc_off + Q.n_near, Q.n_far4);
        Q.n_grp_far = Q.n_grp_far4 + add_groups(h_tc2, Q.tc_off + Q.n_near + Q.n_far4, Q.n_far - Q.n_far4);
        L.quads.push_back(Q);
      }
  }
  // solve tasks: forward (front, row tile) by increasing tile, backward (front,
  // eliminated tile) by decreasing tile, so that every CTA waits only on CTAs
  // with a smaller block index
  std::vector<Task> h_fwd, h_bwd;
  for (auto& L : h->levels) {
    int max_nt = 0, max_nte = 0;
    for (int f : L.ids) {
      max_nt = std::max(max_nt, h->fronts[f].ld / T);
      max_nte = std::max(max_nte, h->fronts[f].ne_pad / T);
    }
    L.fwd_off = (int64_t)h_fwd.size();
    for (int i = 0; i < max_nt; ++i)
      for (int f : L.ids)
        if (i < h->fronts[f].ld / T) h_fwd.push_back(Task{f, i, 0, 0});
    L.n_fwd = (int)((int64_t)h_fwd.size() - L.fwd_off);
    L.bwd_off = (int64_t)h_bwd.size();
    for (int j = max_nte - 1; j >= 0; --j)
      for (int f : L.ids)
        if (j < h->fronts[f].ne_pad / T) h_bwd.push_back(Task{f, j, 0, 0});
    L.n_bwd = (int)((int64_t)h_bwd.size() - L.bwd_off);
  }

  {
    std::vector<int32_t> ne_k(n_front_all), nu_k(n_front_all), par_k(n_front_all);
    for (int x = 0; x < n_front_all; ++x) {
      ne_k[x] = h->fronts[x].ne;
      nu_k[x] = h->fronts[x].nu;
      par_k[x] = par[x];
    }
    h->tune_key = tune_problem_key(n_front_all, par_k.data(), ne_k.data(), nu_k.data(), n_dual, opt.precision,
                                   opt.pivoting);
  }
  if (sym) {
    *sym->n_front = n_front_all;
    if (sym->max_fronts < n_front_all) return DD_ERR_INVALID_ARG;
    int64_t tot = 0;
    for (int x = 0; x < n_front_all; ++x) {
      sym->parent[x] = par[x];
      sym->ne[x] = h->fronts[x].ne;
      sym->nu[x] = h->fronts[x].nu;
      if (sym->upd_ptr) sym->upd_ptr[x] = tot;
      tot += (int64_t)upd[x].size();
    }
    if (sym->upd_ptr) sym->upd_ptr[n_front_all] = tot;
    for (int d = 0; d < n_dual; ++d) sym->dual_front[d] = dual_node[d];
    if (sym->upd_idx) {
      if (sym->upd_cap < tot) return DD_ERR_INVALID_ARG;
      int64_t q = 0;
      for (int x = 0; x < n_front_all; ++x)
        for (int32_t d : upd[x]) sym->upd_idx[q++] = d;
    }
    return DD_OK;
  }

  // ---- sparse domains: the front position of every A_i entry (the front
  // eliminating the earlier of its row and column), of every B_i entry (the
  // root's update rows) and of the padding diagonals, for the initialisation
  std::vector<int64_t> h_sp_dst;
  std::vector<int32_t> h_sp_src;   // >= 0: index into the stacked CSR values; -1: +1; -2: -1
  std::vector<int32_t> h_lvl0;
  h->ld_lam = n_dual;
  if (h->n_sparse) {
    h->ld_lam = (int64_t)n_dual + h->n_loc;
    std::vector<int32_t> rowpos((size_t)h->ld_lam, -1);
    int64_t csr0 = 0, b0 = 0;
    for (int i = 0; i < n_sub; ++i) {
      const SparseDomain& D = spd[i];
      const dd_subdomain& sd = subs[i];
      const int64_t nnz = sd.rowptr[sd.n];
      if (D.nf) {
        std::vector<std::vector<std::pair<int32_t, int32_t>>> by_front(D.nf);   // (CSR entry, its row)
        for (int r = 0; r < sd.n; ++r)
          for (int q = sd.rowptr[r]; q < sd.rowptr[r + 1]; ++q)
            if (D.a_front[q] >= 0) by_front[D.a_front[q]].push_back({q, r});
        for (int x = 0; x < D.nf; ++x) {
          const int g = D.gid[x];
          const FrontDev& G = h->fronts[g];
          for (size_t r = 0; r < sep[g].size(); ++r) rowpos[sep[g][r]] = (int32_t)r;
          if (x != D.root)
            for (size_t r = 0; r < upd[g].size(); ++r) rowpos[upd[g][r]] = G.ne_pad + (int32_t)r;
          for (auto [q, r] : by_front[x]) {
            const int pc = rowpos[vid(i, r)], pr = rowpos[vid(i, sd.colind[q])];
            if (pc < 0 || pc >= G.ne || pr < pc) return DD_ERR_INVALID_ARG;
            h_sp_dst.push_back(G.off + (int64_t)pr * G.ld + pc);
            h_sp_src.push_back((int32_t)(csr0 + q));
          }
          for (int r = G.ne; r < G.ne_pad; ++r) {
            h_sp_dst.push_back(G.off + (int64_t)r * G.ld + r);
            h_sp_src.push_back(-1);
          }
          if (x == D.root)
            for (int k = 0; k < sd.nb; ++k) {
              const int pc = rowpos[vid(i, sd.b_local[k])];
              if (pc < 0 || pc >= G.ne) return DD_ERR_INVALID_ARG;
              h_sp_dst.push_back(G.off + (int64_t)(G.ne_pad + h_brow[b0 + k]) * G.ld + pc);
              h_sp_src.push_back(sd.b_sign[k] > 0 ? -1 : -2);
            }
          for (int32_t id : sep[g]) rowpos[id] = -1;
          if (x != D.root)
            for (int32_t id : upd[g]) rowpos[id] = -1;
          if (height[g] == 0) h_lvl0.push_back(g);
        }
      }
      csr0 += nnz;
      b0 += sd.nb;
    }
  }
  h->n_scatter = (int64_t)h_sp_dst.size();
  h->n_lvl0_sparse = (int)h_lvl0.size();

  // ---- upload (everything above is host-only validation and analysis) -------------
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return DD_ERR_NO_DEVICE;
  }
  if (opt.device >= ndev) return DD_ERR_INVALID_ARG;
  int cur = 0;
  cudaGetDevice(&cur);
  if (cudaSetDevice(h->device) != cudaSuccess) return DD_ERR_CUDA;
  struct Restore { int d; ~Restore() { cudaSetDevice(d); } } restore{cur};
  DeviceArena& A = h->arena;
  DD_CUDA(A.alloc((unsigned char**)&h->pool, h->pool_bytes));
  DD_CUDA(A.upload(&h->d_fronts, h->fronts, s));
  DD_CUDA(A.upload(&h->d_leaves, h_leaves, s));
  DD_CUDA(A.upload(&h->d_rowptr, h_rowptr, s));
  DD_CUDA(A.upload(&h->d_colind, h_colind, s));
  DD_CUDA(A.upload(&h->d_val, h_val, s));
  DD_CUDA(A.upload(&h->d_iperm, h_iperm, s));
  DD_CUDA(A.upload(&h->d_perm, h_perm, s));
  DD_CUDA(A.upload(&h->d_brow, h_brow, s));
  DD_CUDA(A.upload(&h->d_blocal, h_blocal, s));
  DD_CUDA(A.upload(&h->d_bsign, h_bsign, s));
  DD_CUDA(A.upload(&h->d_blptr, h_blptr, s));
  DD_CUDA(A.upload(&h->d_bldual, h_bldual, s));
  DD_CUDA(A.upload(&h->d_blsign, h_blsign, s));
  DD_CUDA(A.upload(&h->d_btptr, h_btptr, s));
  DD_CUDA(A.upload(&h->d_btrow, h_btrow, s));
  DD_CUDA(A.upload(&h->d_btsign, h_btsign, s));
  DD_CUDA(A.upload(&h->d_upd, h_upd, s));
  DD_CUDA(A.upload(&h->d_sep, h_sep, s));
  DD_CUDA(A.upload(&h->d_maps, h_maps, s));
  DD_CUDA(A.upload(&h->d_imaps, h_imaps, s));
  DD_CUDA(A.upload(&h->d_ztiles, h_ztiles, s));
  DD_CUDA(A.upload(&h->d_level_ids, h_level_ids, s));
  DD_CUDA(A.upload(&h->d_diag_ids, h_diag, s));
  DD_CUDA(A.upload(&h->d_trsm, h_trsm, s));
  DD_CUDA(A.upload(&h->d_updt, h_updt, s));
  DD_CUDA(A.upload(&h->d_fwd, h_fwd, s));
  DD_CUDA(A.upload(&h->d_tc, h_tc, s));
  DD_CUDA(A.upload(&h->d_tc2, h_tc2, s));
  DD_CUDA(A.upload(&h->d_grp, h_grp, s));
  if (h->n_sparse) {
    DD_CUDA(A.upload(&h->d_sp_dst, h_sp_dst, s));
    DD_CUDA(A.upload(&h->d_sp_src, h_sp_src, s));
    DD_CUDA(A.upload(&h->d_lvl0_sparse, h_lvl0, s));
  }
  {
    int nl = 0;
    for (auto& L : h->levels) nl += 2 * (int)L.steps.size();
    for (auto& L : h->halves) nl += 2 * (int)L.steps.size();
    h->n_counters = std::max(nl, 1);
    DD_CUDA(A.alloc(&h->d_counters, (size_t)h->n_counters));
  }
  if (h->use_tc) DD_CUDA(A.alloc(&h->d_ws, h->ws_bytes));
  DD_CUDA(cudaStreamCreateWithFlags(&h->s2, cudaStreamNonBlocking));
  // the legacy default stream cannot be captured into a graph: without a caller
  // stream the handle works on its own blocking stream, which is ordered with
  // the legacy stream like the legacy stream itself
  if (!h->stream) {
    DD_CUDA(cudaStreamCreate(&h->own_stream));
    h->stream = h->own_stream;
    s = h->stream;
  }
  DD_CUDA(cudaEventCreateWithFlags(&h->ev_panel, cudaEventDisableTiming));
  DD_CUDA(cudaEventCreateWithFlags(&h->ev_rest, cudaEventDisableTiming));
  // mixed form: L^{-1} of every diagonal tile (panel products and the substitution)
  if (h->prec == DD_PREC_MIXED) DD_CUDA(A.alloc(&h->d_linv, (size_t)std::max<int64_t>(h->n_tiles, 1) * T * T));
  if (h->pivoting) DD_CUDA(A.alloc(&h->d_piv, (size_t)std::max<int64_t>(h->n_tiles, 1) * T));
  DD_CUDA(A.upload(&h->d_bwd, h_bwd, s));
  h->h_leaves_copy = h_leaves;
  if (!h->levels.empty())
    h->h_bwd_leaf.assign(h_bwd.begin() + h->levels[0].bwd_off,
                         h_bwd.begin() + h->levels[0].bwd_off + h->levels[0].n_bwd);
  DD_CUDA(A.alloc(&h->d_flag_f, (size_t)std::max<int64_t>(h->n_tiles, 1)));
  DD_CUDA(A.alloc(&h->d_flag_b, (size_t)std::max<int64_t>(h->n_tiles, 1)));
  DD_CUDA(cudaMemsetAsync(h->d_flag_f, 0, sizeof(int32_t) * std::max<int64_t>(h->n_tiles, 1), s));
  DD_CUDA(cudaMemsetAsync(h->d_flag_b, 0, sizeof(int32_t) * std::max<int64_t>(h->n_tiles, 1), s));
  DD_CUDA(A.alloc(&h->d_solve_status, 1));
  DD_CUDA(cudaMemsetAsync(h->d_solve_status, 0, sizeof(DevStatus), s));
  DD_CUDA(A.alloc(&h->d_status, 1));
  DD_CUDA(A.alloc(&h->d_partials, 2 * kSolveBlock * kNormBlocks));
  DD_CUDA(cudaEventCreate(&h->ev0));
  DD_CUDA(cudaEventCreate(&h->ev1));
  DD_CUDA(cudaStreamSynchronize(s));

  h->stats.n_sub = n_sub;
  h->stats.n_dual = n_dual;
  h->stats.n_fronts = n_front_all;
  h->stats.n_levels = (int)h->levels.size();
  h->stats.n_primal = h->n_loc;
  h->stats.bytes_factor = bytes_factor;
  h->stats.bytes_device = (int64_t)A.bytes;
  // a cached schedule of this problem on this GPU model
  if (opt.tune_cache && opt.tune_cache[0]) {
    h->tune_cache = opt.tune_cache;
    dd_schedule sc{};
    int32_t found = 0;
    if (h->use_tc &&
        dd_tune_cache_lookup(opt.tune_cache, tune_cache_key(h->tune_key, h->device).c_str(), &sc, &found) == DD_OK &&
        found)
      dd_set_schedule(h.get(), &sc);
  }
  h->stats.t_setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_begin).count();
  *out = h.release();
  return DD_OK;
}
}  // namespace

extern "C" {

int dd_setup(dd_handle** out, int32_t n_sub, const dd_subdomain* subs, int32_t n_dual, const dd_options* opt_in) {
  return setup_impl(out, n_sub, subs, n_dual, opt_in, nullptr);
}

int dd_symbolic(int32_t n_sub, const dd_subdomain* subs, int32_t n_dual, const dd_options* opt, int32_t max_fronts,
                int32_t* n_front, int32_t* parent, int32_t* ne, int32_t* nu, int32_t* dual_front, int64_t upd_cap,
                int64_t* upd_ptr, int32_t* upd_idx) {
  if (!n_front || !parent || !ne || !nu || (n_dual > 0 && !dual_front) || (upd_idx && !upd_ptr)) return DD_ERR_INVALID_ARG;
  const SymbolicOut sym{max_fronts, n_front, parent, ne, nu, dual_front, upd_cap, upd_ptr, upd_idx};
  dd_handle* unused = nullptr;
  return setup_impl(&unused, n_sub, subs, n_dual, opt, &sym);
}

int dd_set_values(dd_handle* h, const dd_c128* vals) {
  if (!h || !vals) return DD_ERR_INVALID_ARG;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(h->device);
  const cudaMemcpyKind kind = is_device_ptr(vals) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  cudaError_t e = cudaMemcpyAsync(h->d_val, vals, (size_t)h->nnz_total * 16, kind, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  h->factored = false;
  cudaSetDevice(cur);
  return cuda_status(e);
}

// Enqueues one numeric factorization on stream s (and the look-ahead stream):
// the same launch sequence every call, so it can be captured once as a CUDA
// graph.  With time_kernels, event pairs around every launch (1) or around the
// trailing-update launches only (2).
static int enqueue_factor(dd_handle* h, cudaStream_t s, int& launches, size_t& nev, std::vector<int>& cls_of) {
  const int p = h->prec == DD_PREC_FP64 ? 0 : 1;
  k_status_init<<<1, 1, 0, s>>>(h->d_status);
  launches = 0;
  // optional per-launch timing: an event pair around every launch of a class
  constexpr size_t kMaxTimed = 8192;
  nev = 0;
  cls_of.assign(h->time_kernels ? kMaxTimed : 0, 0);
  auto mark_on = [&](int cls, bool begin, cudaStream_t on) -> cudaError_t {
    if (!h->time_kernels || (h->time_kernels == 2 && cls != DD_K_UPDATE) || nev >= 2 * kMaxTimed) return cudaSuccess;
    if (begin) cls_of[nev / 2] = cls;
    while (h->kev.size() <= nev) {
      cudaEvent_t e;
      cudaError_t err = cudaEventCreate(&e);
      if (err != cudaSuccess) return err;
      h->kev.push_back(e);
    }
    // inside stream capture this becomes an event-record node of the graph
    return cudaEventRecordWithFlags(h->kev[nev++], on, cudaEventRecordExternal);
  };
  auto mark = [&](int cls, bool begin) { return mark_on(cls, begin, s); };
  for (int c = 0; c < DD_K_NCLASS; ++c) {
    h->stats.kernel_ms[c] = 0.0;
    h->stats.kernel_launches[c] = 0;
  }
  auto count = [&](int cls, int n) {
    if (n > 0) {
      launches++;
      h->stats.kernel_launches[cls]++;
    }
  };
  ddk::launch_zero_lower(h->pool, h->elem, h->d_fronts, h->d_ztiles, h->n_ztiles, s);
  if (h->d_counters) ddk::launch_zero(h->d_counters, sizeof(int) * h->n_counters, s);
  int next_counter = 0;
  DD_CUDA(mark(DD_K_INIT, true));
  ddk::launch_leaf_init(p, h->pool, h->d_fronts, h->d_leaves, h->n_sub, h->d_rowptr, h->d_colind, h->d_val,
                        h->d_iperm, h->d_brow, h->d_blocal, h->d_bsign, s);
  ddk::launch_sparse_init(p, h->pool, h->d_sp_dst, h->d_sp_src, h->n_scatter, h->d_val, s);
  DD_CUDA(mark(DD_K_INIT, false));
  count(DD_K_INIT, 1);
  count(DD_K_INIT, h->n_scatter > 0 ? 1 : 0);
  // one level on stream s, or one half of the leaf level (split: no
  // look-ahead, and every update leaves split_sms SMs to the other half's
  // panel chain on the other stream)
  auto run_level = [&](const Level& L, const cudaStream_t s, bool assemble, bool split) -> int {
    const int32_t* ids = h->d_level_ids + L.ids_off;
    const int n = (int)L.ids.size();
    if (assemble) {
      DD_CUDA(mark_on(DD_K_ASSEMBLE, true, s));
      ddk::launch_assemble(p, h->pool, h->d_fronts, ids, n, h->d_imaps, L.max_ld, s);
      ddk::launch_node_init(p, h->pool, h->d_fronts, ids, n, s);
      ddk::launch_extend_add(p, h->pool, h->d_fronts, ids, n, 0, h->d_maps, L.max_child_nu, s);
      ddk::launch_extend_add(p, h->pool, h->d_fronts, ids, n, 1, h->d_maps, L.max_child_nu, s);
      DD_CUDA(mark_on(DD_K_ASSEMBLE, false, s));
      count(DD_K_ASSEMBLE, L.max_ld > 0 ? n : 0);
      count(DD_K_ASSEMBLE, n);
      count(DD_K_ASSEMBLE, n);
      count(DD_K_ASSEMBLE, n);
    }
    // mixed form: wide pivot blocks (double-float, or FP64 with pivoting) for the
    // auxiliary matrix's separator fronts, FP32 for the fronts that eliminate
    // domain unknowns
    const int diag64 = L.n_aux == 0 ? 0 : (L.n_aux == (int)L.ids.size() ? 1 : 2);
    // one-step look-ahead on levels with few fronts: the main stream updates
    // only the next panel columns and factors those panels, while the second
    // stream applies the rest of the trailing update
    const bool ahead = h->use_tc && L.ahead && (int)L.ids.size() <= h->ahead_fronts && L.steps.size() > 1 && !split;
    const int reserve = ahead ? h->reserve_sms : 0;   // SMs left free for the panel chain
    const int capn = split ? h->split_sms : 0;        // main-stream updates: SMs left to the other half
    // image slot of panel k: even / odd panels alternate, the look-ahead levels over four slots
    // four-panel passes (slots k & 3, or k & 7 with look-ahead)
    const bool quad = h->quad_panels && !L.quads.empty();
    auto wsp = [&](int k) -> unsigned char* {
      return h->d_ws + h->ws_slot_off[quad ? (ahead ? (k & 7) : (k & 3)) : (ahead ? (k & 3) : (k & 1))];
    };
    auto panel = [&](const StepRange& R) -> cudaError_t {
      unsigned char* ws = h->use_tc ? wsp(R.k) : nullptr;
      cudaError_t e = mark_on(DD_K_DIAG, true, s);
      if (e != cudaSuccess) return e;
      if (p == 0)
        ddk::launch_diag(p, 0, h->pool, h->d_fronts, h->d_diag_ids + R.diag_off, R.n_diag, R.k, h->d_status, s,
                         h->d_piv);
      else
        ddk::launch_diag_mx(diag64, h->pool, h->d_fronts, h->d_diag_ids + R.diag_off, R.n_diag, R.k, h->d_status,
                            h->d_linv, s, h->d_piv);
      if ((e = mark_on(DD_K_DIAG, false, s)) != cudaSuccess) return e;
      if ((e = mark_on(DD_K_TRSM, true, s)) != cudaSuccess) return e;
      if (p == 0)
        ddk::launch_trsm(p, h->pool, h->d_fronts, h->d_trsm + R.trsm_off, R.n_trsm, R.k, h->d_status, s, nullptr,
                         h->d_piv);
      else
        ddk::launch_trsm_mx(h->pool, h->d_fronts, h->d_trsm + R.trsm_off, R.n_trsm, R.k, h->d_status, h->d_linv, ws,
                            s, h->d_piv, h->use_tc);
      count(DD_K_DIAG, R.n_diag);
      if (p == 1 && diag64 == 2) count(DD_K_DIAG, R.n_diag);
      count(DD_K_TRSM, R.n_trsm);
      return mark_on(DD_K_TRSM, false, s);
    };
    // trailing update of step R.k, tasks [first, first + n) of its lists, on stream `on`
    auto update = [&](const StepRange& R, bool next_part, cudaStream_t on, int cap) -> cudaError_t {
      const unsigned char* ws = h->use_tc ? wsp(R.k) : nullptr;
      const int n = h->use_tc ? (next_part ? R.n_tc_next : R.n_tc - R.n_tc_next)
                              : (next_part ? R.n_upd_next : R.n_upd - R.n_upd_next);
      const int64_t first = h->use_tc ? R.tc_off + (next_part ? 0 : R.n_tc_next)
                                      : R.upd_off + (next_part ? 0 : R.n_upd_next);
      cudaError_t e = mark_on(DD_K_UPDATE, true, on);
      if (e != cudaSuccess) return e;
      if (h->use_tc)
        ddk::launch_update_tc(h->pool, h->d_fronts, h->d_tc, h->d_grp + R.grp_off + (next_part ? 0 : R.n_grp_next),
                              next_part ? R.n_grp_next : R.n_grp_rest, R.k, ddk::PanelImages{{ws, nullptr, nullptr, nullptr}},
                              h->d_status, on, cap, h->d_counters + (next_counter++ % h->n_counters));
      else
        ddk::launch_update(p, h->pool, h->d_fronts, h->d_updt + first, n, R.k, on);
      count(DD_K_UPDATE, n);
      return mark_on(DD_K_UPDATE, false, on);
    };
    // two-panel update of steps P.k, P.k + 1: near (columns k + 2, k + 3) or far (the rest)
    auto pair_update = [&](const PairRange& P, bool near_part, cudaStream_t on, int cap) -> cudaError_t {
      cudaError_t e = mark_on(DD_K_UPDATE, true, on);
      if (e != cudaSuccess) return e;
      ddk::launch_update_tc(h->pool, h->d_fronts, h->d_tc2, h->d_grp + P.grp_off + (near_part ? 0 : P.n_grp_near),
                             near_part ? P.n_grp_near : P.n_grp_far, P.k,
                             ddk::PanelImages{{wsp(P.k), wsp(P.k + 1), nullptr, nullptr}}, h->d_status, on, cap,
                             h->d_counters + (next_counter++ % h->n_counters));
      count(DD_K_UPDATE, near_part ? P.n_near : P.n_far);
      return mark_on(DD_K_UPDATE, false, on);
    };
    // four-panel update of steps Q.k .. Q.k + 3, part 0: columns k + 2, k + 3
    // (panels k, k + 1); 1: columns >= k + 4; 2: columns k + 4 .. k + 7; 3: columns >= k + 8
    auto quad_update = [&](const QuadRange& Q, int part, cudaStream_t on, int cap) -> cudaError_t {
      cudaError_t e = mark_on(DD_K_UPDATE, true, on);
      if (e != cudaSuccess) return e;
      int64_t g0 = Q.grp_off;
      int ng = Q.n_grp_near, nt_ = Q.n_near;
      if (part == 1) { g0 += Q.n_grp_near; ng = Q.n_grp_far; nt_ = Q.n_far; }
      if (part == 2) { g0 += Q.n_grp_near; ng = Q.n_grp_far4; nt_ = Q.n_far4; }
      if (part == 3) { g0 += Q.n_grp_near + Q.n_grp_far4; ng = Q.n_grp_far - Q.n_grp_far4; nt_ = Q.n_far - Q.n_far4; }
      ddk::launch_update_tc(h->pool, h->d_fronts, h->d_tc2, h->d_grp + g0, ng, Q.k,
                             ddk::PanelImages{{wsp(Q.k), wsp(Q.k + 1), wsp(Q.k + 2), wsp(Q.k + 3)}}, h->d_status, on,
                             cap, h->d_counters + (next_counter++ % h->n_counters));
      count(DD_K_UPDATE, nt_);
      return mark_on(DD_K_UPDATE, false, on);
    };
    // the panels of steps q0 .. q0 + 3 with the updates between them that they need
    auto quad_panels = [&](size_t q0) -> cudaError_t {
      const QuadRange& Q = L.quads[q0 / 4];
      cudaError_t e;
      if ((e = panel(L.steps[q0])) != cudaSuccess) return e;
      if ((e = update(L.steps[q0], true, s, capn)) != cudaSuccess) return e;      // column k + 1
      if ((e = panel(L.steps[q0 + 1])) != cudaSuccess) return e;
      if ((e = quad_update(Q, 0, s, capn)) != cudaSuccess) return e;               // columns k + 2, k + 3
      if ((e = panel(L.steps[q0 + 2])) != cudaSuccess) return e;
      if ((e = update(L.steps[q0 + 2], true, s, capn)) != cudaSuccess) return e;  // column k + 3, panel k + 2
      return panel(L.steps[q0 + 3]);
    };
    const size_t ns = L.steps.size();
    if (!h->use_tc || (!h->pair_panels && !ahead)) {
      for (const StepRange& R : L.steps) {
        DD_CUDA(panel(R));
        DD_CUDA(update(R, true, s, capn));
        DD_CUDA(update(R, false, s, capn));
      }
    } else if (!h->pair_panels) {
      // one panel per update pass: the rest of step k on the second stream
      // while the main stream updates column k + 1 and forms panel k + 1
      DD_CUDA(panel(L.steps[0]));
      DD_CUDA(cudaEventRecord(h->ev_panel, s));
      for (size_t q = 0; q < ns; ++q) {
        const StepRange& R = L.steps[q];
        DD_CUDA(cudaStreamWaitEvent(h->s2, h->ev_panel, 0));
        DD_CUDA(update(R, false, h->s2, reserve));            // columns >= k + 2
        DD_CUDA(cudaEventRecord(h->ev_rest, h->s2));
        DD_CUDA(update(R, true, s, capn));                       // column k + 1
        if (q + 1 < ns) {
          DD_CUDA(panel(L.steps[q + 1]));
          DD_CUDA(cudaEventRecord(h->ev_panel, s));
        }
        DD_CUDA(cudaStreamWaitEvent(s, h->ev_rest, 0));
      }
    } else if (quad) {
      // steps in fours: panel k, column k + 1; panel k + 1, columns k + 2, k + 3
      // with panels k, k + 1; panel k + 2, column k + 3 with it; panel k + 3,
      // then the columns >= k + 4 with all four panels (C read and written
      // once per four steps); the last steps in pairs.  With look-ahead the
      // columns >= k + 8 run on the second stream while the main stream
      // applies the four panels to columns k + 4 .. k + 7 and forms the next four.
      size_t q = 0;
      if (ahead) {
        DD_CUDA(cudaEventRecord(h->ev_panel, s));
        DD_CUDA(cudaStreamWaitEvent(h->s2, h->ev_panel, 0));
        DD_CUDA(cudaEventRecord(h->ev_rest, h->s2));
        DD_CUDA(quad_panels(0));
        for (; q + 3 < ns; q += 4) {
          const QuadRange& Q = L.quads[q / 4];
          DD_CUDA(cudaStreamWaitEvent(s, h->ev_rest, 0));     // the previous far part is done
          DD_CUDA(cudaEventRecord(h->ev_panel, s));
          DD_CUDA(cudaStreamWaitEvent(h->s2, h->ev_panel, 0));
          DD_CUDA(quad_update(Q, 3, h->s2, reserve));          // columns >= k + 8
          DD_CUDA(cudaEventRecord(h->ev_rest, h->s2));
          DD_CUDA(quad_update(Q, 2, s, capn));                    // columns k + 4 .. k + 7
          if (q + 7 < ns) DD_CUDA(quad_panels(q + 4));
        }
        DD_CUDA(cudaStreamWaitEvent(s, h->ev_rest, 0));
      }
      for (; q < ns;) {
        const StepRange& R = L.steps[q];
        if (q + 3 < ns) {
          const QuadRange& Q = L.quads[q / 4];
          DD_CUDA(quad_panels(q));
          DD_CUDA(quad_update(Q, 1, s, capn));                    // columns >= k + 4
          q += 4;
        } else {
          DD_CUDA(panel(R));
          DD_CUDA(update(R, true, s, capn));
          if (q + 1 < ns) {
            const PairRange& P = L.pairs[q / 2];
            DD_CUDA(panel(L.steps[q + 1]));
            DD_CUDA(pair_update(P, true, s, capn));
            DD_CUDA(pair_update(P, false, s, capn));
            q += 2;
          } else {
            DD_CUDA(update(R, false, s, capn));
            q += 1;
          }
        }
      }
    } else if (!ahead) {
      // steps in pairs: panel k, column k + 1, panel k + 1, then both panels at once
      for (size_t q = 0; q < ns;) {
        const StepRange& R = L.steps[q];
        DD_CUDA(panel(R));
        DD_CUDA(update(R, true, s, capn));
        if (q + 1 < ns) {
          const PairRange& P = L.pairs[q / 2];
          DD_CUDA(panel(L.steps[q + 1]));
          DD_CUDA(pair_update(P, true, s, capn));
          DD_CUDA(pair_update(P, false, s, capn));
          q += 2;
        } else {
          DD_CUDA(update(R, false, s, capn));
          q += 1;
        }
      }
    } else {
      // the far part of each two-panel update runs on the second stream while
      // the main stream forms the next two panels; before touching columns the
      // far part also updates, the main stream waits for it
      // the second stream joins here (also inside graph capture), with nothing pending
      DD_CUDA(cudaEventRecord(h->ev_panel, s));
      DD_CUDA(cudaStreamWaitEvent(h->s2, h->ev_panel, 0));
      DD_CUDA(cudaEventRecord(h->ev_rest, h->s2));
      DD_CUDA(panel(L.steps[0]));
      for (size_t q = 0; q < ns;) {
        const StepRange& R = L.steps[q];
        DD_CUDA(update(R, true, s, capn));                       // column k + 1 with panel k
        if (q + 1 < ns) {
          const PairRange& P = L.pairs[q / 2];
          DD_CUDA(panel(L.steps[q + 1]));
          DD_CUDA(cudaStreamWaitEvent(s, h->ev_rest, 0));     // the previous far part is done
          DD_CUDA(cudaEventRecord(h->ev_panel, s));
          DD_CUDA(cudaStreamWaitEvent(h->s2, h->ev_panel, 0));
          DD_CUDA(pair_update(P, false, h->s2, reserve));     // columns >= k + 4
          DD_CUDA(cudaEventRecord(h->ev_rest, h->s2));
          DD_CUDA(pair_update(P, true, s, capn));                // columns k + 2, k + 3
          if (q + 2 < ns) DD_CUDA(panel(L.steps[q + 2]));
          q += 2;
        } else {
          DD_CUDA(cudaStreamWaitEvent(s, h->ev_rest, 0));
          DD_CUDA(cudaEventRecord(h->ev_panel, s));
          DD_CUDA(cudaStreamWaitEvent(h->s2, h->ev_panel, 0));
          DD_CUDA(update(R, false, h->s2, reserve));          // columns >= k + 2
          DD_CUDA(cudaEventRecord(h->ev_rest, h->s2));
          q += 1;
        }
      }
      DD_CUDA(cudaStreamWaitEvent(s, h->ev_rest, 0));
    }
    return DD_OK;
  };
  for (size_t l = 0; l < h->levels.size(); ++l) {
    if (l == 0 && h->split_sms > 0 && h->halves.size() == 2) {
      // the leaf level's two halves on the two streams, joined before level 1
      DD_CUDA(cudaEventRecord(h->ev_panel, s));
      DD_CUDA(cudaStreamWaitEvent(h->s2, h->ev_panel, 0));
      int st = run_level(h->halves[0], s, false, true);
      if (st == DD_OK) st = run_level(h->halves[1], h->s2, false, true);
      if (st != DD_OK) return st;
      DD_CUDA(cudaEventRecord(h->ev_rest, h->s2));
      DD_CUDA(cudaStreamWaitEvent(s, h->ev_rest, 0));
      continue;
    }
    const int st = run_level(h->levels[l], s, l > 0, false);
    if (st != DD_OK) return st;
  }
  DD_CUDA(cudaGetLastError());
  return DD_OK;
}

int dd_factor(dd_handle* h) {
  if (!h) return DD_ERR_INVALID_ARG;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(h->device);
  struct Restore { int d; ~Restore() { cudaSetDevice(d); } } restore{cur};
  cudaStream_t s = h->stream;
  h->factored = false;
  // the whole factorization as one CUDA graph, captured on the first call
  // (with time_kernels the graph also records an event pair around every launch)
  if (!h->factor_exec) {
    int launches = 0;
    DD_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed));
    const int st = enqueue_factor(h, s, launches, h->fact_nev, h->fact_cls);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(s, &g);
    if (st != DD_OK || e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      return st != DD_OK ? st : cuda_status(e);
    }
    const cudaError_t ei = cudaGraphInstantiate(&h->factor_exec, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
      h->factor_exec = nullptr;
      return cuda_status(ei);
    }
    h->factor_graph_launches = launches;
  }
  const int launches = h->factor_graph_launches;
  const size_t nev = h->fact_nev;
  const std::vector<int>& cls_of = h->fact_cls;
  DD_CUDA(cudaEventRecord(h->ev0, s));
  DD_CUDA(cudaGraphLaunch(h->factor_exec, s));
  DD_CUDA(cudaGetLastError());
  DD_CUDA(cudaEventRecord(h->ev1, s));
  DevStatus st{};
  DD_CUDA(cudaMemcpyAsync(&st, h->d_status, sizeof(st), cudaMemcpyDeviceToHost, s));
  DD_CUDA(cudaStreamSynchronize(s));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, h->ev0, h->ev1);
  h->stats.t_factor_ms = ms;
  h->stats.launches_factor = launches;
  for (int c = 0; c < DD_K_NCLASS; ++c) h->stats.kernel_ms[c] = 0.0;
  for (size_t q = 0; q + 1 < nev; q += 2) {
    float dt = 0.f;
    if (cudaEventElapsedTime(&dt, h->kev[q], h->kev[q + 1]) == cudaSuccess) h->stats.kernel_ms[cls_of[q / 2]] += dt;
  }
  double maxd, mind, maxl;
  std::memcpy(&maxd, &st.max_abs_d, 8);
  std::memcpy(&mind, &st.min_abs_d, 8);
  std::memcpy(&maxl, &st.max_abs_l, 8);
  h->stats.growth = std::max(maxd, maxl) / h->max_abs_a;
  h->stats.min_pivot = mind;
  h->stats.interchanges = (int64_t)st.n_swap;
  h->stats.pivots_2x2 = (int64_t)st.n_2x2;
  if (st.code == 8) return DD_ERR_TIMEOUT;
  if (st.code != 0) return DD_ERR_SINGULAR_PIVOT;
  h->factored = true;
  return DD_OK;
}

int dd_set_schedule(dd_handle* h, const dd_schedule* sc) {
  if (!h || !sc) return DD_ERR_INVALID_ARG;
  if ((sc->update_panels != 1 && sc->update_panels != 2 && sc->update_panels != 4) || sc->ahead_fronts < 0 ||
      sc->ahead_fronts > kAheadMaxFronts || sc->reserve_sms < 0 || sc->reserve_sms > 64 || sc->split_sms < 0 ||
      sc->split_sms > 120)
    return DD_ERR_INVALID_ARG;
  if (!h->use_tc) return DD_OK;
  h->pair_panels = sc->update_panels >= 2;
  h->quad_panels = sc->update_panels == 4;
  h->ahead_fronts = sc->ahead_fronts;
  h->reserve_sms = sc->reserve_sms;
  h->split_sms = sc->split_sms;
  if (h->factor_exec) cudaGraphExecDestroy(h->factor_exec);   // recaptured by the next dd_factor
  h->factor_exec = nullptr;
  h->fact_nev = 0;
  h->fact_cls.clear();
  return DD_OK;
}

int dd_autotune(dd_handle* h, int32_t repeats, dd_schedule* out) {
  if (!h || !out || repeats < 1) return DD_ERR_INVALID_ARG;
  auto time_it = [&](double* best) -> int {
    *best = 1e300;
    for (int r = 0; r < repeats; ++r) {
      const int st = dd_factor(h);
      if (st != DD_OK) return st;
      *best = std::min(*best, h->stats.t_factor_ms);
    }
    return DD_OK;
  };
  dd_schedule cur{h->quad_panels ? 4 : (h->pair_panels ? 2 : 1), h->ahead_fronts, h->reserve_sms, 0.0, 0,
                  h->split_sms};
  if (!h->use_tc) {
    const int st = time_it(&cur.factor_ms);
    cur.configs_tried = 1;
    *out = cur;
    return st;
  }
  // a cached schedule of this problem on this GPU model: no timing
  const std::string ckey = h->tune_cache.empty() ? std::string() : tune_cache_key(h->tune_key, h->device);
  if (!ckey.empty()) {
    dd_schedule sc{};
    int32_t found = 0;
    if (dd_tune_cache_lookup(h->tune_cache.c_str(), ckey.c_str(), &sc, &found) == DD_OK && found) {
      int st = dd_set_schedule(h, &sc);
      if (st == DD_OK) st = dd_factor(h);
      sc.configs_tried = 0;
      *out = sc;
      return st;
    }
  }
  std::vector<dd_schedule> grid;
  for (int panels : {1, 2, 4})
    for (int ahead : {0, 8, 32, 128, 1024})
      for (int reserve : {8, 16, 32}) {
        if (ahead == 0 && reserve != 16) continue;   // no look-ahead: the reserve is unused
        grid.push_back(dd_schedule{panels, ahead, reserve, 0.0, 0, 0});
      }
  dd_schedule best = cur;
  best.factor_ms = 1e300;
  for (dd_schedule& c : grid) {
    int st = dd_set_schedule(h, &c);
    if (st == DD_OK) st = time_it(&c.factor_ms);
    if (st != DD_OK) return st;
    if (c.factor_ms < best.factor_ms) best = c;
  }
  // then the split leaf level on top of the best schedule
  int tried = (int32_t)grid.size();
  if (h->halves.size() == 2) {
    const dd_schedule base = best;
    for (int split : {24, 40, 64}) {
      dd_schedule c = base;
      c.split_sms = split;
      int st = dd_set_schedule(h, &c);
      if (st == DD_OK) st = time_it(&c.factor_ms);
      if (st != DD_OK) return st;
      ++tried;
      if (c.factor_ms < best.factor_ms) best = c;
    }
  }
  best.configs_tried = tried;
  int st = dd_set_schedule(h, &best);
  if (st == DD_OK) st = dd_factor(h);
  // an unwritable cache path costs the tuning nothing; the schedule is still returned
  if (st == DD_OK && !ckey.empty()) dd_tune_cache_store(h->tune_cache.c_str(), ckey.c_str(), &best);
  *out = best;
  return st;
}

static int solve_block(dd_handle* h, int32_t nrhs, const dd_c128* f, int64_t ldf, dd_c128* u, int64_t ldu,
                       dd_c128* lambda, int64_t ldl);

int dd_solve(dd_handle* h, int32_t nrhs, const dd_c128* f, int64_t ldf, dd_c128* u, int64_t ldu, dd_c128* lambda,
             int64_t ldl) {
  if (!h || nrhs < 0) return DD_ERR_INVALID_ARG;
  if (nrhs == 0) return DD_OK;
  if (!f || !u || ldf < h->n_loc || ldu < h->n_loc) return DD_ERR_INVALID_ARG;
  if (lambda && ldl < h->n_dual) return DD_ERR_INVALID_ARG;
  if (!h->factored) return DD_ERR_NOT_FACTORED;
  // blocks of up to 64 right-hand sides
  int status = DD_OK;
  double t_ms = 0.0, worst = 0.0;
  int iters = 0, launches = 0;
  for (int32_t c0 = 0; c0 < nrhs; c0 += kSolveBlock) {
    const int32_t nb = std::min<int32_t>(kSolveBlock, nrhs - c0);
    const int st = solve_block(h, nb, f + (size_t)c0 * ldf, ldf, u + (size_t)c0 * ldu, ldu,
                               lambda ? lambda + (size_t)c0 * ldl : nullptr, ldl);
    if (st != DD_OK && st != DD_ERR_NOT_CONVERGED) return st;
    if (st == DD_ERR_NOT_CONVERGED) status = st;
    t_ms += h->stats.t_solve_ms;
    worst = std::max(worst, h->stats.refine_last);
    iters = std::max(iters, h->stats.refine_iters);
    launches += h->stats.launches_solve;
  }
  h->stats.t_solve_ms = t_ms;
  h->stats.refine_last = worst;
  h->stats.refine_iters = iters;
  h->stats.launches_solve = launches;
  return status;
}

int dd_solve_subset(dd_handle* h, int32_t nrhs, const dd_c128* f, int64_t ldf, int32_t n_req, const int32_t* req,
                    dd_c128* u, int64_t ldu, dd_c128* lambda, int64_t ldl) {
  if (!h || nrhs < 0 || n_req < 0 || (n_req > 0 && !req)) return DD_ERR_INVALID_ARG;
  if (nrhs == 0) return DD_OK;
  if (!f || ldf < h->n_loc || (lambda && ldl < h->n_dual)) return DD_ERR_INVALID_ARG;
  std::vector<char> seen(h->n_sub, 0);
  int64_t n_rows = 0;
  for (int32_t q = 0; q < n_req; ++q) {
    const int32_t id = req[q];
    if (id < 0 || id >= h->n_sub || seen[id]) return DD_ERR_INVALID_ARG;
    seen[id] = 1;
    n_rows += h->h_leaves_copy[id].n;
  }
  if (n_rows > 0 && (!u || ldu < n_rows)) return DD_ERR_INVALID_ARG;
  if (!h->factored) return DD_ERR_NOT_FACTORED;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(h->device);
  struct Restore { int d; ~Restore() { cudaSetDevice(d); } } restore{cur};
  cudaStream_t s = h->stream;
  // the listed leaves (output offsets in request order), their backward tasks, row segments
  std::vector<LeafDev> sl(n_req);
  std::vector<int64_t> seg(3 * (size_t)n_req);
  std::vector<int> front_listed(h->fronts.size(), 0);
  int64_t off = 0;
  for (int32_t q = 0; q < n_req; ++q) {
    LeafDev L = h->h_leaves_copy[req[q]];
    seg[3 * q] = L.vec_off;
    seg[3 * q + 1] = off;
    seg[3 * q + 2] = L.n;
    L.vec_off = off;
    off += L.n;
    sl[q] = L;
    front_listed[L.front] = 1;
  }
  std::vector<Task> sb;
  for (const Task& t : h->h_bwd_leaf)
    if (front_listed[t.f]) sb.push_back(t);
  // the full solve, then the listed rows: with refinement (the FP64 residual
  // needs every domain) and with sparse domains (whose backward substitution
  // runs over trees of fronts)
  const bool refined = h->max_refine > 0 || h->n_sparse > 0;
  const bool u_dev = n_rows > 0 && is_device_ptr(u);
  const int32_t chunk = std::min<int32_t>(kSolveBlock, nrhs);
  auto al = [](size_t b) { return (b + 255) / 256 * 256; };
  const size_t b_sb = al(sb.size() * sizeof(Task) + 1), b_sl = al(sl.size() * sizeof(LeafDev) + 1),
               b_seg = al(seg.size() * sizeof(int64_t) + 1), b_u = al((size_t)n_rows * chunk * 16 + 1);
  const size_t need = b_sb + b_sl + b_seg + b_u;
  if (need > h->sub_cap) {
    if (h->d_sub) cudaFree(h->d_sub);
    h->d_sub = nullptr;
    h->sub_cap = 0;
    DD_CUDA(cudaMalloc(&h->d_sub, need));
    h->sub_cap = need;
  }
  unsigned char* base = static_cast<unsigned char*>(h->d_sub);
  Task* d_sb = reinterpret_cast<Task*>(base);
  LeafDev* d_sl = reinterpret_cast<LeafDev*>(base + b_sb);
  int64_t* d_seg = reinterpret_cast<int64_t*>(base + b_sb + b_sl);
  double2* d_usub = reinterpret_cast<double2*>(base + b_sb + b_sl + b_seg);
  if (!sb.empty()) DD_CUDA(cudaMemcpyAsync(d_sb, sb.data(), sb.size() * sizeof(Task), cudaMemcpyHostToDevice, s));
  if (n_req) {
    DD_CUDA(cudaMemcpyAsync(d_sl, sl.data(), sl.size() * sizeof(LeafDev), cudaMemcpyHostToDevice, s));
    DD_CUDA(cudaMemcpyAsync(d_seg, seg.data(), seg.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  }
  int status = DD_OK;
  double t_ms = 0.0;
  for (int32_t c0 = 0; c0 < nrhs; c0 += kSolveBlock) {
    const int32_t nb = std::min<int32_t>(kSolveBlock, nrhs - c0);
    const dd_c128* fc = f + (size_t)c0 * ldf;
    dd_c128* lc = lambda ? lambda + (size_t)c0 * ldl : nullptr;
    double2* out = u_dev ? reinterpret_cast<double2*>(u + (size_t)c0 * ldu) : d_usub;
    const int64_t ldo = u_dev ? ldu : n_rows;
    if (refined) {
      const int st = solve_block(h, nb, fc, ldf, nullptr, 0, lc, ldl);
      if (st != DD_OK && st != DD_ERR_NOT_CONVERGED) return st;
      if (st == DD_ERR_NOT_CONVERGED) status = st;
      t_ms += h->stats.t_solve_ms;
      if (n_req) k_gather_rows<<<n_req, 256, 0, s>>>(h->d_u, h->n_loc, out, ldo, d_seg, nb);
    } else {
      const int w = ensure_work(h, nb);
      if (w != DD_OK) return w;
      h->launches = 0;
      const size_t row_b = (size_t)h->n_loc * 16;
      DD_CUDA(cudaEventRecord(h->ev0, s));
      DD_CUDA(cudaMemcpy2DAsync(h->d_f, row_b, fc, (size_t)ldf * 16, row_b, nb,
                                is_device_ptr(fc) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
      LeafSubset sub;
      sub.bwd = d_sb;
      sub.n_bwd = (int)sb.size();
      sub.leaves = d_sl;
      sub.n_leaves = n_req;
      sub.ldu = ldo;
      direct_solve(h, nb, h->d_f, h->n_loc, nullptr, out, h->d_lam, &sub);
      if (lc && h->n_dual)
        DD_CUDA(cudaMemcpy2DAsync(lc, (size_t)ldl * 16, h->d_lam, (size_t)h->n_dual * 16, (size_t)h->n_dual * 16, nb,
                                  is_device_ptr(lc) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
      DD_CUDA(cudaEventRecord(h->ev1, s));
      DevStatus sst{};
      DD_CUDA(cudaMemcpyAsync(&sst, h->d_solve_status, sizeof(sst), cudaMemcpyDeviceToHost, s));
      DD_CUDA(cudaStreamSynchronize(s));
      if (sst.code != 0) {
        DD_CUDA(cudaMemsetAsync(h->d_solve_status, 0, sizeof(DevStatus), s));
        DD_CUDA(cudaStreamSynchronize(s));
        return sst.code == 8 ? DD_ERR_TIMEOUT : DD_ERR_CUDA;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, h->ev0, h->ev1);
      t_ms += ms;
      h->stats.launches_solve = h->launches;
      h->stats.refine_iters = 0;
    }
    if (!u_dev && n_rows > 0)
      DD_CUDA(cudaMemcpy2DAsync(u + (size_t)c0 * ldu, (size_t)ldu * 16, d_usub, (size_t)n_rows * 16,
                                (size_t)n_rows * 16, nb, cudaMemcpyDeviceToHost, s));
  }
  DD_CUDA(cudaGetLastError());
  DD_CUDA(cudaStreamSynchronize(s));
  h->stats.t_solve_ms = t_ms;
  return status;
}

static int solve_block(dd_handle* h, int32_t nrhs, const dd_c128* f, int64_t ldf, dd_c128* u, int64_t ldu,
                       dd_c128* lambda, int64_t ldl) {
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(h->device);
  struct Restore { int d; ~Restore() { cudaSetDevice(d); } } restore{cur};
  cudaStream_t s = h->stream;
  int st = ensure_work(h, nrhs);
  if (st != DD_OK) return st;
  h->launches = 0;
  const size_t row_b = (size_t)h->n_loc * 16;
  const int64_t nu_el = h->n_loc * (int64_t)nrhs;
  const int64_t nl_el = (int64_t)h->n_dual * nrhs;
  // the direct solve (a) and one refinement step (b) are captured once per
  // right-hand-side count and replayed; the host only reads the norms between steps
  dd_handle::SolveGraphs& gr = h->solve_graphs[nrhs];
  auto capture = [&](auto&& body, cudaGraphExec_t* out, int* launches) -> int {
    h->launches = 0;
    DD_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed));
    body();
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(s, &g);
    if (e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      return cuda_status(e);
    }
    const cudaError_t ei = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
      *out = nullptr;
      return cuda_status(ei);
    }
    *launches = h->launches;
    return DD_OK;
  };
  if (!gr.a) {
    const int c = capture([&] { direct_solve(h, nrhs, h->d_f, h->n_loc, nullptr, h->d_u, h->d_lam); }, &gr.a, &gr.la);
    if (c != DD_OK) return c;
  }
  if (h->max_refine > 0 && !gr.b) {
    const int c = capture(
        [&] {
          ddk::launch_residual(h->d_leaves, h->n_sub, h->d_rowptr, h->d_colind, h->d_val, h->d_blptr, h->d_bldual,
                               h->d_blsign, h->d_f, h->n_loc, h->d_u, h->n_loc, h->d_lam, h->n_dual, h->d_r,
                               h->n_loc, nrhs, s);
          ddk::launch_dual_residual(h->n_dual, h->d_btptr, h->d_btrow, h->d_btsign, h->d_u, h->n_loc, h->d_g,
                                    h->n_dual, nrhs, s);
          direct_solve(h, nrhs, h->d_r, h->n_loc, h->d_g, h->d_du, h->d_dlam);
          ddk::launch_sumsq_cols(h->d_du, h->n_loc, nrhs, kNormBlocks, h->d_partials, s);
          ddk::launch_sumsq_cols(h->d_u, h->n_loc, nrhs, kNormBlocks, h->d_partials + kSolveBlock * kNormBlocks, s);
          k_axpy<<<1024, 256, 0, s>>>(h->d_u, h->d_du, nu_el);
          if (nl_el) k_axpy<<<256, 256, 0, s>>>(h->d_lam, h->d_dlam, nl_el);
          h->launches += 6;
        },
        &gr.b, &gr.lb);
    if (c != DD_OK) return c;
  }
  h->launches = 0;
  DD_CUDA(cudaEventRecord(h->ev0, s));
  DD_CUDA(cudaMemcpy2DAsync(h->d_f, row_b, f, (size_t)ldf * 16, row_b, nrhs,
                            is_device_ptr(f) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  DD_CUDA(cudaGraphLaunch(gr.a, s));
  h->launches += gr.la;
  int iters = 0;
  double ratio = 0.0;
  int status = DD_OK;
  // relative size of the previous correction per right-hand side; the direct
  // solve itself is the first correction (from zero), of relative size 1
  double prev_col[kSolveBlock];
  for (int j = 0; j < kSolveBlock; ++j) prev_col[j] = 1.0;
  for (int it = 0; it < h->max_refine; ++it) {
    DD_CUDA(cudaGraphLaunch(gr.b, s));
    h->launches += gr.lb;
    double part[2 * kSolveBlock * kNormBlocks];
    DevStatus sst{};
    DD_CUDA(cudaMemcpyAsync(part, h->d_partials, sizeof(part), cudaMemcpyDeviceToHost, s));
    DD_CUDA(cudaMemcpyAsync(&sst, h->d_solve_status, sizeof(sst), cudaMemcpyDeviceToHost, s));
    DD_CUDA(cudaStreamSynchronize(s));
    if (sst.code != 0) break;  // reported after the loop
    // per right-hand side: |du_j| / |u_j| and, with linear convergence, the
    // error left after this update ~ |du_j| (|du_j| / |du_j previous|)
    iters = it + 1;
    bool all_done = true, finite = true;
    double worst = 0.0;
    for (int j = 0; j < nrhs; ++j) {
      double sdu = 0, su = 0;
      for (int q = 0; q < kNormBlocks; ++q) {
        sdu += part[j * kNormBlocks + q];
        su += part[kSolveBlock * kNormBlocks + j * kNormBlocks + q];
      }
      const double r = su > 0 ? std::sqrt(sdu / su) : 0.0;
      if (!std::isfinite(r)) finite = false;
      double err = r;
      if (prev_col[j] > 0 && r < prev_col[j]) err = std::min(err, r * (r / prev_col[j]));
      prev_col[j] = r;
      worst = std::max(worst, err);
      if (!(err <= h->refine_tol)) all_done = false;
    }
    ratio = worst;
    if (!finite || all_done) break;
  }
  if (h->prec == DD_PREC_MIXED && h->max_refine > 0 && !(ratio <= h->refine_tol)) status = DD_ERR_NOT_CONVERGED;
  if (u)
    DD_CUDA(cudaMemcpy2DAsync(u, (size_t)ldu * 16, h->d_u, row_b, row_b, nrhs,
                              is_device_ptr(u) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
  if (lambda && h->n_dual)
    DD_CUDA(cudaMemcpy2DAsync(lambda, (size_t)ldl * 16, h->d_lam, (size_t)h->n_dual * 16, (size_t)h->n_dual * 16,
                              nrhs, is_device_ptr(lambda) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
  DD_CUDA(cudaGetLastError());
  DD_CUDA(cudaEventRecord(h->ev1, s));
  DevStatus sst{};
  DD_CUDA(cudaMemcpyAsync(&sst, h->d_solve_status, sizeof(sst), cudaMemcpyDeviceToHost, s));
  DD_CUDA(cudaStreamSynchronize(s));
  if (sst.code != 0) {
    DD_CUDA(cudaMemsetAsync(h->d_solve_status, 0, sizeof(DevStatus), s));
    DD_CUDA(cudaStreamSynchronize(s));
    return sst.code == 8 ? DD_ERR_TIMEOUT : DD_ERR_CUDA;
  }
  float ms = 0.f;
  cudaEventElapsedTime(&ms, h->ev0, h->ev1);
  h->stats.t_solve_ms = ms;
  h->stats.refine_iters = iters;
  h->stats.refine_last = ratio;
  h->stats.launches_solve = h->launches;
  return status;
}

int dd_get_schur(const dd_handle* h, int32_t i, dd_c128* out, int32_t* duals, int32_t* m_out) {
  if (!h || i < 0 || i >= h->n_sub) return DD_ERR_INVALID_ARG;
  const FrontDev& F = h->fronts[i];
  const int m = F.nu;
  if (m_out) *m_out = m;
  if (duals) std::copy(h->leaf_duals[i].begin(), h->leaf_duals[i].end(), duals);
  if (!out) return DD_OK;
  if (!h->factored) return DD_ERR_NOT_FACTORED;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(h->device);
  struct Restore { int d; ~Restore() { cudaSetDevice(d); } } restore{cur};
  std::vector<unsigned char> blk((size_t)m * m * h->elem);
  const unsigned char* src = (const unsigned char*)h->pool + ((size_t)F.off + (size_t)F.ne_pad * F.ld + F.ne_pad) * h->elem;
  if (m) {
    DD_CUDA(cudaMemcpy2D(blk.data(), (size_t)m * h->elem, src, (size_t)F.ld * h->elem, (size_t)m * h->elem, m,
                         cudaMemcpyDeviceToHost));
  }
  // the trailing block holds -F_i in its lower triangle, rows in the front's
  // B-row order: pos[a] is the row of the a-th dual in ascending order
  std::vector<int> pos(m);
  for (int r = 0; r < m; ++r)
    pos[std::lower_bound(h->leaf_duals[i].begin(), h->leaf_duals[i].end(), h->leaf_upd[i][r]) -
        h->leaf_duals[i].begin()] = r;
  for (int a = 0; a < m; ++a)
    for (int b = 0; b < m; ++b) {
      const int hi = std::max(pos[a], pos[b]), lo = std::min(pos[a], pos[b]);
      double re, im;
      if (h->elem == 16) {
        const double* v = (const double*)blk.data() + 2 * ((size_t)hi * m + lo);
        re = v[0];
        im = v[1];
      } else {
        const float* v = (const float*)blk.data() + 2 * ((size_t)hi * m + lo);
        re = v[0];
        im = v[1];
      }
      out[(size_t)b * m + a] = dd_c128{-re, -im};
    }
  return DD_OK;
}

int dd_selftest_wait_timeout(void* cuda_stream) {
  cudaStream_t s = (cudaStream_t)cuda_stream;
  int32_t* flag = nullptr;
  DevStatus* st = nullptr;
  if (cudaMalloc(&flag, sizeof(int32_t)) != cudaSuccess) return DD_ERR_OOM;
  if (cudaMalloc(&st, sizeof(DevStatus)) != cudaSuccess) {
    cudaFree(flag);
    return DD_ERR_OOM;
  }
  int code = DD_ERR_CUDA;
  DevStatus host{};
  if (cudaMemsetAsync(flag, 0, sizeof(int32_t), s) == cudaSuccess &&
      cudaMemsetAsync(st, 0, sizeof(DevStatus), s) == cudaSuccess) {
    ddk::launch_wait_probe(flag, st, s);
    if (cudaGetLastError() == cudaSuccess &&
        cudaMemcpyAsync(&host, st, sizeof(host), cudaMemcpyDeviceToHost, s) == cudaSuccess &&
        cudaStreamSynchronize(s) == cudaSuccess)
      code = host.code == 8 ? DD_ERR_TIMEOUT : (host.code == 0 ? DD_OK : DD_ERR_CUDA);
  }
  cudaFree(flag);
  cudaFree(st);
  return code;
}

int dd_selftest_pivot_tile(const float* tile, int32_t precision, float* out_tile, float* out_linv,
                           void* cuda_stream) {
  if (!tile || !out_tile || !out_linv || precision < 0 || precision > 2) return DD_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  constexpr size_t kTile = (size_t)T * T * sizeof(float2);
  float2* pool = nullptr;
  float2* linv = nullptr;
  FrontDev* fr = nullptr;
  int32_t* fid = nullptr;
  DevStatus* st = nullptr;
  int code = DD_ERR_OOM;
  if (cudaMalloc(&pool, kTile) == cudaSuccess && cudaMalloc(&linv, kTile) == cudaSuccess &&
      cudaMalloc(&fr, sizeof(FrontDev)) == cudaSuccess && cudaMalloc(&fid, sizeof(int32_t)) == cudaSuccess &&
      cudaMalloc(&st, sizeof(DevStatus)) == cudaSuccess) {
    FrontDev F{};
    F.ld = T;
    F.ne = T;
    F.ne_pad = T;
    F.kind = 1;
    F.sub = -1;
    F.child[0] = F.child[1] = -1;
    const int32_t zero = 0;
    DevStatus host{};
    code = DD_ERR_CUDA;
    if (cudaMemcpyAsync(pool, tile, kTile, cudaMemcpyHostToDevice, s) == cudaSuccess &&
        cudaMemcpyAsync(fr, &F, sizeof(F), cudaMemcpyHostToDevice, s) == cudaSuccess &&
        cudaMemcpyAsync(fid, &zero, sizeof(zero), cudaMemcpyHostToDevice, s) == cudaSuccess &&
        cudaMemsetAsync(st, 0, sizeof(DevStatus), s) == cudaSuccess) {
      ddk::launch_diag_tile(precision, pool, fr, fid, st, linv, s);
      if (cudaGetLastError() == cudaSuccess &&
          cudaMemcpyAsync(out_tile, pool, kTile, cudaMemcpyDeviceToHost, s) == cudaSuccess &&
          cudaMemcpyAsync(out_linv, linv, kTile, cudaMemcpyDeviceToHost, s) == cudaSuccess &&
          cudaMemcpyAsync(&host, st, sizeof(host), cudaMemcpyDeviceToHost, s) == cudaSuccess &&
          cudaStreamSynchronize(s) == cudaSuccess)
        code = host.code == 3 ? DD_ERR_SINGULAR_PIVOT : (host.code == 0 ? DD_OK : DD_ERR_CUDA);
    }
  }
  cudaFree(pool);
  cudaFree(linv);
  cudaFree(fr);
  cudaFree(fid);
  cudaFree(st);
  return code;
}

int dd_get_stats(const dd_handle* h, dd_stats* out) {
  if (!h || !out) return DD_ERR_INVALID_ARG;
  *out = h->stats;
  out->bytes_device = (int64_t)h->arena.bytes;
  return DD_OK;
}

}  // extern "C"
