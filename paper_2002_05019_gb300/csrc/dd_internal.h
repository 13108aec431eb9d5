// Internal data structures shared by the host driver and the device kernels.
//
// Every elimination in the solver is a partial dense LDL^T of a "front": a
// square, symmetric block stored row-major (lower triangle used) whose first
// ne_pad rows/columns are eliminated and whose trailing block becomes the
// Schur contribution passed to the parent front.
//   * a leaf front is one domain's arrowhead block [A_i B_i^T; B_i 0]
//     (rows: interior unknowns, interface unknowns, identity padding, then the
//     m_i dual unknowns touching the domain); eliminating its n_i primal rows
//     leaves -F_i = -B_i A_i^{-1} B_i^T in the trailing block (Section II:
//     primal elimination and the domain's auxiliary-matrix contribution);
//   * a node front belongs to a node of the domain tree: its separator duals
//     (interfaces whose domains meet first at this node) followed by the
//     ancestor duals it couples to; it assembles its children's trailing
//     blocks and eliminates its separator (Section II: block LDL^T of the
//     block-wise sparse auxiliary matrix, structure from the clique graph).
#pragma once
#include <string>

#include <cuda_runtime.h>
#include <stdint.h>

#define DD_TILE 64

struct FrontDev {
  int64_t off;       // element offset of the front in the front pool
  int64_t roff;      // element offset of its right-hand-side block (ld * nrhs)
  int32_t ld;        // padded order (multiple of DD_TILE)
  int32_t ne;        // eliminated unknowns (unpadded)
  int32_t ne_pad;    // eliminated unknowns padded to DD_TILE (identity padding)
  int32_t nu;        // update (trailing) rows, unpadded
  int32_t n_int;     // leaf: number of interior unknowns (B rows vanish before it); node: 0
  int32_t kind;      // 0 dense domain front, 1 separator front of the auxiliary matrix, 2 front of a
                     // sparse domain's nested-dissection tree (rows given by row ids; the root,
                     // front i of domain i, has the domain's duals as update rows)
  int32_t sub;       // leaf and sparse-domain fronts: domain id; node: -1
  int32_t upd_off;   // offset of the nu dual ids of the update rows
  int32_t sep_off;   // node / sparse-domain front: offset of the ne row ids of its own rows
  int32_t child[2];  // node: child fronts (-1 if absent)
  int32_t map_off[2];// node: offsets of the extend-add maps (child update row -> row here)
  int32_t imap_off[2];// separator front: offsets of the inverse maps (row here -> child update row or -1)
  int32_t tile_off;  // offset of this front's per-tile ready flags (ld / DD_TILE of them)
  int32_t piv;       // 1: its diagonal tiles use restricted Bunch-Kaufman pivoting
  int64_t ws_off;    // mixed form: byte offset of this front's A operand images in the panel workspace
  int64_t ws_boff;   // mixed form: byte offset of its B operand images
};

// Panel operand images for the tensor-core trailing update (mixed form), one
// per trailing 64-row tile t of a panel step, 128B-swizzled K-major, in pieces
// of 128 rows x one K atom (32 tf32) = 16 KB, indexed (split hi/lo, atom):
//   A image (rows of L): within a piece, for each group of 16 tile rows, their
//     real parts then their imaginary parts (piece row 32 (r / 16) + r % 16 and
//     + 16), so the two parts of a row land in one TMEM sub-partition;
//   B image (rows of W = L D, fronts that pivot only): the same layout.
// Unpivoted fronts write only the A image, of M = L D^(1/2), which the update
// reads as both operands (L_i D L_j^T = M_i M_j^T).
#define DD_TC_ATOM 16384
#define DD_TC_ATILE (2 * 2 * DD_TC_ATOM)
#define DD_TC_BTILE (2 * 2 * DD_TC_ATOM)

struct LeafDev {
  int64_t csr_off;   // offset of the domain's nonzeros in the concatenated CSR arrays
  int64_t vec_off;   // offset of the domain's rows in the stacked f / u vectors
  int32_t rowptr_off;// offset of its n+1 row pointers
  int32_t n;         // local unknowns
  int32_t perm_off;  // offset of perm (front row -> local row) and iperm (local row -> front row)
  int32_t b_off;     // offset of its B entries
  int32_t nb;        // number of B entries
  int32_t front;     // front id
};

// Task of the batched partial LDL^T: front f, row tile i, column tile j.
struct Task { int32_t f, i, j, pad; };

// Device status word: first error seen by any kernel.
struct DevStatus {
  int32_t code;      // 0 ok, 3 singular pivot, 8 a bounded wait gave up
  int32_t front;     // front where it happened
  int32_t row;       // row inside the front
  int32_t pad;
  unsigned long long max_abs_d;   // bit pattern of a non-negative double: max |d|
  unsigned long long min_abs_d;   // min |d| over real (unpadded) pivots
  unsigned long long max_abs_l;   // max |l * d| entry written by the panel kernels
  unsigned long long n_swap;      // restricted Bunch-Kaufman: symmetric interchanges
  unsigned long long n_2x2;       // restricted Bunch-Kaufman: 2 x 2 pivots
};

// autotuner schedule cache (dd_tune.cu): the problem key of a front tree and
// the cache key adding the device's name and SM count
uint64_t tune_problem_key(int n_front, const int32_t* parent, const int32_t* ne, const int32_t* nu, int n_dual,
                          int precision, int pivoting);
std::string tune_cache_key(uint64_t problem_key, int device);

namespace ddk {

// ---- factorization (templated on storage: 0 = double2, 1 = float2) -------------
void launch_zero(void* p, size_t bytes, cudaStream_t s);
void launch_leaf_init(int prec, void* pool, const FrontDev* fronts, const LeafDev* leaves, int n_leaves,
                      const int32_t* rowptr, const int32_t* colind, const double2* val,
                      const int32_t* iperm, const int32_t* b_row, const int32_t* b_local,
                      const int8_t* b_sign, cudaStream_t s);
void launch_node_init(int prec, void* pool, const FrontDev* fronts, const int32_t* node_ids, int n,
                      cudaStream_t s);
// sparse-domain fronts: pool[dst[e]] = val[src[e]] (src -1: +1, -2: -1)
void launch_sparse_init(int prec, void* pool, const int64_t* dst, const int32_t* src, int64_t n, const double2* val,
                        cudaStream_t s);
// piv (optional): one byte per pivot position of every diagonal tile (index
// (tile_off + tile) * 64 + c), the permutation of the restricted Bunch-Kaufman
// pivoting of the fronts with FrontDev::piv set; nullptr: no front pivots
// FP64 form only (prec = 0, diag_fp64 = 0): 64 x 64 diagonal tile and panel tiles in FP64
void launch_diag(int prec, int diag_fp64, void* pool, const FrontDev* fronts, const int32_t* fids, int n,
                 int k, DevStatus* st, cudaStream_t s, uint8_t* piv = nullptr);
void launch_trsm(int prec, void* pool, const FrontDev* fronts, const Task* tasks, int n, int k,
                 DevStatus* st, cudaStream_t s, unsigned char* ws = nullptr, const uint8_t* piv = nullptr);
// mixed form: 64 x 64 diagonal tile with 32 x 32 pivot blocks (diag_fp64: 0
// FP32, 1 FP64, 2 FP64 for separator fronts and FP32 for domain fronts) and
// L_kk^{-1} (FP32, 64 x 64 per front id) for the panel product
void launch_diag_mx(int diag_fp64, void* pool, const FrontDev* fronts, const int32_t* fids, int n, int k,
                    DevStatus* st, void* linv, cudaStream_t s, uint8_t* piv = nullptr);
// one 64 x 64 mixed-form diagonal tile (front 0 of `front`, step 0), unpivoted:
// prec 0 FP32 pivot blocks, 1 double-float, 2 FP64 (diagnostics)
void launch_diag_tile(int prec, void* pool, const FrontDev* front, const int32_t* fid, DevStatus* st, void* linv,
                      cudaStream_t s);
// tensor != 0: the product with L_kk^{-1} on the tensor cores (tcgen05 3xTF32), else on the FP32 FMA pipes
void launch_trsm_mx(void* pool, const FrontDev* fronts, const Task* tasks, int n, int k, DevStatus* st,
                    const void* linv, unsigned char* ws, cudaStream_t s, const uint8_t* piv = nullptr,
                    int tensor = 0);
// tensor-core trailing update (mixed form): task (front, row tile i, column
// tile j); .pad bits 0 / 1 store column tiles j / j + 1, bits 2..5 add the
// products of panels k .. k + 3 (images in ws.p[0 .. 3]).
// groups: (first task, count) of runs of tasks of one row tile; n = number of groups;
// counter: a zeroed int in device memory used to claim groups dynamically (one per launch)
struct PanelImages { const unsigned char* p[4]; };
void launch_update_tc(void* pool, const FrontDev* fronts, const Task* tasks, const int2* groups, int n, int k,
                      const PanelImages& ws, DevStatus* st, cudaStream_t s, int reserve_sms, int* counter);
void launch_update(int prec, void* pool, const FrontDev* fronts, const Task* tasks, int n, int k,
                   cudaStream_t s);
void launch_extend_add(int prec, void* pool, const FrontDev* fronts, const int32_t* node_ids, int n,
                       int slot, const int32_t* maps, int max_nu, cudaStream_t s);
// lower-triangular tiles (tile row t: columns [0, 64 (t + 1))) of the listed
// (front, tile row) pairs set to zero; elem = bytes per complex entry
void launch_zero_lower(void* pool, int elem, const FrontDev* fronts, const int2* tiles, int64_t n, cudaStream_t s);
// assembly of the separator fronts (kind 1) of a level by pulling their
// children's trailing blocks: every entry of the lower-triangular tiles written
// once (no zeroing, no read-modify-write); other fronts are skipped
void launch_assemble(int prec, void* pool, const FrontDev* fronts, const int32_t* node_ids, int n,
                     const int32_t* imaps, int max_ld, cudaStream_t s);

// ---- solve --------------------------------------------------------------------
void launch_rhs_leaf(int prec, void* rpool, const FrontDev* fronts, const LeafDev* leaves, int n_leaves,
                     const int32_t* perm, const double2* f, int64_t ldf, int nrhs, cudaStream_t s);
// separator fronts: own rows <- g (NULL: zero); sparse-domain fronts: own rows <- f
// by row id (n_dual + stacked row); dense domain fronts are left alone
void launch_rhs_node(int prec, void* rpool, const FrontDev* fronts, const int32_t* node_ids, int n,
                     const int32_t* sep, const double2* g, int64_t ldg, const double2* f, int64_t ldf, int n_dual,
                     int nrhs, cudaStream_t s);
void launch_rhs_extend_add(int prec, void* rpool, const FrontDev* fronts, const int32_t* node_ids, int n,
                           int slot, const int32_t* maps, int nrhs, cudaStream_t s);
// tile-parallel substitution: one CTA per (front, tile) task of a level; a
// CTA waits (bounded) on the ready flags of the tiles it depends on
// linv (mixed form, optional): FP32 inverses of the unit-lower diagonal tiles,
// index tile_off + tile; when given, the in-tile triangular solves are products
// tensor != 0 (mixed form, 4..64 right-hand sides): the tile products on the
// tensor cores (tcgen05 3xTF32), else on the FP32 FMA pipes
void launch_forward(int prec, const void* pool, void* rpool, const FrontDev* fronts, const Task* tasks, int n,
                    int nrhs, int32_t* flags, int epoch, DevStatus* st, cudaStream_t s,
                    const void* linv = nullptr, const uint8_t* piv = nullptr, int tensor = 0);
// upart (optional, separator levels): scratch for the update-row partial sums
// (n x nsplit x nrhs x 64 elements); the update-row product then runs as a
// separate launch split nsplit ways.  Returns the number of kernels launched.
int launch_backward(int prec, const void* pool, void* rpool, const FrontDev* fronts, const Task* tasks, int n,
                    int nrhs, const int32_t* upd, const int32_t* sep, void* lam_work, int64_t ld_lam,
                    int32_t* flags, int epoch, DevStatus* st, cudaStream_t s, const void* linv = nullptr,
                    const uint8_t* piv = nullptr, void* upart = nullptr, int nsplit = 0, int tensor = 0);
// u of every listed domain: from its dense front (rows through perm) or, for a
// sparse domain, from the row-id vector lam (ld_lam, rows n_dual + stacked row)
void launch_leaf_out(int prec, const void* rpool, const FrontDev* fronts, const LeafDev* leaves,
                     int n_leaves, const int32_t* perm, double2* u, int64_t ldu, int nrhs, int accumulate,
                     cudaStream_t s, const void* lam, int64_t ld_lam, int n_dual);
void launch_lam_out(int prec, const void* lam_work, int64_t ld_work, int n_dual, int nrhs, double2* lam,
                    int64_t ldl, int accumulate, cudaStream_t s);

// ---- FP64 arrowhead residual and refinement helpers -----------------------------
void launch_residual(const LeafDev* leaves, int n_leaves, const int32_t* rowptr, const int32_t* colind,
                     const double2* val, const int32_t* b_dual_glob, const int32_t* b_local,
                     const int8_t* b_sign, const double2* f, int64_t ldf, const double2* u, int64_t ldu,
                     const double2* lam, int64_t ldl, double2* r, int64_t ldr, int nrhs, cudaStream_t s);
void launch_dual_residual(int n_dual, const int32_t* bt_ptr, const int64_t* bt_row, const int8_t* bt_sign,
                          const double2* u, int64_t ldu, double2* rl, int64_t ldrl, int nrhs,
                          cudaStream_t s);
// diagnostic: one CTA waits (bounded) on *flag >= 1
void launch_wait_probe(const int32_t* flag, DevStatus* st, cudaStream_t s);
// per-column partial sums of |x|^2: out[col * blocks + b]
void launch_sumsq_cols(const double2* x, int64_t n, int ncols, int blocks, double* out, cudaStream_t s);
// partial sums of |x|^2 per block into out[blocks]; returns block count used
int launch_sumsq(const double2* x, int64_t n, double* out, int max_blocks, cudaStream_t s);

}  // namespace ddk
