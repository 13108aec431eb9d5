/*
 * dd.h - C ABI of the GB300 direct domain-decomposition (DD) solver.
 *
 * The solver implements the direct DD strategy of Moshfegh & Vouvakis,
 * "Direct Solution of FEM Models: Are Sparse Direct Solvers the Best
 * Strategy?" (ICEAA 2017), Section II:
 *   - the FEM problem is decomposed into domains with primal unknowns u_i in
 *     each domain volume and dual unknowns lambda on the interfaces, giving the
 *     sparse arrowhead system
 *         [ blkdiag(A_i)  B^T ] [ u      ]   [ f ]
 *         [ B             0   ] [ lambda ] = [ g ]             (g = 0 here);
 *   - the primal unknowns are eliminated by many independent factorizations
 *     A_i = L_i D_i L_i^T;
 *   - the resulting auxiliary matrix F = sum_i B_i A_i^{-1} B_i^T is symmetric,
 *     much smaller, and sparse at the level of dense blocks; its block structure is found by a symbolic step on the clique
 *     graph of the domains and it is factored by a block LDL^T;
 *   - the primal unknowns are recovered by many small forward/backward
 *     substitutions, one per domain.
 * Matrices are complex symmetric (A = A^T, no conjugation).  The paper defers
 * the exact decomposed formulation to its references; this library uses the
 * FETI-style arrowhead above with lossy (nonsingular) domains.
 *
 * Threading: one handle per CUDA stream; calls on one handle are not
 * reentrant.  Every call returns a dd_status code and never throws.
 */
#ifndef DD_GB300_H
#define DD_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Interleaved complex double, layout-compatible with C99 double _Complex,
 * numpy complex128 and torch.complex128. */
typedef struct { double re, im; } dd_c128;

typedef struct dd_handle dd_handle;

typedef enum {
  DD_OK = 0,
  DD_ERR_INVALID_ARG = 1,     /* bad size, NULL pointer, index out of range      */
  DD_ERR_NOT_SYMMETRIC = 2,   /* a domain CSR is not structurally/numerically symmetric */
  DD_ERR_SINGULAR_PIVOT = 3,  /* a zero or non-finite pivot appeared in dd_factor */
  DD_ERR_OOM = 4,             /* device or host allocation failed                */
  DD_ERR_CUDA = 5,            /* a CUDA runtime call failed                      */
  DD_ERR_NOT_FACTORED = 6,    /* dd_solve before a successful dd_factor          */
  DD_ERR_NOT_CONVERGED = 7,   /* refinement stopped above refine_tol (best iterate written) */
  DD_ERR_TIMEOUT = 8,         /* a bounded device wait gave up                   */
  DD_ERR_NO_DEVICE = 9        /* no usable CUDA device                           */
} dd_status;

typedef enum { DD_PREC_FP64 = 0, DD_PREC_MIXED = 1 } dd_precision;

/* One domain of the arrowhead system (Section II: primal unknowns live in
 * the domain volumes, dual unknowns on the domain interfaces).
 *   n        local primal unknowns (rows of A_i), n >= 1
 *   rowptr   n+1 entries, 0-based CSR row pointers of A_i
 *   colind   rowptr[n] column indices, sorted and unique within each row
 *   val      rowptr[n] complex values; the pattern must be symmetric and
 *            A_i = A_i^T to a relative 1e-12 (checked: DD_ERR_NOT_SYMMETRIC)
 *   nb       number of nonzeros of B_i
 *   b_dual   nb dual (multiplier) ids in [0, n_dual)
 *   b_local  nb local rows in [0, n)
 *   b_sign   nb entries, +1 or -1: B_i[b_dual[k], b_local[k]] = b_sign[k]
 * All arrays are HOST memory; dd_setup deep-copies them. */
typedef struct {
  int32_t n;
  const int32_t* rowptr;
  const int32_t* colind;
  const dd_c128* val;
  int32_t nb;
  const int32_t* b_dual;
  const int32_t* b_local;
  const int8_t* b_sign;
} dd_subdomain;

typedef struct {
  int32_t precision;        /* DD_PREC_FP64: every step in FP64 complex.
                               DD_PREC_MIXED: complex64 factors and solves,
                               wide pivot blocks of the auxiliary matrix (double-float,
                               an FP32 pair of about 48 bits; FP64 with pivoting) and
                               FP64 iterative refinement on the arrowhead system. */
  double refine_tol;        /* MIXED: stop when |du|/|u| <= refine_tol, or when the error left
                               after the update, estimated from the contraction of successive
                               corrections (|du_k|^2 / |du_k-1|, the direct solve being du_0
                               of relative size 1), is <= refine_tol (default 1e-13) */
  int32_t max_refine;       /* MIXED: refinement iteration cap (default 10); FP64: extra
                               FP64 refinement steps after the direct solve (default 0) */
  int32_t pivoting;         /* 0: unpivoted LDL^T everywhere (it exists for lossy domains).
                               1: restricted Bunch-Kaufman pivoting (Section II) in the diagonal
                                  blocks of the auxiliary-matrix fronts: 64 x 64 tiles (FP64 form)
                                  or 32 x 32 FP64 pivot blocks (mixed form); the domains unpivoted.
                               2: the same in the domain fronts too.
                               Pivots never leave their diagonal block, so the symbolic structure
                               is unchanged; other values: DD_ERR_INVALID_ARG. */
  const int32_t* tree_parent; /* optional, 2*n_sub-1 entries: binary domain tree, leaves
                                 0..n_sub-1 are the domains, internal nodes n_sub.. with every
                                 parent id larger than its children's, root parent = -1.
                                 NULL: built by recursive bisection of `centroids`. */
  const double* centroids;  /* optional, 3*n_sub: domain centres used when tree_parent is NULL;
                               NULL too: bisection by domain index */
  void* cuda_stream;        /* cudaStream_t for every device call; NULL = legacy default stream */
  int32_t device;           /* CUDA device ordinal */
  int32_t time_kernels;     /* 1: dd_factor brackets every launch with CUDA events and reports
                               per-kernel-class device time in dd_stats (slower; default 0);
                               2: only the trailing-update launches (DD_K_UPDATE, the dominant
                               kernel), the other classes reporting 0 */
  int32_t simt_update;      /* MIXED: 1 runs the trailing updates on the FP32 FMA pipes instead of
                               the tensor cores (comparison baseline; default 0) */
  int32_t update_panels;    /* MIXED, tensor cores: panels fused per trailing-update pass, 1 (C read
                               and written after every 64-wide panel), 2 (after every pair of
                               panels, K = 128; default) or 4 (after every four panels, K = 256,
                               on tree levels without look-ahead; the others use pairs); other
                               values: DD_ERR_INVALID_ARG */
  int32_t sparse_min;       /* Section II factors each domain with a sparse direct solver: domains of
                               at least sparse_min unknowns are split into a tree of fronts by nested
                               dissection of their matrix graph (interface unknowns last, in the
                               domain's root front, whose update rows are the domain's duals), the
                               others stay one dense front.  0 (default): every domain is one dense
                               front; negative: DD_ERR_INVALID_ARG */
  int32_t sparse_leaf;      /* largest leaf front of that dissection (0: 256); negative: DD_ERR_INVALID_ARG */
  const char* tune_cache;   /* optional path of the autotuner's schedule cache (JSON lines, one per
                               tuned problem and GPU model; see dd_tune_cache_lookup): dd_setup
                               applies a cached schedule of this problem, dd_autotune returns it
                               without timing (configs_tried = 0) or tunes and appends one line.
                               NULL (default): no cache.  The string is copied at setup. */
} dd_options;

/* Kernel classes of dd_stats.kernel_ms / kernel_launches / kernel_flops. */
enum { DD_K_DIAG = 0, DD_K_TRSM = 1, DD_K_UPDATE = 2, DD_K_ASSEMBLE = 3, DD_K_INIT = 4, DD_K_NCLASS = 5 };

/* Per-handle statistics filled by dd_factor / dd_solve. */
typedef struct {
  int32_t n_sub, n_dual, n_fronts, n_levels;
  int64_t n_primal;          /* sum of n_i */
  int32_t max_front;         /* largest dual front (rows) */
  double flops_factor;       /* algorithmic real flops of one dd_factor (8 per complex multiply-add) */
  double flops_solve;        /* algorithmic real flops of one direct solve with one right-hand side */
  int64_t bytes_factor;      /* bytes of the stored factors (L, D of every front) */
  int64_t bytes_device;      /* device bytes held by the handle */
  double t_setup_ms;          /* dd_setup wall time: validation, symbolic analysis, device uploads */
  double t_factor_ms, t_solve_ms;   /* last call, device-timed */
  double growth;             /* max |L D| entry / max |A| entry over all fronts (pivot growth) */
  double min_pivot;          /* min |d| over all pivots */
  int32_t refine_iters;      /* last dd_solve */
  double refine_last;        /* last |du|/|u| */
  int32_t launches_factor;   /* kernels launched by one dd_factor */
  int32_t launches_solve;    /* kernels launched by the last dd_solve */
  double kernel_ms[DD_K_NCLASS];        /* time_kernels: summed device time per class, last dd_factor */
  int32_t kernel_launches[DD_K_NCLASS]; /* launches per class in one dd_factor */
  double kernel_flops[DD_K_NCLASS];     /* algorithmic real flops per class in one dd_factor, counted on
                                           the fronts' exact sizes (tile padding not counted) */
  int64_t interchanges;      /* pivoting: symmetric interchanges in the last dd_factor */
  int64_t pivots_2x2;        /* pivoting: 2 x 2 pivot blocks in the last dd_factor */
} dd_stats;

/* Schedule of the tensor-core factorization path (MIXED form). */
typedef struct {
  int32_t update_panels;  /* panels fused per trailing-update pass: 1, 2 or 4 */
  int32_t ahead_fronts;   /* one-step look-ahead on tree levels with at most this many fronts (0: none) */
  int32_t reserve_sms;    /* SMs the look-ahead update leaves to the panel chain */
  double factor_ms;       /* dd_autotune: device time of one dd_factor with this schedule */
  int32_t configs_tried;  /* dd_autotune: schedules timed */
  int32_t split_sms;      /* 0: the leaf level (the domain fronts) as one launch sequence; 1..120: as
                             two halves of about equal work on two streams, every trailing update of
                             a half leaving this many SMs to the other half's panel chain, so that
                             one half's bandwidth-bound panels overlap the other's tensor-core
                             updates */
} dd_schedule;

/* Fill `opt` with defaults (FP64, no tree, default stream, device 0). */
int dd_default_options(dd_options* opt);

/* Analyse and upload the arrowhead system (Section II: decomposed BVP with
 * primal and dual unknowns; the symbolic factorization on the clique graph
 * of the block-wise sparse auxiliary matrix).  Validates every input, orders
 * each domain's unknowns interior-first / interface-last, builds the
 * separator tree of the dual unknowns from the domain tree, computes the
 * dense-block structure of the auxiliary factor, and copies all values to
 * the device.  n_sub >= 1, n_dual >= 0.  On success *out owns all device
 * memory of the solve; on failure *out is NULL and nothing is leaked. */
int dd_setup(dd_handle** out, int32_t n_sub, const dd_subdomain* subs, int32_t n_dual,
             const dd_options* opt);

/* Replace the numeric values of every A_i (same patterns as at setup): `vals`
 * holds sum_i rowptr_i[n_i] complex values, domain after domain, host or
 * device memory (detected).  The handle becomes unfactored. */
int dd_set_values(dd_handle* h, const dd_c128* vals);

/* Set the schedule of the tensor-core path (update_panels 1, 2 or 4, ahead_fronts
 * in [0, 1024], reserve_sms in [0, 64], split_sms in [0, 120]); factor_ms and
 * configs_tried are ignored.
 * The factors already computed stay valid; the next dd_factor uses the new
 * schedule.  No effect in the FP64 form or with simt_update.
 * DD_ERR_INVALID_ARG for values out of range. */
int dd_set_schedule(dd_handle* h, const dd_schedule* sched);

/* Autotuner: times dd_factor (the minimum over `repeats` runs each) under every
 * schedule of the grid update_panels {1, 2, 4} x ahead_fronts {0, 8, 32, 128, 1024} x
 * reserve_sms {8, 16, 32} (look-ahead off: reserve not varied) with split_sms 0,
 * then the best of those with split_sms {24, 40, 64} (when the leaf level has
 * two fronts or more), keeps the fastest for this handle and returns it in
 * *out; the handle is left factored with it.  FP64 form / simt_update: one
 * dd_factor, configs_tried = 1.
 * Errors: as dd_factor; DD_ERR_INVALID_ARG for repeats < 1 or out == NULL. */
int dd_autotune(dd_handle* h, int32_t repeats, dd_schedule* out);

/* Numeric factorization (Section II): A_i = L_i D_i L_i^T for every domain
 * together with its Schur contribution -F_i, assembly of the auxiliary matrix
 * into dense blocks, and the block LDL^T of the auxiliary matrix.  Runs on
 * the handle's stream and returns after the stream has finished it. */
int dd_factor(dd_handle* h);

/* Solve the arrowhead system for nrhs right-hand sides (Section II: primal
 * elimination, auxiliary solve, recovery of the primal unknowns).
 *   f       (sum_i n_i) x nrhs, column-major, leading dimension ldf: the local
 *           loads f_i stacked domain after domain, each in the caller's local
 *           row order given at setup
 *   u       same layout (ldu): the local solutions u_i
 *   lambda  n_dual x nrhs, column-major (ldl), or NULL: the dual solution
 * Pointers may be host or device memory (detected per pointer).  In MIXED
 * precision the result is refined in FP64 on the arrowhead system; if it does
 * not reach refine_tol the best iterate is written and DD_ERR_NOT_CONVERGED
 * returned. */
int dd_solve(dd_handle* h, int32_t nrhs, const dd_c128* f, int64_t ldf, dd_c128* u, int64_t ldu,
             dd_c128* lambda, int64_t ldl);

/* Solve as dd_solve but recover the primal unknowns of the listed domains only
 * (Section II: only the requested subdomains' primal unknowns need be
 * recovered after the auxiliary solve).
 *   f       all domains' loads, as for dd_solve
 *   req     n_req distinct domain ids in [0, n_sub), host memory
 *   u       (sum over req of n_i) x nrhs, column-major (ldu): u_i of the listed
 *           domains stacked in the order of req, each in its caller row order
 *   lambda  as for dd_solve (all duals), or NULL
 * Without refinement (FP64 form, max_refine = 0) the backward substitution
 * and output run for the listed domains only; with refinement every domain
 * is solved (the FP64 residual needs all of u) and the listed rows returned.
 * Errors: DD_ERR_INVALID_ARG for a bad, repeated or out-of-range id or a short
 * ldu; otherwise as dd_solve. */
int dd_solve_subset(dd_handle* h, int32_t nrhs, const dd_c128* f, int64_t ldf, int32_t n_req, const int32_t* req,
                    dd_c128* u, int64_t ldu, dd_c128* lambda, int64_t ldl);

/* Copy F_i = B_i A_i^{-1} B_i^T of domain i (Section II: the domain's
 * contribution to the auxiliary matrix) into host memory `out`
 * (m_i x m_i, column-major, ld m_i), with `duals` (m_i entries, may be NULL)
 * receiving the ascending dual ids of its rows.  *m_out receives m_i; call
 * with out == NULL to query m_i only.  Requires a factored handle. */
int dd_get_schur(const dd_handle* h, int32_t i, dd_c128* out, int32_t* duals, int32_t* m_out);

int dd_get_stats(const dd_handle* h, dd_stats* out);

/* Static description of a status code. */
const char* dd_strerror(int code);

/* Release the handle and all its device memory.  NULL is a no-op. */
void dd_free(dd_handle* h);

/* ---------------------------------------------------------------------------
 * Allocation-free dense solve.  The paper has no counterpart: this is a
 * service for callers that cannot allocate device memory once they are
 * running (an application whose own allocator owns all device memory, or a
 * loop that cannot afford cudaMalloc's implicit synchronisation or failure).
 *
 * Solves A X = B for one dense complex-symmetric A (A = A^T, lower triangle
 * read, unpivoted LDL^T in FP64 with the same kernels as dd_factor/dd_solve).
 *   n      1..DD_NOALLOC_MAX_N;  nrhs  1..DD_NOALLOC_MAX_NRHS
 *   A      device memory, n x n column-major, leading dimension lda >= n
 *   b      device memory, n x nrhs column-major (ldb >= n)
 *   x      device memory, n x nrhs column-major (ldx >= n), written
 *   cuda_stream  stream for all work (NULL = legacy default stream)
 * A, b and x must be device memory of the CURRENT device (or managed memory);
 * host memory and device memory of another GPU are refused. 
 * Allocates nothing: all scratch is one static device array of about 4.3 MB
 * that every GPU loading this library holds until the process exits.  The
 * first call on a device looks up that array's device address; make that
 * first call before any stream capture.  Every call clears what must start
 * at zero, but all calls share the one array: calls that overlap on the GPU
 * (other streams, other host threads) race and must be serialised by the
 * caller.  Returns after the stream has finished the solve.  Errors:
 * DD_ERR_INVALID_ARG (sizes beyond the limits, NULL pointers, host memory or
 * another device's memory),
 * DD_ERR_SINGULAR_PIVOT, DD_ERR_TIMEOUT, DD_ERR_CUDA.
 * ------------------------------------------------------------------------- */
#define DD_NOALLOC_MAX_N 512
#define DD_NOALLOC_MAX_NRHS 16
int dd_dense_solve_noalloc(int32_t n, const dd_c128* A, int64_t lda, int32_t nrhs, const dd_c128* b,
                           int64_t ldb, dd_c128* x, int64_t ldx, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* DD_GB300_H */
