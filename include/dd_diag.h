/*
 * dd_diag.h - diagnostics of the GB300 direct domain-decomposition solver.
 *
 * Not part of the method's data path: a check that the library's bounded
 * device-side waits give up and report an error instead of hanging, so that
 * failure detection can be tested without a GPU fault; and the front tree of
 * the symbolic analysis, so that it can be checked on a host without a GPU.
 */
#ifndef DD_GB300_DIAG_H
#define DD_GB300_DIAG_H

#include "dd.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Launch one CTA that waits on a device flag nothing ever sets, using the same
 * bounded wait as the tile-parallel substitution (about 2^24 polls, one to a
 * few seconds).  Returns DD_ERR_TIMEOUT (8) when the wait gave up and the
 * status word reached the host; the CUDA context stays usable.  Allocates a
 * few bytes of device memory for the flag and the status word; runs on
 * `cuda_stream` (NULL = legacy default stream) and synchronises it. */
int dd_selftest_wait_timeout(void* cuda_stream);

/* Factor one 64 x 64 diagonal tile with the mixed form's diagonal kernel, as
 * a separator front of the auxiliary matrix would be (Section II: the block
 * LDL^T of the auxiliary matrix; unpivoted): the two 32 x 32 pivot blocks in
 * FP32 (precision 0), double-float (1: an FP32 pair, about 48 bits, the
 * library's choice for unpivoted separator fronts) or FP64 (2), the rest in
 * FP32.  tile: host, 64 x 64 complex64 interleaved (re, im), row-major, lower
 * triangle read.  out_tile (host, same layout): the factor, D on the
 * diagonal and L strictly below it (unit diagonal implied); the upper
 * triangle is left as it came in.  out_linv (host, same layout): L^-1, lower
 * triangular, zeros above.  Diagnostics for testing the pivot-block
 * precision; allocates and frees a few KB of device memory, runs on
 * `cuda_stream` (NULL = legacy default stream) and synchronises it.
 * Returns DD_OK, DD_ERR_SINGULAR_PIVOT (a zero or non-finite pivot),
 * DD_ERR_INVALID_ARG, DD_ERR_OOM or DD_ERR_CUDA. */
int dd_selftest_pivot_tile(const float* tile, int32_t precision, float* out_tile, float* out_linv,
                           void* cuda_stream);

/* The symbolic analysis of dd_setup alone (Section II: the auxiliary matrix
 * is factored after a symbolic factorization on the clique graph of the
 * domain interfaces), on the host, touching no device.  Same inputs and
 * validation as dd_setup (the same error codes for bad inputs).
 *
 * Fronts: 0 .. n_sub-1 are the domains (front i eliminates the n_i unknowns of
 * domain i), n_sub .. n_sub+n_sep-1 the separator fronts of the domain tree in
 * post-order (children before parents).  With opt->sparse_min > 0, front i of
 * a domain of at least sparse_min unknowns is the root of its nested-dissection
 * tree (it eliminates the interface unknowns) and the tree's other fronts
 * follow the separator fronts, domain after domain, children before parents;
 * their rows are given by row ids n_dual + (the row's index in the stacked
 * primal vector).  Outputs, all caller-allocated:
 *   n_front            number of fronts (also written when max_fronts is too small)
 *   parent[max_fronts] parent front, -1 at the root
 *   ne[max_fronts]     unknowns eliminated in the front (domain size, or separator duals)
 *   nu[max_fronts]     update rows of the front (duals passed on to ancestors)
 *   dual_front[n_dual] front that eliminates each dual (the lowest common
 *                      ancestor of the domains it touches)
 *   upd_ptr[max_fronts + 1], upd_idx[upd_cap] (optional, NULL to skip): the
 *                      update-row duals (or row ids) of front x are
 *                      upd_idx[upd_ptr[x] .. upd_ptr[x + 1]), in the library's row order
 * Returns DD_OK, DD_ERR_INVALID_ARG (bad inputs, a NULL output, max_fronts <
 * n_front or upd_cap too small), or dd_setup's other validation codes. */
int dd_symbolic(int32_t n_sub, const dd_subdomain* subs, int32_t n_dual, const dd_options* opt,
                int32_t max_fronts, int32_t* n_front, int32_t* parent, int32_t* ne, int32_t* nu,
                int32_t* dual_front, int64_t upd_cap, int64_t* upd_ptr, int32_t* upd_idx);

/* Nested-dissection symbolic analysis of one domain matrix, for domains
 * beyond the dense-front range (Section II factors each domain with a sparse
 * direct solver); host only, touching no device.  dd_setup uses the same
 * analysis for the domains selected by dd_options.sparse_min.  The rows flagged in is_last (the
 * interface rows that B couples to the duals; NULL: none) are eliminated last,
 * in the root front; the others by nested dissection -- separators are middle
 * levels of breadth-first level structures from pseudo-peripheral vertices --
 * down to leaves of at most leaf_max rows.
 *
 * Input: the n x n pattern in CSR (rowptr[n + 1], colind; 0-based, symmetric,
 * the diagonal optional).  Outputs, caller-allocated:
 *   n_front              fronts of the tree (also written when max_fronts is too small)
 *   parent[max_fronts]   parent front, -1 at the root; children precede parents
 *   ne[max_fronts]       rows eliminated in the front
 *   nu[max_fronts]       its update rows (later rows coupled to it or its subtree)
 *   order[n]             elimination order (row eliminated at position k)
 *   front_of[n]          front eliminating each row
 *   stored               entries of the fronts' strictly lower L: sum ne(ne-1)/2 + ne nu
 *   upd_ptr[max_fronts + 1], upd_idx[upd_cap] (optional, NULL to skip): the
 *                        update rows of front x, ascending
 * Returns DD_OK, DD_ERR_NOT_SYMMETRIC (pattern), or DD_ERR_INVALID_ARG (bad
 * sizes or indices, a NULL output, max_fronts or upd_cap too small). */
int dd_domain_symbolic(int32_t n, const int32_t* rowptr, const int32_t* colind, const int8_t* is_last,
                       int32_t leaf_max, int32_t max_fronts, int32_t* n_front, int32_t* parent, int32_t* ne,
                       int32_t* nu, int32_t* order, int32_t* front_of, int64_t* stored, int64_t upd_cap,
                       int64_t* upd_ptr, int32_t* upd_idx);

/* The assembly maps of the same analysis, for a multifrontal factorization
 * of the domain over its front tree.  Front x holds rows[rows_ptr[x] ..
 * rows_ptr[x + 1]): its ne[x] own rows, then its update rows, both in
 * elimination order.  Outputs, caller-allocated (call once with rows = NULL
 * for the sizes: n_front, parent, ne and rows_ptr are then written):
 *   parent[max_fronts], ne[max_fronts], rows_ptr[max_fronts + 1]
 *   rows[rows_cap]     the domain row of every front row
 *   ea_map[rows_cap]   for an update row of a front, its row in the parent
 *                      front (extend-add); -1 for own rows and at the root
 *   a_front[nnz], a_row[nnz], a_col[nnz]  for CSR entry q = (r, c): the front
 *                      and the (row, column) there that receive a_rc, column
 *                      r being an own row of that front; -1 for the entries
 *                      left to their mirror (c eliminated before r)
 * Returns as dd_domain_symbolic (DD_ERR_INVALID_ARG also for rows_cap too
 * small or a NULL map with rows given). */
int dd_domain_assembly(int32_t n, const int32_t* rowptr, const int32_t* colind, const int8_t* is_last,
                       int32_t leaf_max, int32_t max_fronts, int32_t* n_front, int32_t* parent, int32_t* ne,
                       int64_t rows_cap, int64_t* rows_ptr, int32_t* rows, int32_t* ea_map, int32_t* a_front,
                       int32_t* a_row, int32_t* a_col);

/* Shard plan of the front tree over n_ranks ranks (host only, touching no
 * device; multi-GPU sharding of Section II's independent domain factorizations
 * and of the tree of the auxiliary matrix's dense blocks).  The front tree is
 * dd_symbolic's (same inputs and options); it is cut into n_ranks subtrees of
 * about equal algorithmic work by repeatedly splitting the subtree of largest
 * work into its children.  Rank r owns the subtree rooted at rank_root[r]
 * (its domains and fronts); rank 0 also owns the fronts above the cuts.  The
 * exchange this implies: each cut subtree's root passes its Schur complement
 * (on its update duals, dd_symbolic's upd_idx) to the owner of its parent
 * front, and in a solve the right-hand side of those duals up and their
 * solved values down.
 * Outputs, caller-allocated: n_front; front_rank[max_fronts] (the owner of
 * every front); rank_root[n_ranks] (ascending front ids).
 * Returns DD_OK, DD_ERR_INVALID_ARG (n_ranks < 1, more ranks than the tree can
 * be cut into, a NULL output, max_fronts too small) or dd_symbolic's codes. */
int dd_shard_plan(int32_t n_sub, const dd_subdomain* subs, int32_t n_dual, const dd_options* opt, int32_t n_ranks,
                  int32_t max_fronts, int32_t* n_front, int32_t* front_rank, int32_t* rank_root);

/* Autotuner schedule cache (host only, no device).
 *
 * dd_tune_key: the problem key under which dd_setup and dd_autotune file a
 * schedule: a 64-bit FNV-1a hash of dd_symbolic's front tree (parent, ne, nu
 * of every front, in order), n_dual, opt->precision and opt->pivoting.  Same
 * arguments as dd_symbolic; *key written on DD_OK; dd_symbolic's errors.
 * The cache key adds the GPU: "<key as 16 hex digits>:<device name>:<SMs>".
 *
 * The cache file holds JSON lines, one per tuned problem and GPU:
 *   {"key": "...", "update_panels": P, "ahead_fronts": A, "reserve_sms": R,
 *    "split_sms": S, "factor_ms": T}
 * dd_tune_cache_lookup: *found = 1 and *out filled (configs_tried = 0) from
 * the last well-formed line whose key equals `key` and whose values are in
 * dd_set_schedule's ranges; *found = 0 when there is none or no file.
 * Returns DD_OK, or DD_ERR_INVALID_ARG for a NULL argument.
 * dd_tune_cache_store: appends one line for `key` (no '"' or newline in it)
 * and `*s` in one write; DD_ERR_INVALID_ARG if the file cannot be written. */
int dd_tune_key(int32_t n_sub, const dd_subdomain* subs, int32_t n_dual, const dd_options* opt, uint64_t* key);
int dd_tune_cache_lookup(const char* path, const char* key, dd_schedule* out, int32_t* found);
int dd_tune_cache_store(const char* path, const char* key, const dd_schedule* s);

#ifdef __cplusplus
}
#endif

#endif /* DD_GB300_DIAG_H */
