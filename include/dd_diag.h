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

/* The symbolic analysis of dd_setup alone (Section II: the auxiliary matrix
 * is factored after a symbolic factorization on the clique graph of the
 * domain interfaces), on the host, touching no device.  Same inputs and
 * validation as dd_setup (the same error codes for bad inputs).
 *
 * Fronts: 0 .. n_sub-1 are the domains (front i eliminates the n_i unknowns of
 * domain i), n_sub .. n_front-1 the separator fronts of the domain tree in
 * post-order (children before parents).  Outputs, all caller-allocated:
 *   n_front            number of fronts (also written when max_fronts is too small)
 *   parent[max_fronts] parent front, -1 at the root
 *   ne[max_fronts]     unknowns eliminated in the front (domain size, or separator duals)
 *   nu[max_fronts]     update rows of the front (duals passed on to ancestors)
 *   dual_front[n_dual] front that eliminates each dual (the lowest common
 *                      ancestor of the domains it touches)
 *   upd_ptr[max_fronts + 1], upd_idx[upd_cap] (optional, NULL to skip): the
 *                      update-row duals of front x are upd_idx[upd_ptr[x] ..
 *                      upd_ptr[x + 1]), in the library's row order
 * Returns DD_OK, DD_ERR_INVALID_ARG (bad inputs, a NULL output, max_fronts <
 * n_front or upd_cap too small), or dd_setup's other validation codes. */
int dd_symbolic(int32_t n_sub, const dd_subdomain* subs, int32_t n_dual, const dd_options* opt,
                int32_t max_fronts, int32_t* n_front, int32_t* parent, int32_t* ne, int32_t* nu,
                int32_t* dual_front, int64_t upd_cap, int64_t* upd_ptr, int32_t* upd_idx);

#ifdef __cplusplus
}
#endif

#endif /* DD_GB300_DIAG_H */
