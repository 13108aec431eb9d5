/*
 * dd_diag.h - diagnostics of the GB300 direct domain-decomposition solver.
 *
 * Not part of the method (the paper has no counterpart): a check that the
 * library's bounded device-side waits give up and report an error instead of
 * hanging, so that failure detection can be tested without a GPU fault.
 */
#ifndef DD_GB300_DIAG_H
#define DD_GB300_DIAG_H

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

#ifdef __cplusplus
}
#endif

#endif /* DD_GB300_DIAG_H */
