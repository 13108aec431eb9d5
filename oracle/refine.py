"""Residuals in double-double arithmetic and iterative refinement.

Test infrastructure only.  r = b - A x is accumulated exactly enough that the
refined FP64 solution is accurate to about cond(A) * 1e-16 * 1e-16 + 1 ulp,
so that comparisons at 1e-12 measure the solver under test, not the oracle.
Error-free transformations: TwoSum (Knuth, TAOCP vol. 2, 4.2.2) and
TwoProduct with Dekker's splitting (Dekker, Numer. Math. 18 (1971) 224-242).
"""
from __future__ import annotations

import numpy as np

_SPLIT = 134217729.0  # 2^27 + 1


def two_sum(a, b):
    s = a + b
    bb = s - a
    return s, (a - (s - bb)) + (b - bb)


def _split(a):
    c = _SPLIT * a
    hi = c - (c - a)
    return hi, a - hi


def two_prod(a, b):
    p = a * b
    ah, al = _split(a)
    bh, bl = _split(b)
    return p, ((ah * bh - p) + ah * bl + al * bh) + al * bl


def _dd_add(sh, sl, ph, pl):
    s, e = two_sum(sh, ph)
    e = e + (sl + pl)
    hi = s + e
    return hi, e - (hi - s)


def residual_dd(indptr, indices, data, x, b):
    """r = b - A x for CSR A (complex), accumulated in double-double, rounded to FP64."""
    n = indptr.size - 1
    x = np.asarray(x, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    vec = x.ndim == 1
    X = x[:, None] if vec else x
    B = b[:, None] if vec else b
    cnt = np.diff(indptr)
    width = int(cnt.max()) if n else 0
    rows = np.repeat(np.arange(n), cnt)
    pos = np.arange(indices.size) - np.repeat(indptr[:-1], cnt)
    V = np.zeros((n, width), dtype=np.complex128)
    C = np.zeros((n, width), dtype=np.int64)
    V[rows, pos] = data
    C[rows, pos] = indices
    out = np.empty_like(B)
    for c in range(B.shape[1]):
        rh, rl = B[:, c].real.copy(), np.zeros(n)
        ih, il = B[:, c].imag.copy(), np.zeros(n)
        for k in range(width):
            a = V[:, k]
            xv = X[C[:, k], c]
            for (u, v, sgn_r, part) in ((a.real, xv.real, -1.0, "r"), (a.imag, xv.imag, 1.0, "r"),
                                        (a.real, xv.imag, -1.0, "i"), (a.imag, xv.real, -1.0, "i")):
                ph, pl = two_prod(u, v)
                if part == "r":
                    rh, rl = _dd_add(rh, rl, sgn_r * ph, sgn_r * pl)
                else:
                    ih, il = _dd_add(ih, il, sgn_r * ph, sgn_r * pl)
        out[:, c] = (rh + rl) + 1j * (ih + il)
    return out[:, 0] if vec else out


def refine(indptr, indices, data, b, solve, x0=None, tol=1e-16, max_iter=10):
    """x <- x + solve(b - A x) with double-double residuals until |dx| <= tol |x|."""
    x = solve(b) if x0 is None else np.array(x0, dtype=np.complex128)
    hist = []
    for _ in range(max_iter):
        r = residual_dd(indptr, indices, data, x, b)
        dx = solve(r)
        x = x + dx
        ratio = np.linalg.norm(dx) / max(np.linalg.norm(x), 1e-300)
        hist.append(ratio)
        if ratio <= tol:
            break
    return x, hist


def backward_error(indptr, indices, data, x, b):
    """|b - A x| / (|A|_F |x| + |b|), 2-norms with the residual in double-double."""
    r = residual_dd(indptr, indices, data, x, b)
    anorm = np.sqrt(np.sum(np.abs(data) ** 2))
    return float(np.linalg.norm(r) / (anorm * np.linalg.norm(x) + np.linalg.norm(b)))
