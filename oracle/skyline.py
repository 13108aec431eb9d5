"""Undecomposed sparse reference solve: RCM ordering + band-profile LDL^T.

Test infrastructure only.  This is the "conventional one-shot" route that the
paper compares its decomposition method against (Section I, Fig. 1): factor
the whole assembled FEM matrix.  The ordering is reverse Cuthill-McKee
(Cuthill & McKee 1969; George & Liu 1981, pseudo-peripheral start node); the
factor is the unpivoted complex-symmetric LDL^T (the matrix is lossy, so it
exists), stored in a band of the permuted matrix's half-bandwidth.  Fill of
LDL^T never leaves the profile, so the band holds every nonzero of L.
"""
from __future__ import annotations

from collections import deque

import numpy as np


def _bfs_levels(indptr, indices, start, n):
    level = np.full(n, -1, dtype=np.int64)
    level[start] = 0
    q = deque([start])
    last = start
    while q:
        v = q.popleft()
        last = v
        for w in indices[indptr[v]:indptr[v + 1]]:
            if level[w] < 0:
                level[w] = level[v] + 1
                q.append(w)
    return level, last


def rcm(indptr: np.ndarray, indices: np.ndarray) -> np.ndarray:
    """Reverse Cuthill-McKee permutation (new position -> old index)."""
    n = indptr.size - 1
    deg = np.diff(indptr).astype(np.int64)
    order = []
    seen = np.zeros(n, dtype=bool)
    for comp_start in np.argsort(deg, kind="stable"):
        if seen[comp_start]:
            continue
        # pseudo-peripheral node: repeat BFS from the last level's min-degree node
        s = int(comp_start)
        level, _ = _bfs_levels(indptr, indices, s, n)
        ecc = level.max()
        while True:
            far = np.nonzero(level == level.max())[0]
            t = int(far[np.argmin(deg[far])])
            lv2, _ = _bfs_levels(indptr, indices, t, n)
            if lv2.max() > ecc:
                s, level, ecc = t, lv2, lv2.max()
            else:
                break
        q = deque([s])
        seen[s] = True
        while q:
            v = q.popleft()
            order.append(v)
            nb = [w for w in indices[indptr[v]:indptr[v + 1]] if not seen[w]]
            nb.sort(key=lambda w: (deg[w], w))
            for w in nb:
                seen[w] = True
                q.append(w)
    return np.array(order[::-1], dtype=np.int64)


class BandLDLT:
    """LDL^T of a permuted sparse complex-symmetric matrix in band storage.

    S[i, t] holds entry (i, i - t) of the permuted matrix for t = 0..beta;
    after factor(), S[:, 0] is D and S[i, t] (t > 0) is L[i, i - t].
    """

    def __init__(self, indptr, indices, data, perm=None):
        n = indptr.size - 1
        if perm is None:
            perm = rcm(indptr, indices)
        self.perm = perm
        inv = np.empty(n, dtype=np.int64)
        inv[perm] = np.arange(n)
        rows = np.repeat(np.arange(n), np.diff(indptr))
        pi = inv[rows]
        pj = inv[indices]
        low = pi >= pj
        self.beta = int(np.max(pi - pj)) if n else 0
        self.n = n
        self.S = np.zeros((n, self.beta + 1), dtype=np.complex128)
        self.S[pi[low], (pi - pj)[low]] = data[low]
        self.growth = None

    def factor(self):
        """Right-looking elimination restricted to the band (Golub & Van Loan 4.3)."""
        S, n, beta = self.S, self.n, self.beta
        amax = np.abs(S).max() if S.size else 0.0
        # window offsets: rows a >= cols b inside a beta x beta window
        a_idx, b_idx = np.tril_indices(beta)
        for k in range(n):
            dk = S[k, 0]
            if dk == 0:
                raise np.linalg.LinAlgError(f"zero pivot at {k}")
            w = min(beta, n - k - 1)
            if w == 0:
                continue
            ra = k + 1 + np.arange(w)
            ta = np.arange(1, w + 1)
            l = S[ra, ta] / dk                                # column k: A[k+1+a, k]
            S[ra, ta] = l
            if w < beta:
                m = (a_idx < w) & (b_idx < w)
                aa, bb = a_idx[m], b_idx[m]
            else:
                aa, bb = a_idx, b_idx
            S[k + 1 + aa, aa - bb] -= l[aa] * dk * l[bb]
        self.growth = float(np.abs(S).max() / amax) if amax else 0.0
        return self

    def solve(self, b: np.ndarray) -> np.ndarray:
        S, n, beta = self.S, self.n, self.beta
        b = np.asarray(b, dtype=np.complex128)
        vec = b.ndim == 1
        z = (b[:, None] if vec else b)[self.perm].copy()
        for k in range(n):
            w = min(beta, n - k - 1)
            if w:
                z[k + 1:k + 1 + w] -= S[k + 1 + np.arange(w), np.arange(1, w + 1)][:, None] * z[k]
        z /= S[:, 0][:, None]
        for k in range(n - 1, -1, -1):
            w = min(beta, n - k - 1)
            if w:
                z[k] -= S[k + 1 + np.arange(w), np.arange(1, w + 1)] @ z[k + 1:k + 1 + w]
        x = np.empty_like(z)
        x[self.perm] = z
        return x[:, 0] if vec else x


def envelope_entries(indptr: np.ndarray, indices: np.ndarray, perm: np.ndarray | None = None) -> int:
    """Stored entries of a skyline (envelope) LDL^T factor after the ordering
    perm (RCM by default): for each row i of the permuted matrix, the entries
    from its first nonzero column to the diagonal.  The profile holds all fill
    of an LDL^T without pivoting, so this is the factor memory of O2."""
    n = indptr.size - 1
    if n == 0:
        return 0
    if perm is None:
        perm = rcm(indptr, indices)
    inv = np.empty(n, dtype=np.int64)
    inv[perm] = np.arange(n)
    rows = np.repeat(np.arange(n), np.diff(indptr))
    pi, pj = inv[rows], inv[indices]
    first = np.arange(n, dtype=np.int64)
    np.minimum.at(first, pi, pj)
    return int(np.sum(np.arange(n) - first + 1))
