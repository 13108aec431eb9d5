"""Seeded indefinite arrowhead inputs for the pivoting path.

The FEM workloads are lossy, so every domain matrix and the auxiliary matrix
admit an unpivoted LDL^T.  These inputs do not: each domain matrix is the
interleaved form of [[eps I, C_i], [C_i^T, eps I]] (unknown 2s is row s of the
first block, unknown 2t+1 row t of the second), with C_i complex and well
conditioned.  With eps = 0 the diagonal is exactly zero, so an unpivoted
elimination meets a zero pivot at once, and so is the diagonal of every
A_i^{-1} and hence of the auxiliary matrix.  With a small eps > 0 the domains
still factor without pivoting, but the auxiliary matrix has an O(eps) diagonal
under O(1) couplings.

Domains form a chain: domain i shares n_if unknowns with domain i + 1 (its
last n_if to the first n_if of i + 1), tied by n_if multipliers each with
sign +1 in domain i and -1 in domain i + 1.  m and n_if are even, so after the
solver's interior-first / interface-last reordering every aligned pivot block
holds as many even as odd unknowns.  Nothing here factors or solves anything.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class ArrowDomain:
    n: int
    indptr: np.ndarray      # CSR of A_i, int32, full pattern, sorted columns
    indices: np.ndarray
    data: np.ndarray        # complex128
    f: np.ndarray           # (n, nrhs) complex128
    b_dual: np.ndarray      # int32
    b_local: np.ndarray     # int32
    b_sign: np.ndarray      # int8


@dataclass
class ArrowProblem:
    subs: list
    n_dual: int

    @property
    def n_sub(self) -> int:
        return len(self.subs)


def indefinite_chain(n_sub: int = 4, m: int = 96, n_if: int = 8, eps: float = 0.0, nrhs: int = 1,
                     seed: int = 0) -> ArrowProblem:
    if m % 2 or n_if % 2 or 2 * n_if > m:
        raise ValueError("m and n_if must be even with 2 n_if <= m")
    rng = np.random.default_rng(seed)
    h = m // 2
    subs = []
    for i in range(n_sub):
        C = (rng.normal(size=(h, h)) + 1j * rng.normal(size=(h, h))) / np.sqrt(h) + 2.0 * np.eye(h)
        A = np.zeros((m, m), dtype=np.complex128)
        A[0::2, 1::2] = C
        A[1::2, 0::2] = C.T
        A[np.diag_indices(m)] = eps
        rows, cols = np.nonzero(np.ones((m, m), dtype=bool))   # dense pattern, zero diagonal stored
        indptr = np.searchsorted(rows, np.arange(m + 1)).astype(np.int32)
        f = rng.normal(size=(m, nrhs)) + 1j * rng.normal(size=(m, nrhs))
        bd, bl, bs = [], [], []
        if i > 0:                       # first n_if unknowns tie to domain i - 1
            for t in range(n_if):
                bd.append((i - 1) * n_if + t); bl.append(t); bs.append(-1)
        if i + 1 < n_sub:               # last n_if unknowns tie to domain i + 1
            for t in range(n_if):
                bd.append(i * n_if + t); bl.append(m - n_if + t); bs.append(1)
        subs.append(ArrowDomain(m, indptr, cols.astype(np.int32), A[rows, cols].copy(), f,
                                np.array(bd, np.int32), np.array(bl, np.int32), np.array(bs, np.int8)))
    return ArrowProblem(subs, (n_sub - 1) * n_if)
