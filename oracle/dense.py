"""Dense reference factorizations (FP64, complex).  Test infrastructure only.

* lu_solve: Gaussian elimination with partial pivoting (the plain definition of
  x = A^{-1} b for a small undecomposed system; Golub & Van Loan, Alg. 3.4.1).
* ldlt / ldlt_solve: unpivoted A = L D L^T of a complex symmetric matrix
  (A = A^T, no conjugation), column by column (Golub & Van Loan, Alg. 4.1.2).
  The paper factors both the domain matrices and the auxiliary matrix as
  symmetric LDL^T (Section II); existence without pivoting follows from the
  lossy domains: Im(x^H A x) > 0 for every x != 0, so every leading principal
  submatrix is nonsingular.
* ldlt_bk_restricted / ldlt_bk_solve: complex-symmetric LDL^T with the
  Bunch-Kaufman pivot choice (Bunch & Kaufman 1977, partial pivoting with
  1x1 and 2x2 pivots, alpha = (1 + sqrt 17) / 8) whose search is restricted to
  the diagonal block holding the current column, the "restricted
  Bunch-Kaufman" of the block LDL^T of the auxiliary matrix (Section II).
  Right-looking, one column (or column pair) at a time, with the interchanges
  applied to the whole matrix.
"""
from __future__ import annotations

import numpy as np


def lu_solve(A: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Solve A x = b by LU with row partial pivoting.  A (n, n), b (n,) or (n, k)."""
    U = np.array(A, dtype=np.complex128, copy=True)
    x = np.array(b, dtype=np.complex128, copy=True)
    vec = x.ndim == 1
    if vec:
        x = x[:, None]
    n = U.shape[0]
    for k in range(n):
        p = k + int(np.argmax(np.abs(U[k:, k])))
        if U[p, k] == 0:
            raise np.linalg.LinAlgError("singular matrix")
        if p != k:
            U[[k, p], :] = U[[p, k], :]
            x[[k, p], :] = x[[p, k], :]
        m = U[k + 1:, k] / U[k, k]
        U[k + 1:, k:] -= np.outer(m, U[k, k:])
        x[k + 1:, :] -= np.outer(m, x[k, :])
    for k in range(n - 1, -1, -1):
        x[k, :] = (x[k, :] - U[k, k + 1:] @ x[k + 1:, :]) / U[k, k]
    return x[:, 0] if vec else x


def ldlt(A: np.ndarray):
    """Unpivoted complex-symmetric LDL^T.  Returns (L unit lower (n, n), d (n,)).

    Column j: d_j = a_jj - sum_k L_jk^2 d_k and
    L_ij = (a_ij - sum_k L_ik d_k L_jk) / d_j for i > j.
    """
    A = np.asarray(A, dtype=np.complex128)
    n = A.shape[0]
    L = np.eye(n, dtype=np.complex128)
    d = np.zeros(n, dtype=np.complex128)
    for j in range(n):
        v = L[j, :j] * d[:j]
        d[j] = A[j, j] - L[j, :j] @ v
        if d[j] == 0:
            raise np.linalg.LinAlgError(f"zero pivot at {j}")
        L[j + 1:, j] = (A[j + 1:, j] - L[j + 1:, :j] @ v) / d[j]
    return L, d


def forward_unit(L: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Solve L z = b for unit lower-triangular L, row by row."""
    z = np.array(b, dtype=np.complex128, copy=True)
    for i in range(L.shape[0]):
        z[i] -= L[i, :i] @ z[:i]
    return z


def backward_unit_t(L: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Solve L^T x = b (plain transpose) for unit lower-triangular L."""
    x = np.array(b, dtype=np.complex128, copy=True)
    n = L.shape[0]
    for i in range(n - 1, -1, -1):
        x[i] -= L[i + 1:, i] @ x[i + 1:]
    return x


def ldlt_solve(L: np.ndarray, d: np.ndarray, b: np.ndarray) -> np.ndarray:
    """x = L^{-T} D^{-1} L^{-1} b."""
    z = forward_unit(L, b)
    z = z / (d[:, None] if z.ndim == 2 else d)
    return backward_unit_t(L, z)


BK_ALPHA = (1.0 + np.sqrt(17.0)) / 8.0


def ldlt_bk_restricted(A: np.ndarray, nb: int):
    """A[perm][:, perm] = L D L^T with restricted Bunch-Kaufman pivoting.

    The diagonal blocks are [b, b + nb) for b = 0, nb, 2 nb, ...; at column j
    (block end e) with S the trailing matrix:
      lambda = max_{j < i < e} |S_ij| (first maximiser r); if lambda = 0 or
      |S_jj| >= alpha lambda: 1x1 pivot at j; else with
      sigma = max_{j <= i < e, i != r} |S_ir|: 1x1 at j if |S_jj| sigma >=
      alpha lambda^2, else 1x1 at j after interchanging j and r if
      |S_rr| >= alpha sigma, else a 2x2 pivot on (j, j+1) after
      interchanging j+1 and r.
    Returns (perm, L unit lower, D block diagonal, interchanges, 2x2 pivots).
    """
    S = np.array(A, dtype=np.complex128, copy=True)
    n = S.shape[0]
    perm = np.arange(n)
    L = np.eye(n, dtype=np.complex128)
    D = np.zeros((n, n), dtype=np.complex128)
    n_swap = n_2x2 = 0
    j = 0
    while j < n:
        e = min((j // nb + 1) * nb, n)
        step, q = 1, -1
        col = np.abs(S[j + 1:e, j])
        if col.size and col.max() > 0:
            lam = col.max()
            r = j + 1 + int(np.argmax(col))
            ajj = abs(S[j, j])
            if ajj < BK_ALPHA * lam:
                sig = max(abs(S[i, r]) for i in range(j, e) if i != r)
                if ajj * sig >= BK_ALPHA * lam * lam:
                    pass
                elif abs(S[r, r]) >= BK_ALPHA * sig:
                    q = r
                else:
                    step = 2
                    q = r if r != j + 1 else -1
        if q >= 0:
            p = j + step - 1
            S[[p, q], :] = S[[q, p], :]
            S[:, [p, q]] = S[:, [q, p]]
            L[[p, q], :j] = L[[q, p], :j]
            perm[[p, q]] = perm[[q, p]]
            n_swap += 1
        if step == 1:
            D[j, j] = S[j, j]
            if S[j, j] == 0:
                raise np.linalg.LinAlgError(f"zero pivot at {j}")
            w = S[j + 1:, j].copy()                   # d_j l_ij
            L[j + 1:, j] = w / S[j, j]
            S[j + 1:, j + 1:] -= np.outer(L[j + 1:, j], w)
        else:
            Db = S[j:j + 2, j:j + 2].copy()
            D[j:j + 2, j:j + 2] = Db
            W = S[j + 2:, j:j + 2].copy()               # L_b D_b
            Lb = np.linalg.solve(Db.T, W.T).T          # W D_b^{-1}
            L[j + 2:, j:j + 2] = Lb
            S[j + 2:, j + 2:] -= Lb @ W.T
            n_2x2 += 1
        j += step
    return perm, L, D, n_swap, n_2x2


def ldlt_bk_solve(perm, L, D, b: np.ndarray) -> np.ndarray:
    """x = A^{-1} b from A[perm][:, perm] = L D L^T."""
    b = np.asarray(b, dtype=np.complex128)
    z = forward_unit(L, b[perm])
    z = np.linalg.solve(D, z)
    y = backward_unit_t(L, z)
    x = np.empty_like(y)
    x[perm] = y
    return x
