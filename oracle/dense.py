"""Dense reference factorizations (FP64, complex).  Test infrastructure only.

* lu_solve: Gaussian elimination with partial pivoting (the plain definition of
  x = A^{-1} b for a small undecomposed system; Golub & Van Loan, Alg. 3.4.1).
* ldlt / ldlt_solve: unpivoted A = L D L^T of a complex symmetric matrix
  (A = A^T, no conjugation), column by column (Golub & Van Loan, Alg. 4.1.2).
  The paper factors both the domain matrices and the auxiliary matrix as
  symmetric LDL^T (Section II); existence without pivoting follows from the
  lossy domains: Im(x^H A x) > 0 for every x != 0, so every leading principal
  submatrix is nonsingular.
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
