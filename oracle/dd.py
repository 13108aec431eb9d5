"""Reference domain-decomposition direct solve (FP64).  Test infrastructure only.

Follows the paper's approach (Section II) in its plainest form:

1. the decomposed problem is the arrowhead system
       [blkdiag(A_i)  B^T] [u     ]   [f]
       [B             0  ] [lambda] = [g]
   with primal unknowns u_i per domain and dual unknowns lambda on the
   interfaces (g = 0 for the torn FEM problem);
2. the primal unknowns are eliminated by independent factorizations
   A_i = L_i D_i L_i^T, one per domain;
3. the auxiliary (interface) matrix F = sum_i B_i A_i^{-1} B_i^T is formed by
   explicit solves; it is symmetric (F = F^T) and much smaller than A;
4. F is factored (LDL^T) and F lambda = sum_i B_i A_i^{-1} f_i - g is solved;
5. the primal unknowns are recovered independently: u_i = A_i^{-1}(f_i - B_i^T lambda).

The method is exact in exact arithmetic (the paper's "numerically exact"
claim), so its result must equal the undecomposed solve up to rounding.
"""
from __future__ import annotations

import numpy as np

from .dense import ldlt, ldlt_solve, lu_solve


def local_B(sub) -> np.ndarray:
    """Dense B_i^T restricted to the duals touching domain i: (n_i, m_i), and the dual ids (m_i,)."""
    duals = np.unique(sub.b_dual)
    col = np.searchsorted(duals, sub.b_dual)
    Bt = np.zeros((sub.n, duals.size), dtype=np.complex128)
    Bt[sub.b_local, col] = sub.b_sign
    return Bt, duals


def factor_subdomain(sub):
    """Step 2: A_i = L_i D_i L_i^T (unpivoted)."""
    return ldlt(sub.dense())


def subdomain_schur(sub, fac=None):
    """Step 3 for one domain: F_i = B_i A_i^{-1} B_i^T (m_i x m_i) and its dual ids."""
    L, d = factor_subdomain(sub) if fac is None else fac
    Bt, duals = local_B(sub)
    X = ldlt_solve(L, d, Bt)
    return Bt.T @ X, duals


class DDOracle:
    """Factor once, solve for any right-hand side (f, g)."""

    def __init__(self, problem):
        self.p = problem
        self.facs = [factor_subdomain(s) for s in problem.subs]
        nd = problem.n_dual
        F = np.zeros((nd, nd), dtype=np.complex128)
        self.Bt = []
        for s, fac in zip(problem.subs, self.facs):
            Fi, duals = subdomain_schur(s, fac)
            F[np.ix_(duals, duals)] += Fi
            self.Bt.append(local_B(s))
        self.F = F
        self.LF, self.dF = ldlt(F) if nd else (np.zeros((0, 0)), np.zeros(0))
        d_sub = [np.abs(fac[1]) for fac in self.facs]
        self.min_pivot = float(min(x.min() for x in d_sub))

    def solve(self, f_list, g=None):
        """Return (u_list, lambda) for local loads f_i (n_i, k) and dual rhs g (n_dual, k)."""
        p = self.p
        k = f_list[0].shape[1]
        d = np.zeros((p.n_dual, k), dtype=np.complex128)
        y = []
        for (L, dd), (Bt, duals), f in zip(self.facs, self.Bt, f_list):
            yi = ldlt_solve(L, dd, f)
            y.append(yi)
            d[duals] += Bt.T @ yi
        if g is not None:
            d -= g
        lam = ldlt_solve(self.LF, self.dF, d) if p.n_dual else d
        u = []
        for (L, dd), (Bt, duals), f in zip(self.facs, self.Bt, f_list):
            u.append(ldlt_solve(L, dd, f - Bt @ lam[duals]))
        return u, lam

    def gather(self, u_list):
        """Global vector from the local copies (lowest-index domain's copy) and the copy mismatch."""
        return gather_copies(self.p, u_list)


def gather_copies(p, u_list):
    """Global vector from the local copies (lowest-index domain's copy) and the copy mismatch."""
    k = u_list[0].shape[1]
    x = np.zeros((p.n, k), dtype=np.complex128)
    seen = np.zeros(p.n, dtype=bool)
    mismatch = 0.0
    for s, ui in zip(p.subs, u_list):
        new = ~seen[s.l2g]
        old = ~new
        if old.any():
            mismatch = max(mismatch, float(np.abs(x[s.l2g[old]] - ui[old]).max()))
        x[s.l2g[new]] = ui[new]
        seen[s.l2g] = True
    return x, mismatch


class SparseDDOracle:
    """The same decomposition route with sparse domain factorizations (Section
    II: the domains are factored by sparse direct solvers), for domains far
    beyond the dense oracle's reach.  Library routines serve as steps: SuperLU
    (scipy.sparse.linalg.splu, LU with its own fill-reducing column order) for
    each A_i, and LAPACK's LU (scipy.linalg.lu_factor) for the dense F.  Steps
    2-5 are those of DDOracle."""

    def __init__(self, problem):
        import scipy.linalg as sla
        import scipy.sparse as sp
        import scipy.sparse.linalg as spla
        self.p = problem
        nd = problem.n_dual
        F = np.zeros((nd, nd), dtype=np.complex128)
        self.lus, self.Bt = [], []
        for s in problem.subs:
            A = sp.csr_matrix((s.data, s.indices, s.indptr), shape=(s.n, s.n)).tocsc()
            lu = spla.splu(A)
            Bt, duals = local_B(s)
            F[np.ix_(duals, duals)] += Bt.T @ lu.solve(Bt)        # F_i = B_i A_i^{-1} B_i^T
            self.lus.append(lu)
            self.Bt.append((Bt, duals))
        self.F = F
        self.F_lu = sla.lu_factor(F) if nd else None

    def solve(self, f_list, g=None):
        """Return (u_list, lambda) for local loads f_i (n_i, k) and dual rhs g (n_dual, k)."""
        import scipy.linalg as sla
        p = self.p
        k = f_list[0].shape[1]
        d = np.zeros((p.n_dual, k), dtype=np.complex128)
        for lu, (Bt, duals), f in zip(self.lus, self.Bt, f_list):
            d[duals] += Bt.T @ lu.solve(np.ascontiguousarray(f))
        if g is not None:
            d -= g
        lam = sla.lu_solve(self.F_lu, d) if p.n_dual else d
        u = [lu.solve(np.ascontiguousarray(f - Bt @ lam[duals])) for lu, (Bt, duals), f in zip(self.lus, self.Bt, f_list)]
        return u, lam

    def gather(self, u_list):
        return gather_copies(self.p, u_list)


def csr_matvec(indptr, indices, data, x):
    """y = A x for a CSR matrix, row sums in FP64."""
    rows = np.repeat(np.arange(indptr.size - 1), np.diff(indptr))
    y = np.zeros((indptr.size - 1,) + x.shape[1:], dtype=np.complex128)
    np.add.at(y, rows, (data[:, None] * x[indices]) if x.ndim == 2 else data * x[indices])
    return y


def arrow_residual(problem, u_list, lam, g=None):
    """Residual of the arrowhead system: (r_i = f_i - A_i u_i - B_i^T lambda per domain, B u - g)."""
    rp = []
    ru = np.zeros((problem.n_dual, lam.shape[1]), dtype=np.complex128)
    for s, ui in zip(problem.subs, u_list):
        Au = csr_matvec(s.indptr, s.indices, s.data, ui)
        Bt, duals = local_B(s)
        rp.append(s.f - Au - Bt @ lam[duals])
        ru[duals] += Bt.T @ ui
    if g is not None:
        ru -= g
    return rp, ru


def _csr_dense(sub) -> np.ndarray:
    A = np.zeros((sub.n, sub.n), dtype=np.complex128)
    rows = np.repeat(np.arange(sub.n), np.diff(sub.indptr))
    A[rows, sub.indices] = sub.data
    return A


def arrow_dense(subs, n_dual: int) -> np.ndarray:
    """Step 1 written out: the dense arrowhead matrix [blkdiag(A_i) B^T; B 0]."""
    n_loc = sum(s.n for s in subs)
    K = np.zeros((n_loc + n_dual, n_loc + n_dual), dtype=np.complex128)
    off = 0
    for s in subs:
        K[off:off + s.n, off:off + s.n] = _csr_dense(s)
        K[n_loc + s.b_dual, off + s.b_local] = s.b_sign
        K[off + s.b_local, n_loc + s.b_dual] = s.b_sign
        off += s.n
    return K


def arrow_solve(subs, n_dual: int, f: np.ndarray):
    """The arrowhead system solved as one undecomposed system by LU with partial
    pivoting (no LDL^T, so no pivoting assumption): (stacked u, lambda) for the
    stacked loads f (n_loc, k) and g = 0."""
    n_loc = sum(s.n for s in subs)
    rhs = np.zeros((n_loc + n_dual, f.shape[1]), dtype=np.complex128)
    rhs[:n_loc] = f
    x = lu_solve(arrow_dense(subs, n_dual), rhs)
    return x[:n_loc], x[n_loc:]
