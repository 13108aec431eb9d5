"""The decomposition route with the auxiliary matrix eliminated block by block
over the domain tree.  TEST INFRASTRUCTURE ONLY (see the package docstring).

Section II: the auxiliary matrix F = sum_i B_i A_i^{-1} B_i^T is symmetric and
sparse at the level of dense blocks; its block structure follows from a
symbolic factorization on the clique graph of the domain interfaces, and it is
factored block by block.  DDOracle forms F as one dense matrix, which at the
10^5 duals of the 512-domain mesh would need about 200 GB; this route holds
only the dense blocks the elimination creates, so it reaches the 512- and
2048-domain workloads.  Its steps:

  1. every domain: A_i factored by LAPACK's LU with partial pivoting
     (scipy.linalg.lu_factor, a library routine standing for A_i^{-1}), and
     F_i = B_i A_i^{-1} B_i^T by explicit solves;
  2. the front tree of F from the domain tree (symbolic.fronts_by_tree: a dual
     is eliminated at the lowest common ancestor of its domains; separators
     after their subtrees, i.e. nested dissection);
  3. block Gaussian elimination in that order: the front of tree node v sums
     the blocks its children pass up (a domain passes F_i on its duals) into
     [F_ss F_us^T; F_us F_uu] over its separator duals s and update duals u,
     and passes up the Schur complement F_uu - F_us F_ss^{-1} F_us^T;
  4. F lambda = d by the same elimination applied to d (in order,
     d_u -= F_us F_ss^{-1} d_s), then back substitution in reverse order,
     lambda_s = F_ss^{-1} (d_s - F_us^T lambda_u);
  5. primal recovery u_i = A_i^{-1} (f_i - B_i^T lambda).

Each step is a definition (a Schur complement, a block solve) with LAPACK
solves and matrix products as its steps; nothing is fused, blocked or
reordered beyond the elimination order of step 2.  The route is exact in
exact arithmetic, so it equals DDOracle and the undecomposed solve to
rounding (tests/test_oracle_tree.py).

`subtree=v` restricts every step to the domains and fronts below tree node v
(v included): the same arithmetic as the whole-tree run on that part, with the
Schur complement of v left unfactored (`passed_up`) and lambda of v's update
duals taken as zero in the solve.  It serves as a bounded sample of a large
workload for timing.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .dd import gather_copies, local_B
from .symbolic import fronts_by_tree


def subtree_nodes(parent, node: int) -> np.ndarray:
    """Nodes of the subtree rooted at `node`, ascending (children before parents)."""
    parent = np.asarray(parent)
    inside = np.zeros(parent.size, dtype=bool)
    inside[node] = True
    for x in range(node - 1, -1, -1):          # a parent's id is larger than its children's
        q = parent[x]
        if 0 <= q <= node and inside[q]:
            inside[x] = True
    return np.nonzero(inside)[0]


def eliminate_fronts(n_dual, fronts, sep, upd, children, passed):
    """Step 3 over `fronts` (children first): each front sums the blocks its
    children pass up (popped from `passed`: child -> (duals, block)) and
    passes up its Schur complement (stored in `passed` under its id).
    Returns the LU of every F_ss, every F_us, and every front's order."""
    pos = np.full(n_dual, -1, dtype=np.int64)
    Fss, Fus_all, front_rows = {}, {}, {}
    for v in fronts:
        S, U = sep[v], upd[v]
        rows = np.concatenate([S, U])
        pos[rows] = np.arange(rows.size)
        W = np.zeros((rows.size, rows.size), dtype=np.complex128)
        for c in children[v]:
            duals, M = passed.pop(c)
            ix = pos[duals]
            if (ix < 0).any():
                raise ValueError(f"front {v}: a child passes a dual outside the front")
            W[np.ix_(ix, ix)] += M
        pos[rows] = -1
        ns = S.size
        Fus = W[ns:, :ns].copy()
        if ns:
            lu = sla.lu_factor(W[:ns, :ns], check_finite=False)
            schur = W[ns:, ns:] - Fus @ sla.lu_solve(lu, Fus.T, check_finite=False)
        else:
            lu = None
            schur = W[ns:, ns:]
        Fss[v], Fus_all[v] = lu, Fus
        front_rows[v] = rows.size
        passed[v] = (U, schur)
    return Fss, Fus_all, front_rows


def forward_fronts(fronts, sep, upd, Fss, Fus, d):
    """Step 4, the elimination of d over `fronts` in order (in place)."""
    for v in fronts:
        S, U = sep[v], upd[v]
        if S.size:
            d[U] -= Fus[v] @ sla.lu_solve(Fss[v], d[S], check_finite=False)


def backward_fronts(fronts, sep, upd, Fss, Fus, d, lam):
    """Step 4, the back substitution over `fronts` in reverse order (in place)."""
    for v in reversed(fronts):
        S, U = sep[v], upd[v]
        if S.size:
            lam[S] = sla.lu_solve(Fss[v], d[S] - Fus[v].T @ lam[U], check_finite=False)


class TreeDDOracle:
    """Factor once (steps 1-3), solve for any loads (steps 4-5)."""

    def __init__(self, problem, parent=None, subtree=None):
        p = self.p = problem
        parent = np.asarray(p.rcb.parent if parent is None else parent, dtype=np.int64)
        n_sub = p.n_sub
        ft = fronts_by_tree(parent, p.subs, p.n_dual)
        nodes = np.arange(parent.size) if subtree is None else subtree_nodes(parent, int(subtree))
        self.domains = [int(x) for x in nodes if x < n_sub]
        self.fronts = [int(x) for x in nodes if x >= n_sub]
        self.sep = {v: np.asarray(ft["sep"][v], dtype=np.int64) for v in self.fronts}
        self.upd = {v: np.asarray(ft["upd"][v], dtype=np.int64) for v in self.fronts}
        children = {v: [] for v in self.fronts}
        for x in nodes:
            q = int(parent[x])
            if q in children:
                children[q].append(int(x))

        # step 1: domain factorizations and their contributions F_i
        self.lu, self.Bt = {}, {}
        passed = {}
        for i in self.domains:
            s = p.subs[i]
            lu = sla.lu_factor(s.dense(), check_finite=False)
            Bt, duals = local_B(s)
            Fi = Bt.T @ sla.lu_solve(lu, Bt, check_finite=False)
            self.lu[i] = lu
            self.Bt[i] = (Bt, duals.astype(np.int64))
            passed[i] = (duals.astype(np.int64), Fi)

        # step 3: block elimination of F over the front tree, children first
        self.Fss, self.Fus, self.front_rows = eliminate_fronts(p.n_dual, self.fronts, self.sep, self.upd, children,
                                                               passed)
        # what is left: the Schur complement handed to the ancestors of the top
        # node (empty for the whole tree, whose root has no update duals)
        self.passed_up = passed

    def forward(self, f_list, g=None):
        """d = sum_i B_i A_i^{-1} f_i - g over this tree's domains (n_dual, k),
        then step 4's elimination over this tree's fronts."""
        p = self.p
        k = f_list[self.domains[0]].shape[1]
        d = np.zeros((p.n_dual, k), dtype=np.complex128)
        for i in self.domains:                                   # d = sum_i B_i A_i^{-1} f_i
            Bt, duals = self.Bt[i]
            d[duals] += Bt.T @ sla.lu_solve(self.lu[i], f_list[i], check_finite=False)
        if g is not None:
            d -= g
        forward_fronts(self.fronts, self.sep, self.upd, self.Fss, self.Fus, d)
        return d

    def backward(self, d, lam):
        """Back substitution over this tree's fronts (reverse order); lam holds
        the values of the update duals of the top front on entry."""
        backward_fronts(self.fronts, self.sep, self.upd, self.Fss, self.Fus, d, lam)
        return lam

    def recover(self, f_list, lam):
        """Step 5 for this tree's domains: u_i = A_i^{-1} (f_i - B_i^T lambda)."""
        u = []
        for i in self.domains:
            Bt, duals = self.Bt[i]
            u.append(sla.lu_solve(self.lu[i], f_list[i] - Bt @ lam[duals], check_finite=False))
        return u

    def solve(self, f_list, g=None):
        """Loads f_i (n_i, k), indexed by domain id (all domains of the problem),
        and the dual right-hand side g (n_dual, k) or None.  Returns (u_list in
        the order of self.domains, lambda (n_dual, k))."""
        d = self.forward(f_list, g)
        lam = self.backward(d, np.zeros_like(d))
        return self.recover(f_list, lam), lam

    def gather(self, u_list):
        """Global vector from the local copies (whole tree only) and the copy mismatch."""
        if len(self.domains) != self.p.n_sub:
            raise ValueError("gather needs every domain")
        return gather_copies(self.p, u_list)

    def stored_entries(self) -> int:
        """Complex entries of the separator fronts' stored blocks (F_ss and F_us)."""
        return int(sum(self.sep[v].size ** 2 + self.sep[v].size * self.upd[v].size for v in self.fronts))
