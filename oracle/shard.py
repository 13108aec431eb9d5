"""The tree route of the decomposition method sharded over ranks along
subtrees of the front tree.  TEST INFRASTRUCTURE ONLY (see the package
docstring).

Section II: the domain factorizations are independent of one another, and the
block elimination of the auxiliary matrix over the front tree runs
independently in disjoint subtrees.  So the work splits along a cut of the
tree: each rank owns one subtree (its domains and the fronts below the cut),
rank 0 also owns the fronts above the cut, and the ranks exchange only

  * in the factorization, the Schur complement each cut subtree's root passes
    up (on the root's update duals), sent to rank 0;
  * in a solve, the eliminated right-hand side of those duals, sent to rank 0,
    and their solved values, sent back.

`plan` is the cut: the subtree of largest algorithmic work is split into its
children until there are as many subtrees as ranks.  A front of e eliminated
and u update rows costs (4/3)e^3 + 4e^2 u + 4e u^2 real flops (8 per complex
multiply-add: LDL^T of the pivot block, the triangular solve of the update
rows, the symmetric update); 3x that is an integer, which is what is summed,
so equal subtrees tie exactly and the first one in the cut list wins.

`ShardedTreeDD` runs the tree route (TreeDDOracle) on such a cut over a
torch.distributed process group (gloo on the CPU); every step is the
one-rank route's, on the rank's part of the tree, so the result equals the
one-rank solve to rounding.
"""
from __future__ import annotations

import numpy as np

from .symbolic import fronts_by_tree
from .tree import TreeDDOracle, backward_fronts, eliminate_fronts, forward_fronts, subtree_nodes


def front_work(ne, nu) -> list:
    """3x the real flops of every front (exact Python integers)."""
    return [4 * int(e) ** 3 + 12 * int(e) ** 2 * int(u) + 12 * int(e) * int(u) ** 2 for e, u in zip(ne, nu)]


def plan(parent, ne, nu, n_ranks: int) -> dict:
    """Cut of the front tree (parent ids larger than their children's) into
    n_ranks subtrees.  Returns rank_root (ascending front ids), front_rank
    (the owner of every front: the rank whose subtree holds it, rank 0 above
    the cut) and the subtree work of every front."""
    parent = np.asarray(parent, dtype=np.int64)
    n = parent.size
    if n_ranks < 1:
        raise ValueError("n_ranks < 1")
    children = [[] for _ in range(n)]
    for x in range(n):
        if parent[x] >= 0:
            children[int(parent[x])].append(x)
    roots = [x for x in range(n) if parent[x] < 0]
    if len(roots) != 1:
        raise ValueError("the front tree must have one root")
    total = front_work(ne, nu)
    for x in range(n):                       # children before parents
        if parent[x] >= 0:
            total[int(parent[x])] += total[x]
    cut = [roots[0]]
    while len(cut) < n_ranks:
        best = -1
        for q, x in enumerate(cut):
            if children[x] and (best < 0 or total[x] > total[cut[best]]):
                best = q
        if best < 0:
            raise ValueError("the tree has fewer subtrees than ranks")
        x = cut.pop(best)
        cut.extend(children[x])
    if len(cut) != n_ranks:
        raise ValueError("a split gave more subtrees than ranks")
    rank_root = np.array(sorted(cut), dtype=np.int64)
    front_rank = np.zeros(n, dtype=np.int64)
    for r, v in enumerate(rank_root):
        front_rank[subtree_nodes(parent, int(v))] = r
    return {"rank_root": rank_root, "front_rank": front_rank, "work": total}


def plan_problem(problem, n_ranks: int) -> dict:
    """plan() on the front tree of a femgen problem's domain tree."""
    parent = np.asarray(problem.rcb.parent, dtype=np.int64)
    ft = fronts_by_tree(parent, problem.subs, problem.n_dual)
    return plan(parent, ft["ne"], ft["nu"], n_ranks)


class ShardedTreeDD:
    """The tree route on one rank of a process group (all ranks construct it
    together): factor in the constructor, solve() for any loads."""

    def __init__(self, problem, shard: dict, group=None):
        import torch.distributed as dist
        self.dist, self.group = dist, group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        p = self.p = problem
        roots = shard["rank_root"]
        if len(roots) != self.world:
            raise ValueError("the cut has a subtree per rank")
        parent = self.parent = np.asarray(p.rcb.parent, dtype=np.int64)
        self.front_rank = np.asarray(shard["front_rank"], dtype=np.int64)
        ft = fronts_by_tree(parent, p.subs, p.n_dual)
        self.owner = self.front_rank[np.asarray(ft["dual_front"], dtype=np.int64)]   # the rank solving each dual
        self.root = int(roots[self.rank])

        # the rank's subtree: domain factorizations and block elimination
        self.T = TreeDDOracle(p, parent=parent, subtree=self.root)
        self.U = self.T.passed_up[self.root][0]          # duals the subtree hands to its ancestors
        blocks = [None] * self.world
        dist.all_gather_object(blocks, (self.root, self.T.passed_up[self.root]), group=group)

        # rank 0: the fronts above the cut, children first
        self.top = []
        if self.rank == 0:
            below = set()
            for v in roots:
                below.update(int(x) for x in subtree_nodes(parent, int(v)))
            self.top = [x for x in range(p.n_sub, parent.size) if x not in below]
            self.sep = {v: np.asarray(ft["sep"][v], dtype=np.int64) for v in self.top}
            self.upd = {v: np.asarray(ft["upd"][v], dtype=np.int64) for v in self.top}
            children = {v: [int(x) for x in np.nonzero(parent == v)[0]] for v in self.top}
            passed = {v: blk for v, blk in blocks}
            self.Fss, self.Fus, _ = eliminate_fronts(p.n_dual, self.top, self.sep, self.upd, children, passed)
            left = [v for v, (duals, _) in passed.items() if duals.size]
            if left:
                raise ValueError(f"blocks left over above the cut: {left}")
        self.U_all = [None] * self.world
        dist.all_gather_object(self.U_all, self.U, group=group)

    def solve(self, f_list, g=None):
        """Loads f_i (n_i, k) indexed by domain id (a rank reads only its own)
        and g (n_dual, k) or None.  Returns ({domain: u_i} of this rank's
        domains, lambda on the duals this rank solves, as (duals, values))."""
        dist, p = self.dist, self.p
        k = f_list[self.T.domains[0]].shape[1]
        gr = None
        if g is not None:                      # each rank subtracts g on the duals it solves
            gr = np.where((self.owner == self.rank)[:, None], g, 0)
        d = self.T.forward(f_list, gr)
        # the cut roots' eliminated right-hand sides go up to rank 0
        ups = [None] * self.world
        dist.all_gather_object(ups, d[self.U], group=self.group)
        lam = np.zeros((p.n_dual, k), dtype=np.complex128)
        downs = [None] * self.world
        if self.rank == 0:
            for r in range(1, self.world):
                d[self.U_all[r]] += ups[r]
            forward_fronts(self.top, self.sep, self.upd, self.Fss, self.Fus, d)
            backward_fronts(self.top, self.sep, self.upd, self.Fss, self.Fus, d, lam)
            downs = [lam[self.U_all[r]] for r in range(self.world)]
        # their solved values come back down
        mine = [None]
        dist.scatter_object_list(mine, downs if self.rank == 0 else None, src=0, group=self.group)
        lam[self.U] = mine[0]
        self.T.backward(d, lam)
        u = dict(zip(self.T.domains, self.T.recover(f_list, lam)))
        duals = np.nonzero(self.owner == self.rank)[0]
        return u, (duals, lam[duals])

    def gather(self, part):
        """Rank 0: the whole solution (u_list by domain id, lambda) from every
        rank's solve() result; the other ranks get None."""
        parts = [None] * self.world
        self.dist.all_gather_object(parts, part, group=self.group)
        if self.rank != 0:
            return None
        u = [None] * self.p.n_sub
        lam = None
        for ud, (duals, vals) in parts:
            for i, ui in ud.items():
                u[i] = ui
            if lam is None:
                lam = np.zeros((self.p.n_dual, vals.shape[1]), dtype=np.complex128)
            lam[duals] = vals
        return u, lam
