"""Symbolic analysis of the auxiliary (dual) matrix over the domain tree.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Section II: the auxiliary matrix is symmetric and block-wise sparse, and it
is LDL^T-factored after a symbolic factorization on the clique graph of the
domain interfaces (every domain couples all the duals on its boundary, so the
Schur complement F_i of domain i is a dense clique over its duals).  The
elimination order is a nested dissection along the domain tree: a dual is
eliminated at the lowest common ancestor of the domains it touches, and
tree nodes are eliminated children first.

Two independent routes to the same front tree:

  * fronts_by_elimination: the definition.  Build the clique graph, then
    eliminate each tree node's separator duals in post-order, adding the fill
    (the separator's remaining neighbours become a clique).  A front's update
    rows are the separator's not yet eliminated neighbours at that moment.
  * fronts_by_tree: from the tree alone.  A leaf's update rows are its
    domain's duals; a node's are its children's update rows less the duals
    it eliminates.

Both return a dict with, per front (domains 0 .. n_sub-1, then the tree's
internal nodes in post-order): parent, ne (unknowns eliminated: the domain
size, or the separator size), nu and upd (update-row duals, sorted), sep
(separator duals, sorted), and dual_front (the front eliminating each dual).
Parity status: pinned by the equality of the two routes and by structural
invariants (tests/test_symbolic.py); the paper prints no example.
"""
import numpy as np


def dual_domains(subs, n_dual: int):
    """Sorted list of the domains each dual touches (from the B entries)."""
    doms = [set() for _ in range(n_dual)]
    for i, s in enumerate(subs):
        for d in np.asarray(s.b_dual):
            doms[int(d)].add(i)
    return [sorted(x) for x in doms]


def _depths(parent):
    # parents carry larger ids than their children
    depth = np.zeros(len(parent), dtype=np.int64)
    for x in range(len(parent) - 1, -1, -1):
        if parent[x] >= 0:
            depth[x] = depth[parent[x]] + 1
    return depth


def lca_fronts(parent, n_sub: int, doms):
    """Front eliminating each dual: the lowest common ancestor of its domains
    (a dual touching a single domain goes to that domain's parent)."""
    depth = _depths(parent)

    def lca(a, b):
        while a != b:
            if depth[a] >= depth[b]:
                a = parent[a]
            else:
                b = parent[b]
        return a

    out = np.empty(len(doms), dtype=np.int64)
    for d, ds in enumerate(doms):
        if not ds:
            raise ValueError(f"dual {d} touches no domain")
        a = ds[0]
        for b in ds[1:]:
            a = lca(a, b)
        if a < n_sub:
            a = parent[a]
        out[d] = a
    return out


def _children(parent):
    ch = [[] for _ in range(len(parent))]
    for x, p in enumerate(parent):
        if p >= 0:
            ch[p].append(x)
    return ch


def _result(parent, subs, n_sub, df, sep, upd):
    n_front = len(parent)
    ne = [int(subs[i].n) for i in range(n_sub)] + [len(sep[v]) for v in range(n_sub, n_front)]
    return {"n_front": n_front, "parent": np.asarray(parent, dtype=np.int64), "ne": np.asarray(ne),
            "nu": np.asarray([len(u) for u in upd]), "upd": [sorted(u) for u in upd],
            "sep": [sorted(s) for s in sep], "dual_front": df}


def fronts_by_tree(parent, subs, n_dual: int):
    """Front tree from the domain tree: update rows passed up child to parent."""
    parent = [int(p) for p in parent]
    n_sub = len(subs)
    doms = dual_domains(subs, n_dual)
    df = lca_fronts(parent, n_sub, doms)
    sep = [set() for _ in parent]
    for d, v in enumerate(df):
        sep[v].add(d)
    ch = _children(parent)
    upd = [set(int(d) for d in np.asarray(subs[i].b_dual)) for i in range(n_sub)] + \
          [None] * (len(parent) - n_sub)
    for v in range(n_sub, len(parent)):
        u = set()
        for c in ch[v]:
            u |= upd[c]
        upd[v] = u - sep[v]
    return _result(parent, subs, n_sub, df, sep, upd)


def fronts_by_elimination(parent, subs, n_dual: int, fill: bool = True):
    """Front tree by symbolic elimination of the interfaces' clique graph
    (fill=False leaves the fill out: only for showing that the fill matters)."""
    parent = [int(p) for p in parent]
    n_sub = len(subs)
    doms = dual_domains(subs, n_dual)
    df = lca_fronts(parent, n_sub, doms)
    # the domain eliminations: each domain's duals form a clique
    adj = [set() for _ in range(n_dual)]
    for s in subs:
        ds = set(int(d) for d in np.asarray(s.b_dual))
        for d in ds:
            adj[d] |= ds
    for d in range(n_dual):
        adj[d].discard(d)
    sep = [set() for _ in parent]
    for d, v in enumerate(df):
        sep[v].add(d)
    eliminated = np.zeros(n_dual, dtype=bool)
    ch = _children(parent)
    upd = [set(int(d) for d in np.asarray(subs[i].b_dual)) for i in range(n_sub)] + \
          [None] * (len(parent) - n_sub)
    for v in range(n_sub, len(parent)):
        S = sep[v]
        if not S:
            # nothing eliminated here: the node only assembles its children's rows
            u = set()
            for c in ch[v]:
                u |= upd[c]
            upd[v] = {d for d in u if not eliminated[d]}
            continue
        nb = set()
        for d in S:
            nb |= adj[d]
        nb = {d for d in nb - S if not eliminated[d]}
        upd[v] = nb
        for d in nb if fill else ():   # fill: the remaining neighbours become a clique
            adj[d] |= nb
            adj[d].discard(d)
        for d in S:
            eliminated[d] = True
    return _result(parent, subs, n_sub, df, sep, upd)
