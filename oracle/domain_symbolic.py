"""Symbolic factorization of one domain matrix under a nested dissection.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Section II factors each domain with a sparse direct solver.  A nested
dissection is not unique (it is a heuristic), so what is checked is:

  * check_dissection: the tree is a valid dissection of the domain's graph --
    every row eliminated once, children before parents, the flagged interface
    rows in the root, leaves within the size bound, and no edge of the graph
    between two fronts unless one is an ancestor of the other (each separator
    separates);
  * the front structure that the dissection implies, which is unique, by two
    routes: fronts_by_elimination eliminates the graph one row at a time in
    the given order (the definition: the not yet eliminated neighbours of a
    row become a clique), a front's update rows being the later rows its own
    rows reach; fronts_by_reach takes a front's update rows as the later rows
    adjacent to its own rows or passed up by its children.

Parity status: pinned by the equality of the two routes, the validity checks,
and planted mistakes that they catch (tests/test_domain_symbolic.py).
"""
import numpy as np


def _adjacency(indptr, indices):
    n = len(indptr) - 1
    adj = [set() for _ in range(n)]
    for i in range(n):
        for j in indices[indptr[i]:indptr[i + 1]]:
            if j != i:
                adj[i].add(int(j))
    return adj


def _ancestor(parent, a, x):
    """Is a an ancestor of x (or x itself)."""
    while x >= 0:
        if x == a:
            return True
        x = parent[x]
    return False


def check_dissection(t, indptr, indices, is_last, leaf_max: int):
    """Raise AssertionError unless t (front tree of one domain) is a valid dissection."""
    n = len(indptr) - 1
    parent = [int(p) for p in t["parent"]]
    nf = t["n_front"]
    order, front_of = np.asarray(t["order"]), np.asarray(t["front_of"])
    assert sorted(order.tolist()) == list(range(n)), "every row eliminated exactly once"
    assert all(parent[x] > x or parent[x] == -1 for x in range(nf)), "children precede parents"
    assert sum(1 for p in parent if p < 0) == 1 and parent[nf - 1] == -1, "one root, last"
    # the order lists the fronts' rows front after front
    pos = 0
    for x in range(nf):
        rows = order[pos:pos + t["ne"][x]]
        assert (front_of[rows] == x).all()
        pos += t["ne"][x]
    if is_last is not None:
        il = np.asarray(is_last).astype(bool)
        assert (front_of[il] == nf - 1).all() and (front_of[~il] != nf - 1).all(), "interface rows in the root"
    has_child = np.zeros(nf, dtype=bool)
    for x in range(nf):
        if parent[x] >= 0:
            has_child[parent[x]] = True
    for x in range(nf - 1):
        if not has_child[x]:
            assert t["ne"][x] <= leaf_max, f"leaf {x} too large"
    adj = _adjacency(indptr, indices)
    for i in range(n):
        for j in adj[i]:
            a, b = int(front_of[i]), int(front_of[j])
            assert _ancestor(parent, a, b) or _ancestor(parent, b, a), f"edge {i}-{j} crosses subtrees"


def fronts_by_elimination(indptr, indices, order, front_of, parent):
    """Update rows of every front, by eliminating the graph row by row in the
    given order (a front that eliminates no row only assembles its children's
    update rows and passes them on); also the stored entries
    sum ne(ne-1)/2 + ne nu and the row-by-row nnz of L (no larger)."""
    parent = [int(p) for p in parent]
    n_front = len(parent)
    adj = _adjacency(indptr, indices)
    n = len(adj)
    done = np.zeros(n, dtype=bool)
    struct = [None] * n
    for v in order:
        v = int(v)
        nb = {w for w in adj[v] if not done[w]}
        struct[v] = nb
        for w in nb:
            adj[w] |= nb
            adj[w].discard(w)
        done[v] = True
    front_of = np.asarray(front_of)
    rows = [[] for _ in range(n_front)]
    for v in order:
        rows[int(front_of[v])].append(int(v))
    upd = []
    for x in range(n_front):
        own = set(rows[x])
        u = set()
        for v in rows[x]:
            u |= struct[v]
        if not rows[x]:
            for c in range(x):
                if parent[c] == x:
                    u |= set(upd[c])
        upd.append(sorted(u - own))
    ne = np.asarray([len(r) for r in rows])
    nu = np.asarray([len(u) for u in upd])
    stored = int(sum(e * (e - 1) // 2 + e * a for e, a in zip(ne.tolist(), nu.tolist())))
    return {"upd": upd, "ne": ne, "nu": nu, "stored": stored, "nnz_L": int(sum(len(s) for s in struct))}


def fronts_by_reach(indptr, indices, front_of, parent):
    """Update rows of every front from its own rows' neighbours and its children's update rows."""
    adj = _adjacency(indptr, indices)
    parent = [int(p) for p in parent]
    nf = len(parent)
    front_of = np.asarray(front_of)
    rows = [[] for _ in range(nf)]
    for v in range(len(adj)):
        rows[int(front_of[v])].append(v)
    children = [[] for _ in range(nf)]
    for x, p in enumerate(parent):
        if p >= 0:
            children[p].append(x)
    upd = [None] * nf
    for x in range(nf):
        u = set()
        for v in rows[x]:
            u |= {w for w in adj[v] if int(front_of[w]) != x and _ancestor(parent, int(front_of[w]), x)}
        for c in children[x]:
            u |= {w for w in upd[c] if int(front_of[w]) != x}
        upd[x] = sorted(u)
    return {"upd": upd, "nu": np.asarray([len(u) for u in upd])}
