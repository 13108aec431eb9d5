"""Domain partition and tearing into an arrowhead (FETI-style) system.

The paper decomposes the boundary value problem into domains, keeps primal
unknowns in the domain volumes and dual unknowns on the domain interfaces, and
so obtains a sparse arrowhead matrix (Section II).  It defers the formulation
to its cited works, so the tearing here is the FETI one: every domain keeps its
own copy of each edge it touches, and each edge shared by domains
s_1 < s_2 < ... < s_m carries m - 1 Lagrange multipliers enforcing
u_{s_1}(e) - u_{s_k}(e) = 0 (sign +1 in B_{s_1}, -1 in B_{s_k}).  That choice is
non-redundant, so B has full row rank.

The partition is recursive coordinate bisection on whole cubes of the mesh
(all six tetrahedra of a cube go to the same domain), splitting the longest
side of the current box at a cube plane, at a seeded random fraction.  The
recursion tree is kept: it is the separator tree that orders the dual unknowns.
"""
from __future__ import annotations

from dataclasses import dataclass
from functools import lru_cache

import numpy as np

from .mesh import kuhn_edge_count

# fallback cuts stay within this fraction of the side
_CUT_LIMIT = (0.3, 0.7)


def _cut_range(n_ax: int):
    lo = max(1, int(np.ceil(_CUT_LIMIT[0] * n_ax)))
    hi = min(n_ax - 1, int(np.floor(_CUT_LIMIT[1] * n_ax)))
    return range(lo, hi + 1)


@dataclass
class RcbTree:
    cell_sub: np.ndarray   # (n^3,) domain id of every cube
    boxes: list            # per domain: (lo (3,), hi (3,)) in cube units
    parent: np.ndarray     # (2 ns - 1,) parent node id; leaves 0..ns-1, internal ns.. in post-order; root -1
    children: np.ndarray   # (2 ns - 1, 2) children of internal nodes, -1 for leaves


def rcb_cells(n: int, levels: int, split_range=None, rng=None, size_range=None,
              max_tries: int = 500) -> RcbTree:
    """Recursive coordinate bisection of an n^3 cube grid into 2**levels boxes.

    split_range=None cuts every box in half (rounded down); otherwise the cut
    fraction is drawn from U[split_range] with `rng`.  With size_range=(lo, hi)
    a draw is redrawn while a final box would hold fewer than lo or more than
    hi edges, or while an intermediate box could not reach that range.
    """
    leaves: list = []
    parent: list = []
    children: list = []
    internal_ids: list = []

    @lru_cache(maxsize=None)
    def _feasible(ext, rem):
        lo, hi = size_range
        if rem == 0:
            return lo <= kuhn_edge_count(*ext) <= hi
        ax = int(np.argmax(ext))
        n_ax = ext[ax]
        for c in _cut_range(n_ax):
            e1 = list(ext)
            e1[ax] = c
            e2 = list(ext)
            e2[ax] = n_ax - c
            if _feasible(tuple(e1), rem - 1) and _feasible(tuple(e2), rem - 1):
                return True
        return False

    def feasible(ext, rem):
        """Can this box still be cut into 2**rem leaves of lo..hi edges?"""
        if size_range is None:
            return True
        return _feasible(tuple(int(v) for v in ext), rem)

    def rec(lo, hi, rem):
        if rem == 0:
            leaves.append((lo.copy(), hi.copy()))
            return ("leaf", len(leaves) - 1)
        ext = hi - lo
        ax = int(np.argmax(ext))
        if ext[ax] < 2:
            raise ValueError("box too small to split")
        for _ in range(max_tries):
            f = 0.5 if split_range is None else rng.uniform(*split_range)
            cut = lo[ax] + int(np.floor(f * ext[ax] + (0.0 if split_range is None else 0.5)))
            cut = min(max(cut, lo[ax] + 1), hi[ax] - 1)
            hi1 = hi.copy()
            hi1[ax] = cut
            lo2 = lo.copy()
            lo2[ax] = cut
            if feasible(hi1 - lo, rem - 1) and feasible(hi - lo2, rem - 1):
                break
        else:
            # no random draw worked: take the feasible cut closest to the middle
            cuts = sorted((lo[ax] + c for c in _cut_range(ext[ax])), key=lambda c: (abs(c - lo[ax] - 0.5 * ext[ax]), c))
            for cut in cuts:
                hi1 = hi.copy()
                hi1[ax] = cut
                lo2 = lo.copy()
                lo2[ax] = cut
                if feasible(hi1 - lo, rem - 1) and feasible(hi - lo2, rem - 1):
                    break
            else:
                raise RuntimeError(f"no feasible split of box {lo}-{hi} with {rem} levels left")
        a = rec(lo, hi1, rem - 1)
        b = rec(lo2, hi, rem - 1)
        node = len(internal_ids)
        internal_ids.append((a, b))
        return ("int", node)

    rec(np.zeros(3, dtype=np.int64), np.full(3, n, dtype=np.int64), levels)
    ns = len(leaves)
    nn = 2 * ns - 1
    parent = np.full(nn, -1, dtype=np.int64)
    children = np.full((nn, 2), -1, dtype=np.int64)

    def gid(ref):
        kind, idx = ref
        return idx if kind == "leaf" else ns + idx

    for k, (a, b) in enumerate(internal_ids):
        p = ns + k
        for slot, ch in enumerate((a, b)):
            c = gid(ch)
            parent[c] = p
            children[p, slot] = c

    cell_sub = np.empty(n ** 3, dtype=np.int64)
    for s, (lo, hi) in enumerate(leaves):
        ci = np.arange(lo[0], hi[0])
        cj = np.arange(lo[1], hi[1])
        ck = np.arange(lo[2], hi[2])
        I, J, K = np.meshgrid(ci, cj, ck, indexing="ij")
        cell_sub[(I + n * (J + n * K)).ravel()] = s
    return RcbTree(cell_sub=cell_sub, boxes=leaves, parent=parent, children=children)


@dataclass
class Tearing:
    l2g: list                # per domain: sorted global edge ids of its local copies
    n_dual: int
    dual_edge: np.ndarray    # (n_dual,) global edge of each multiplier
    dual_pair: np.ndarray    # (n_dual, 2) domains (s_1, s_k) it couples
    b_dual: list             # per domain: multiplier ids of its B entries
    b_local: list            # per domain: local index of the edge copy
    b_sign: list             # per domain: +1 / -1
    edge_mult: np.ndarray    # (E,) number of domains touching each edge


def tear(tet_edges: np.ndarray, tet_sub: np.ndarray, n_edges: int, n_sub: int) -> Tearing:
    """Local edge copies per domain and the star-to-lowest multipliers."""
    l2g = []
    for s in range(n_sub):
        l2g.append(np.unique(tet_edges[tet_sub == s]))
    # (edge, domain) incidence, sorted by edge then domain
    pe = np.concatenate(l2g)
    ps = np.concatenate([np.full(len(g), s, dtype=np.int64) for s, g in enumerate(l2g)])
    o = np.lexsort((ps, pe))
    pe = pe[o]
    ps = ps[o]
    mult = np.bincount(pe, minlength=n_edges)
    first = np.r_[True, pe[1:] != pe[:-1]]
    owner = ps[first]                       # s_1 per touched edge, in edge order
    owner_of_edge = np.full(n_edges, -1, dtype=np.int64)
    owner_of_edge[pe[first]] = owner
    others = ~first                          # (edge, s_k) pairs with k >= 2
    dual_edge = pe[others]
    dual_pair = np.stack([owner_of_edge[dual_edge], ps[others]], axis=1)
    n_dual = int(dual_edge.size)

    b_dual, b_local, b_sign = [], [], []
    did = np.arange(n_dual, dtype=np.int64)
    for s in range(n_sub):
        g = l2g[s]
        plus = dual_pair[:, 0] == s
        minus = dual_pair[:, 1] == s
        d = np.concatenate([did[plus], did[minus]])
        e = np.concatenate([dual_edge[plus], dual_edge[minus]])
        sg = np.concatenate([np.ones(plus.sum(), dtype=np.int8), -np.ones(minus.sum(), dtype=np.int8)])
        o = np.argsort(d, kind="stable")
        b_dual.append(d[o].astype(np.int32))
        b_local.append(np.searchsorted(g, e[o]).astype(np.int32))
        b_sign.append(sg[o])
    return Tearing(l2g=l2g, n_dual=n_dual, dual_edge=dual_edge, dual_pair=dual_pair,
                   b_dual=b_dual, b_local=b_local, b_sign=b_sign, edge_mult=mult)
