"""Symbolic analysis of the auxiliary matrix (Section II: symbolic
factorization on the clique graph of the domain interfaces, nested dissection
along the domain tree).  CPU only.

* the oracle's two routes to the front tree agree: symbolic elimination of the
  clique graph (the definition) and the update rows passed up the tree;
* structural invariants: the separators partition the duals, every dual is
  eliminated at the lowest tree node holding all its domains, the root passes
  nothing on, update rows belong to ancestors' separators;
* planted mistakes (in the oracle) are caught: the elimination without fill,
  and duals assigned to the wrong tree node;
* the library's symbolic analysis (dd_symbolic, host only) equals the oracle's
  front tree exactly: parents, sizes, the front of every dual and every
  front's update-row set.
"""
import numpy as np
import pytest

import femgen
import oracle
import paper_2002_05019_gb300 as dd

SMALL = [("tiny 2/1", lambda: femgen.tiny(2, 1)), ("tiny 2/3", lambda: femgen.tiny(2, 3)),
         ("tiny 3/2", lambda: femgen.tiny(3, 2)), ("tiny 3/3 jittered", lambda: femgen.tiny(3, 3, jittered=True)),
         ("8 domains", femgen.plain_c1)]


def _same_tree(a, b):
    assert a["n_front"] == b["n_front"]
    assert np.array_equal(a["parent"], b["parent"])
    assert np.array_equal(a["ne"], b["ne"])
    assert np.array_equal(a["nu"], b["nu"])
    assert np.array_equal(np.asarray(a["dual_front"]), np.asarray(b["dual_front"]))
    for x in range(a["n_front"]):
        assert set(int(d) for d in a["upd"][x]) == set(int(d) for d in b["upd"][x]), f"front {x}"


def _subtree_leaves(parent, n_sub):
    leaves = [set() for _ in parent]
    for i in range(n_sub):
        x = i
        while x >= 0:
            leaves[x].add(i)
            x = parent[x]
    return leaves


def _check_invariants(t, p):
    parent = [int(x) for x in t["parent"]]
    n_sub, n_front = p.n_sub, t["n_front"]
    doms = oracle.dual_domains(p.subs, p.n_dual)
    below = _subtree_leaves(parent, n_sub)
    # the separators partition the duals
    seen = np.zeros(p.n_dual, dtype=int)
    for v in range(n_sub, n_front):
        for d in t["sep"][v]:
            seen[d] += 1
    assert (seen == 1).all()
    assert int(sum(t["ne"][n_sub:])) == p.n_dual
    # every dual at the lowest node whose subtree holds all its domains
    for d, v in enumerate(t["dual_front"]):
        v = int(v)
        assert v >= n_sub and set(doms[d]) <= below[v], f"dual {d}"
        for c in range(n_front):
            if parent[c] == v and c >= n_sub:
                assert not set(doms[d]) <= below[c], f"dual {d} could go lower"
    # the root passes nothing on; update rows are ancestors' separator duals
    roots = [x for x in range(n_front) if parent[x] < 0]
    assert len(roots) == 1 and t["nu"][roots[0]] == 0
    for x in range(n_front):
        anc, y = set(), parent[x]
        while y >= 0:
            anc.add(y)
            y = parent[y]
        for d in t["upd"][x]:
            assert int(t["dual_front"][d]) in anc, f"front {x} dual {d}"
    # leaves eliminate their domain, and pass on exactly its duals
    for i in range(n_sub):
        assert t["ne"][i] == p.subs[i].n
        assert set(t["upd"][i]) == set(int(d) for d in p.subs[i].b_dual)


@pytest.mark.parametrize("name,make", SMALL)
def test_oracle_routes_agree(name, make):
    p = make()
    a = oracle.fronts_by_elimination(p.rcb.parent, p.subs, p.n_dual)
    b = oracle.fronts_by_tree(p.rcb.parent, p.subs, p.n_dual)
    _same_tree(a, b)
    for x in range(a["n_front"]):
        assert a["sep"][x] == b["sep"][x]
    _check_invariants(b, p)


def test_oracle_routes_agree_64_domains():
    p = femgen.medium()
    a = oracle.fronts_by_elimination(p.rcb.parent, p.subs, p.n_dual)
    b = oracle.fronts_by_tree(p.rcb.parent, p.subs, p.n_dual)
    _same_tree(a, b)
    _check_invariants(b, p)
    # the top separators are duals on the first cut planes: the root eliminates the most
    assert a["ne"][-1] == max(a["ne"][p.n_sub:])


def test_planted_mistakes_are_caught():
    p = femgen.medium()
    b = oracle.fronts_by_tree(p.rcb.parent, p.subs, p.n_dual)
    # 1. elimination without the fill misses update rows of the upper fronts
    nf = oracle.fronts_by_elimination(p.rcb.parent, p.subs, p.n_dual, fill=False)
    assert any(set(nf["upd"][x]) != set(b["upd"][x]) for x in range(b["n_front"]))
    # 2. duals at the parent of their lowest domain instead of the common ancestor
    doms = oracle.dual_domains(p.subs, p.n_dual)
    wrong = dict(b)
    wrong["dual_front"] = np.asarray([int(p.rcb.parent[ds[0]]) for ds in doms])
    with pytest.raises(AssertionError):
        _check_invariants(wrong, p)


@pytest.mark.parametrize("name,make", SMALL + [("64 domains", femgen.medium), ("512 domains", femgen.batched_c2)])
def test_library_symbolic_equals_oracle(name, make):
    p = make()
    lib = dd.symbolic_problem(p)
    ref = oracle.fronts_by_tree(p.rcb.parent, p.subs, p.n_dual)
    _same_tree(lib, ref)
