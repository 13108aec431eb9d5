"""Nested-dissection symbolic analysis of one domain matrix (the sparse-domain
route; Section II factors each domain with a sparse direct solver).  CPU only:
dd_domain_symbolic runs on the host.

* the library's dissection is valid (oracle.domain_symbolic.check_dissection);
* the front structure it implies is unique, and the library's equals the
  oracle's by row-by-row graph elimination and by reach, index for index;
* the stored front entries never undercount the row-by-row nnz of L;
* planted mistakes are caught: a separator row moved into a child, and update
  rows computed without the children's.
"""
import numpy as np
import pytest

import femgen
from oracle import domain_symbolic as ods
import paper_2002_05019_gb300 as dd


def _iface(sub):
    il = np.zeros(sub.n, np.int8)
    il[np.asarray(sub.b_local)] = 1
    return il


CASES = [("8 domains, domain 0", lambda: femgen.plain_c1().subs[0], 32),
         ("8 domains, domain 5", lambda: femgen.plain_c1().subs[5], 64),
         ("tiny 3/1", lambda: femgen.tiny(3, 1).subs[0], 16),
         ("jittered tiny 4/2", lambda: femgen.tiny(4, 2, jittered=True).subs[1], 24),
         ("2,863-row domain", lambda: femgen.big_domains(14).subs[0], 128)]


@pytest.mark.parametrize("name,make,leaf_max", CASES)
def test_library_dissection_and_fronts(name, make, leaf_max):
    s = make()
    il = _iface(s)
    t = dd.domain_symbolic(s.indptr, s.indices, il, leaf_max=leaf_max)
    assert t["n_front"] > 1
    ods.check_dissection(t, s.indptr, s.indices, il, leaf_max)
    reach = ods.fronts_by_reach(s.indptr, s.indices, t["front_of"], t["parent"])
    for x in range(t["n_front"]):
        assert list(t["upd"][x]) == reach["upd"][x], f"front {x}"
    if s.n <= 1000:   # row-by-row elimination: the definition, small graphs only
        el = ods.fronts_by_elimination(s.indptr, s.indices, t["order"], t["front_of"], t["parent"])
        assert el["upd"] == reach["upd"]
        assert np.array_equal(el["ne"], t["ne"]) and el["stored"] == t["stored"]
        assert el["nnz_L"] <= el["stored"]


def test_no_interface_and_pattern_errors():
    s = femgen.tiny(3, 1).subs[0]
    t = dd.domain_symbolic(s.indptr, s.indices, None, leaf_max=16)
    ods.check_dissection(t, s.indptr, s.indices, None, 16)
    assert t["ne"][-1] == 0 and t["nu"][-1] == 0   # no interface rows: an empty root over the dissection
    # an unsymmetric pattern is rejected
    rp = np.array([0, 2, 3], np.int32)
    ci = np.array([0, 1, 1], np.int32)
    with pytest.raises(dd.DDError) as e:
        dd.domain_symbolic(rp, ci)
    assert e.value.code == 2


def test_planted_mistakes_are_caught():
    s = femgen.plain_c1().subs[0]
    il = _iface(s)
    t = dd.domain_symbolic(s.indptr, s.indices, il, leaf_max=32)
    # 1. a separator row moved into one child's front: some edge now crosses subtrees
    parent = t["parent"]
    sep_front = next(x for x in range(t["n_front"] - 1) if any(parent[c] == x for c in range(x)) and t["ne"][x] > 0)
    child = next(c for c in range(sep_front) if parent[c] == sep_front)
    bad = dict(t)
    bad["front_of"] = t["front_of"].copy()
    row = int(np.flatnonzero(t["front_of"] == sep_front)[0])
    bad["front_of"][row] = child
    with pytest.raises(AssertionError):
        ods.check_dissection(bad, s.indptr, s.indices, il, 32)
    # 2. update rows without the children's: the root-ward fronts lose rows
    adj_only = []
    for x in range(t["n_front"]):
        rows = np.flatnonzero(t["front_of"] == x)
        u = set()
        for v in rows:
            for w in s.indices[s.indptr[v]:s.indptr[v + 1]]:
                fw = int(t["front_of"][w])
                if fw != x and ods._ancestor(parent, fw, x):
                    u.add(int(w))
        adj_only.append(sorted(u))
    el = ods.fronts_by_elimination(s.indptr, s.indices, t["order"], t["front_of"], t["parent"])
    assert adj_only != el["upd"]


def _multifrontal_solve(s, mp, b):
    """Unpivoted multifrontal LDL^T of A_i over the library's front tree, driven
    only by its assembly maps (entries scattered to fronts, update blocks
    extend-added into parents), then the forward, diagonal and backward
    substitutions over the same tree."""
    nf, parent, ne = mp["n_front"], mp["parent"], mp["ne"]
    rp, rows, ea = mp["rows_ptr"], mp["rows"], mp["ea_map"]
    rowid = np.repeat(np.arange(s.n), np.diff(s.indptr))
    fronts, upd_blocks, facs = [], [None] * nf, [None] * nf
    for x in range(nf):
        m = int(rp[x + 1] - rp[x])
        fronts.append(np.zeros((m, m), dtype=np.complex128))
    for q in np.flatnonzero(mp["a_front"] >= 0):
        x, r, c = mp["a_front"][q], mp["a_row"][q], mp["a_col"][q]
        assert r >= c
        fronts[x][r, c] += s.data[q]
    for x in range(nf):
        Fm = fronts[x]
        for c in range(x):
            if parent[c] == x and upd_blocks[c] is not None:
                idx = ea[rp[c] + ne[c]:rp[c + 1]]
                assert (idx >= 0).all() and (np.diff(idx) > 0).all()   # increasing rows of the parent
                Fm[np.ix_(idx, idx)] += upd_blocks[c]
        Fm = np.tril(Fm) + np.tril(Fm, -1).T
        e = ne[x]
        L = np.eye(e, dtype=np.complex128)
        d = np.zeros(e, dtype=np.complex128)
        A11 = Fm[:e, :e].copy()
        for j in range(e):          # unpivoted LDL^T of the own block
            d[j] = A11[j, j]
            L[j + 1:, j] = A11[j + 1:, j] / d[j]
            A11[j + 1:, j + 1:] -= np.outer(L[j + 1:, j], A11[j, j + 1:])
        L21 = np.linalg.solve(L, Fm[e:, :e].T).T / d       # F21 L11^{-T} D^{-1}
        upd_blocks[x] = np.tril(Fm[e:, e:] - (L21 * d) @ L21.T)
        facs[x] = (L, d, L21)
    y = b.astype(np.complex128).copy()
    for x in range(nf):             # forward
        L, d, L21 = facs[x]
        r = rows[rp[x]:rp[x + 1]]
        w = np.linalg.solve(L, y[r[:ne[x]]])
        y[r[:ne[x]]] = w
        y[r[ne[x]:]] -= L21 @ w
    for x in range(nf):
        y[rows[rp[x]:rp[x] + ne[x]]] /= facs[x][1][:, None]
    for x in range(nf - 1, -1, -1):  # backward
        L, d, L21 = facs[x]
        r = rows[rp[x]:rp[x + 1]]
        y[r[:ne[x]]] = np.linalg.solve(L.T, y[r[:ne[x]]] - L21.T @ y[r[ne[x]:]])
    return y


@pytest.mark.parametrize("name,make,leaf_max", CASES)
def test_assembly_maps_drive_a_correct_factorization(name, make, leaf_max):
    s = make()
    il = _iface(s)
    mp = dd.domain_assembly(s.indptr, s.indices, il, leaf_max=leaf_max)
    t = dd.domain_symbolic(s.indptr, s.indices, il, leaf_max=leaf_max)
    assert np.array_equal(mp["parent"], t["parent"]) and np.array_equal(mp["ne"], t["ne"])
    # every front's rows: its own rows in elimination order, then its update rows
    for x in range(mp["n_front"]):
        r = mp["rows"][mp["rows_ptr"][x]:mp["rows_ptr"][x + 1]]
        assert np.array_equal(np.sort(r[mp["ne"][x]:]), np.sort(t["upd"][x]))
    # each unordered entry pair assembled exactly once
    assert int((mp["a_front"] >= 0).sum()) == (s.indices.size + s.n) // 2
    b = np.random.default_rng(3).standard_normal((s.n, 2)) + 0j
    x = _multifrontal_solve(s, mp, b)
    ref = np.linalg.solve(s.dense(), b)
    assert np.linalg.norm(x - ref) <= 1e-10 * np.linalg.norm(ref)
