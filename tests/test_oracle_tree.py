"""The oracle's tree route (oracle.TreeDDOracle: the auxiliary matrix
eliminated block by block over the domain tree), the route that reaches the
512- and 2048-domain workloads.  CPU only.

Pinned by what the method and the mathematics fix, not by itself:
  * Section II's exactness: it equals the dense decomposition route (DDOracle,
    whose F is one dense matrix factored by the oracle's own LDL^T) on tiny
    meshes and on 8 and 64 domains, and the undecomposed sparse solve
    (SuperLU of the assembled global matrix) on 64 domains;
  * a closed form: with the linear field a + b x r as exact solution it
    returns the field's edge interpolant;
  * the subtree restriction: the block its top node passes up equals the
    Schur complement, written out densely, of the subtree's part of F onto
    the duals that leave the subtree;
  * planted mistakes in the oracle (B without its signs; Hermitian instead of
    complex-symmetric solves; a front that drops a child's block) fail these
    pins.
"""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse.linalg as spla

import femgen
import oracle
import oracle.tree as otree


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _solve(o, p):
    u, lam = o.solve([s.f for s in p.subs])
    return o.gather(u)[0], lam


@pytest.mark.parametrize("n,levels,jit", [(2, 1, False), (3, 2, False), (4, 3, True), (6, 4, True)])
def test_tree_route_equals_dense_route_tiny(n, levels, jit):
    p = femgen.tiny(n, levels, jittered=jit, eps="random" if jit else "uniform")
    xa, la = _solve(oracle.DDOracle(p), p)
    xb, lb = _solve(otree.TreeDDOracle(p), p)
    assert _rel(xb, xa) <= 1e-12
    assert _rel(lb, la) <= 1e-12


def test_tree_route_equals_dense_route_8_domains(c1):
    xa, la = _solve(oracle.DDOracle(c1), c1)
    t = otree.TreeDDOracle(c1)
    xb, lb = _solve(t, c1)
    assert _rel(xb, xa) <= 1e-12
    assert _rel(lb, la) <= 1e-12
    assert t.passed_up[max(t.fronts)][0].size == 0      # the root passes nothing on


@pytest.fixture(scope="module")
def p64():
    """64 jittered-bisection domains of 10^3 cubes (7,930 unknowns, 3,150 duals)."""
    return femgen.build_problem("t64", 10, 6, split_range=(0.37, 0.63), eps="random")


def test_tree_route_64_domains_equals_dense_route_and_global_solve(p64):
    p = p64
    xg = spla.splu(p.A_csr().tocsc()).solve(p.b)
    xa, la = _solve(oracle.DDOracle(p), p)
    xb, lb = _solve(otree.TreeDDOracle(p), p)
    assert _rel(xb, xa) <= 1e-12
    assert _rel(lb, la) <= 1e-12
    assert _rel(xb, xg) <= 1e-11
    assert np.abs(xb - xg).max() <= 1e-11 * np.abs(xg).max()


def test_tree_route_linear_field_closed_form():
    p = femgen.build_problem("t64-linear", 10, 6, split_range=(0.37, 0.63), eps="random", rhs="linear")
    x, _ = _solve(otree.TreeDDOracle(p), p)
    assert _rel(x, p.x_exact) <= 1e-11


def test_subtree_passes_up_the_dense_schur_complement(p64):
    p = p64
    parent = np.asarray(p.rcb.parent)
    # a node two levels below the root: 16 domains
    root = parent.size - 1
    node = max(x for x in range(parent.size) if parent[x] >= 0 and parent[parent[x]] == root)
    t = otree.TreeDDOracle(p, subtree=node)
    assert len(t.domains) == 16
    up_duals, S = t.passed_up[node]
    # definition: F_sub = sum over the subtree's domains of B_i A_i^{-1} B_i^T on
    # their duals; eliminate every dual of the subtree's fronts
    duals = np.unique(np.concatenate([np.asarray(p.subs[i].b_dual) for i in t.domains]))
    F = np.zeros((duals.size, duals.size), dtype=np.complex128)
    for i in t.domains:
        Bt, di = oracle.local_B(p.subs[i])
        ix = np.searchsorted(duals, di)
        F[np.ix_(ix, ix)] += Bt.T @ np.linalg.solve(p.subs[i].dense(), Bt)
    inner = np.concatenate([t.sep[v] for v in t.fronts])
    a = np.searchsorted(duals, inner)
    b = np.searchsorted(duals, up_duals)
    assert np.array_equal(np.sort(np.concatenate([inner, up_duals])), duals)
    S_def = F[np.ix_(b, b)] - F[np.ix_(b, a)] @ np.linalg.solve(F[np.ix_(a, a)], F[np.ix_(a, b)])
    assert _rel(S, S_def) <= 1e-12


def test_planted_unsigned_B_is_caught(c1, monkeypatch):
    xa, _ = _solve(oracle.DDOracle(c1), c1)
    real = otree.local_B

    def unsigned(sub):
        Bt, duals = real(sub)
        return np.abs(Bt), duals

    monkeypatch.setattr(otree, "local_B", unsigned)
    xb, _ = _solve(otree.TreeDDOracle(c1), c1)
    assert _rel(xb, xa) > 1e-6


def test_planted_hermitian_solves_are_caught(c1, monkeypatch):
    """Solving with A^H instead of A (a conjugation the complex-symmetric,
    non-Hermitian systems must not have)."""
    xa, _ = _solve(oracle.DDOracle(c1), c1)

    class HermitianSolves:
        lu_factor = staticmethod(sla.lu_factor)

        @staticmethod
        def lu_solve(lu, b, **kw):
            return sla.lu_solve(lu, b, trans=2, **kw)

    monkeypatch.setattr(otree, "sla", HermitianSolves)
    xb, _ = _solve(otree.TreeDDOracle(c1), c1)
    assert _rel(xb, xa) > 1e-6


def test_planted_dropped_child_block_is_caught(p64, monkeypatch):
    """Update rows that leave out the fill (a front built from its separator's
    direct neighbours only): a child then passes duals its parent does not
    hold, which the assembly refuses."""
    real = otree.fronts_by_tree

    def no_fill(parent, subs, n_dual):
        ft = real(parent, subs, n_dual)
        top = len(parent) - 1
        for v in range(len(subs), top):
            if ft["upd"][v]:
                ft["upd"][v] = ft["upd"][v][: len(ft["upd"][v]) // 2]
        return ft

    monkeypatch.setattr(otree, "fronts_by_tree", no_fill)
    with pytest.raises(ValueError):
        otree.TreeDDOracle(p64)
