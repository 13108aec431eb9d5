"""GPU: domains factored sparsely (Section II: the primal unknowns are
eliminated by sparse direct factorizations of the domains).

With dd_options.sparse_min, a domain of at least that many unknowns becomes a
tree of fronts ordered by nested dissection (interface unknowns last, in the
domain's root front, which carries the domain's duals as update rows), inside
the same front tree as the auxiliary matrix.  Checked through the C ABI:

* 8 domains of 2,863 unknowns against the oracle's sparse route
  (oracle.SparseDDOracle: SuperLU per domain), element by element, both forms,
  unpivoted and with restricted Bunch-Kaufman pivoting in every front; F_i of
  every domain against the oracle's;
* 64 domains of 500..2,500 unknowns with the larger half sparse and the rest
  dense fronts, against the oracle's tree route;
* 8 domains of 13,428 unknowns (the dense route's fronts would be 13k wide):
  the linear-field closed form, and fewer stored factor entries than the dense
  route;
* new values (dd_set_values) and the listed-domain solve.
"""
import numpy as np
import pytest

import femgen
import oracle
import paper_2002_05019_gb300 as dd

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "mixed": 1e-10}
OPTS = {"fp64": {}, "mixed": {"refine_tol": 1e-11}}


def _gather(p, u):
    x = np.zeros((p.n,) + u.shape[1:], dtype=np.complex128)
    seen = np.zeros(p.n, dtype=bool)
    off = 0
    for s in p.subs:
        new = ~seen[s.l2g]
        x[s.l2g[new]] = u[off:off + s.n][new]
        seen[s.l2g] = True
        off += s.n
    return x


def _check(p, u, lam, u_o, lam_o, tol):
    x, x_o = _gather(p, u), _gather(p, u_o)
    assert np.linalg.norm(x - x_o) <= tol * np.linalg.norm(x_o)
    assert np.abs(u - u_o).max() <= tol * np.abs(u_o).max()
    assert np.linalg.norm(lam - lam_o) <= 10 * tol * np.linalg.norm(lam_o)


@pytest.fixture(scope="module")
def big14():
    p = femgen.big_domains(14)
    o = oracle.SparseDDOracle(p)
    u, lam = o.solve([s.f for s in p.subs])
    return p, o, np.concatenate(u, axis=0), lam


@pytest.mark.parametrize("precision,pivoting", [("fp64", 0), ("mixed", 0), ("fp64", 2), ("mixed", 2)])
def test_sparse_domains_against_oracle(big14, precision, pivoting):
    p, o, u_o, lam_o = big14
    s = dd.Solver.from_problem(p, precision=precision, sparse_min=1000, pivoting=pivoting, **OPTS[precision])
    st = s.stats()
    assert st["n_fronts"] > 2 * p.n_sub      # the domains became trees of fronts
    s.factor()
    u, lam = s.solve(dd.stacked_loads(p))
    _check(p, u, lam, u_o, lam_o, TOL[precision])
    if pivoting == 0:
        for i, sub in enumerate(p.subs):
            Fi, duals = s.schur(i)
            lu = o.lus[i]
            Bt, do = o.Bt[i]
            Fo = Bt.T @ lu.solve(Bt)
            assert np.array_equal(duals, do)
            tol = 1e-12 if precision == "fp64" else float(np.linalg.cond(sub.dense())) * 2.0 ** -21
            assert np.linalg.norm(Fi - Fo) <= tol * np.linalg.norm(Fo)
    s.free()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_mixed_dense_and_sparse_domains_against_oracle(precision):
    p = femgen.medium()
    t = oracle.TreeDDOracle(p)
    u_o, lam_o = t.solve([s.f for s in p.subs])
    u_o = np.concatenate(u_o, axis=0)
    sizes = np.array([sub.n for sub in p.subs])
    cut = int(np.median(sizes))
    s = dd.Solver.from_problem(p, precision=precision, sparse_min=cut, **OPTS[precision])
    s.factor()
    u, lam = s.solve(dd.stacked_loads(p))
    _check(p, u, lam, u_o, lam_o, TOL[precision])
    # new values (twice the matrices: half the primal solution, the same
    # multipliers since 2 A (u / 2) + B^T lambda = f), same analysis
    s.set_values(np.concatenate([2.0 * sub.data for sub in p.subs]))
    s.factor()
    u2, lam2 = s.solve(dd.stacked_loads(p))
    _check(p, u2, lam2, 0.5 * u_o, lam_o, TOL[precision])
    # listed domains: a sparse one and a dense one
    ids = [int(np.argmax(sizes)), int(np.argmin(sizes))]
    us, _ = s.solve_subset(dd.stacked_loads(p), ids)
    offs = np.cumsum([0] + list(sizes))
    ref = np.concatenate([0.5 * u_o[offs[i]:offs[i + 1]] for i in ids], axis=0)
    assert np.abs(us - ref).max() <= TOL[precision] * np.abs(u_o).max()
    s.free()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_large_sparse_domains_closed_form(precision):
    """8 domains of 13,428 unknowns: linear-field closed form, and the stored
    factor against the dense route's."""
    p = femgen.big_domains(24, rhs="linear")
    s = dd.Solver.from_problem(p, precision=precision, sparse_min=2000, **OPTS[precision])
    s.factor()
    u, _ = s.solve(dd.stacked_loads(p))
    x = _gather(p, u)
    assert np.linalg.norm(x - p.x_exact) <= TOL[precision] * np.linalg.norm(p.x_exact)
    sparse_bytes = s.stats()["bytes_factor"]
    s.free()
    dense = dd.Solver.from_problem(p, precision=precision)
    dense_bytes = dense.stats()["bytes_factor"]
    dense.free()
    print(f"\n{precision}: factor bytes sparse domains {sparse_bytes / 1e9:.2f} GB, dense {dense_bytes / 1e9:.2f} GB")
    assert sparse_bytes < dense_bytes / 3
