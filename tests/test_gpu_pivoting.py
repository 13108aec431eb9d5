"""GPU parity of the restricted Bunch-Kaufman pivoting option (Section II:
the diagonal blocks of the block LDL^T pivot inside the block only).

* single dense domain, FP64 form, every front pivoting: the number of
  interchanges and of 2x2 pivots equals the oracle's restricted Bunch-Kaufman
  with 64-wide blocks (FP64 decisions on both sides), and the solution matches
  the undecomposed solve;
* indefinite chain with a zero diagonal (femgen.indefinite): without domain
  pivoting the factorization stops with DD_ERR_SINGULAR_PIVOT; with it the
  result equals the oracle's undecomposed arrowhead solve;
* O(eps) auxiliary diagonal: pivoting in the auxiliary fronts only fires 2x2
  pivots there and keeps the result within tolerance;
* the FEM workloads give the same results with pivoting on as the oracle.
Tolerances: 1e-12 (FP64), 1e-10 (mixed after FP64 refinement).
"""
import numpy as np
import pytest

import femgen
import oracle
import paper_2002_05019_gb300 as dd
from femgen.indefinite import indefinite_chain
from oracle import dense as odense

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "mixed": 1e-10}


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def _dense_domain(A):
    n = A.shape[0]
    rows, cols = np.nonzero(np.ones((n, n), dtype=bool))
    return dict(n=n, indptr=np.arange(0, n * n + 1, n, dtype=np.int32), indices=cols.astype(np.int32),
                data=A[rows, cols], b_dual=np.zeros(0, np.int32), b_local=np.zeros(0, np.int32),
                b_sign=np.zeros(0, np.int8))


def _domains(p):
    return [dict(n=s.n, indptr=s.indptr, indices=s.indices, data=s.data, b_dual=s.b_dual, b_local=s.b_local,
                 b_sign=s.b_sign) for s in p.subs]


def _small_diag(n, seed):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    A = (X + X.T) / 2
    A[np.diag_indices(n)] *= 0.05
    return A


@pytest.mark.parametrize("n", [200, 64, 37])
def test_single_domain_decisions_match_oracle(n):
    A = _small_diag(n, seed=n)
    B = np.random.default_rng(1).normal(size=(n, 2)) + 1j * np.random.default_rng(2).normal(size=(n, 2))
    perm, L, D, n_swap, n_2x2 = odense.ldlt_bk_restricted(A, 64)
    xo = odense.ldlt_bk_solve(perm, L, D, B)
    assert rel(xo, oracle.lu_solve(A, B)) <= 1e-12
    s = dd.Solver([_dense_domain(A)], 0, precision="fp64", pivoting=2)
    s.factor()
    st = s.stats()
    assert (st["interchanges"], st["pivots_2x2"]) == (n_swap, n_2x2)
    assert n_swap + n_2x2 > 0
    X, _ = s.solve(B)
    assert rel(X, xo) <= TOL["fp64"]
    s.free()
    # mixed form: FP32 domain pivot blocks, refined in FP64
    s = dd.Solver([_dense_domain(A)], 0, precision="mixed", pivoting=2)
    s.factor()
    X, _ = s.solve(B)
    assert rel(X, xo) <= TOL["mixed"]
    s.free()


def test_zero_diagonal_needs_pivoting():
    A = _small_diag(96, seed=4)
    A[np.diag_indices(96)] = 0
    for mode in (0, 1):   # domain fronts unpivoted
        s = dd.Solver([_dense_domain(A)], 0, precision="fp64", pivoting=mode)
        with pytest.raises(dd.DDError) as e:
            s.factor()
        assert e.value.code == 3
        s.free()
    s = dd.Solver([_dense_domain(A)], 0, precision="fp64", pivoting=2)
    s.factor()
    b = np.ones((96, 1), dtype=np.complex128)
    x, _ = s.solve(b)
    assert rel(x, oracle.lu_solve(A, b)) <= TOL["fp64"]
    s.free()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("n_sub,m,n_if", [(4, 96, 8), (9, 150, 34)])
def test_indefinite_chain_against_oracle(precision, n_sub, m, n_if):
    p = indefinite_chain(n_sub=n_sub, m=m, n_if=n_if, eps=0.0, nrhs=2, seed=n_sub)
    f = np.concatenate([s.f for s in p.subs], axis=0)
    uo, lo = oracle.arrow_solve(p.subs, p.n_dual, f)
    s = dd.Solver(_domains(p), p.n_dual, precision=precision, pivoting=1)
    with pytest.raises(dd.DDError) as e:
        s.factor()
    assert e.value.code == 3
    s.free()
    s = dd.Solver(_domains(p), p.n_dual, precision=precision, pivoting=2)
    s.factor()
    st = s.stats()
    assert st["pivots_2x2"] > 0
    u, lam = s.solve(f)
    assert rel(u, uo) <= TOL[precision]
    assert rel(lam, lo) <= TOL[precision] * 10
    s.free()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_small_auxiliary_diagonal_pivots_in_auxiliary_fronts(precision):
    p = indefinite_chain(n_sub=8, m=128, n_if=40, eps=1e-2, nrhs=1, seed=11)
    f = np.concatenate([s.f for s in p.subs], axis=0)
    uo, lo = oracle.arrow_solve(p.subs, p.n_dual, f)
    s = dd.Solver(_domains(p), p.n_dual, precision=precision, pivoting=1)
    s.factor()
    st = s.stats()
    assert st["pivots_2x2"] > 0
    u, lam = s.solve(f)
    assert rel(u, uo) <= TOL[precision]
    assert rel(lam, lo) <= TOL[precision] * 10
    s.free()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("mode", [1, 2])
def test_fem_with_pivoting_against_oracle(precision, mode):
    p = femgen.plain_c1()
    o = oracle.DDOracle(p)
    uo, lo = o.solve([s.f for s in p.subs])
    xo, _ = o.gather(uo)
    s = dd.Solver.from_problem(p, precision=precision, pivoting=mode)
    s.factor()
    u, lam = s.solve(dd.stacked_loads(p))
    x, _ = o.gather(dd.unstack(p, u))
    assert rel(x, xo) <= TOL[precision]
    assert rel(lam, lo) <= TOL[precision] * 10
    s.free()
