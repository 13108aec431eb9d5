"""The oracle's sparse-domain route (oracle.SparseDDOracle: SuperLU for each
A_i, LAPACK LU for the dense F), for domains beyond the dense route's reach
(Section II: the domains are factored by sparse direct solvers).  CPU only.

Pinned by the method's exactness: it equals the dense decomposition route on
the 8-domain mesh, and the undecomposed global solve on a mesh whose domains
exceed 2,500 unknowns; F is symmetric with Im(z^H F z) < 0 (lossy domains);
and a planted mistake (B without its signs) is caught.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import femgen
import oracle
import oracle.dd as odd


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_sparse_route_equals_dense_route():
    p = femgen.plain_c1()
    f = [s.f for s in p.subs]
    a, b = oracle.DDOracle(p), oracle.SparseDDOracle(p)
    ua, la = a.solve(f)
    ub, lb = b.solve(f)
    assert _rel(b.F, a.F) <= 1e-12
    assert _rel(lb, la) <= 1e-12
    assert _rel(b.gather(ub)[0], a.gather(ua)[0]) <= 1e-12


@pytest.fixture(scope="module")
def large():
    p = femgen.big_domains(14)
    assert min(s.n for s in p.subs) > 2500
    return p, spla.splu(p.A_csr().tocsc()).solve(p.b)


def test_sparse_route_equals_global_solve(large):
    p, xg = large
    o = oracle.SparseDDOracle(p)
    u, lam = o.solve([s.f for s in p.subs])
    x, mismatch = o.gather(u)
    assert _rel(x, xg) <= 1e-11
    assert mismatch <= 1e-12 * np.abs(x).max()
    assert _rel(o.F.T, o.F) <= 1e-13
    z = np.random.default_rng(7).standard_normal((p.n_dual, 4)) + 1j * np.random.default_rng(8).standard_normal((p.n_dual, 4))
    assert (np.einsum("ij,ik,kj->j", z.conj(), o.F, z).imag < 0).all()


def test_planted_sign_mistake_is_caught(large, monkeypatch):
    p, xg = large
    real_local_B = odd.local_B

    def unsigned_B(sub):
        Bt, duals = real_local_B(sub)
        return np.abs(Bt), duals

    monkeypatch.setattr(odd, "local_B", unsigned_B)
    o = odd.SparseDDOracle(p)
    u, _ = o.solve([s.f for s in p.subs])
    assert _rel(o.gather(u)[0], xg) > 1e-6
