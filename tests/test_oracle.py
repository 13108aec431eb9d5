"""Pins of the CPU oracle against what the paper and the mathematics fix.

* library special cases: dense LU == LAPACK (numpy.linalg.solve);
* invariants: L D L^T reconstructs A; F = F^T; Im(z^H F z) < 0;
* the paper's exactness claim (Section II): the decomposition route equals the
  undecomposed solve to rounding, on tiny meshes by brute force and on the
  8-domain mesh;
* closed form: with the linear field a + b x r as exact solution the oracle's
  DD route returns its interpolant;
* exact arithmetic: the double-double residual matches rational arithmetic;
* planted mistakes in the oracle are caught by the pins above.
"""
from fractions import Fraction

import numpy as np
import pytest

import femgen
import oracle
from oracle import dd as odd
from oracle import dense as odense


def _rand_csym(n, rng, lossy=True):
    X = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    A = X + X.T
    if lossy:  # Im part positive definite -> all leading minors nonsingular
        Y = rng.normal(size=(n, n))
        A = A + 1j * (Y @ Y.T + n * np.eye(n))
    return A


@pytest.mark.parametrize("n", [1, 5, 37])
def test_lu_matches_lapack(n):
    rng = np.random.default_rng(n)
    A = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    A[0, 0] = 0.0  # forces a row exchange
    b = rng.normal(size=(n, 3)) + 1j * rng.normal(size=(n, 3))
    if n == 1:
        A[0, 0] = 2.0 - 1j
    x = oracle.lu_solve(A, b)
    assert np.allclose(x, np.linalg.solve(A, b), rtol=1e-12, atol=1e-13)


def test_ldlt_reconstructs_and_solves():
    rng = np.random.default_rng(7)
    A = _rand_csym(60, rng)
    L, d = oracle.ldlt(A)
    assert np.allclose(np.diag(L), 1) and np.allclose(np.triu(L, 1), 0)
    assert np.abs(L @ np.diag(d) @ L.T - A).max() < 1e-11 * np.abs(A).max()
    b = rng.normal(size=(60, 2)) + 1j * rng.normal(size=(60, 2))
    assert np.allclose(oracle.ldlt_solve(L, d, b), np.linalg.solve(A, b), rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("n,levels", [(2, 1), (3, 2)])
def test_band_ldlt_equals_dense_lu(n, levels):
    p = femgen.tiny(n, levels)
    A = p.A_csr().toarray()
    x1 = oracle.lu_solve(A, p.b)
    bl = oracle.BandLDLT(p.A_indptr, p.A_indices, p.A_data).factor()
    assert sorted(bl.perm.tolist()) == list(range(p.n))
    x2 = bl.solve(p.b)
    assert np.linalg.norm(x2 - x1) <= 1e-13 * np.linalg.norm(x1)


@pytest.mark.parametrize("n,levels,jit", [(2, 1, False), (2, 2, False), (2, 3, False), (3, 3, False),
                                          (4, 3, True), (5, 4, True)])
def test_dd_equals_undecomposed_tiny(n, levels, jit):
    """The paper's 'numerically exact' claim on brute-force-sized meshes."""
    p = femgen.tiny(n, levels, jittered=jit, eps="random" if jit else "uniform")
    A = p.A_csr().toarray()
    x1 = oracle.lu_solve(A, p.b)
    o = oracle.DDOracle(p)
    u, lam = o.solve([s.f for s in p.subs])
    x3, mism = o.gather(u)
    assert np.linalg.norm(x3 - x1) <= 1e-12 * np.linalg.norm(x1)
    assert mism <= 1e-13 * np.abs(x1).max()
    # F = B A^{-1} B^T from a library solve of the block-diagonal system
    offs = np.cumsum([0] + [s.n for s in p.subs])
    N = offs[-1]
    Ablk = np.zeros((N, N), dtype=complex)
    B = np.zeros((p.n_dual, N))
    for o_, s in zip(offs, p.subs):
        Ablk[o_:o_ + s.n, o_:o_ + s.n] = s.dense()
        B[s.b_dual, o_ + s.b_local] = s.b_sign
    F_lib = B @ np.linalg.solve(Ablk, B.T)
    assert np.abs(o.F - F_lib).max() <= 1e-12 * np.abs(F_lib).max()
    assert np.abs(o.F - o.F.T).max() <= 1e-13 * np.abs(o.F).max()
    rng = np.random.default_rng(0)
    for _ in range(4):
        z = rng.normal(size=p.n_dual) + 1j * rng.normal(size=p.n_dual)
        assert (z.conj() @ o.F @ z).imag < 0


def test_dd_equals_undecomposed_c1(c1):
    bl = oracle.BandLDLT(c1.A_indptr, c1.A_indices, c1.A_data).factor()
    x2 = bl.solve(c1.b)
    o = oracle.DDOracle(c1)
    u, lam = o.solve([s.f for s in c1.subs])
    x3, mism = o.gather(u)
    assert np.linalg.norm(x3 - x2) <= 1e-12 * np.linalg.norm(x2)
    assert oracle.backward_error(c1.A_indptr, c1.A_indices, c1.A_data, x3, c1.b) < 1e-15
    rp, ru = oracle.arrow_residual(c1, u, lam)
    assert max(np.abs(r).max() for r in rp) < 1e-12 and np.abs(ru).max() < 1e-13


def test_dd_reproduces_linear_field(c1_linear):
    p = c1_linear
    o = oracle.DDOracle(p)
    u, lam = o.solve([s.f for s in p.subs])
    x, _ = o.gather(u)
    assert np.linalg.norm(x - p.x_exact) <= 1e-12 * np.linalg.norm(p.x_exact)


def _exact_residual(indptr, indices, data, x, b):
    out = []
    for i in range(indptr.size - 1):
        re = Fraction(b[i].real)
        im = Fraction(b[i].imag)
        for k in range(indptr[i], indptr[i + 1]):
            a = data[k]
            xv = x[indices[k]]
            re -= Fraction(a.real) * Fraction(xv.real) - Fraction(a.imag) * Fraction(xv.imag)
            im -= Fraction(a.real) * Fraction(xv.imag) + Fraction(a.imag) * Fraction(xv.real)
        out.append(complex(float(re), float(im)))
    return np.array(out)


def test_double_double_residual_is_exact():
    p = femgen.tiny(2, 1)
    x = np.linalg.solve(p.A_csr().toarray(), p.b[:, 0])   # residual ~ 1e-16: cancellation heavy
    r_dd = oracle.residual_dd(p.A_indptr, p.A_indices, p.A_data, x, p.b[:, 0])
    r_ex = _exact_residual(p.A_indptr, p.A_indices, p.A_data, x, p.b[:, 0])
    scale = np.abs(r_ex).max()
    assert np.abs(r_dd - r_ex).max() <= 1e-14 * scale


def test_refinement_recovers_solution():
    p = femgen.tiny(3, 1)
    A = p.A_csr().toarray()
    x1 = np.linalg.solve(A, p.b[:, 0])
    # a deliberately sloppy inner solver (single precision) still refines to FP64 accuracy
    A32 = A.astype(np.complex64)

    def solve32(r):
        return np.linalg.solve(A32, r.astype(np.complex64)).astype(np.complex128)
    x, hist = oracle.refine(p.A_indptr, p.A_indices, p.A_data, p.b[:, 0], solve32, tol=1e-15)
    assert np.linalg.norm(x - x1) <= 1e-13 * np.linalg.norm(x1)
    assert hist[0] > 1e-9 and hist[-1] <= 1e-15


# ---------------------------------------------------------------------------
# planted mistakes: each must make one of the pins above fail
# ---------------------------------------------------------------------------
def _ldlt_conj(A):
    """Hermitian-style LDL^H applied to a complex-symmetric matrix (wrong here)."""
    A = np.asarray(A, dtype=np.complex128)
    n = A.shape[0]
    L = np.eye(n, dtype=np.complex128)
    d = np.zeros(n, dtype=np.complex128)
    for j in range(n):
        v = L[j, :j].conj() * d[:j]
        d[j] = A[j, j] - L[j, :j] @ v
        L[j + 1:, j] = (A[j + 1:, j] - L[j + 1:, :j] @ v) / d[j]
    return L, d


def _solve_without_dual_term(self, f_list, g=None):
    p = self.p
    u = [odense.ldlt_solve(L, dd, f) for (L, dd), f in zip(self.facs, f_list)]
    return u, np.zeros((p.n_dual, f_list[0].shape[1]), dtype=complex)


def _schur_sign_flip(sub, fac=None):
    Fi, duals = odd.__dict__["_orig_schur"](sub, fac)
    return -Fi, duals


@pytest.mark.parametrize("mistake", ["conjugated_ldlt", "dropped_dual_term", "schur_sign"])
def test_planted_mistakes_are_caught(monkeypatch, mistake):
    p = femgen.tiny(3, 2)
    x1 = oracle.lu_solve(p.A_csr().toarray(), p.b)
    if mistake == "conjugated_ldlt":
        monkeypatch.setattr(odd, "ldlt", _ldlt_conj)
    elif mistake == "dropped_dual_term":
        monkeypatch.setattr(odd.DDOracle, "solve", _solve_without_dual_term)
    else:
        monkeypatch.setitem(odd.__dict__, "_orig_schur", odd.subdomain_schur)
        monkeypatch.setattr(odd, "subdomain_schur", _schur_sign_flip)
    o = odd.DDOracle(p)
    u, lam = o.solve([s.f for s in p.subs])
    x3, _ = o.gather(u)
    assert np.linalg.norm(x3 - x1) > 1e-6 * np.linalg.norm(x1)


# ---------------------------------------------------------------------------
# the undecomposed arrowhead route (inputs that need pivoting have no
# unpivoted DD route): pinned against the decomposition route and against the
# global LU on FEM problems, and by its residual on an indefinite input
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n,levels", [(2, 1), (3, 2)])
def test_arrow_solve_equals_dd_route(n, levels):
    p = femgen.tiny(n, levels)
    o = oracle.DDOracle(p)
    uo, lo = o.solve([s.f for s in p.subs])
    f = np.concatenate([s.f for s in p.subs], axis=0)
    u, lam = oracle.arrow_solve(p.subs, p.n_dual, f)
    assert np.linalg.norm(u - np.concatenate(uo)) <= 1e-12 * np.linalg.norm(u)
    assert np.linalg.norm(lam - lo) <= 1e-11 * np.linalg.norm(lam)
    x1 = oracle.lu_solve(p.A_csr().toarray(), p.b)
    x3, _ = o.gather(np.split(u, np.cumsum([s.n for s in p.subs])[:-1]))
    assert np.linalg.norm(x3 - x1) <= 1e-12 * np.linalg.norm(x1)


def test_arrow_solve_on_indefinite_chain():
    from femgen.indefinite import indefinite_chain
    p = indefinite_chain(n_sub=3, m=40, n_if=4, eps=0.0, nrhs=2, seed=5)
    f = np.concatenate([s.f for s in p.subs], axis=0)
    u, lam = oracle.arrow_solve(p.subs, p.n_dual, f)
    offs = np.cumsum([0] + [s.n for s in p.subs])
    rp, ru = oracle.arrow_residual(p, [u[offs[k]:offs[k + 1]] for k in range(p.n_sub)], lam)
    assert max(np.abs(r).max() for r in rp) <= 1e-12 * np.abs(f).max()
    assert np.abs(ru).max() <= 1e-12 * np.abs(u).max()
    # exactly zero diagonal: the unpivoted LDL^T of a domain breaks down at once
    with pytest.raises(np.linalg.LinAlgError):
        oracle.ldlt(odd._csr_dense(p.subs[0]))


# ---------------------------------------------------------------------------
# skyline (envelope) factor size of O2, the memory the paper compares against
# ---------------------------------------------------------------------------
def _csr(A):
    import scipy.sparse as sp
    M = sp.csr_matrix(A)
    M.sort_indices()
    return M.indptr.astype(np.int64), M.indices.astype(np.int64)


def test_envelope_closed_forms():
    n = 9
    ident = np.arange(n)
    ip, ix = _csr(np.eye(n))
    assert oracle.envelope_entries(ip, ix, ident) == n                       # diagonal: n
    T = np.eye(n) + np.eye(n, k=1) + np.eye(n, k=-1)
    ip, ix = _csr(T)
    assert oracle.envelope_entries(ip, ix, ident) == 2 * n - 1               # tridiagonal: 2n - 1
    ip, ix = _csr(np.ones((n, n)))
    assert oracle.envelope_entries(ip, ix, ident) == n * (n + 1) // 2        # dense: n(n+1)/2
    # arrow pointing down-right (last row full): n + (n - 1)(n)/2 ... its reversal is 2n - 1
    Ar = np.eye(n)
    Ar[-1, :] = Ar[:, -1] = 1
    ip, ix = _csr(Ar)
    assert oracle.envelope_entries(ip, ix, ident) == 2 * n - 1
    assert oracle.envelope_entries(ip, ix, ident[::-1].copy()) == n * (n + 1) // 2


def test_envelope_holds_the_band_factor():
    # the unpivoted LDL^T of the RCM-ordered matrix has no fill outside the envelope
    p = femgen.tiny(3, 2)
    A = p.A_csr().toarray()
    perm = oracle.rcm(p.A_indptr, p.A_indices)
    L, _ = oracle.ldlt(A[np.ix_(perm, perm)])
    nz = np.abs(np.tril(L)) > 0
    first = np.argmax(nz, axis=1)
    assert int(np.sum(np.arange(A.shape[0]) - first + 1)) <= oracle.envelope_entries(p.A_indptr, p.A_indices, perm)
