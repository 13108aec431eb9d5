"""Pins of the oracle's restricted Bunch-Kaufman LDL^T (Section II: pivoting
restricted to the diagonal blocks of the block LDL^T; pivot rule of Bunch and
Kaufman 1977 with alpha = (1 + sqrt 17) / 8).

* invariants: A[perm][:, perm] = L D L^T with L unit lower, D block diagonal
  with 1x1 / 2x2 blocks, perm a permutation that never leaves a block;
* library special case: the solve equals LAPACK (numpy.linalg.solve);
* special case nb = 1: no pivoting at all, the factors equal the unpivoted
  column LDL^T;
* the decision rule on hand-made matrices whose pivot choice follows from the
  rule by hand (2x2 on a zero diagonal, interchange, the alpha threshold on both
  sides, a large entry outside the block that must be ignored);
* planted mistakes (a wrong alpha, an unrestricted search) fail these pins.
"""
import numpy as np
import pytest

from oracle import dense as odense


def _csym_small_diag(n, seed, scale=0.05):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    A = (X + X.T) / 2
    A[np.diag_indices(n)] *= scale
    return A


def _check_structure(perm, L, D, nb):
    n = L.shape[0]
    assert sorted(perm.tolist()) == list(range(n))
    assert all(perm[i] // nb == i // nb for i in range(n)), "an interchange left its diagonal block"
    assert np.allclose(np.diag(L), 1) and np.allclose(np.triu(L, 1), 0)
    off = np.abs(D) > 0
    for i in range(n):
        for j in range(n):
            if off[i, j] and i != j:
                assert abs(i - j) == 1 and i // nb == j // nb   # 2x2 blocks only, inside a block
                assert L[max(i, j), min(i, j)] == 0


@pytest.mark.parametrize("n,nb", [(70, 16), (130, 64), (45, 32)])
def test_bk_reconstructs_and_solves(n, nb):
    A = _csym_small_diag(n, seed=n)
    perm, L, D, n_swap, n_2x2 = odense.ldlt_bk_restricted(A, nb)
    _check_structure(perm, L, D, nb)
    assert n_swap > 0 and n_2x2 > 0          # the small diagonal makes both kinds of pivot fire
    assert np.abs(A[perm][:, perm] - L @ D @ L.T).max() < 1e-12 * np.abs(A).max() * n
    b = np.random.default_rng(1).normal(size=(n, 2)) + 0j
    x = odense.ldlt_bk_solve(perm, L, D, b)
    assert np.linalg.norm(x - np.linalg.solve(A, b)) <= 1e-11 * np.linalg.norm(x)


def test_bk_with_unit_blocks_is_unpivoted_ldlt():
    rng = np.random.default_rng(3)
    X = rng.normal(size=(30, 30)) + 1j * rng.normal(size=(30, 30))
    Y = rng.normal(size=(30, 30))
    A = X + X.T + 1j * (Y @ Y.T + 30 * np.eye(30))
    perm, L, D, n_swap, n_2x2 = odense.ldlt_bk_restricted(A, 1)
    L0, d0 = odense.ldlt(A)
    assert n_swap == 0 and n_2x2 == 0 and (perm == np.arange(30)).all()
    assert np.allclose(L, L0, rtol=1e-12, atol=1e-13) and np.allclose(np.diag(D), d0, rtol=1e-12)


def test_bk_decisions_by_hand():
    c = np.complex128
    # zero diagonal: lambda = 1 > 0 = |a00|, sigma = 0, |a11| = 0 < alpha sigma fails -> 2x2
    perm, L, D, ns, n2 = odense.ldlt_bk_restricted(np.array([[0, 1], [1, 0]], c), 64)
    assert (ns, n2) == (0, 1) and D[0, 1] == 1
    # |a00| = 1e-3 < alpha, sigma = 1, |a11| = 2 >= alpha -> 1x1 after interchanging 0 and 1
    perm, L, D, ns, n2 = odense.ldlt_bk_restricted(np.array([[1e-3, 1], [1, 2]], c), 64)
    assert (ns, n2) == (1, 0) and perm.tolist() == [1, 0] and D[0, 0] == 2
    # alpha = 0.6404: |a00| = 0.65 lambda keeps the 1x1 pivot, 0.63 lambda goes on to a 2x2
    hi = np.array([[0.65, 1, 0], [1, 0.1, 0], [0, 0, 1]], c)
    lo = np.array([[0.63, 1, 0], [1, 0.1, 0], [0, 0, 1]], c)
    assert odense.ldlt_bk_restricted(hi, 64)[3:] == (0, 0)
    assert odense.ldlt_bk_restricted(lo, 64)[3:] == (0, 1)
    # |a00| sigma >= alpha lambda^2 keeps the 1x1: a00 = 0.5, lambda = 1 (r = 1), sigma = |a21| = 1.5
    keep = np.array([[0.5, 1, 0.2], [1, 0.1, 1.5], [0.2, 1.5, 1]], c)
    assert odense.ldlt_bk_restricted(keep, 64)[3:] == (0, 0)


def test_bk_search_is_restricted_to_the_block():
    # the large a20 lies outside the first 2 x 2 block: only a10 = 0.01 is seen
    A = np.array([[1e-3, 0.01, 1, 0], [0.01, 1, 0, 0], [1, 0, 1, 0], [0, 0, 0, 1]], np.complex128)
    perm, L, D, ns, n2 = odense.ldlt_bk_restricted(A, 2)
    assert perm.tolist() == [1, 0, 2, 3] and (ns, n2) == (1, 0)
    # lambda = 0 inside the block: no interchange at all, whatever lies outside
    B = np.array([[1e-3, 0, 1], [0, 1, 0], [1, 0, 1]], np.complex128)
    assert odense.ldlt_bk_restricted(B, 2)[3:] == (0, 0)


@pytest.mark.parametrize("mistake", ["alpha_half", "unrestricted"])
def test_planted_bk_mistakes_are_caught(monkeypatch, mistake):
    lo = np.array([[0.63, 1, 0], [1, 0.1, 0], [0, 0, 1]], np.complex128)
    A = np.array([[1e-3, 0.01, 1, 0], [0.01, 1, 0, 0], [1, 0, 1, 0], [0, 0, 0, 1]], np.complex128)
    if mistake == "alpha_half":
        monkeypatch.setattr(odense, "BK_ALPHA", 0.5)
        assert odense.ldlt_bk_restricted(lo, 64)[3:] != (0, 1)
    else:
        perm = odense.ldlt_bk_restricted(A, 4)[0]      # the search sees the whole matrix
        assert perm.tolist() != [1, 0, 2, 3]
