"""The mixed form's diagonal-tile kernel on one 64 x 64 tile
(dd_selftest_pivot_tile), against the oracle's unpivoted LDL^T of the same
complex64 tile in FP64.

The tile is L0 D0 L0^T with two pivots of the first 32 x 32 pivot block about
1e-5 times the others, rounded to complex64: their elimination cancels five
digits, so FP32 pivot-block arithmetic loses them (about 1e-2 relative error
on those pivots, 2e-1 on the L column below), while the double-float form
(about 48 bits, the library's choice for unpivoted separator fronts) and
FP64 must keep them to the FP32 rounding of the output.  Outside the pivot
blocks the kernel computes in FP32 in every form, so the second block is
held to FP32 accuracy only (the L21 column below a cancelled pivot is formed
in FP32 and is right only in the backward sense: L D L^T reproduces the tile
to FP32 rounding), and the double-float and FP64 forms agree there.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

dd = pytest.importorskip("paper_2002_05019_gb300")


def _tile(seed=7, tiny=(7, 20), mag=1e-5):
    r = np.random.default_rng(seed)
    n = 64
    L0 = np.tril(0.3 * (r.normal(size=(n, n)) + 1j * r.normal(size=(n, n))), -1) + np.eye(n)
    d0 = (0.5 + r.random(n)) * np.exp(1j * r.uniform(-0.3, 0.3, n))
    for j in tiny:
        d0[j] *= mag
    return ((L0 * d0) @ L0.T).astype(np.complex64)


def _split(out):
    d = np.diag(out).astype(np.complex128)
    L = np.tril(out.astype(np.complex128), -1) + np.eye(64)
    return L, d


@pytest.fixture(scope="module")
def case():
    A = _tile()
    L, d = oracle.ldlt(A.astype(np.complex128))
    return A, L, d


@pytest.mark.parametrize("prec", ["dfloat", "fp64"])
def test_wide_pivot_blocks_keep_the_cancelled_pivots(case, prec):
    A, L, d = case
    out, linv = dd.pivot_tile(A, prec)
    Lk, dk = _split(out)
    rel_d = np.abs(dk - d) / np.abs(d)
    assert rel_d[:32].max() <= 1e-5, rel_d[:32].max()                 # first pivot block, both tiny pivots
    assert np.abs(Lk[:32, :32] - L[:32, :32]).max() <= 1e-5 * np.abs(L).max()
    assert rel_d[32:].max() <= 1e-3                                   # second block: FP32 Schur update
    # the whole tile to FP32 backward error (L21 below a tiny pivot is formed
    # in FP32 and is accurate only in this sense)
    R = (Lk * dk) @ Lk.T - A
    assert np.abs(R).max() <= 1e-5 * np.abs(A).max()
    # the stored inverse of the unit-lower factor
    N = linv.astype(np.complex128)
    assert np.abs(np.triu(N, 1)).max() == 0
    assert np.abs(N @ Lk - np.eye(64)).max() <= 1e-4


def test_fp32_pivot_blocks_lose_them(case):
    A, L, d = case
    out, _ = dd.pivot_tile(A, "fp32")
    _, dk = _split(out)
    rel = np.abs(dk - d) / np.abs(d)
    assert rel[[7, 20]].max() > 1e-3          # the tile does tell the precisions apart
    assert np.delete(rel[:32], [7, 20]).max() <= 1e-4


def test_double_float_agrees_with_fp64(case):
    A, _, _ = case
    a, na = dd.pivot_tile(A, "dfloat")
    b, nb = dd.pivot_tile(A, "fp64")
    La, da = _split(a)
    Lb, db = _split(b)
    rel = np.abs(da - db) / np.abs(db)
    assert rel[:32].max() <= 1e-6                     # both round the same pivots to FP32
    assert np.abs(La[:32, :32] - Lb[:32, :32]).max() <= 1e-6 * np.abs(Lb).max()
    # the second block sees the FP32 Schur update of both, which amplifies
    # last-bit differences of the first block: agreement to FP32 accuracy
    assert rel[32:].max() <= 1e-3
    assert np.abs(na[:32, :32].astype(np.complex128) - nb[:32, :32]).max() <= 1e-5 * np.abs(nb).max()


def test_rejects_bad_precision():
    with pytest.raises(KeyError):
        dd.pivot_tile(np.eye(64), "fp16")
