"""Failure detection without a GPU fault.

A device-side wait on a flag that nothing sets must give up after its bound
(about a second), report DD_ERR_TIMEOUT to the host, and leave the CUDA
context usable for the next solve.  Bad inputs are rejected on the host
(tests/test_abi.py); a singular pivot is reported as a status code.
"""
import numpy as np
import pytest

import femgen
import paper_2002_05019_gb300 as dd

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_context_survives():
    lib = dd.load()
    assert lib.dd_selftest_wait_timeout(None) == 8
    p = femgen.tiny(3, 2)
    s = dd.Solver.from_problem(p)
    s.factor()
    u, lam = s.solve(dd.stacked_loads(p))
    assert np.all(np.isfinite(u))
    s.free()


def test_zero_pivot_is_reported():
    """A domain matrix with a zero leading pivot (lossless, singular block)."""
    n = 3
    A = np.array([[0.0, 1.0, 0.0], [1.0, 2.0, 1.0], [0.0, 1.0, 2.0]], dtype=complex)
    indptr = np.array([0, 3, 6, 9], np.int32)
    indices = np.tile(np.arange(3, dtype=np.int32), 3)
    s = dd.Solver([dict(n=n, indptr=indptr, indices=indices, data=A.ravel(), b_dual=np.zeros(0, np.int32),
                        b_local=np.zeros(0, np.int32), b_sign=np.zeros(0, np.int8))], 0)
    with pytest.raises(dd.DDError) as e:
        s.factor()
    assert e.value.code == 3
    with pytest.raises(dd.DDError) as e:
        s.solve(np.ones(3))
    assert e.value.code == 6
    s.free()
