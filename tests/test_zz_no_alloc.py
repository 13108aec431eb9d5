"""dd_dense_solve_noalloc: the allocation-free dense solve, through the C ABI.

This entry point serves callers that cannot allocate device memory once they
are running (an application whose allocator owns all device memory, or a loop
that cannot afford cudaMalloc's synchronisation or failure); its scratch is a
static device array.  The test checks it against the allocating entry points
(dd_setup / dd_factor / dd_solve on the same system as a single domain) within
the FP64 tolerance, on calls in a row with different systems (small, the
largest, small again), and checks
that sizes beyond its limit and host pointers are rejected.  It sits in its own
file, collected last, and passes alone or after the other tests.
"""
import ctypes as C

import numpy as np
import pytest

import femgen
import paper_2002_05019_gb300 as dd

pytestmark = pytest.mark.gpu

TOL = 1e-12


def _lossy_symmetric(n, seed):
    """Random complex-symmetric matrix with a positive-definite imaginary part."""
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    Y = rng.normal(size=(n, n))
    return (X + X.T) / np.sqrt(n) + 1j * (Y @ Y.T / n + np.eye(n))


def _allocating_solve(A, B):
    n = A.shape[0]
    rows, cols = np.nonzero(np.ones_like(A, dtype=bool))
    indptr = np.arange(0, n * n + 1, n, dtype=np.int32)
    s = dd.Solver([dict(n=n, indptr=indptr, indices=cols.astype(np.int32), data=A[rows, cols],
                        b_dual=np.zeros(0, np.int32), b_local=np.zeros(0, np.int32),
                        b_sign=np.zeros(0, np.int8))], 0)
    s.factor()
    X, _ = s.solve(B)
    s.free()
    return X


def _noalloc_solve(A, B):
    import torch
    lib = dd.load()
    n, nrhs = B.shape
    At = torch.from_numpy(np.ascontiguousarray(A.T)).cuda()        # column-major A
    Bt = torch.from_numpy(np.ascontiguousarray(B.T)).cuda()        # column-major B (n x nrhs)
    Xt = torch.full_like(Bt, float("nan"))
    code = lib.dd_dense_solve_noalloc(n, C.c_void_p(At.data_ptr()), n, nrhs, C.c_void_p(Bt.data_ptr()), n,
                                      C.c_void_p(Xt.data_ptr()), n, None)
    return code, Xt.cpu().numpy().T


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_noalloc_matches_allocating_path_twice():
    # a FEM domain matrix (ragged size), then the maximum size, then a smaller
    # system again: the shared scratch still holds the large call's front and
    # right-hand sides (another padded order), which must not leak into it
    p = femgen.tiny(3, 1)
    A1 = p.subs[0].dense()
    B1 = np.random.default_rng(1).normal(size=(A1.shape[0], 3)) + 0j
    A2 = _lossy_symmetric(512, seed=2)
    B2 = np.random.default_rng(3).normal(size=(512, 16)) + 1j * np.random.default_rng(4).normal(size=(512, 16))
    A3 = _lossy_symmetric(77, seed=5)
    B3 = np.random.default_rng(6).normal(size=(77, 2)) + 0j
    for A, B in ((A1, B1), (A2, B2), (A3, B3)):
        code, X = _noalloc_solve(A, B)
        assert code == 0
        Xref = _allocating_solve(A, B)
        assert rel(X, Xref) <= TOL
        assert rel(A @ X, B) <= 1e-10


def test_noalloc_rejects_out_of_range_and_host_pointers():
    import torch
    lib = dd.load()
    n = 513
    A = torch.zeros((n, n), dtype=torch.complex128, device="cuda")
    b = torch.zeros((1, n), dtype=torch.complex128, device="cuda")
    x = torch.zeros_like(b)
    assert lib.dd_dense_solve_noalloc(n, C.c_void_p(A.data_ptr()), n, 1, C.c_void_p(b.data_ptr()), n,
                                      C.c_void_p(x.data_ptr()), n, None) == 1
    assert lib.dd_dense_solve_noalloc(8, C.c_void_p(A.data_ptr()), n, 17, C.c_void_p(b.data_ptr()), n,
                                      C.c_void_p(x.data_ptr()), n, None) == 1
    hb = np.zeros(8, dtype=np.complex128)
    assert lib.dd_dense_solve_noalloc(8, C.c_void_p(A.data_ptr()), n, 1, C.c_void_p(hb.ctypes.data), 8,
                                      C.c_void_p(x.data_ptr()), n, None) == 1
