"""The C-ABI library builds, loads and exports every declared entry point.

CPU-only: no compute call reaches a GPU.  dd_setup validates its inputs and
runs the whole symbolic analysis on the host before it looks for a device,
so the error codes of bad inputs, and the success of the analysis on good
ones (reported as DD_ERR_NO_DEVICE here), are checked without a GPU.
"""
import ctypes as C
import os
import re

import numpy as np
import pytest

import femgen
import paper_2002_05019_gb300 as dd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _gpu_present():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def _declared():
    names = []
    inc = os.path.join(ROOT, "include")
    for f in sorted(os.listdir(inc)):
        if f.endswith(".h"):
            src = open(os.path.join(inc, f)).read()
            names += re.findall(r"^(?:int|void|const char\*)\s+(dd_\w+)\s*\(", src, re.M)
    return names


def test_every_declared_symbol_is_exported():
    lib = dd.load()
    names = _declared()
    assert set(names) == set(dd.EXPORTS)
    for n in names:
        assert getattr(lib, n) is not None


def test_strerror_covers_all_codes():
    lib = dd.load()
    seen = set()
    for code in range(10):
        s = lib.dd_strerror(code).decode()
        assert s and s != "unknown status"
        seen.add(s)
    assert len(seen) == 10
    assert lib.dd_strerror(99).decode() == "unknown status"


def test_null_handles_are_rejected():
    lib = dd.load()
    lib.dd_free(None)
    assert lib.dd_factor(None) == 1
    assert lib.dd_solve(None, 1, None, 1, None, 1, None, 1) == 1
    assert lib.dd_solve_subset(None, 1, None, 1, 0, None, None, 1, None, 1) == 1
    assert lib.dd_autotune(None, 1, None) == 1
    assert lib.dd_set_schedule(None, None) == 1
    assert lib.dd_get_stats(None, None) == 1
    # dd_symbolic: NULL outputs
    assert lib.dd_symbolic(1, None, 0, None, 4, None, None, None, None, None, 0, None, None) == 1
    assert lib.dd_domain_symbolic(4, None, None, None, 16, 8, None, None, None, None, None, None, None, 0, None,
                                  None) == 1
    assert lib.dd_domain_assembly(4, None, None, None, 16, 8, None, None, None, 0, None, None, None, None, None,
                                  None) == 1


def test_symbolic_output_limits():
    """dd_symbolic reports the front count when max_fronts is too small, and
    rejects an update-row buffer that cannot hold the rows."""
    import ctypes as C
    lib = dd.load()
    p = femgen.tiny(2, 2)
    subs, opt, keep = dd._marshal(dd._problem_subs(p), tree_parent=p.rcb.parent)
    nf = C.c_int32(0)
    small = np.zeros(2, np.int32)
    dual_front = np.zeros(p.n_dual, np.int32)
    st = lib.dd_symbolic(p.n_sub, subs, p.n_dual, C.byref(opt), 2, C.byref(nf), small.ctypes.data, small.ctypes.data,
                         small.ctypes.data, dual_front.ctypes.data, 0, None, None)
    assert st == 1 and nf.value == 2 * p.n_sub - 1
    cap = nf.value
    par, ne, nu = (np.zeros(cap, np.int32) for _ in range(3))
    ptr = np.zeros(cap + 1, np.int64)
    idx = np.zeros(1, np.int32)
    st = lib.dd_symbolic(p.n_sub, subs, p.n_dual, C.byref(opt), cap, C.byref(nf), par.ctypes.data, ne.ctypes.data,
                         nu.ctypes.data, dual_front.ctypes.data, 1, ptr.ctypes.data, idx.ctypes.data)
    assert st == 1 and ptr[cap] > 1
    del keep


def _subs(p):
    return [dict(n=s.n, indptr=s.indptr, indices=s.indices, data=s.data, b_dual=s.b_dual,
                 b_local=s.b_local, b_sign=s.b_sign) for s in p.subs]


def _setup_code(subs, n_dual, **kw):
    try:
        s = dd.Solver(subs, n_dual, **kw)
        s.free()
        return 0
    except dd.DDError as e:
        return e.code


@pytest.mark.skipif(_gpu_present(), reason="checks the host-only path of dd_setup")
def test_setup_host_analysis_succeeds_without_device():
    p = femgen.tiny(3, 2, jittered=False)
    assert _setup_code(_subs(p), p.n_dual, tree_parent=p.rcb.parent) == 9      # NO_DEVICE: analysis passed
    assert _setup_code(_subs(p), p.n_dual, centroids=p.centroids()) == 9
    assert _setup_code(_subs(p), p.n_dual) == 9
    assert _setup_code(_subs(p), p.n_dual, pivoting=2) == 9                      # every pivoting mode accepted


def test_setup_rejects_bad_inputs():
    p = femgen.tiny(2, 1)
    good = _subs(p)
    # non-symmetric values
    bad = [dict(d) for d in good]
    data = bad[0]["data"].copy()
    r, c = 0, int(bad[0]["indices"][bad[0]["indptr"][0] + 1])
    data[bad[0]["indptr"][0] + 1] += 1.0
    bad[0]["data"] = data
    assert _setup_code(bad, p.n_dual) == 2
    # column index out of range
    bad = [dict(d) for d in good]
    ind = bad[1]["indices"].copy()
    ind[-1] = bad[1]["n"] + 5
    bad[1]["indices"] = ind
    assert _setup_code(bad, p.n_dual) == 1
    # dual id out of range
    bad = [dict(d) for d in good]
    bd = bad[0]["b_dual"].copy()
    bd[0] = p.n_dual
    bad[0]["b_dual"] = bd
    assert _setup_code(bad, p.n_dual) == 1
    # sign other than +-1
    bad = [dict(d) for d in good]
    bs = bad[0]["b_sign"].copy()
    bs[0] = 2
    bad[0]["b_sign"] = bs
    assert _setup_code(bad, p.n_dual) == 1
    # a dual that no domain touches
    assert _setup_code(good, p.n_dual + 1) == 1
    # malformed tree (parent before child)
    assert _setup_code(good, p.n_dual, tree_parent=np.array([2, 0, -1])) == 1
    # unsupported options
    assert _setup_code(good, p.n_dual, precision="fp64", refine_tol=-1.0) == 1
    assert _setup_code(good, p.n_dual, pivoting=3) == 1
    assert _setup_code(good, p.n_dual, pivoting=-1) == 1
