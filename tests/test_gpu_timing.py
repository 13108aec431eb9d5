"""GPU: per-launch kernel timing of the factorization (dd_options.time_kernels):
0 none, 1 every launch (a device time per kernel class), 2 the trailing-update
launches only.  The event nodes change neither the launches nor the result;
the setup and factor times are reported whatever the mode."""
import numpy as np
import pytest

import femgen
import paper_2002_05019_gb300 as dd

pytestmark = pytest.mark.gpu


def test_kernel_timing_modes():
    p = femgen.plain_c1()
    f = dd.stacked_loads(p)
    res = {}
    for mode in (0, 1, 2):
        s = dd.Solver.from_problem(p, precision="mixed", time_kernels=mode)
        s.factor()
        st = s.stats()
        u, _ = s.solve(f)
        assert st["t_setup_ms"] > 0 and st["t_factor_ms"] > 0
        res[mode] = (st["kernel_ms"], st["kernel_launches"], u)
        s.free()
    (km0, kl0, u0), (km1, kl1, u1), (km2, kl2, u2) = res[0], res[1], res[2]
    assert all(v == 0 for v in km0.values())
    assert km1["update"] > 0 and km1["diag"] > 0 and km1["trsm"] > 0
    assert km2["update"] > 0 and km2["diag"] == 0 and km2["trsm"] == 0 and km2["assemble"] == 0
    assert kl0 == kl1 == kl2
    for u in (u1, u2):
        assert np.linalg.norm(u - u0) <= 1e-12 * np.linalg.norm(u0)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_class_flops_add_up_to_the_factor_count(precision):
    """The per-class algorithmic flops (diagonal blocks, panels, trailing
    updates; exact front sizes, no tile padding) add up to the factorization's
    algorithmic count (4/3 n^3 per elimination plus the Schur terms), within
    the interior columns that share a tile with interface columns."""
    p = femgen.medium()
    s = dd.Solver.from_problem(p, precision=precision)
    s.factor()
    st = s.stats()
    kf = st["kernel_flops"]
    total = kf["diag"] + kf["trsm"] + kf["update"]
    assert kf["update"] > 0.9 * total
    assert abs(total - st["flops_factor"]) <= 0.03 * st["flops_factor"]
    s.free()
