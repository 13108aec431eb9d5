"""GPU: recovery of a subset of the primal unknowns (Section II: only the
requested subdomains are recovered after the auxiliary solve) and the factor
memory report.

* FP64 form, no refinement: the listed domains' u and lambda equal the full
  solve's bit for bit (the same kernels run on the same data; the other
  domains are simply not back-substituted), on 8 and 512 domains;
* mixed form (refined on every domain): the listed rows of the full refined
  solution;
* both forms against the oracle (DDOracle) on the 8-domain mesh, element by
  element (the 512-domain comparison is in test_gpu_parity_c2.py);
* bad, repeated and out-of-range ids are rejected;
* factor memory: dd_stats.bytes_factor against the skyline (envelope) factor
  of the undecomposed RCM-ordered system (the oracle's O2), reported.
"""
import numpy as np
import pytest

import femgen
import oracle
import paper_2002_05019_gb300 as dd

pytestmark = pytest.mark.gpu


def _rows(p, ids):
    offs = np.cumsum([0] + [s.n for s in p.subs])
    return np.concatenate([np.arange(offs[i], offs[i + 1]) for i in ids]) if len(ids) else np.zeros(0, int)


@pytest.mark.parametrize("name", ["plain", "batched"])
def test_fp64_subset_equals_full_solve(name):
    p = femgen.plain_c1(rhs="edges") if name == "plain" else femgen.batched_c2()
    s = dd.Solver.from_problem(p, precision="fp64")
    s.factor()
    f = dd.stacked_loads(p)
    u, lam = s.solve(f)
    rng = np.random.default_rng(0)
    for ids in ([5, 2, 7], list(rng.choice(p.n_sub, size=min(17, p.n_sub), replace=False)), [0], []):
        us, ls = s.solve_subset(f, ids)
        assert np.array_equal(ls, lam)
        assert np.array_equal(us, u[_rows(p, ids)])
    s.free()


def test_mixed_subset_is_the_refined_solution():
    p = femgen.plain_c1(rhs="edges")
    s = dd.Solver.from_problem(p, precision="mixed")
    s.factor()
    f = dd.stacked_loads(p)
    u, lam = s.solve(f)
    ids = [6, 1]
    us, ls = s.solve_subset(f, ids)
    rows = _rows(p, ids)
    assert np.linalg.norm(us - u[rows]) <= 1e-14 * np.linalg.norm(u[rows])
    assert np.linalg.norm(ls - lam) <= 1e-14 * np.linalg.norm(lam)
    s.free()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_subset_against_oracle_8_domains(c1, precision):
    o = oracle.DDOracle(c1)
    uo, lo = o.solve([s.f for s in c1.subs])
    s = dd.Solver.from_problem(c1, precision=precision)
    s.factor()
    ids = [6, 1, 3]
    us, ls = s.solve_subset(dd.stacked_loads(c1), ids)
    ref = np.concatenate([uo[i] for i in ids], axis=0)
    tol = 1e-12 if precision == "fp64" else 1e-10
    scale = max(np.abs(u).max() for u in uo)
    assert np.abs(us - ref).max() <= tol * scale
    assert np.linalg.norm(ls - lo) <= 10 * tol * np.linalg.norm(lo)
    s.free()


def test_subset_rejects_bad_ids():
    p = femgen.tiny(3, 2)
    s = dd.Solver.from_problem(p, precision="fp64")
    s.factor()
    f = dd.stacked_loads(p)
    for ids in ([0, 0], [p.n_sub], [-1]):
        with pytest.raises(dd.DDError) as e:
            s.solve_subset(f, ids)
        assert e.value.code == 1
    s.free()


def test_factor_memory_against_skyline():
    p = femgen.plain_c1()
    s = dd.Solver.from_problem(p, precision="fp64")
    s.factor()
    st = s.stats()
    env = oracle.envelope_entries(p.A_indptr, p.A_indices)
    sky_bytes = 16 * env
    print(f"\n8 domains, {p.n} DoFs: DD factor {st['bytes_factor'] / 1e6:.1f} MB, "
          f"skyline (RCM envelope) {sky_bytes / 1e6:.1f} MB")
    # every front stores at least its own lower triangle of the domain unknowns
    assert st["bytes_factor"] >= 16 * sum(sub.n * (sub.n + 1) // 2 for sub in p.subs)
    assert st["bytes_factor"] <= st["bytes_device"]
    s.free()
