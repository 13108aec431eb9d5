"""GPU: the schedule autotuner of the tensor-core factorization path and the
schedules it chooses among.

Every schedule (one, two or four panels per update pass, look-ahead on levels with
at most 0 / 8 / 32 / 128 fronts, 8 / 16 / 32 SMs left to the panel chain) is a
different launch order of the same arithmetic: each must give the oracle's
solution to the mixed tolerance; the tuner must leave the handle factored with
the schedule it reports."""
import numpy as np
import pytest

import femgen
import oracle
import paper_2002_05019_gb300 as dd

pytestmark = pytest.mark.gpu

TOL = 1e-10


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def c1():
    p = femgen.plain_c1()
    o = oracle.DDOracle(p)
    uo, lo = o.solve([s.f for s in p.subs])
    return p, o.gather(uo)[0]


def _x(p, u):
    x = np.zeros((p.n,) + u.shape[1:], dtype=np.complex128)
    off = 0
    for s in p.subs:
        x[s.l2g] = u[off:off + s.n]
        off += s.n
    return x


@pytest.mark.parametrize("sched", [(1, 0, 16), (2, 0, 16), (4, 0, 16), (1, 128, 8), (2, 128, 32), (2, 8, 16),
                                   (2, 1024, 16), (4, 8, 16), (4, 128, 16, 40), (2, 0, 16, 24), (1, 8, 8, 64),
                                   (4, 1024, 32, 120)])
def test_every_schedule_solves(c1, sched):
    p, xo = c1
    s = dd.Solver.from_problem(p, precision="mixed")
    s.set_schedule(*sched)
    s.factor()
    u, _ = s.solve(dd.stacked_loads(p))
    assert rel(_x(p, u), xo) <= TOL
    s.free()


def test_autotune_picks_and_keeps_a_schedule(c1):
    p, xo = c1
    s = dd.Solver.from_problem(p, precision="mixed")
    r = s.autotune(repeats=1)
    assert r["configs_tried"] == 39 + 3 and r["factor_ms"] > 0      # the grid, then three leaf splits
    assert r["split_sms"] in (0, 24, 40, 64)
    assert r["update_panels"] in (1, 2, 4) and r["ahead_fronts"] in (0, 8, 32, 128, 1024)
    u, _ = s.solve(dd.stacked_loads(p))          # factored by the tuner with its choice
    assert rel(_x(p, u), xo) <= TOL
    with pytest.raises(dd.DDError) as e:
        s.set_schedule(3, 0, 16)
    assert e.value.code == 1
    with pytest.raises(dd.DDError) as e:
        s.set_schedule(4, 0, 16, 121)
    assert e.value.code == 1
    s.free()
    f = dd.Solver.from_problem(p, precision="fp64")
    assert f.autotune(repeats=1)["configs_tried"] == 1
    f.free()


def test_autotune_schedule_cache(c1, tmp_path):
    """A tuned schedule is filed under the problem's key and this GPU; a
    second handle of the same problem gets it at setup, and its autotune
    returns it without timing."""
    p, xo = c1
    path = str(tmp_path / "tune.jsonl")
    s = dd.Solver.from_problem(p, precision="mixed", tune_cache=path)
    r = s.autotune(repeats=1)
    assert r["configs_tried"] == 42
    s.free()
    lines = open(path).read().splitlines()
    assert len(lines) == 1 and ("%016x" % dd.tune_key_problem(p)) in lines[0]
    t = dd.Solver.from_problem(p, precision="mixed", tune_cache=path)
    r2 = t.autotune(repeats=1)
    assert r2["configs_tried"] == 0
    assert [r2[k] for k in ("update_panels", "ahead_fronts", "reserve_sms", "split_sms")] == \
           [r[k] for k in ("update_panels", "ahead_fronts", "reserve_sms", "split_sms")]
    u, _ = t.solve(dd.stacked_loads(p))
    assert rel(_x(p, u), xo) <= TOL
    t.free()
    assert len(open(path).read().splitlines()) == 1     # a hit appends nothing
