"""The tree route sharded over ranks along subtrees of the front tree
(oracle.shard), run as gloo ranks on the CPU, and the library's host-side
shard plan (dd_shard_plan).  CPU only.

Pinned by:
  * the one-rank tree route (itself pinned against the dense route, the
    global sparse solve and a closed form): the sharded solve over 2 and 4
    ranks, with a dual right-hand side g that every rank must subtract only
    on the duals it solves, equals it to rounding on 8 and 64 domains;
  * the cut's definition: each rank's fronts are the subtree of its root,
    the subtrees are disjoint and hold every domain, the fronts above the cut
    are exactly the roots' ancestors and belong to rank 0, and on the 8 equal
    domains of the 2x2x2 box the cut into 8 is the domains themselves;
  * the library's plan equals the oracle's, bit for bit, for 1..16 ranks;
  * a planted mistake (rank 0 skips the elimination of the right-hand side
    over the fronts above the cut) fails the first pin.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

import femgen  # noqa: E402
import oracle.shard as oshard  # noqa: E402
import oracle.tree as otree  # noqa: E402


def _problem(name):
    if name == "c1":
        return femgen.plain_c1()
    return femgen.build_problem("t64", 10, 6, split_range=(0.37, 0.63), eps="random")


def _dual_rhs(p, k):
    r = np.random.default_rng(11)
    return r.normal(size=(p.n_dual, k)) + 1j * r.normal(size=(p.n_dual, k))


def _loads(p):
    return [s.f for s in p.subs]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


_THREADS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")


def _rank_main(rank, world, port, name, plant, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    torch.distributed.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p = _problem(name)
        if plant == "skip_top_forward":
            oshard.forward_fronts = lambda *a, **k: None
        sh = oshard.ShardedTreeDD(p, oshard.plan_problem(p, world))
        f = _loads(p)
        g = _dual_rhs(p, f[0].shape[1])
        res = sh.gather(sh.solve(f, g))
        if rank == 0:
            u, lam = res
            out.put((np.concatenate([x[:, 0] for x in u]), lam[:, 0], len(sh.top), len(sh.T.domains)))
        torch.distributed.barrier()
    finally:
        torch.distributed.destroy_process_group()


def _run(world, name, plant=None):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, name, plant, q)) for r in range(world)]
    saved = {k: os.environ.get(k) for k in _THREADS}
    os.environ.update({k: str(max(1, (os.cpu_count() or 1) // world)) for k in _THREADS})   # no oversubscription
    try:
        for pr in procs:
            pr.start()
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    res = q.get(timeout=300)
    for pr in procs:
        pr.join(timeout=120)
        assert pr.exitcode == 0
    return res


def _one_rank(name):
    p = _problem(name)
    f = _loads(p)
    u, lam = otree.TreeDDOracle(p).solve(f, _dual_rhs(p, f[0].shape[1]))
    return np.concatenate([x[:, 0] for x in u]), lam[:, 0]


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("name,world", [("c1", 2), ("c1", 4), ("t64", 4)])
def test_sharded_route_equals_one_rank(name, world):
    u1, l1 = _one_rank(name)
    u, lam, n_top, n_dom0 = _run(world, name)
    assert n_top >= 1 and n_dom0 >= 1
    assert _rel(u, u1) <= 1e-12
    assert _rel(lam, l1) <= 1e-12


def test_planted_skipped_top_forward_is_caught():
    u1, l1 = _one_rank("c1")
    u, lam, _, _ = _run(4, "c1", plant="skip_top_forward")      # above the cut: fronts with update duals
    assert _rel(lam, l1) > 1e-6


def _check_cut(parent, sh, n_ranks):
    parent = np.asarray(parent)
    roots = sh["rank_root"]
    fr = np.asarray(sh["front_rank"])
    assert len(roots) == n_ranks and np.all(np.diff(roots) > 0)
    below = np.zeros(parent.size, dtype=int)
    for r, v in enumerate(roots):
        nodes = otree.subtree_nodes(parent, int(v))
        below[nodes] += 1
        assert np.all(fr[nodes] == r)
    assert below.max() == 1                              # disjoint subtrees
    leaves = np.setdiff1d(np.arange(parent.size), parent[parent >= 0])
    assert np.all(below[leaves] == 1)                    # every domain below the cut
    above = set(int(x) for x in np.nonzero(below == 0)[0])
    anc = set()
    for v in roots:
        anc.update(_ancestors(parent, int(v)))
    assert above == anc                                  # above the cut: the roots' ancestors, on rank 0
    assert all(fr[x] == 0 for x in above)


def _ancestors(parent, v):
    out = []
    while parent[v] >= 0:
        v = int(parent[v])
        out.append(v)
    return out


@pytest.mark.parametrize("name", ["c1", "t64"])
def test_plan_is_a_cut(name):
    p = _problem(name)
    for n_ranks in (1, 2, 3, 4, 7, 8):
        _check_cut(p.rcb.parent, oshard.plan_problem(p, n_ranks), n_ranks)
    c = oshard.plan_problem(p, 1)
    assert list(c["rank_root"]) == [len(p.rcb.parent) - 1]


def test_plan_of_equal_domains_is_the_domains(c1):
    sh = oshard.plan_problem(c1, 8)
    assert list(sh["rank_root"]) == list(range(8))
    with pytest.raises(ValueError):
        oshard.plan_problem(c1, 9)


@pytest.mark.parametrize("name", ["c1", "t64"])
def test_library_plan_equals_oracle_plan(name):
    import paper_2002_05019_gb300 as dd
    p = _problem(name)
    for n_ranks in range(1, 17 if name == "t64" else 9):
        lib = dd.shard_plan_problem(p, n_ranks)
        ora = oshard.plan_problem(p, n_ranks)
        assert np.array_equal(lib["rank_root"], ora["rank_root"]), n_ranks
        assert np.array_equal(lib["front_rank"], ora["front_rank"]), n_ranks
    with pytest.raises(dd.DDError):
        dd.shard_plan_problem(p, 0)
