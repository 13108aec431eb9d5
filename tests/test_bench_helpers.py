"""Host logic of bench.py (CPU): the subtree sample of the CPU baseline, the
traffic figure read from the committed ncu summary, and the whole-job value."""
import numpy as np

import bench
import femgen
import oracle


def test_pick_subtree_holds_the_requested_domains():
    p = femgen.build_problem("t64", 10, 6, split_range=(0.37, 0.63), eps="random")
    parent = np.asarray(p.rcb.parent)
    for want in (1, 2, 8, 16, 64):
        node = bench.pick_subtree(parent, p.n_sub, want)
        doms = [x for x in oracle.subtree_nodes(parent, node) if x < p.n_sub]
        assert len(doms) == want


def test_update_traffic_scales_by_flops_and_tracks_the_kernel_source():
    t, bpf = bench.update_traffic(1e9)
    if t is None:       # the kernel changed since the counters were taken: no figure
        assert bpf is None
    else:
        assert abs(t - 1e9 * bpf) < 1e-3 * t and 0.001 < bpf < 1.0


def test_job_value_is_the_whole_job_throughput():
    assert bench.job_value(100, 4, 2.0) == 200.0
