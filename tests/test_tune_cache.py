"""The autotuner's schedule cache on the host: the problem key
(dd_tune_key) and the cache file (dd_tune_cache_lookup / _store).  CPU only.

The key is a hash of the symbolic analysis's front tree with the number of
duals, the form and the pivoting mode, so it is pinned by what must and
must not change it: the same problem gives the same key in two calls and
from two copies of its input; another decomposition, another form or
pivoting mode gives another key; new matrix values with the same patterns
give the same key (a schedule depends on sizes, not values).
"""
import numpy as np
import pytest

import femgen
import paper_2002_05019_gb300 as dd


def test_key_is_a_function_of_the_front_tree_and_the_form(c1):
    k = dd.tune_key_problem(c1)
    assert k == dd.tune_key_problem(c1)
    assert k == dd.tune_key_problem(femgen.plain_c1())              # a fresh copy of the same problem
    assert k != dd.tune_key_problem(c1, precision="fp64")
    assert k != dd.tune_key_problem(c1, pivoting=1)
    assert k != dd.tune_key_problem(femgen.tiny(4, 3, jittered=True))
    subs = dd._problem_subs(c1)
    scaled = [dict(s, data=2.0 * np.asarray(s["data"])) for s in subs]   # values change, patterns do not
    assert dd.tune_key(scaled, c1.n_dual, tree_parent=c1.rcb.parent) == k


def test_cache_file_round_trip(tmp_path):
    path = str(tmp_path / "tune.jsonl")
    assert dd.tune_cache_lookup(path, "0123:GPU:152") is None          # no file yet
    dd.tune_cache_store(path, "0123:GPU:152", {"update_panels": 4, "ahead_fronts": 32, "reserve_sms": 16,
                                                "split_sms": 24, "factor_ms": 461.9})
    dd.tune_cache_store(path, "4567:GPU:152", {"update_panels": 2, "ahead_fronts": 0, "reserve_sms": 16})
    got = dd.tune_cache_lookup(path, "0123:GPU:152")
    assert (got["update_panels"], got["ahead_fronts"], got["reserve_sms"], got["split_sms"]) == (4, 32, 16, 24)
    assert abs(got["factor_ms"] - 461.9) < 1e-3 and got["configs_tried"] == 0
    assert dd.tune_cache_lookup(path, "0123:GPU:148") is None          # another GPU model
    # the last line of a key wins; malformed or out-of-range lines are skipped
    with open(path, "a") as fh:
        fh.write('{"key": "0123:GPU:152", "update_panels": 1, "ahead_fronts": 8, "reserve_sms": 8, '
                 '"split_sms": 0, "factor_ms": 500}\n')
        fh.write('{"key": "0123:GPU:152", "update_panels": 3, "ahead_fronts": 8, "reserve_sms": 8, '
                 '"split_sms": 0, "factor_ms": 1}\n')
        fh.write('{"key": "0123:GPU:152", "update_panels": 4\n')
        fh.write("not json at all\n")
    got = dd.tune_cache_lookup(path, "0123:GPU:152")
    assert (got["update_panels"], got["ahead_fronts"], got["reserve_sms"]) == (1, 8, 8)
    with pytest.raises(dd.DDError):
        dd.tune_cache_store(path, 'bad"key', {"update_panels": 4, "ahead_fronts": 0, "reserve_sms": 16})
    with pytest.raises(dd.DDError):
        dd.tune_cache_store(str(tmp_path / "no_such_dir" / "t.jsonl"), "k",
                            {"update_panels": 4, "ahead_fronts": 0, "reserve_sms": 16})
