"""Autotuner of the batched products: selection rules and the JSON cache on
the CPU; on the GPU, a tuned batch solves to the untuned batch's solution and
a second call is served from the cache."""
import os

import numpy as np
import pytest

from paper_2308_00637_gb300 import autotune as at


def test_bucket_of():
    assert [at.bucket_of(n) for n in (1, 2, 3, 64, 127, 128, 4096, 4097)] == [0, 1, 1, 6, 6, 7, 12, 12]


def test_choose_team_smallest_near_best():
    # 8 CTAs is within 10 % of the fastest (16): prefer it, the rest go to other QPs
    assert at.choose_team({1: 100.0, 2: 52.0, 4: 28.0, 8: 16.0, 16: 15.0, 32: 15.5}) == 8
    assert at.choose_team({1: 1.0, 2: 1.2}) == 1


def test_choose_colpass_threshold():
    # the column pass wins from bucket 9 (n = 512) upwards
    assert at.choose_colpass({7: (2.0, 1.0), 8: (1.1, 1.0), 9: (0.8, 1.0), 10: (0.5, 1.0)}) == 512
    # a loss above a win stops the run of wins
    assert at.choose_colpass({8: (0.9, 1.0), 9: (1.2, 1.0), 10: (0.5, 1.0)}) == 1024
    assert at.choose_colpass({8: (2.0, 1.0)}) == 512


def test_table_arrays_fill_from_nearest_bucket():
    table = {"buckets": {"6": {"team_cap": 1, "t_prod_us": 10.0},
                         "9": {"team_cap": 8, "t_prod_us": 200.0}}, "colpass_min_n": 512}
    caps, times = at.table_arrays(table)
    assert len(caps) == 10 and caps[6] == 1 and caps[9] == 8
    assert caps[0] == 1 and caps[8] == 8          # nearest tuned bucket (ties to the lower)
    assert times[6] == 10.0 and times[7] == 40.0  # borrowed times scale with n^2
    assert times[8] == pytest.approx(200.0 / 4)


def test_cache_round_trip(tmp_path):
    path = os.path.join(str(tmp_path), "sub", "tune.json")
    assert at.load_cache(path) == {}
    data = {at.cache_key("GB300", 2, 1, 1): {"buckets": {"7": {"team_cap": 2, "t_prod_us": 3.0}},
                                              "colpass_min_n": 512}}
    at.save_cache(path, data)
    assert at.load_cache(path) == data


@pytest.mark.gpu
def test_autotuned_batch_matches_default(tmp_path):
    import qpgen
    import __graft_entry__ as g
    g.build()
    import paper_2308_00637_gb300 as kq
    sizes = qpgen.batch_sizes(20, 32, 900, size_seed=13)
    qps = [qpgen.batch_qp(k, n) for k, n in enumerate(sizes)]
    cache = os.path.join(str(tmp_path), "tune.json")
    table = at.autotune(qps, precision=1, reps=3, cache=cache)
    assert not table["from_cache"]
    assert {int(k) for k in table["buckets"]} == {at.bucket_of(n) for n in sizes}
    for k, v in table["buckets"].items():
        assert v["team_cap"] >= 1 and v["t_prod_us"] > 0
    again = at.autotune(qps, precision=1, reps=3, cache=cache)
    assert again["from_cache"] and again["buckets"] == table["buckets"]
    objs = {}
    for tuned in (False, True):
        b = kq.qp_create_batch(qps)
        if tuned:
            at.apply_tuning(b, table)
        xs = [np.zeros(q.n) for q in qps]
        rc, status, st = kq.ipm_solve_batch(b, kq.default_ipm_opts(precision=1), xs)
        assert rc == kq.KQ_OK
        objs[tuned] = [q.objective(x) for q, x in zip(qps, xs)]
        kq.qp_batch_destroy(b)
    for f0, f1 in zip(objs[False], objs[True]):
        assert abs(f0 - f1) <= 1e-6 * (1 + abs(f0))
