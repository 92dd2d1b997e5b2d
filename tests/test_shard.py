"""Trial-sharded multi-process mode: world-size-2 gloo runs equal the single-process result.

Trials are independent functions of (rng_seed, trial), so the ranks' spreads
concatenated in rank order and their summed counts must equal one run over all
trials exactly.  The CPU tests drive the sharding and exchange logic with the
oracle as each rank's simulator; the GPU test runs libcnd on each rank.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
from paper_2404_17059_gb300 import inputs as I
from paper_2404_17059_gb300.shard import trial_shard

import _shard_worker as W


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_trial_shard_partitions():
    for T in [0, 1, 63, 64, 65, 1000, 10000, 12345]:
        for world in [1, 2, 3, 4, 8]:
            ranges = [trial_shard(T, r, world) for r in range(world)]
            pos = 0
            for first, cnt in ranges:
                assert cnt >= 0
                if cnt:
                    assert first == pos and first % 64 == 0
                pos += cnt
            assert pos == T
            sizes = [c for _, c in ranges]
            assert max(sizes) - min(sizes) <= 64
    with pytest.raises(ValueError):
        trial_shard(10, 2, 2)


def _run_world(tmp_path, backend, case, world=2):
    port = _free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=W.run, args=(r, world, port, backend, str(tmp_path), case)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    return [np.load(os.path.join(tmp_path, f"rank{r}.npz"), allow_pickle=True) for r in range(world)]


def _run_world2(tmp_path, backend, case):
    return _run_world(tmp_path, backend, case, 2)


def _single(case):
    g = I.erdos_renyi_m(400, 3000, graph_seed=3)
    seeds = I.uniform_seeds(g.n, 5, 4)
    kw = {"ic_prob": I.ic_uniform(g, 0.12)} if case["model"] == "ic" else {"lt_weight": I.lt_weighted_cascade(g)}
    return oracle.simulate(case["model"], g, seeds, case["n_trials"], case["rng_seed"], level_counts_len=32, **kw)


@pytest.mark.parametrize("case", [{"model": "ic", "n_trials": 1000, "rng_seed": 7},
                                  {"model": "lt", "n_trials": 130, "rng_seed": 2**40 + 5}])
def test_world2_gloo_matches_single_process(tmp_path, case):
    outs = _run_world2(tmp_path, "oracle", case)
    ref = _single(case)
    assert outs[0]["first"] == 0 and outs[1]["first"] == outs[0]["count"]
    assert int(outs[0]["count"]) + int(outs[1]["count"]) == case["n_trials"]
    for o in outs:  # every rank holds the full exchanged result
        np.testing.assert_array_equal(o["spread"], ref.spread)
        np.testing.assert_array_equal(o["node_count"], ref.node_count)
        assert int(o["edge_checks"]) == ref.edge_checks
        np.testing.assert_array_equal(o["level_counts"], ref.level_counts[:32])


def test_world3_uneven_ranges(tmp_path):
    """Three ranks, a trial count that leaves the last rank a short range."""
    case = {"model": "ic", "n_trials": 200, "rng_seed": 3}
    outs = _run_world(tmp_path, "oracle", case, 3)
    ref = _single(case)
    assert [int(o["count"]) for o in outs] == [64, 64, 72]
    for o in outs:
        np.testing.assert_array_equal(o["spread"], ref.spread)
        np.testing.assert_array_equal(o["node_count"], ref.node_count)
        assert int(o["edge_checks"]) == ref.edge_checks


def test_trial_shard_properties():
    hypothesis = pytest.importorskip("hypothesis")
    st = hypothesis.strategies

    @hypothesis.given(st.integers(0, 10**7), st.integers(1, 64))
    @hypothesis.settings(max_examples=200, deadline=None)
    def check(T, world):
        ranges = [trial_shard(T, r, world) for r in range(world)]
        assert sum(c for _, c in ranges) == T
        pos = 0
        for first, cnt in ranges:
            if cnt:
                assert first == pos and first % 64 == 0
            pos += cnt
        counts = [c for _, c in ranges]
        assert max(counts) - min(counts) <= 64

    check()


@pytest.mark.gpu
def test_world2_gpu_ranks_match_oracle(tmp_path):
    case = {"model": "ic", "n_trials": 1000, "rng_seed": 11}
    outs = _run_world2(tmp_path, "gpu", case)
    ref = _single(case)
    for o in outs:
        np.testing.assert_array_equal(o["spread"], ref.spread)
        np.testing.assert_array_equal(o["node_count"], ref.node_count)
        assert int(o["edge_checks"]) == ref.edge_checks
