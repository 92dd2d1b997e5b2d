"""GPU engine vs CPU oracle at the full sizes of the two large workloads, on sampled outputs.

R-MAT scale 24 (edge factor 16: 263 M directed edges, n = 2^24; IC p = 0.01, LT weighted cascade,
the 100 highest-out-degree seeds) and the batched R-MAT scale 20 workload (2^24 samples; IC p ~
U[0, 0.1); the first 64 of the 4,096 seed sets) run on the GPU as bench.py times them: seeds in device
memory, one call per model of 1,024 trials over a contiguous trial range, the pass width the engine
picks; also 16,384 IC trials (three passes of 86 words at n = 2^24) and LT split into two passes.
The oracle cannot run every trial at this size, so:

- sampled trials are recomputed one by one (``first_trial = t``, one trial each) and their spreads
  must be identical -- trial ids at word, lane and pass boundaries and at the top of the 100,000;
- four trials per model are also run alone on the GPU (one-trial calls) and every output of each is
  compared with the oracle's: the activated set over all n nodes, the edge checks, the activations
  per step;
- the outputs no sample can check are tied by identities that hold at any size: the per-node counts
  sum to the summed spreads (both count the (trial, active node) pairs), edge checks equal the sum of
  out-degree times per-node count (the oracle's definition: out-edges of every active node in every
  trial), every seed is active in every trial, and every count lies in [0, trials].
"""
import concurrent.futures as cf
import os

import numpy as np
import pytest

import oracle
import paper_2404_17059_gb300 as P
from paper_2404_17059_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _oracle_trials(model, g, seeds, rng_seed, trial_ids, p=None, w=None):
    """Spread of each listed trial, one oracle call per trial, on the host's cores."""
    def one(t):
        r = oracle.simulate(model, g, seeds, 1, rng_seed, ic_prob=p, lt_weight=w, first_trial=int(t),
                            level_counts_len=0)
        assert r.status >= 0
        return int(r.spread[0])
    threads = max(1, min(len(os.sched_getaffinity(0)), len(trial_ids), 16))
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        return np.array(list(ex.map(one, trial_ids)), dtype=np.int32)


def _identities(g, seeds, spread, count, checks, T):
    outdeg = np.diff(g.row_ptr).astype(np.int64)
    assert int(count.astype(np.int64).sum()) == int(spread.astype(np.int64).sum())
    assert int((count.astype(np.int64) * outdeg).sum()) == checks
    assert np.all(count[np.unique(seeds)] == T)
    assert count.min() >= 0 and count.max() <= T
    assert spread.min() >= np.unique(seeds).size and spread.max() <= g.n


@pytest.fixture(scope="module")
def rmat24():
    g = I.rmat(24, 16 << 24, graph_seed=1)
    p = I.ic_uniform(g, 0.01)
    w = I.lt_weighted_cascade(g)
    seeds = I.top_degree_seeds(g, 100)
    G = P.cnd_graph_create(g.n, g.row_ptr, g.col, p, w)
    yield g, G, p, w, seeds
    G.close()


def test_rmat24_ic_sampled_trials(rmat24):
    """16,384 IC trials, the top of the 100,000 (trials 83,584 .. 99,967)."""
    g, G, p, _, seeds = rmat24
    T, first = 16_384, 83_584
    r = P.cnd_ic_simulate_ex(G, torch.as_tensor(seeds, device="cuda"), T, 1, first_trial=first,
                             edge_checks=True, stats=1)
    torch.cuda.synchronize()
    assert r.status == P.CND_OK
    assert r.stats["passes"] == 3 and r.stats["word_bits"] == 86 * 64
    spread, count = r.spread.cpu().numpy(), r.node_count.cpu().numpy()
    _identities(g, seeds, spread, count, r.edge_checks, T)
    rng = np.random.default_rng(24)
    local = np.unique(np.concatenate([[0, 1, 63, 64, 5503, 5504, 11007, 11008, 16383],
                                      rng.integers(0, T, 7)]))
    want = _oracle_trials("ic", g, seeds, 1, first + local, p=p)
    assert np.array_equal(spread[local], want), (local, spread[local], want)


@pytest.mark.parametrize("model", ["ic", "lt"])
def test_rmat24_bench_step_sampled_trials(rmat24, model):
    """One call of bench.py's default step: 1,024 trials, a contiguous range of trial ids (the range of
    step 8 of the rotation, trials 8,192 .. 9,215), device seeds, the engine's own pass width; LT in the
    counting form.  Sampled trials at word and lane boundaries and random ones."""
    g, G, p, w, seeds = rmat24
    T, first = 1024, 8 * 1024
    f = P.cnd_ic_simulate_ex if model == "ic" else P.cnd_lt_simulate_ex
    r = f(G, torch.as_tensor(seeds, device="cuda"), T, 1, first_trial=first, edge_checks=True,
          stats=P.CND_STATS_COUNT)
    torch.cuda.synchronize()
    assert r.status == P.CND_OK and r.stats["passes"] == 1
    if model == "lt":
        assert r.stats["lt_counters"] == 1
    spread, count = r.spread.cpu().numpy(), r.node_count.cpu().numpy()
    _identities(g, seeds, spread, count, r.edge_checks, T)
    rng = np.random.default_rng(26 if model == "ic" else 27)
    local = np.unique(np.concatenate([[0, 1, 63, 64, 511, 512, 1023], rng.integers(0, T, 9)]))
    want = _oracle_trials(model, g, seeds, 1, first + local, p=p, w=w)
    assert np.array_equal(spread[local], want), (local, spread[local], want)


@pytest.mark.parametrize("model", ["ic", "lt"])
def test_rmat24_single_trials_every_output(rmat24, model):
    """Four trials of the configuration, each run alone on the GPU (first_trial = t, one trial), against
    the oracle's run of the same trial: the activated set over all 16.7 M nodes (per-node counts of the
    one trial), the edge checks and the activations per step are identical."""
    g, G, p, w, seeds = rmat24
    ts, L = (0, 64, 50_048, 99_968), 1024  # a call's first trial is a multiple of 64
    f = P.cnd_ic_simulate_ex if model == "ic" else P.cnd_lt_simulate_ex
    got = []
    for t in ts:
        r = f(G, torch.as_tensor(seeds, device="cuda"), 1, 1, first_trial=t, edge_checks=True, level_counts_len=L)
        torch.cuda.synchronize()
        assert r.status == P.CND_OK
        got.append((r.node_count.cpu().numpy(), r.edge_checks, r.level_counts.cpu().numpy()))

    def one(t):
        return oracle.simulate(model, g, seeds, 1, 1, ic_prob=p, lt_weight=w, first_trial=int(t), level_counts_len=L)

    with cf.ThreadPoolExecutor(max_workers=len(ts)) as ex:
        want = list(ex.map(one, ts))
    for t, (count, checks, levels), o in zip(ts, got, want):
        assert o.status >= 0
        assert np.array_equal(count, o.node_count), t
        assert checks == o.edge_checks, (t, checks, o.edge_checks)
        assert np.array_equal(levels, o.level_counts), t
        assert levels[L - 1] == 0  # every cascade ended within the recorded steps


def test_rmat24_lt_two_passes(rmat24):
    """1,024 LT trials at the top of the 100,000 (98,944 .. 99,967) split into two passes of 8 words, so
    the counting form re-initialises its counters and seeds between passes at full size."""
    g, G, _, w, seeds = rmat24
    T, first = 1024, 98_944
    r = P.cnd_lt_simulate_ex(G, torch.as_tensor(seeds, device="cuda"), T, 1, first_trial=first,
                             edge_checks=True, word_bits=512, stats=P.CND_STATS_COUNT)
    torch.cuda.synchronize()
    assert r.status == P.CND_OK and r.stats["passes"] == 2 and r.stats["lt_counters"] == 1
    spread, count = r.spread.cpu().numpy(), r.node_count.cpu().numpy()
    _identities(g, seeds, spread, count, r.edge_checks, T)
    rng = np.random.default_rng(25)
    local = np.unique(np.concatenate([[0, 63, 511, 512, 575, 1023], rng.integers(0, T, 2)]))
    want = _oracle_trials("lt", g, seeds, 1, first + local, w=w)
    assert np.array_equal(spread[local], want), (local, spread[local], want)


def test_rmat20_batch_sampled_trials():
    """The batched step: the first 64 of the 4,096 seed sets in one call; two sampled trials of each
    of 8 items, and the identities per item."""
    g = I.rmat(20, 1 << 24, graph_seed=1)
    p = I.ic_uniform_random(g, 0.1, graph_seed=1)
    so, sd, tr, keys = I.batch_items(g.n, 4096, 1, 100, (256, 1024, 4096), graph_seed=1)
    k = 64
    so, sd, tr, keys = so[:k + 1], sd[:so[k]], tr[:k], keys[:k]
    G = P.cnd_graph_create(g.n, g.row_ptr, g.col, p, None)
    a = P.cnd_ic_simulate_batch(G, so, torch.as_tensor(sd, device="cuda"), tr, keys, edge_checks=True)
    b = P.cnd_ic_simulate_batch(G, so, torch.as_tensor(sd, device="cuda"), tr, keys, edge_checks=True,
                                node_count=True)
    torch.cuda.synchronize()
    G.close()
    spread = a.spread.cpu().numpy()
    assert np.array_equal(spread, b.spread.cpu().numpy()) and a.edge_checks == b.edge_checks
    counts = b.node_count.cpu().numpy().reshape(k, g.n)
    off = np.concatenate([[0], np.cumsum(tr.astype(np.int64))])
    outdeg = np.diff(g.row_ptr).astype(np.int64)
    checks = 0
    for i in range(k):
        s_i = sd[so[i]:so[i + 1]]
        sp_i = spread[off[i]:off[i + 1]]
        assert int(counts[i].astype(np.int64).sum()) == int(sp_i.astype(np.int64).sum())
        assert np.all(counts[i][np.unique(s_i)] == tr[i]) and counts[i].max() <= tr[i]
        checks += int((counts[i].astype(np.int64) * outdeg).sum())
    assert checks == a.edge_checks
    rng = np.random.default_rng(20)
    for i in rng.choice(k, 8, replace=False):
        ts = np.array([0, tr[i] - 1]) if i % 2 else rng.integers(0, tr[i], 2)
        want = _oracle_trials("ic", g, sd[so[i]:so[i + 1]], int(keys[i]), ts, p=p)
        got = spread[off[i] + ts]
        assert np.array_equal(got, want), (int(i), ts, got, want)
