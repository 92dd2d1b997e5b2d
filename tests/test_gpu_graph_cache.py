"""Graph-mode calls reuse the executable graph of an earlier call of the same shape.

A graph-mode call (opts.graph = 1) runs as one CUDA graph launch.  Each host
thread keeps the executables of its recent call shapes and updates a matching
one in place with the new call's parameters (seeds, keys, trial offsets,
buffers) instead of instantiating a new one.  The results must stay exactly
the oracle's whatever was cached before: same shape with other seeds, keys and
trial offsets; other shapes in between; batches of other compositions.
"""
import numpy as np
import pytest

import oracle
import paper_2404_17059_gb300 as P
from paper_2404_17059_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _same(a, b):
    assert np.array_equal(a.spread, b.spread)
    assert np.array_equal(a.node_count, b.node_count)
    assert a.edge_checks == b.edge_checks


def test_repeated_calls_reuse_and_stay_exact():
    g = I.erdos_renyi_m(1000, 10_000, graph_seed=1)
    p, w = I.ic_uniform(g, 0.1), I.lt_weighted_cascade(g)
    G = P.cnd_graph_create(g.n, g.row_ptr, g.col, p, w)
    h = I.barabasi_albert(5000, 3, graph_seed=4)
    H = P.cnd_graph_create(h.n, h.row_ptr, h.col, I.ic_weighted_cascade(h), I.lt_weighted_cascade(h))
    reused = []
    for i, (seeds, rng, first) in enumerate([(I.uniform_seeds(g.n, 10, 1), 1, 0), (I.uniform_seeds(g.n, 4, 2), 77, 640),
                                             (I.uniform_seeds(g.n, 25, 3), 5, 64 * 999)]):
        for model in ("ic", "lt"):
            f = P.cnd_ic_simulate_ex if model == "ic" else P.cnd_lt_simulate_ex
            a = f(G, seeds, 1000, rng, first_trial=first, graph=1, edge_checks=True, stats=P.CND_STATS_COUNT)
            kw = {"ic_prob": p} if model == "ic" else {"lt_weight": w}
            _same(a, oracle.simulate_threads(model, g, seeds, 1000, rng, first_trial=first, level_counts_len=0, **kw))
            reused.append(a.stats["graph_reused"])
            # another graph (another shape) in between
            b = f(H, [0, 1, 2], 300, rng, graph=1, edge_checks=True)
            kw = {"ic_prob": I.ic_weighted_cascade(h)} if model == "ic" else {"lt_weight": I.lt_weighted_cascade(h)}
            _same(b, oracle.simulate_threads(model, h, [0, 1, 2], 300, rng, level_counts_len=0, **kw))
    # the second and third rounds find the executables of the first
    assert reused[:2] == [0, 0] and all(r == 1 for r in reused[2:]), reused


def test_batches_of_other_compositions():
    g = I.rmat(12, 16 << 12, graph_seed=3)
    p = I.ic_uniform_random(g, 0.1, graph_seed=3)
    G = P.cnd_graph_create(g.n, g.row_ptr, g.col, p, None)
    so, seeds, tr, keys = I.batch_items(g.n, 24, 1, 30, (64, 128, 640), graph_seed=5)
    for a0, a1 in ((0, 8), (8, 20), (3, 11), (0, 8)):
        s2 = so[a0:a1 + 1] - so[a0]
        r = P.cnd_ic_simulate_batch(G, s2, seeds[so[a0]:so[a1]], tr[a0:a1], keys[a0:a1], graph=1, node_count=True,
                                    edge_checks=True)
        off = np.concatenate([[0], np.cumsum(tr[a0:a1])])
        checks = 0
        for i in range(a1 - a0):
            b = oracle.simulate("ic", g, seeds[so[a0 + i]:so[a0 + i + 1]], int(tr[a0 + i]), int(keys[a0 + i]),
                                ic_prob=p, level_counts_len=0)
            assert np.array_equal(r.spread[off[i]:off[i + 1]], b.spread)
            assert np.array_equal(np.asarray(r.node_count).reshape(a1 - a0, g.n)[i], b.node_count)
            checks += b.edge_checks
        assert r.edge_checks == checks
