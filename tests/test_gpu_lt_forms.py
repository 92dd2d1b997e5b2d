"""LT in its two device forms vs the CPU oracle, bit-exact, through the C ABI.

Where every node's non-zero in-weights are equal (the weighted cascade, Sec. 4
"Benchmarks"), the engine counts active in-neighbours in bit-sliced counters
instead of summing 32-bit weights: k * w_v > theta <=> k > floor(theta / w_v).
Elsewhere, or with lt_accumulate=1, it keeps the per-trial sums.  Both must give
the oracle's per-trial spreads, node counts, edge checks and per-step counts.
"""
import numpy as np
import pytest

import oracle
import paper_2404_17059_gb300 as P
from paper_2404_17059_gb300 import inputs as I

pytestmark = pytest.mark.gpu
LC = 160


def sim(G, seeds, T, rng, **kw):
    kw.setdefault("edge_checks", True)
    kw.setdefault("level_counts_len", LC)
    return P.cnd_lt_simulate_ex(G, seeds, T, rng, stats=P.CND_STATS_COUNT, **kw)


def ref(g, w, seeds, T, rng, **kw):
    return oracle.simulate_threads("lt", g, seeds, T, rng, lt_weight=w, level_counts_len=LC, **kw)


def assert_same(a, b):
    assert a.status == (P.CND_ELIMIT if b.status == oracle.LIMIT else P.CND_OK)
    assert np.array_equal(a.spread, b.spread), np.nonzero(a.spread != b.spread)[0][:10]
    assert np.array_equal(a.node_count, b.node_count)
    assert a.edge_checks == b.edge_checks
    assert np.array_equal(a.level_counts, b.level_counts)


@pytest.fixture(scope="module")
def wc_graphs():
    out = []
    for g, seeds in ((I.erdos_renyi_m(1000, 10_000, graph_seed=1), I.uniform_seeds(1000, 10, 1)),
                     (I.barabasi_albert(20_000, 5, graph_seed=2), None),
                     (I.rmat(14, 16 << 14, graph_seed=3), None)):
        seeds = I.top_degree_seeds(g, 20) if seeds is None else seeds
        w = I.lt_weighted_cascade(g)
        out.append((g, w, P.cnd_graph_create(g.n, g.row_ptr, g.col, None, w), seeds))
    return out


@pytest.mark.parametrize("acc", [0, 1])
def test_both_forms_match_the_oracle(wc_graphs, acc):
    for g, w, G, seeds in wc_graphs:
        a = sim(G, seeds, 1000, 3, lt_accumulate=acc)
        assert a.stats["lt_counters"] == (0 if acc else 1)
        assert_same(a, ref(g, w, seeds, 1000, 3))


def test_unequal_weights_use_the_sums(wc_graphs):
    for g, _, _, seeds in wc_graphs[:2]:
        for total in (1.0, 0.6):
            w = I.lt_random(g, total=total, graph_seed=5)
            G = P.cnd_graph_create(g.n, g.row_ptr, g.col, None, w)
            a = sim(G, seeds, 700, 9)
            assert a.stats["lt_counters"] == 0
            assert_same(a, ref(g, w, seeds, 700, 9))


def test_counting_form_options(wc_graphs):
    """Passes of several widths, trial offsets, level caps, deferral and graph mode in the counting form."""
    g, w, G, seeds = wc_graphs[1]
    for kw, okw in (({"word_bits": 128}, {}), ({"word_bits": 64 * 7, "first_trial": 64 * 1001},
                                               {"first_trial": 64 * 1001}),
                    ({"max_levels": 3}, {"max_levels": 3}), ({"graph": 1}, {})):
        a = sim(G, seeds, 900, 11, **kw)
        assert a.stats["lt_counters"] == 1
        assert_same(a, ref(g, w, seeds, 900, 11, **okw))
    a = P.cnd_lt_simulate_ex(G, seeds, 900, 11, edge_checks=True, defer_bits=6)
    b = ref(g, w, seeds, 900, 11)
    assert np.array_equal(a.spread, b.spread) and np.array_equal(a.node_count, b.node_count)
    assert a.edge_checks == b.edge_checks


def test_counter_width_boundaries():
    """In-stars whose centre has k in-edges around the plane-count boundaries (2^L - 1, 2^L), with
    zero-weight extra in-edges (which leave the counting form usable) and random leaf seed sets of
    every size, so that the activation test k * w > theta is taken at every count."""
    rng = np.random.default_rng(17)
    for k in (1, 2, 3, 4, 7, 8, 15, 16, 31, 32, 255, 256, 1000):
        # node 0 is the centre; leaves 1..k point to it; node k+1 points to it with weight 0 and
        # to every leaf (so leaves have equal in-weights too)
        src = np.concatenate([np.arange(1, k + 1), [k + 1], np.full(k, k + 1)])
        dst = np.concatenate([np.zeros(k, np.int64), [0], np.arange(1, k + 1)])
        g = I.csr_from_edges(k + 2, src, dst, sort=False)
        w = I.lt_weighted_cascade(g).astype(np.uint64)
        zero = (g.src() == k + 1) & (g.col == 0)
        w[zero] = 0
        # the centre's in-weights: k leaves of floor((2^32-1)/k) (recomputed without the zero edge)
        w[(g.col == 0) & ~zero] = 0xFFFFFFFF // k
        w = w.astype(np.uint32)
        G = P.cnd_graph_create(g.n, g.row_ptr, g.col, None, w)
        for size in sorted({1, max(1, k // 3), max(1, k // 2), k - 1, k} - {0}):
            seeds = rng.choice(np.arange(1, k + 1), size=size, replace=False).astype(np.int32)
            a = sim(G, seeds, 640, 1000 + k)
            assert a.stats["lt_counters"] == 1
            assert_same(a, ref(g, w, seeds, 640, 1000 + k))


def test_counting_form_batches(wc_graphs):
    g, w, G, _ = wc_graphs[2]
    so, seeds, tr, keys = I.batch_items(g.n, 12, 1, 40, (64, 200, 1000), graph_seed=7)
    a = P.cnd_lt_simulate_batch(G, so, seeds, tr, keys, node_count=True, edge_checks=True)
    off = np.concatenate([[0], np.cumsum(tr)])
    checks = 0
    for i in range(len(tr)):
        b = ref(g, w, seeds[so[i]:so[i + 1]], int(tr[i]), int(keys[i]))
        assert np.array_equal(a.spread[off[i]:off[i + 1]], b.spread)
        assert np.array_equal(np.asarray(a.node_count).reshape(len(tr), g.n)[i], b.node_count)
        checks += b.edge_checks
    assert a.edge_checks == checks
