"""The paper's run-time table workloads (Sec. 4 "Benchmarks", Table 1) on the GPU vs the oracle.

Undirected G(n=2000, p=0.002) and Watts-Strogatz (n=10,000, k=10, p=0.007)
graphs, every undirected edge stored both ways, with the three edge-weight
models of the table: trivalency (p from {0.1, 0.01, 0.001}), uniform random on
[0, 1] and weighted cascade (1 / in-degree); 100 uniform seeds and 1,000
trials, as in the table.  Uniform [0, 1] drives the cascades to nearly the
whole graph: the dense-frontier regime.  Spreads, node counts, edge checks and
per-step counts must be identical, pushing and pulling, and LT with weighted-
cascade weights on the same graphs too.
"""
import numpy as np
import pytest

import oracle
import paper_2404_17059_gb300 as P
from paper_2404_17059_gb300 import inputs as I

pytestmark = pytest.mark.gpu
LC = 64
T = 1000


@pytest.fixture(scope="module", params=["gnp", "ws"])
def graph(request):
    if request.param == "gnp":
        return I.erdos_renyi_gnp(2000, 0.002, graph_seed=1)
    return I.watts_strogatz(10_000, 10, 0.007, graph_seed=1)


def assert_same(a, b):
    assert a.status == P.CND_OK and b.status == oracle.OK
    assert np.array_equal(a.spread, b.spread), np.nonzero(a.spread != b.spread)[0][:10]
    assert np.array_equal(a.node_count, b.node_count)
    assert a.edge_checks == b.edge_checks
    assert np.array_equal(a.level_counts, b.level_counts)


@pytest.mark.parametrize("ewm", ["TV", "UR", "WC"])
def test_ic_edge_weight_models(graph, ewm):
    g = graph
    p = {"TV": lambda: I.ic_trivalency(g, graph_seed=1), "UR": lambda: I.ic_uniform_random(g, 1.0, graph_seed=1),
         "WC": lambda: I.ic_weighted_cascade(g)}[ewm]()
    seeds = I.uniform_seeds(g.n, 100, 1)
    G = P.cnd_graph_create(g.n, g.row_ptr, g.col, p, None)
    b = oracle.simulate_threads("ic", g, seeds, T, 1, ic_prob=p, level_counts_len=LC)
    for direction in ("push", "pull"):
        a = P.cnd_ic_simulate_ex(G, seeds, T, 1, edge_checks=True, level_counts_len=LC, direction=direction)
        assert_same(a, b)
    if ewm == "UR":
        # the near-saturating regime: most trials reach most of the graph
        assert b.spread.mean() > 0.5 * g.n


def test_lt_weighted_cascade(graph):
    g = graph
    w = I.lt_weighted_cascade(g)
    seeds = I.uniform_seeds(g.n, 100, 1)
    G = P.cnd_graph_create(g.n, g.row_ptr, g.col, None, w)
    b = oracle.simulate_threads("lt", g, seeds, T, 1, lt_weight=w, level_counts_len=LC)
    for acc in (0, 1):
        assert_same(P.cnd_lt_simulate_ex(G, seeds, T, 1, edge_checks=True, level_counts_len=LC, lt_accumulate=acc), b)
