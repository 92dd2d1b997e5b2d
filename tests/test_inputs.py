"""Synthetic workload generators: the structural properties the workloads rely on."""
import numpy as np

from paper_2404_17059_gb300 import inputs as I


def _simple(g):
    src = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    assert not np.any(src == g.col)
    k = src.astype(np.int64) * g.n + g.col
    assert np.unique(k).size == k.size
    return src


def test_random_regular_is_simple_regular_and_symmetric():
    for n, d, seed in [(5000, 7, 1), (50, 3, 2), (11, 4, 3)]:
        g = I.random_regular(n, d, graph_seed=seed)
        assert g.m == n * d
        assert np.all(np.diff(g.row_ptr) == d) and np.all(g.in_degree() == d)
        src = _simple(g)
        fwd = set(zip(src.tolist(), g.col.tolist()))
        assert all((v, u) in fwd for u, v in fwd)
    a = I.random_regular(200, 5, graph_seed=9)
    b = I.random_regular(200, 5, graph_seed=9)
    assert np.array_equal(a.col, b.col)


def test_erdos_renyi_and_ba_shapes():
    g = I.erdos_renyi_m(1000, 10_000, graph_seed=1)
    assert g.m == 10_000
    _simple(g)
    b = I.barabasi_albert(2000, 5, graph_seed=1)
    assert b.m == 2 * (2000 - 5) * 5
    _simple(b)
