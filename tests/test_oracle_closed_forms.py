"""Oracle expectations against closed forms (Monte Carlo within 5 sigma).

Each case is a graph whose expected spread is known exactly in terms of the
effective live probability q = thr / 2^32 (IC) or the fixed-point weight
w / 2^32 (LT).  Both traversal modes of the oracle are checked.
"""
import numpy as np
import pytest

import oracle
from paper_2404_17059_gb300 import inputs as I

T = 200_000
TWO32 = float(1 << 32)


def q_of(p):
    return float(oracle.ic_threshold([p])[0]) / TWO32 if p < 1 else 1.0


def within(samples, expected, k=5.0):
    samples = np.asarray(samples, dtype=np.float64)
    se = samples.std(ddof=1) / np.sqrt(samples.size)
    se = max(se, 1e-12)
    assert abs(samples.mean() - expected) <= k * se, (samples.mean(), expected, se)


@pytest.mark.parametrize("mode", ["bfs", "sweep"])
@pytest.mark.parametrize("p,L", [(0.5, 6), (0.3, 4), (0.9, 10)])
def test_ic_path(mode, p, L):
    g = I.path_graph(L)
    r = oracle.simulate("ic", g, [0], T, 1, ic_prob=I.ic_uniform(g, p), mode=mode)
    q = q_of(p)
    within(r.spread, sum(q ** i for i in range(L + 1)))
    # node i is active with probability q^i
    for i in range(L + 1):
        P = q ** i
        se = np.sqrt(P * (1 - P) / T) if 0 < P < 1 else 0
        assert abs(r.node_count[i] / T - P) <= 5 * se + 1e-12


@pytest.mark.parametrize("mode", ["bfs", "sweep"])
def test_ic_out_star(mode):
    k, p = 25, 0.3
    g = I.out_star(k)
    r = oracle.simulate("ic", g, [0], T, 3, ic_prob=I.ic_uniform(g, p), mode=mode)
    within(r.spread, 1 + k * q_of(p))
    assert r.edge_checks == T * k  # only the centre has out-edges


@pytest.mark.parametrize("mode", ["bfs", "sweep"])
def test_ic_in_star(mode):
    k = 8
    g = I.in_star(k)
    p = np.array([0.05, 0.1, 0.2, 0.3, 0.4, 0.5, 0.6, 0.7], dtype=np.float32)
    prob = np.zeros(g.m, dtype=np.float32)
    src = g.src()
    prob[:] = p[src - 1]
    seeds = [1, 3, 4, 7]
    r = oracle.simulate("ic", g, seeds, T, 5, ic_prob=prob, mode=mode)
    P = 1.0 - np.prod([1.0 - q_of(p[s - 1]) for s in seeds])
    se = np.sqrt(P * (1 - P) / T)
    assert abs(r.node_count[0] / T - P) <= 5 * se
    assert np.all(r.node_count[[1, 3, 4, 7]] == T)
    assert np.all(r.node_count[[2, 5, 6, 8]] == 0)


@pytest.mark.parametrize("mode", ["bfs", "sweep"])
def test_ic_tree(mode):
    # complete binary tree of depth 4 with per-edge probabilities; E = sum over nodes of the
    # product of q along the root path
    depth = 4
    n = 2 ** (depth + 1) - 1
    src = np.array([(v - 1) // 2 for v in range(1, n)])
    dst = np.arange(1, n)
    g = I.csr_from_edges(n, src, dst)
    rng = np.random.default_rng(5)
    pv = rng.uniform(0.2, 0.95, size=n).astype(np.float32)  # probability of the edge into v
    prob = pv[g.col]
    r = oracle.simulate("ic", g, [0], T, 9, ic_prob=prob, mode=mode)
    reach = np.zeros(n)
    reach[0] = 1.0
    for v in range(1, n):
        reach[v] = reach[(v - 1) // 2] * q_of(pv[v])
    within(r.spread, reach.sum())


@pytest.mark.parametrize("mode", ["bfs", "sweep"])
@pytest.mark.parametrize("wfrac,L", [(0.5, 6), (0.8, 8)])
def test_lt_path(mode, wfrac, L):
    g = I.path_graph(L)
    W = int(wfrac * 0xFFFFFFFF)
    w = np.full(g.m, W, dtype=np.uint32)
    r = oracle.simulate("lt", g, [0], T, 2, lt_weight=w, mode=mode)
    x = W / TWO32
    within(r.spread, sum(x ** i for i in range(L + 1)))


@pytest.mark.parametrize("mode", ["bfs", "sweep"])
def test_lt_in_star(mode):
    k = 6
    g = I.in_star(k)
    wl = np.array([0.05, 0.1, 0.15, 0.2, 0.2, 0.25]) * 0xFFFFFFFF
    wl = wl.astype(np.uint64)
    assert wl.sum() <= 0xFFFFFFFF
    w = wl[g.src() - 1].astype(np.uint32)
    seeds = [2, 3, 6]
    r = oracle.simulate("lt", g, seeds, T, 4, lt_weight=w, mode=mode)
    P = float(sum(int(wl[s - 1]) for s in seeds)) / TWO32
    se = np.sqrt(P * (1 - P) / T)
    assert abs(r.node_count[0] / T - P) <= 5 * se


@pytest.mark.parametrize("mode", ["bfs", "sweep"])
def test_lt_out_star(mode):
    k = 10
    g = I.out_star(k)
    wl = (np.linspace(0.1, 1.0, k) * 0xFFFFFFFF).astype(np.uint64).astype(np.uint32)
    w = wl[g.col - 1]
    r = oracle.simulate("lt", g, [0], T, 6, lt_weight=w, mode=mode)
    within(r.spread, 1 + float(wl.astype(np.float64).sum()) / TWO32)
