"""Exact per-trial properties of the oracle (common random numbers).

* Both traversal modes give the same activation step for every node of every trial.
* p = 0 gives the distinct seeds; p = 1 gives breadth-first reachability and
  distances (networkx, an independent library routine).
* Monotone in the seed set and in the probabilities / weights; IC coverage is
  submodular per trial.
* Observation 1 (Sec. 3): every active non-seed node at step L has an
  in-neighbour active at step L-1; for LT, the active in-weight at L-1
  exceeds the node's threshold while the weight at L-2 does not.
* Edge checks, level counts, node counts and spreads agree with the
  activation sets; trial ranges compose; bad input is rejected.
"""
import numpy as np
import pytest

import oracle
from paper_2404_17059_gb300 import inputs as I


@pytest.fixture(scope="module")
def er():
    return I.erdos_renyi_m(300, 1500, graph_seed=5)


@pytest.fixture(scope="module")
def ba():
    return I.barabasi_albert(400, 3, graph_seed=2)


def _ic(g, seeds, p, T=64, **kw):
    return oracle.simulate("ic", g, seeds, T, 7, ic_prob=p, want_sets=True, **kw)


def _lt(g, seeds, w, T=64, **kw):
    return oracle.simulate("lt", g, seeds, T, 7, lt_weight=w, want_sets=True, **kw)


@pytest.mark.parametrize("gname", ["er", "ba"])
def test_bfs_equals_sweep(request, gname):
    g = request.getfixturevalue(gname)
    seeds = I.uniform_seeds(g.n, 5, 3)
    for p in (0.05, 0.2):
        a = _ic(g, seeds, I.ic_uniform(g, p), mode="bfs")
        b = _ic(g, seeds, I.ic_uniform(g, p), mode="sweep")
        assert np.array_equal(a.level, b.level)
    a = _ic(g, seeds, I.ic_weighted_cascade(g), mode="bfs")
    b = _ic(g, seeds, I.ic_weighted_cascade(g), mode="sweep")
    assert np.array_equal(a.level, b.level)
    w = I.lt_weighted_cascade(g)
    a = _lt(g, seeds, w, mode="bfs")
    b = _lt(g, seeds, w, mode="sweep")
    assert np.array_equal(a.level, b.level)


def test_p_zero_and_duplicates(er):
    seeds = [3, 3, 7, 11, 7]
    r = _ic(er, seeds, I.ic_uniform(er, 0.0))
    assert np.all(r.spread == 3)
    assert np.all(r.active[:, [3, 7, 11]] == 1)
    r = oracle.simulate("ic", er, [], 10, 1, ic_prob=I.ic_uniform(er, 0.5))
    assert np.all(r.spread == 0) and r.edge_checks == 0


def test_p_one_is_bfs(er):
    nx = pytest.importorskip("networkx")
    G = nx.DiGraph()
    G.add_nodes_from(range(er.n))
    G.add_edges_from(zip(er.src().tolist(), er.col.tolist()))
    seeds = [0, 17, 99]
    dist = nx.multi_source_dijkstra_path_length(G, set(seeds))
    r = _ic(er, seeds, I.ic_uniform(er, 1.0), T=4)
    want = np.full(er.n, -1)
    for v, d in dist.items():
        want[v] = d
    for t in range(4):
        assert np.array_equal(r.level[t], want)


def test_monotone_in_seeds(er, ba):
    for g in (er, ba):
        S = I.uniform_seeds(g.n, 3, 1)
        Tset = np.concatenate([S, I.uniform_seeds(g.n, 6, 2)])
        p = I.ic_uniform(g, 0.15)
        a, b = _ic(g, S, p), _ic(g, Tset, p)
        assert np.all(a.active <= b.active)
        w = I.lt_weighted_cascade(g)
        a, b = _lt(g, S, w), _lt(g, Tset, w)
        assert np.all(a.active <= b.active)


def test_monotone_in_probability(er):
    rng = np.random.default_rng(1)
    p1 = (rng.random(er.m) * 0.2).astype(np.float32)
    p2 = np.minimum(p1 + (rng.random(er.m) * 0.1).astype(np.float32), 1).astype(np.float32)
    seeds = [1, 2]
    a, b = _ic(er, seeds, p1), _ic(er, seeds, p2)
    assert np.all(a.active <= b.active)
    w1 = I.lt_weighted_cascade(er)
    w2 = w1.copy()
    w1 = (w1.astype(np.uint64) * 3 // 4).astype(np.uint32)
    a, b = _lt(er, seeds, w1), _lt(er, seeds, w2)
    assert np.all(a.active <= b.active)


def test_ic_submodular_per_trial(er):
    p = I.ic_uniform(er, 0.12)
    S = [5]
    Tset = [5, 40, 77]
    for v in (120, 3, 250):
        rS, rSv = _ic(er, S, p), _ic(er, S + [v], p)
        rT, rTv = _ic(er, Tset, p), _ic(er, Tset + [v], p)
        assert np.all(rSv.spread - rS.spread >= rTv.spread - rT.spread)


def test_observation1_ic(ba):
    seeds = [0, 1]
    r = _ic(ba, seeds, I.ic_weighted_cascade(ba))
    src = ba.src()
    for t in range(r.level.shape[0]):
        lv = r.level[t]
        for v in np.nonzero(lv > 0)[0]:
            preds = src[ba.col == v]
            assert np.any(lv[preds] == lv[v] - 1)


def test_lt_threshold_rule(ba):
    w = I.lt_weighted_cascade(ba)
    seeds = [0, 1, 2]
    T = 16
    r = _lt(ba, seeds, w, T=T)
    src = ba.src()
    for t in range(T):
        lv = r.level[t]
        for v in range(ba.n):
            if lv[v] == 0:
                continue
            ins = np.nonzero(ba.col == v)[0]
            theta = oracle.lt_theta(7, t, v)
            final_in = sum(int(w[e]) for e in ins if lv[src[e]] >= 0)
            if lv[v] < 0:
                assert final_in <= theta  # never crossed
                continue
            L = lv[v]
            before = sum(int(w[e]) for e in ins if 0 <= lv[src[e]] <= L - 1)
            earlier = sum(int(w[e]) for e in ins if 0 <= lv[src[e]] <= L - 2)
            assert before > theta >= earlier


def test_counts_checks_levels(ba):
    p = I.ic_weighted_cascade(ba)
    r = oracle.simulate("ic", ba, [0, 5, 9], 50, 3, ic_prob=p, want_sets=True, level_counts_len=200)
    deg = ba.out_degree()
    assert np.array_equal(r.spread, r.active.sum(axis=1))
    assert np.array_equal(r.node_count, r.active.sum(axis=0))
    assert r.edge_checks == int((r.active.astype(np.int64) * deg[None, :]).sum())
    lv = r.level[r.level >= 0]
    assert np.array_equal(r.level_counts[: lv.max() + 1], np.bincount(lv))
    assert r.level_counts.sum() == r.spread.sum()


def test_trial_ranges_compose(er):
    p = I.ic_uniform(er, 0.1)
    seeds = [0, 9]
    full = oracle.simulate("ic", er, seeds, 200, 11, ic_prob=p)
    part = oracle.simulate("ic", er, seeds, 70, 11, ic_prob=p, first_trial=64)
    assert np.array_equal(part.spread, full.spread[64:134])
    thr = oracle.simulate_threads("ic", er, seeds, 200, 11, ic_prob=p, threads=3)
    assert np.array_equal(thr.spread, full.spread)
    assert np.array_equal(thr.node_count, full.node_count)
    assert thr.edge_checks == full.edge_checks
    assert np.array_equal(thr.level_counts, full.level_counts)
    w = I.lt_weighted_cascade(er)
    full = oracle.simulate("lt", er, seeds, 200, 11, lt_weight=w)
    thr = oracle.simulate_threads("lt", er, seeds, 200, 11, lt_weight=w, threads=4)
    assert np.array_equal(thr.spread, full.spread)


def test_level_cap():
    g = I.path_graph(6)
    p = I.ic_uniform(g, 1.0)
    r = oracle.simulate("ic", g, [0], 3, 1, ic_prob=p, max_levels=2, want_sets=True)
    assert r.status == oracle.LIMIT
    assert np.all(r.spread == 3) and r.level.max() == 2
    r = oracle.simulate("ic", g, [0], 3, 1, ic_prob=p, max_levels=6)
    assert r.status == oracle.LIMIT  # node 6 sits at level 6
    r = oracle.simulate("ic", g, [0], 3, 1, ic_prob=p, max_levels=7)
    assert r.status == oracle.OK and np.all(r.spread == 7)
    for mode in ("bfs", "sweep"):
        r = oracle.simulate("lt", g, [0], 3, 1, lt_weight=np.full(g.m, 0xFFFFFFFF, np.uint32),
                            max_levels=3, mode=mode, want_sets=True)
        assert r.level.max() <= 3


def test_rejects_bad_input(er):
    p = I.ic_uniform(er, 0.1)
    for bad in (np.nan, -0.1, 1.5):
        q = p.copy()
        q[17] = bad
        assert oracle.simulate("ic", er, [0], 2, 1, ic_prob=q).status == oracle.EINVAL
    assert oracle.simulate("ic", er, [er.n], 2, 1, ic_prob=p).status == oracle.EINVAL
    assert oracle.simulate("ic", er, [-1], 2, 1, ic_prob=p).status == oracle.EINVAL
    w = np.full(er.m, 0xFFFFFFFF, dtype=np.uint32)
    assert oracle.simulate("lt", er, [0], 2, 1, lt_weight=w).status == oracle.EOVERFLOW
    bad_g = I.Graph(n=er.n, row_ptr=er.row_ptr.copy(), col=er.col.copy())
    bad_g.col[3] = er.n
    assert oracle.simulate("ic", bad_g, [0], 2, 1, ic_prob=p).status == oracle.EINVAL
