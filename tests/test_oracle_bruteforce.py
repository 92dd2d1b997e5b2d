"""Oracle expectations against exhaustive enumeration on tiny graphs.

IC: the process equals reachability from S in a random live-edge graph in
which edge e is live independently with probability q_e = thr_e / 2^32, so
the expected spread is a sum over all 2^m live-edge subsets (Kempe et al.).

LT: with thresholds uniform and activation probability linear in the active
in-weight (P = W / 2^32 exactly, in fixed point), the process equals
reachability in a live-edge graph where every node keeps at most one in-edge,
edge e with probability w_e / 2^32 and none with the rest (Kempe et al.'s LT
equivalence); enumeration covers all prod_v (indeg_v + 1) choices.

Monte Carlo means of the oracle must land within 5 sigma of the exact value,
for the spread and for every node's activation probability.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_2404_17059_gb300 import inputs as I

T = 100_000
TWO32 = float(1 << 32)


def reach(n, edges, seeds):
    adj = [[] for _ in range(n)]
    for (u, v) in edges:
        adj[u].append(v)
    seen = set(seeds)
    stack = list(seen)
    while stack:
        u = stack.pop()
        for v in adj[u]:
            if v not in seen:
                seen.add(v)
                stack.append(v)
    return seen


def exact_ic(g, thr, seeds):
    src = g.src()
    m = g.m
    q = [float(t) / TWO32 if t != 0xFFFFFFFF else 1.0 for t in thr]
    node_p = np.zeros(g.n)
    for mask in range(1 << m):
        pr = 1.0
        live = []
        for e in range(m):
            if mask >> e & 1:
                pr *= q[e]
                live.append((int(src[e]), int(g.col[e])))
            else:
                pr *= 1.0 - q[e]
        if pr == 0.0:
            continue
        for v in reach(g.n, live, seeds):
            node_p[v] += pr
    return node_p


def exact_lt(g, w, seeds):
    src = g.src()
    in_edges = [[] for _ in range(g.n)]
    for e in range(g.m):
        in_edges[int(g.col[e])].append(e)
    options = []
    for v in range(g.n):
        opts = [(None, 1.0 - sum(float(w[e]) for e in in_edges[v]) / TWO32)]
        opts += [(e, float(w[e]) / TWO32) for e in in_edges[v]]
        options.append(opts)
    node_p = np.zeros(g.n)
    for choice in itertools.product(*options):
        pr = 1.0
        live = []
        for (e, pe) in choice:
            pr *= pe
            if e is not None:
                live.append((int(src[e]), int(g.col[e])))
        if pr == 0.0:
            continue
        for v in reach(g.n, live, seeds):
            node_p[v] += pr
    return node_p


def small_graph(seed, n, m):
    rng = np.random.default_rng(seed)
    pairs = [(u, v) for u in range(n) for v in range(n) if u != v]
    idx = rng.choice(len(pairs), size=m, replace=False)
    e = np.array([pairs[i] for i in idx])
    return I.csr_from_edges(n, e[:, 0], e[:, 1])


def check(result, node_p):
    # spread
    s = result.spread.astype(np.float64)
    se = max(s.std(ddof=1) / np.sqrt(s.size), 1e-12)
    assert abs(s.mean() - node_p.sum()) <= 5 * se, (s.mean(), node_p.sum(), se)
    # every node
    for v, P in enumerate(node_p):
        P = min(max(P, 0.0), 1.0)
        got = result.node_count[v] / T
        sev = np.sqrt(P * (1 - P) / T)
        assert abs(got - P) <= 5 * sev + 1e-9, (v, got, P)


@pytest.mark.parametrize("case", range(5))
@pytest.mark.parametrize("mode", ["bfs", "sweep"])
def test_ic_bruteforce(case, mode):
    n, m = [(5, 8), (6, 10), (6, 12), (7, 11), (4, 9)][case]
    g = small_graph(100 + case, n, m)
    rng = np.random.default_rng(200 + case)
    p = rng.uniform(0.05, 0.95, size=m).astype(np.float32)
    if case == 4:
        p[0] = 1.0
        p[1] = 0.0
    seeds = [0] if case % 2 == 0 else [0, 2, 2]
    thr = oracle.ic_threshold(p)
    node_p = exact_ic(g, thr, sorted(set(seeds)))
    r = oracle.simulate("ic", g, seeds, T, 1000 + case, ic_prob=p, mode=mode)
    assert r.status == oracle.OK
    check(r, node_p)


@pytest.mark.parametrize("case", range(4))
@pytest.mark.parametrize("mode", ["bfs", "sweep"])
def test_lt_bruteforce(case, mode):
    n, m = [(5, 8), (6, 10), (6, 9), (5, 12)][case]
    g = small_graph(300 + case, n, m)
    rng = np.random.default_rng(400 + case)
    # random in-weights scaled so that each node's total lies in [0.3, 1]
    raw = rng.uniform(0.1, 1.0, size=m)
    tot = np.bincount(g.col, weights=raw, minlength=n)
    scale = rng.uniform(0.3, 1.0, size=n)
    w = np.floor(raw / tot[g.col] * scale[g.col] * 0xFFFFFFFF).astype(np.uint64)
    assert np.all(np.bincount(g.col, weights=w, minlength=n) <= 0xFFFFFFFF)
    w = w.astype(np.uint32)
    seeds = [1] if case % 2 == 0 else [1, 3]
    node_p = exact_lt(g, w, seeds)
    r = oracle.simulate("lt", g, seeds, T, 2000 + case, lt_weight=w, mode=mode)
    assert r.status == oracle.OK
    check(r, node_p)
