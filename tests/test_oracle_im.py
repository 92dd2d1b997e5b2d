"""Pins of the oracle's lazy-greedy (CELF) influence maximisation (Sec. 2 "Influence Maximization").

With common random numbers the IC objective F(X) = sum of spreads over fixed
trials is a coverage function of the trials' live-edge graphs, so it is
submodular and CELF must choose exactly what plain greedy chooses.  Plain
greedy is checked against exhaustive search (its (1 - 1/e) guarantee holds
for the exact F) and against closed forms on stars and paths.
"""
import itertools

import numpy as np
import pytest

import oracle
from oracle import im
from paper_2404_17059_gb300 import inputs as I


def _F(model, g, X, T, key, **kw):
    return int(oracle.simulate(model, g, np.asarray(X, dtype=np.int32), T, key, level_counts_len=0,
                               **kw).spread.astype(np.int64).sum())


@pytest.fixture(scope="module")
def er():
    return I.erdos_renyi_m(120, 480, graph_seed=5)


@pytest.mark.parametrize("batch", [1, 3, 64])
def test_ic_celf_equals_plain_greedy(er, batch):
    p = I.ic_uniform(er, 0.15)
    s1, f1, ev = im.celf("ic", er, 6, 96, 3, eval_batch=batch, ic_prob=p)
    s2, f2 = im.greedy("ic", er, 6, 96, 3, ic_prob=p)
    np.testing.assert_array_equal(s1, s2)
    np.testing.assert_array_equal(f1, f2)
    assert ev < 6 * er.n  # lazy evaluation saved work


def test_celf_values_are_the_objective(er):
    w = I.lt_weighted_cascade(er)
    seeds, f, _ = im.celf("lt", er, 4, 64, 9, eval_batch=2, lt_weight=w)
    for j in range(4):
        assert f[j] == _F("lt", er, seeds[:j + 1], 64, 9, lt_weight=w)
    assert len(set(seeds.tolist())) == 4


def test_greedy_against_exhaustive_search():
    g = I.erdos_renyi_m(14, 40, graph_seed=8)
    p = I.ic_uniform(g, 0.3)
    T = 128
    seeds, f = im.greedy("ic", g, 2, T, 5, ic_prob=p)
    best = max(_F("ic", g, list(X), T, 5, ic_prob=p) for X in itertools.combinations(range(g.n), 2))
    best1 = max(_F("ic", g, [v], T, 5, ic_prob=p) for v in range(g.n))
    assert f[0] == best1                              # the first greedy pick is exact
    assert best >= f[1] >= (1 - (1 - 1 / 2) ** 2) * best  # k=2 greedy bound 1-(1-1/k)^k


def test_out_star_closed_form():
    g = I.out_star(9)  # centre 0 -> leaves 1..9
    p = I.ic_uniform(g, 1.0)
    seeds, f, _ = im.celf("ic", g, 3, 64, 1, ic_prob=p)
    assert seeds[0] == 0 and f[0] == 64 * 10
    # every leaf is already active: the next picks gain nothing and ties go to the lowest id
    assert seeds.tolist() == [0, 1, 2] and f.tolist() == [640, 640, 640]


def test_path_closed_form():
    g = I.path_graph(6)  # 6 edges: 0 -> 1 -> ... -> 6
    p = I.ic_uniform(g, 1.0)
    seeds, f, _ = im.celf("ic", g, 2, 32, 1, ic_prob=p)
    assert seeds.tolist() == [0, 1] and f.tolist() == [7 * 32, 7 * 32]


def test_candidates_restrict_the_choice(er):
    p = I.ic_uniform(er, 0.15)
    cand = list(range(0, er.n, 7))
    seeds, _, _ = im.celf("ic", er, 3, 64, 2, candidates=cand, ic_prob=p)
    assert set(seeds.tolist()) <= set(cand)
    with pytest.raises(ValueError):
        im.celf("ic", er, len(cand) + 1, 8, 2, candidates=cand, ic_prob=p)


def test_lt_celf_first_pick_is_the_exhaustive_best(er):
    """Round 0 evaluates every candidate, so the first LT pick is argmax F({v}) (ties: lower id)
    even though the LT objective over fixed trials need not be submodular."""
    w = I.lt_weighted_cascade(er)
    seeds, f, _ = im.celf("lt", er, 2, 48, 4, lt_weight=w)
    single = np.array([_F("lt", er, [v], 48, 4, lt_weight=w) for v in range(er.n)])
    assert seeds[0] == int(np.argmax(single)) and f[0] == single.max()
    pair = np.array([_F("lt", er, [seeds[0], v], 48, 4, lt_weight=w) if v != seeds[0] else -1
                     for v in range(er.n)])
    assert f[1] <= pair.max()                          # the second pick's value is a real F(S + v)
    assert f[1] == _F("lt", er, seeds[:2], 48, 4, lt_weight=w)
