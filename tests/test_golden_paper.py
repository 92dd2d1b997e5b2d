"""The paper's printed activation-over-time curves against the oracle.

Fixture: tests/golden/fig_activation_over_time.txt (Sec. 4, figure "Mean number of nodes activated
over time": 10 seeds, 1,000 simulations, a NetworkX random regular graph).  The paper's CELF benchmark
graph is a random 7-regular graph with 5,000 nodes; with trivalency probabilities there, the oracle's
CELF seeds (k = 10, 1,000 common trials) give a curve within 3 % of the printed CELF curve at every
iteration, and 10 uniform seeds (on a regular graph every node ties for the highest degree) give the
printed "highest degree" curve within 3 %.  The tolerance covers Monte Carlo noise (1,000 trials) and
the different graph instance and random numbers; a wrong activation rule, a per-step instead of
cumulative count, seeds left out of the count or a wrong edge-probability model miss it by far more.
The printed "random sampling" curve is not reproduced: the paper does not say how those seeds were
drawn, and uniform draws match its "highest degree" curve instead (its step-0 value still pins that
seeds count).
"""
import os

import numpy as np
import pytest

import oracle
from oracle import im
from paper_2404_17059_gb300 import inputs as I

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def fig():
    rows = [ln.split() for ln in open(os.path.join(HERE, "golden", "fig_activation_over_time.txt"))
            if ln.strip() and not ln.startswith("#")]
    a = np.array(rows, dtype=np.float64)
    return {"iter": a[:, 0], "celf": a[:, 1], "random": a[:, 2], "degree": a[:, 3]}


@pytest.fixture(scope="module")
def rr7():
    g = I.random_regular(5000, 7, graph_seed=1)
    return g, I.ic_trivalency(g, graph_seed=1)


def _curve(g, p, seeds, T=1000, key=77):
    r = oracle.simulate_threads("ic", g, np.asarray(seeds, dtype=np.int32), T, key, ic_prob=p, level_counts_len=12)
    return np.cumsum(r.level_counts)[:8] / T


def test_printed_curves_start_at_the_seed_count(fig):
    for name in ("celf", "random", "degree"):
        c = fig[name]
        assert c[0] == 10.0                      # iteration 0 counts the 10 seeds
        assert np.all(np.diff(c) >= 0)           # cumulative counts
        assert c[-1] == c[-2]                    # the cascade has stopped


def test_celf_curve(fig, rr7):
    g, p = rr7
    seeds, _, _ = im.celf("ic", g, 10, 1000, 1, ic_prob=p)
    ours = _curve(g, p, seeds)
    assert ours[0] == 10.0
    np.testing.assert_allclose(ours[1:], fig["celf"][1:], rtol=0.03)


def test_highest_degree_curve_on_a_regular_graph(fig, rr7):
    g, p = rr7
    assert np.all(np.diff(g.row_ptr) == 7)
    ours = np.mean([_curve(g, p, I.uniform_seeds(g.n, 10, 100 + d)) for d in range(5)], axis=0)
    np.testing.assert_allclose(ours[1:], fig["degree"][1:], rtol=0.03)
