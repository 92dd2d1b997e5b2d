"""The README's usage example, on small inputs: every call it shows works as shown."""
import numpy as np
import pytest

import paper_2404_17059_gb300 as P
from paper_2404_17059_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def test_readme_usage():
    g = I.barabasi_albert(2_000, 5)
    G = P.cnd_graph_create(g.n, g.row_ptr, g.col, I.ic_weighted_cascade(g), I.lt_weighted_cascade(g))
    seeds = I.top_degree_seeds(g, 50)
    r = P.cnd_ic_simulate_ex(G, seeds, 1_000, rng_seed=1, edge_checks=True, graph=1)
    assert r.spread.shape == (1_000,) and r.node_count.shape == (g.n,)
    assert np.all(r.spread >= 50) and np.all(r.node_count[seeds] == 1_000) and r.edge_checks > 0
    lt = P.cnd_lt_simulate(G, seeds, 1_000, 1)
    assert np.all(lt.spread >= 50)
    celf = P.cnd_ic_im_celf(G, k=5, n_trials=256, rng_seed=1)
    assert len(set(celf.seeds.tolist())) == 5 and np.all(np.diff(celf.f) >= 0)
    sur = P.cnd_sur_create(G, I.surrogate_init(1))
    out = P.cnd_sur_train(sur, 512, n_trials=256)
    assert out["loss"].size == 32 and np.all(np.isfinite(out["loss"]))
    res, t = P.cnd_ic_im_screened(G, sur, 5, 256, 1, n_screen=8, n_exact=8, mode="onehop")
    assert len(set(res.seeds.tolist())) == 5 and res.evaluations == 40 and t["sim_ms"] > 0
