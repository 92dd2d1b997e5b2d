"""Lazy-greedy (CELF) influence maximisation on the GPU batch engine vs the oracle's CELF, exactly.

The chosen seeds and every F(S_j) (sum of spreads over the common trials) must
be identical: the lazy rule is fixed (include/cnd.h) and each F is an exact
integer computed bit-exactly by the engine.
"""
import numpy as np
import pytest

import oracle
from oracle import im
import paper_2404_17059_gb300 as P
from paper_2404_17059_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def er0():
    g = I.erdos_renyi_m(1000, 10_000, graph_seed=1)
    p = I.ic_uniform(g, 0.1)
    w = I.lt_weighted_cascade(g)
    return g, P.cnd_graph_create(g.n, g.row_ptr, g.col, p, w), p, w


@pytest.mark.parametrize("batch", [1, 64])
def test_ic_celf_er(er0, batch):
    g, G, p, _ = er0
    r = P.cnd_ic_im_celf(G, 5, 256, 1, eval_batch=batch)
    s, f, ev = im.celf("ic", g, 5, 256, 1, eval_batch=batch, ic_prob=p)
    np.testing.assert_array_equal(r.seeds, s)
    np.testing.assert_array_equal(r.f, f)
    assert r.evaluations <= ev and r.edge_checks > 0


def test_lt_celf_er(er0):
    g, G, _, w = er0
    r = P.cnd_lt_im_celf(G, 4, 128, 5, eval_batch=8)
    s, f, _ = im.celf("lt", g, 4, 128, 5, eval_batch=8, lt_weight=w)
    np.testing.assert_array_equal(r.seeds, s)
    np.testing.assert_array_equal(r.f, f)


def test_celf_candidates_chunking_and_engine_options(er0):
    g, G, p, _ = er0
    cand = np.arange(3, g.n, 5, dtype=np.int32)[::-1].copy()
    r = P.cnd_ic_im_celf(G, 4, 200, 2**40 + 3, candidates=cand, eval_batch=3, max_items=7, first_trial=1024,
                         word_bits=128, chunk_edges=3)
    s, f, _ = im.celf("ic", g, 4, 200, 2**40 + 3, candidates=cand, eval_batch=3, first_trial=1024, ic_prob=p)
    np.testing.assert_array_equal(r.seeds, s)
    np.testing.assert_array_equal(r.f, f)


def test_celf_random_regular_wc():
    """The paper's CELF benchmark graph shape: random 7-regular, n=5,000 (35,000 edges), WC IC."""
    g = I.random_regular(5000, 7, graph_seed=1)
    p = I.ic_weighted_cascade(g)
    G = P.cnd_graph_create(g.n, g.row_ptr, g.col, p, None)
    r = P.cnd_ic_im_celf(G, 6, 128, 1, graph=1)
    s, f, _ = im.celf("ic", g, 6, 128, 1, ic_prob=p)
    np.testing.assert_array_equal(r.seeds, s)
    np.testing.assert_array_equal(r.f, f)


def test_celf_rejects_bad_arguments(er0):
    g, G, _, _ = er0
    with pytest.raises(P.CndError):
        P.cnd_ic_im_celf(G, 3, 64, 1, candidates=[1, 2])
    with pytest.raises(P.CndError):
        P.cnd_ic_im_celf(G, 1, 64, 1, candidates=[1, 1])
    with pytest.raises(P.CndError):
        P.cnd_ic_im_celf(G, 1, 0, 1)
    with pytest.raises(P.CndError):
        P.cnd_ic_im_celf(G, 1, 64, 1, candidates=[g.n])


def test_screened_greedy_without_screening_is_plain_greedy(er0):
    """With every candidate passed to the simulator the surrogate decides nothing: plain greedy."""
    g, G, p, _ = er0
    cand = np.arange(0, g.n, 4, dtype=np.int32)
    sur = P.cnd_sur_create(G, I.surrogate_init(2))
    r, tm = P.cnd_ic_im_screened(G, sur, 3, 256, 7, n_screen=cand.size, n_exact=cand.size, candidates=cand)
    s, f = im.greedy("ic", g, 3, 256, 7, candidates=cand, ic_prob=p)
    np.testing.assert_array_equal(r.seeds, s)
    np.testing.assert_array_equal(r.f, f)
    assert tm["sim_ms"] > 0 and tm["sur_ms"] > 0


def test_screened_greedy_values_are_exact(er0):
    g, G, p, _ = er0
    sur = P.cnd_sur_create(G, I.surrogate_init(3))
    r, _ = P.cnd_ic_im_screened(G, sur, 5, 128, 3, n_screen=32, n_exact=3)
    assert len(set(r.seeds.tolist())) == 5 and r.evaluations == 5 * 3
    for j in range(5):
        ref = oracle.simulate("ic", g, r.seeds[:j + 1], 128, 3, ic_prob=p, level_counts_len=0)
        assert r.f[j] == int(ref.spread.astype(np.int64).sum())


def test_screened_greedy_degree_mode_needs_no_network(er0):
    g, G, p, _ = er0
    r, tm = P.cnd_ic_im_screened(G, None, 3, 128, 5, n_screen=16, n_exact=2, mode="degree")
    deg = np.diff(g.row_ptr)
    assert r.seeds[0] in np.argsort(-deg, kind="stable")[:2]
    assert r.evaluations == 3 * 2 and tm["sur_ms"] >= 0


def test_celf_takes_every_candidate_and_isolated_nodes(er0):
    g, G, p, _ = er0
    cand = np.array([5, 17, 42, 99, 600], dtype=np.int32)
    r = P.cnd_ic_im_celf(G, len(cand), 64, 9, candidates=cand)
    s, f, _ = im.celf("ic", g, len(cand), 64, 9, candidates=cand, ic_prob=p)
    np.testing.assert_array_equal(r.seeds, s)
    np.testing.assert_array_equal(r.f, f)
    assert sorted(r.seeds.tolist()) == sorted(cand.tolist())
    # isolated nodes: every candidate spreads to itself only; ties go to the lowest id
    h = I.csr_from_edges(6, np.zeros(0, dtype=np.int64), np.zeros(0, dtype=np.int64))
    H = P.cnd_graph_create(h.n, h.row_ptr, h.col, np.zeros(0, dtype=np.float32), None)
    r = P.cnd_ic_im_celf(H, 3, 32, 1)
    assert r.seeds.tolist() == [0, 1, 2] and r.f.tolist() == [32, 64, 96]
