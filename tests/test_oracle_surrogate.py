"""Pins of the surrogate network's fp64 oracle (forward, backward, screening score, Adam).

The gradient pins are central finite differences of the oracle's own forward
with the bf16 rounding switched off (the function is then smooth), so a
dropped term, a wrong sign, a transposed weight or a reversed edge direction
in the backward fails them.  The forward is pinned by closed forms and by the
receptive field of a 3-layer network on a path (information flows along
edge direction, three hops).
"""
import numpy as np
import pytest

import oracle.surrogate as S
from paper_2404_17059_gb300 import inputs as I


@pytest.fixture
def smooth(monkeypatch):
    monkeypatch.setattr(S, "bf16", lambda x: np.asarray(x, dtype=np.float64))


def _graph(n=40, m=160, seed=3):
    g = I.erdos_renyi_m(n, m, graph_seed=seed)
    rng = np.random.default_rng(seed)
    p = rng.uniform(0.05, 0.9, size=g.m).astype(np.float32)
    return g, S.Graph(g, p)


def _params(seed=1, scale=1.0):
    return I.surrogate_init(seed).astype(np.float64) * scale


def test_param_layout_matches_generator():
    assert S.N_PARAMS == I.SURROGATE_N_PARAMS == 18689
    names = [n for n, _ in S.param_shapes()]
    assert names == [n for n, _, _ in I.SURROGATE_SHAPES]


def test_bf16_rounding_against_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.normal(size=4000) * 10.0 ** rng.integers(-6, 6, size=4000),
                        [1 + 2 ** -8, 1 + 3 * 2 ** -8, -(1 + 2 ** -8), 0.0, 1.0, 2 ** -130]])
    x = x.astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(S.bf16(x), ref)
    assert S.bf16(1 + 2 ** -8) == 1.0 and S.bf16(1 + 3 * 2 ** -8) == 1 + 2 ** -6


def test_edge_q_is_the_ic_live_probability():
    p = np.array([0.0, 0.1, 0.5, 1.0, 2 ** -33], dtype=np.float32)
    q = S.edge_q(p)
    assert q[0] == 0 and q[2] == 0.5 and q[3] == 1.0 and q[4] == 0.0
    assert abs(q[1] - 0.1) < 1e-7


def test_zero_weights_closed_form():
    g, G = _graph()
    flat = np.zeros(S.N_PARAMS)
    flat[-1] = 0.7  # b_o
    seeds = [1, 5, 9]
    c = S.forward(flat, G, seeds)
    sig = 1 / (1 + np.exp(-0.7))
    want = np.full(g.n, sig)
    want[seeds] = 1.0
    np.testing.assert_allclose(c["yhat"], want, rtol=0, atol=1e-15)
    y = np.zeros(g.n)
    loss, grad, _ = S.loss_and_grad(flat, G, seeds, y)
    np.testing.assert_allclose(loss, ((g.n - 3) * sig ** 2 + 3) / g.n, rtol=1e-14)
    # only the bias of the head sees a gradient when every hidden activation is zero
    assert np.count_nonzero(grad[:-1]) == 0
    np.testing.assert_allclose(grad[-1], (2 / g.n) * (g.n - 3) * sig * sig * (1 - sig), rtol=1e-12)


def test_receptive_field_follows_edge_direction():
    g = I.path_graph(6)  # 0 -> 1 -> ... -> 6
    G = S.Graph(g, I.ic_uniform(g, 0.5))
    flat = _params(2)
    base = S.forward(flat, G, [])["o"]
    with0 = S.forward(flat, G, [0])["o"]
    changed = np.nonzero(np.abs(with0 - base) > 0)[0].tolist()
    assert 0 in changed and 4 not in changed and 5 not in changed and 6 not in changed
    with6 = S.forward(flat, G, [6])["o"]
    assert np.array_equal(with6[:6], base[:6])  # a sink influences nobody upstream


def test_loss_gradient_finite_differences(smooth):
    g, G = _graph()
    flat = _params(4, scale=2.0)
    rng = np.random.default_rng(7)
    y = rng.uniform(0, 1, size=g.n)
    seeds = [0, 3, 17, 22]
    _, grad, _ = S.loss_and_grad(flat, G, seeds, y)
    idx = np.concatenate([rng.choice(S.N_PARAMS - 65, 60, replace=False), np.arange(S.N_PARAMS - 65, S.N_PARAMS)])
    h = 1e-6
    for i in idx:
        e = np.zeros(S.N_PARAMS)
        e[i] = h
        fd = (S.loss_and_grad(flat + e, G, seeds, y)[0] - S.loss_and_grad(flat - e, G, seeds, y)[0]) / (2 * h)
        assert abs(fd - grad[i]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (i, fd, grad[i])


def test_every_parameter_block_gets_gradient():
    g, G = _graph()
    rng = np.random.default_rng(1)
    _, grad, _ = S.loss_and_grad(_params(5, 2.0), G, [1, 2, 3], rng.uniform(size=g.n))
    o = 0
    for name, shape in S.param_shapes():
        k = int(np.prod(shape))
        assert np.any(grad[o:o + k] != 0), name
        o += k


def test_screen_score_finite_differences(smooth):
    g, G = _graph(30, 120, seed=9)
    flat = _params(6, scale=2.0)
    seeds = [2, 11]
    score, _ = S.screen_scores(flat, G, seeds)
    s0 = S.seed_indicator(g.n, seeds)
    h = 1e-6
    for c in [0, 1, 5, 13, 29]:
        e = np.zeros(g.n)
        e[c] = h
        fp = S.forward(flat, G, s0 + e)["yhat"].sum()
        fm = S.forward(flat, G, s0 - e)["yhat"].sum()
        fd = (fp - fm) / (2 * h)
        assert abs(fd - score[c]) <= 1e-6 * max(1.0, abs(fd)), (c, fd, score[c])


def test_adam_first_step_is_signed_lr():
    rng = np.random.default_rng(2)
    w = rng.normal(size=50)
    g = rng.normal(size=50)
    w1, m, v = S.adam(w, g, np.zeros(50), np.zeros(50), 1, 0.01)
    # at t = 1 the bias corrections give m_hat = g and v_hat = g^2
    np.testing.assert_allclose(w1, w - 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.001 * g * g)


def test_onehop_score_closed_form():
    """Out-star centre 0 -> leaves 1..5 with q = 1/2: with a network predicting 0 everywhere off the seeds,
    the centre's score is 1 + 5/2 and a leaf's is 1; with the centre seeded, leaves still score 1, centre 0."""
    g = I.out_star(5)
    G = S.Graph(g, I.ic_uniform(g, 0.5))
    flat = np.zeros(S.N_PARAMS)
    flat[-1] = -80.0  # sigmoid(o) = e^-80: zero to double precision next to 1
    sc, _ = S.onehop_scores(flat, G, [])
    np.testing.assert_allclose(sc, [3.5, 1, 1, 1, 1, 1], rtol=1e-12)
    sc, _ = S.onehop_scores(flat, G, [0])
    np.testing.assert_allclose(sc, [0, 1, 1, 1, 1, 1], rtol=1e-12)
