"""Surrogate network on the GPU (tensor-core kernels through the C ABI) vs the fp64 oracle.

Both sides round to bf16 at the same points (weights, activations, aggregates
and the backward's dz); they differ only in fp32 vs fp64 accumulation order,
which can move a stored bf16 value by one unit in the last place (2^-8
relative) where the exact value sits near a rounding boundary.  The
tolerances are set from that: 5e-3 absolute on predicted frequencies, and 2 %
of a tensor's largest entry on gradients and screening scores (a transposed
operand, a dropped term or a reversed edge direction produces errors of the
order of the entries themselves).
"""
import numpy as np
import pytest

import oracle.surrogate as S
import paper_2404_17059_gb300 as P
from paper_2404_17059_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _graph(kind):
    if kind == "er":
        g = I.erdos_renyi_m(301, 2400, graph_seed=4)  # 301 rows: a ragged last 16-row tile
    else:  # R-MAT hubs: in-rows longer than one 256-edge work item
        g = I.rmat(12, 16 << 12, graph_seed=2)
    rng = np.random.default_rng(5)
    p = rng.uniform(0.02, 0.6, size=g.m).astype(np.float32)
    p[::97] = 1.0
    return g, p


@pytest.fixture(scope="module", params=["er", "rmat"])
def setup(request):
    g, p = _graph(request.param)
    G = P.cnd_graph_create(g.n, g.row_ptr, g.col, p, None)
    params = I.surrogate_init(3) * 3.0  # larger weights: more active units, larger gradients
    sur = P.cnd_sur_create(G, params)
    return g, S.Graph(g, p), G, sur, params.astype(np.float32)


def _seeds(g, k, seed):
    return I.uniform_seeds(g.n, k, seed)


def test_rmat_fixture_has_split_rows():
    g, _ = _graph("rmat")
    assert g.in_degree().max() > 256


def test_forward_matches_oracle(setup):
    g, OG, G, sur, params = setup
    for k, sd in [(0, 1), (1, 2), (10, 3), (60, 4)]:
        seeds = _seeds(g, k, sd)
        yh, tot = P.cnd_sur_forward(sur, seeds)
        ref = S.forward(params.astype(np.float64), OG, seeds)["yhat"]
        np.testing.assert_allclose(yh, ref, rtol=0, atol=5e-3)
        assert abs(tot - ref.sum()) <= 5e-3 * g.n
        if k:
            assert np.all(yh[seeds] == 1.0)


def test_duplicate_seeds_count_once(setup):
    g, OG, G, sur, params = setup
    a, _ = P.cnd_sur_forward(sur, [3, 7, 3, 7, 7])
    b, _ = P.cnd_sur_forward(sur, [7, 3])
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-3)  # split rows add with atomics: order may vary


def test_state_is_restored_between_calls(setup):
    g, OG, G, sur, params = setup
    a, _ = P.cnd_sur_forward(sur, [])
    P.cnd_sur_forward(sur, _seeds(g, 30, 9))
    P.cnd_sur_loss_grad(sur, _seeds(g, 5, 8), np.zeros(g.n))
    P.cnd_sur_scores(sur, _seeds(g, 5, 8))
    b, _ = P.cnd_sur_forward(sur, [])
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-3)


def _close(a, b, frac=0.02):
    scale = max(np.abs(b).max(), 1e-12)
    err = np.abs(a - b).max()
    assert err <= frac * scale + 1e-7, (err, scale)


def test_loss_and_gradient_match_oracle(setup):
    g, OG, G, sur, params = setup
    rng = np.random.default_rng(11)
    for k in (1, 12):
        seeds = _seeds(g, k, 20 + k)
        y = rng.uniform(0, 1, size=g.n).astype(np.float32)
        loss, grad = P.cnd_sur_loss_grad(sur, seeds, y)
        rl, rg, _ = S.loss_and_grad(params.astype(np.float64), OG, seeds, y.astype(np.float64))
        assert abs(loss - rl) <= 1e-3 * rl
        o = 0
        for name, shape in S.param_shapes():
            kk = int(np.prod(shape))
            _close(grad[o:o + kk], rg[o:o + kk])
            o += kk


def test_screen_scores_match_oracle(setup):
    g, OG, G, sur, params = setup
    seeds = _seeds(g, 7, 31)
    sc = P.cnd_sur_scores(sur, seeds)
    ref, _ = S.screen_scores(params.astype(np.float64), OG, seeds)
    _close(sc, ref)
    assert np.all(sc[seeds] == pytest.approx(ref[seeds], abs=0.02 * np.abs(ref).max() + 1e-6))


def test_adam_step_matches_oracle(setup):
    g, OG, G, sur, params = setup
    rng = np.random.default_rng(3)
    p0 = params.astype(np.float64)
    m = np.zeros_like(p0)
    v = np.zeros_like(p0)
    cur = p0
    for t in (1, 2, 3):
        gr = (rng.normal(size=p0.size) * 10.0 ** rng.integers(-6, 0, size=p0.size)).astype(np.float32)
        P.cnd_sur_adam(sur, gr, 1e-3)
        cur, m, v = S.adam(cur, gr.astype(np.float64), m, v, t, 1e-3)
    got = P.cnd_sur_get_params(sur).astype(np.float64)
    np.testing.assert_allclose(got, cur, rtol=0, atol=2e-6)
    P.cnd_sur_set_params(sur, params)  # restore for the other tests


def test_training_reduces_loss():
    g = I.erdos_renyi_m(800, 6400, graph_seed=6)
    p = I.ic_weighted_cascade(g)
    G = P.cnd_graph_create(g.n, g.row_ptr, g.col, p, None)
    sur = P.cnd_sur_create(G, I.surrogate_init(1))
    r = P.cnd_sur_train(sur, 2048, set_size=(1, 20), n_trials=256, batch_sets=16, sim_chunk=256, lr=3e-3)
    loss = r["loss"]
    assert loss.size == 128 and np.all(np.isfinite(loss))
    assert loss[-16:].mean() < 0.5 * loss[:4].mean()


def test_bit_reproducible():
    """Every reduction runs in a fixed order: two trainings from the same start on the same data end in the
    same bits, and forward passes, gradients and screening scores repeat bit for bit (R-MAT hubs: in-rows
    and out-rows split over several work items, many seeds sharing out-neighbours)."""
    g, p = _graph("rmat")
    G = P.cnd_graph_create(g.n, g.row_ptr, g.col, p, None)
    init = I.surrogate_init(3)
    runs = []
    for _ in range(2):
        sur = P.cnd_sur_create(G, init)
        r = P.cnd_sur_train(sur, 512, set_size=(1, 30), n_trials=128, batch_sets=16, lr=3e-3, hub_frac=0.5)
        runs.append((P.cnd_sur_get_params(sur), r["loss"], sur))
    assert np.array_equal(runs[0][0], runs[1][0]) and np.array_equal(runs[0][1], runs[1][1])
    sur = runs[0][2]
    seeds = I.top_degree_seeds(g, 40)
    y = np.random.default_rng(3).uniform(0, 1, size=g.n).astype(np.float32)
    a = [P.cnd_sur_forward(sur, seeds) for _ in range(2)]
    assert np.array_equal(a[0][0], a[1][0]) and a[0][1] == a[1][1]
    b = [P.cnd_sur_loss_grad(sur, seeds, y) for _ in range(2)]
    assert b[0][0] == b[1][0] and np.array_equal(b[0][1], b[1][1])
    c = [P.cnd_sur_scores(sur, seeds) for _ in range(2)]
    assert np.array_equal(c[0], c[1])


def test_onehop_scores_match_oracle(setup):
    g, OG, G, sur, params = setup
    seeds = _seeds(g, 9, 41)
    sc = P.cnd_sur_onehop(sur, seeds)
    ref, _ = S.onehop_scores(params.astype(np.float64), OG, seeds)
    np.testing.assert_allclose(sc, ref, rtol=1e-2, atol=1e-2)


def test_degenerate_graphs_match_oracle():
    """Edgeless graph, a single node, and every node a seed."""
    params = I.surrogate_init(5) * 2.0
    for n, src, dst in ((50, [], []), (1, [], []), (40, list(range(39)), list(range(1, 40)))):
        g = I.csr_from_edges(n, np.asarray(src, dtype=np.int64), np.asarray(dst, dtype=np.int64))
        p = np.full(g.m, 0.5, dtype=np.float32)
        G = P.cnd_graph_create(g.n, g.row_ptr, g.col, p, None)
        sur = P.cnd_sur_create(G, params)
        OG = S.Graph(g, p)
        for seeds in ([], [0], list(range(n))):
            yh, tot = P.cnd_sur_forward(sur, seeds)
            ref = S.forward(params.astype(np.float32).astype(np.float64), OG, seeds)["yhat"]
            np.testing.assert_allclose(yh, ref, rtol=0, atol=5e-3)
            if len(seeds) == n:
                assert np.all(yh == 1.0) and abs(tot - n) < 1e-9
            y = np.zeros(n, dtype=np.float32)
            loss, grad = P.cnd_sur_loss_grad(sur, seeds, y)
            rl, rg, _ = S.loss_and_grad(params.astype(np.float32).astype(np.float64), OG, seeds, y.astype(np.float64))
            assert abs(loss - rl) <= 1e-3 * max(rl, 1e-12) + 1e-12
            assert np.abs(grad - rg).max() <= 0.02 * max(np.abs(rg).max(), 1e-12) + 1e-7


def test_bad_arguments_are_rejected(setup):
    g, OG, G, sur, params = setup
    with pytest.raises(P.CndError):
        P.cnd_sur_forward(sur, [g.n])
    with pytest.raises(P.CndError):
        P.cnd_sur_forward(sur, [-1])
    bad = params.copy()
    bad[7] = np.nan
    with pytest.raises(P.CndError):
        P.cnd_sur_set_params(sur, bad)
    G2 = P.cnd_graph_create(g.n, g.row_ptr, g.col, None, I.lt_weighted_cascade(g))
    with pytest.raises(P.CndError):
        P.cnd_sur_create(G2, params)  # no IC probabilities
