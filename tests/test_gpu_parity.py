"""GPU engine vs CPU oracle, bit-exact, through the C ABI (libcnd).

Per-trial spreads, per-node activation counts, edge checks and per-step
activation counts must be identical: a trial is a pure function of
(graph, seeds, rng_seed, trial id), so any grouping of trials into words or
passes, any chunking of rows and any traversal order gives the same result.
"""
import numpy as np
import pytest

import oracle
import paper_2404_17059_gb300 as P
from paper_2404_17059_gb300 import inputs as I

pytestmark = pytest.mark.gpu
LC = 128


def sim(model, G, seeds, T, rng, **kw):
    f = P.cnd_ic_simulate_ex if model == "ic" else P.cnd_lt_simulate_ex
    kw.setdefault("edge_checks", True)
    kw.setdefault("level_counts_len", LC)
    return f(G, seeds, T, rng, **kw)


def ref(model, g, seeds, T, rng, p=None, w=None, **kw):
    kw.setdefault("level_counts_len", LC)
    if model == "ic":
        return oracle.simulate_threads("ic", g, seeds, T, rng, ic_prob=p, **kw)
    return oracle.simulate_threads("lt", g, seeds, T, rng, lt_weight=w, **kw)


def assert_same(a, b, counts=True):
    assert a.status == (P.CND_ELIMIT if b.status == oracle.LIMIT else P.CND_OK)
    assert np.array_equal(a.spread, b.spread), np.nonzero(a.spread != b.spread)[0][:10]
    if counts:
        assert np.array_equal(a.node_count, b.node_count)
        assert a.edge_checks == b.edge_checks
        assert np.array_equal(a.level_counts, b.level_counts)


def both(model, g, G, seeds, T, rng, p=None, w=None, oracle_kw=None, **kw):
    a = sim(model, G, seeds, T, rng, **kw)
    okw = dict(oracle_kw or {})
    if "first_trial" in kw:
        okw["first_trial"] = kw["first_trial"]
    if "max_levels" in kw:
        okw["max_levels"] = kw["max_levels"]
    b = ref(model, g, seeds, T, rng, p=p, w=w, **okw)
    assert_same(a, b)
    return a, b


# ------------------------------------------------------------------ fixtures
@pytest.fixture(scope="module")
def er0():
    """Directed ER n=1000, m=10,000, p=0.1, 10 uniform seeds (the small IC workload)."""
    g = I.erdos_renyi_m(1000, 10_000, graph_seed=1)
    p = I.ic_uniform(g, 0.1)
    w = I.lt_weighted_cascade(g)
    G = P.cnd_graph_create(g.n, g.row_ptr, g.col, p, w)
    return g, G, p, w, I.uniform_seeds(g.n, 10, 1)


@pytest.fixture(scope="module")
def ba():
    """BA n=100,000, 5 attachments, symmetrised; WC IC (fp32) and WC LT (fixed point); 50 top-degree seeds."""
    g = I.barabasi_albert(100_000, 5, graph_seed=1)
    p = I.ic_weighted_cascade(g)
    w = I.lt_weighted_cascade(g)
    G = P.cnd_graph_create(g.n, g.row_ptr, g.col, p, w)
    return g, G, p, w, I.top_degree_seeds(g, 50)


@pytest.fixture(scope="module")
def rmat14():
    """R-MAT scale 14 (hubs with thousands of out-edges: exercises row chunking)."""
    g = I.rmat(14, 16 << 14, graph_seed=3)
    p = I.ic_uniform_random(g, 0.1, graph_seed=3)
    w = I.lt_weighted_cascade(g)
    G = P.cnd_graph_create(g.n, g.row_ptr, g.col, p, w)
    return g, G, p, w, I.top_degree_seeds(g, 20)


# ------------------------------------------------------------------ tests
def test_device_philox_matches_oracle():
    rng = np.random.default_rng(5)
    ctr = rng.integers(0, 1 << 32, size=(4096, 4), dtype=np.uint64).astype(np.uint32)
    for s in (0, 1, 0xDEADBEEFCAFEF00D, (1 << 64) - 1):
        assert np.array_equal(P.cnd_philox4x32_10(s, ctr), oracle.philox(ctr, s))


@pytest.mark.parametrize("model", ["ic", "lt"])
def test_er_small_workload(er0, model):
    g, G, p, w, seeds = er0
    both(model, g, G, seeds, 1000, 1, p=p, w=w)


@pytest.mark.parametrize("model", ["ic", "lt"])
def test_ba_workload_all_trials(ba, model):
    g, G, p, w, seeds = ba
    both(model, g, G, seeds, 10_000, 1, p=p, w=w)


@pytest.mark.parametrize("model", ["ic", "lt"])
def test_rmat_hubs(rmat14, model):
    g, G, p, w, seeds = rmat14
    both(model, g, G, seeds, 640, 9, p=p, w=w)
    both(model, g, G, seeds, 130, 9, p=p, w=w, chunk_edges=3)


@pytest.mark.parametrize("model", ["ic", "lt"])
def test_word_widths_and_chunks(er0, model):
    g, G, p, w, seeds = er0
    b = ref(model, g, seeds, 1000, 4, p=p, w=w)
    for wb in (64, 128, 192, 256, 576, 1024, 16384):
        assert_same(sim(model, G, seeds, 1000, 4, word_bits=wb), b)
    for ch in (1, 5, 32, 4096):
        assert_same(sim(model, G, seeds, 1000, 4, chunk_edges=ch), b)


@pytest.mark.parametrize("model", ["ic", "lt"])
def test_wide_passes(er0, model):
    """Passes wider than 256 words: dirty masks of more than 4 words (up to 32) and push items
    with more frontier words than a warp stages in shared memory."""
    g, G, p, w, seeds = er0
    b = ref(model, g, seeds, 40_000, 12, p=p, w=w)  # 625 words
    for wb in (0, 64 * 625, 64 * 300, 64 * 2048):
        assert_same(sim(model, G, seeds, 40_000, 12, word_bits=wb), b)
    assert_same(sim(model, G, seeds, 40_000, 12, chunk_edges=2), b)


@pytest.mark.parametrize("model", ["ic", "lt"])
def test_wide_batch_passes(rmat14, model):
    """Many small items in one pass of up to 2048 words."""
    g, G, p, w, _ = rmat14
    seed_off, seeds, trials, keys = I.batch_items(g.n, 150, 1, 30, (64, 128, 1000, 640), graph_seed=8)
    f = P.cnd_ic_simulate_batch if model == "ic" else P.cnd_lt_simulate_batch
    want_sp, want_nc, want_ck = _batch_ref(model, g, p, w, seed_off, seeds, trials, keys)
    for wb in (0, 64 * 1500):
        a = f(G, seed_off, seeds, trials, keys, node_count=True, edge_checks=True, word_bits=wb, stats=1)
        assert np.array_equal(a.spread, want_sp)
        assert np.array_equal(a.node_count, want_nc)
        assert a.edge_checks == want_ck
        assert a.stats["word_bits"] > 64 * 256


@pytest.mark.parametrize("model", ["ic", "lt"])
def test_ragged_trial_counts(ba, model):
    g, G, p, w, seeds = ba
    for T in (1, 3, 63, 64, 65, 130, 257):
        both(model, g, G, seeds, T, 2, p=p, w=w)


@pytest.mark.parametrize("model", ["ic", "lt"])
def test_first_trial_offsets(er0, model):
    g, G, p, w, seeds = er0
    for ft in (64, 6400, (1 << 34) - 128, (1 << 36) + 64):
        both(model, g, G, seeds, 200, 3, p=p, w=w, first_trial=ft)


@pytest.mark.parametrize("model", ["ic", "lt"])
def test_rng_seeds(er0, model):
    g, G, p, w, seeds = er0
    for s in (0, 0xFFFFFFFF, 1 << 32, (1 << 63) + 5):
        both(model, g, G, seeds, 100, s, p=p, w=w)


def test_edge_cases_ic_lt():
    # isolated nodes, zero-out-degree seeds, a self-loop, parallel edges, p = 0 and p = 1 edges
    src = np.array([0, 0, 0, 1, 2, 2, 3, 5, 5, 6, 7, 7])
    dst = np.array([1, 1, 2, 3, 2, 4, 5, 6, 7, 8, 8, 0])
    g = I.csr_from_edges(10, src, dst, sort=False)
    p = np.array([0.5, 0.5, 1.0, 0.0, 0.7, 1.0, 0.9, 0.3, 0.6, 1.0, 0.2, 0.4], dtype=np.float32)
    w = I.lt_weighted_cascade(g)
    G = P.cnd_graph_create(g.n, g.row_ptr, g.col, p, w)
    for seeds in ([0], [9], [0, 0, 3, 3], [4, 8, 9], list(range(10))):
        for model in ("ic", "lt"):
            both(model, g, G, seeds, 300, 5, p=p, w=w)
    for model in ("ic", "lt"):
        a = sim(model, G, [], 100, 1)
        assert np.all(a.spread == 0) and np.all(a.node_count == 0) and a.edge_checks == 0
        a = sim(model, G, [0], 0, 1)
        assert a.spread.size == 0 and np.all(a.node_count == 0)


def test_no_edges_graph():
    g = I.Graph(n=5, row_ptr=np.zeros(6, np.int32), col=np.zeros(0, np.int32))
    G = P.cnd_graph_create(g.n, g.row_ptr, g.col, np.zeros(0, np.float32), np.zeros(0, np.uint32))
    for model in ("ic", "lt"):
        a = sim(model, G, [1, 3], 77, 1)
        assert np.all(a.spread == 2) and a.edge_checks == 0
        assert np.array_equal(a.node_count, np.array([0, 77, 0, 77, 0]))


def test_p_one_is_reachability(er0):
    g, _, _, _, seeds = er0
    p1 = I.ic_uniform(g, 1.0)
    G = P.cnd_graph_create(g.n, g.row_ptr, g.col, p1, None)
    both("ic", g, G, seeds, 70, 1, p=p1)
    p0 = I.ic_uniform(g, 0.0)
    G0 = P.cnd_graph_create(g.n, g.row_ptr, g.col, p0, None)
    a = sim("ic", G0, seeds, 70, 1)
    assert np.all(a.spread == len(set(seeds.tolist())))


@pytest.mark.parametrize("model", ["ic", "lt"])
def test_level_cap(ba, model):
    g, G, p, w, seeds = ba
    for cap in (1, 3, 10):
        a, b = both(model, g, G, seeds, 200, 7, p=p, w=w, max_levels=cap)
        assert a.status == P.CND_ELIMIT


@pytest.mark.parametrize("model", ["ic", "lt"])
def test_device_pointers_match_host(ba, model):
    torch = pytest.importorskip("torch")
    g, G, p, w, seeds = ba
    host = sim(model, G, seeds, 1000, 11)
    d = sim(model, G, torch.as_tensor(seeds, device="cuda"), 1000, 11)
    torch.cuda.synchronize()
    assert np.array_equal(d.spread.cpu().numpy(), host.spread)
    assert np.array_equal(d.node_count.cpu().numpy(), host.node_count)
    assert d.edge_checks == host.edge_checks
    assert np.array_equal(d.level_counts.cpu().numpy(), host.level_counts)


def test_bad_device_seed_rejected(er0):
    torch = pytest.importorskip("torch")
    g, G, p, w, seeds = er0
    s = torch.tensor([1, 2, g.n + 5], dtype=torch.int32, device="cuda")
    with pytest.raises(P.CndError) as ei:
        sim("ic", G, s, 64, 1)
    assert ei.value.status == P.CND_EINVAL
    # the context is still usable
    both("ic", g, G, seeds, 64, 1, p=p, w=w)


def test_plain_entry_points(er0):
    g, G, p, w, seeds = er0
    a = P.cnd_ic_simulate(G, seeds, 500, 1)
    b = ref("ic", g, seeds, 500, 1, p=p)
    assert np.array_equal(a.spread, b.spread) and np.array_equal(a.node_count, b.node_count)
    a = P.cnd_lt_simulate(G, seeds, 500, 1)
    b = ref("lt", g, seeds, 500, 1, w=w)
    assert np.array_equal(a.spread, b.spread) and np.array_equal(a.node_count, b.node_count)


@pytest.mark.parametrize("model", ["ic", "lt"])
def test_deferred_expansion_same_results(ba, rmat14, model):
    """Words that wait for more bits before expansion (defer_bits) change no result."""
    for fx in (ba, rmat14):
        g, G, p, w, seeds = fx
        b = ref(model, g, seeds, 640, 3, p=p, w=w, level_counts_len=0)
        for tau, ds in ((1, 0), (2, 0), (5, 0), (17, 0), (64, 0), (64, 1), (64, 3), (8, 2), (33, 255)):
            a = sim(model, G, seeds, 640, 3, defer_bits=tau, defer_steps=ds, level_counts_len=0)
            assert a.status == P.CND_OK
            assert np.array_equal(a.spread, b.spread)
            assert np.array_equal(a.node_count, b.node_count)
            assert a.edge_checks == b.edge_checks


def test_deferred_expansion_refuses_levels(er0):
    g, G, p, w, seeds = er0
    with pytest.raises(P.CndError) as ei:
        sim("ic", G, seeds, 64, 1, defer_bits=4)  # level counts requested by default here
    assert ei.value.status == P.CND_EINVAL
    with pytest.raises(P.CndError):
        sim("ic", G, seeds, 64, 1, defer_bits=4, level_counts_len=0, max_levels=3)


def _batch_ref(model, g, p, w, seed_off, seeds, trials, keys, first_trial=0, want_counts=False):
    spreads, counts, checks = [], [], 0
    for i in range(len(trials)):
        S = seeds[seed_off[i]:seed_off[i + 1]]
        r = ref(model, g, S, int(trials[i]), int(keys[i]), p=p, w=w, first_trial=first_trial, level_counts_len=0)
        spreads.append(r.spread)
        counts.append(r.node_count)
        checks += r.edge_checks
    return np.concatenate(spreads) if spreads else np.zeros(0, np.int32), np.stack(counts), checks


@pytest.mark.parametrize("model", ["ic", "lt"])
def test_batch_matches_items_one_by_one(rmat14, model):
    """Items of uneven seed-set size and trial count, packed into shared passes."""
    g, G, p, w, _ = rmat14
    seed_off, seeds, trials, keys = I.batch_items(g.n, 23, 1, 40, (64, 100, 256, 7, 1000), graph_seed=4)
    trials[3] = 0  # an empty item
    f = P.cnd_ic_simulate_batch if model == "ic" else P.cnd_lt_simulate_batch
    want_sp, want_nc, want_ck = _batch_ref(model, g, p, w, seed_off, seeds, trials, keys)
    for wb in (0, 128, 640):
        a = f(G, seed_off, seeds, trials, keys, node_count=True, edge_checks=True, word_bits=wb)
        assert np.array_equal(a.spread, want_sp)
        assert np.array_equal(a.node_count, want_nc)
        assert a.edge_checks == want_ck


def test_batch_device_pointers_and_offsets(ba):
    torch = pytest.importorskip("torch")
    g, G, p, w, _ = ba
    seed_off, seeds, trials, keys = I.batch_items(g.n, 9, 1, 100, (256, 1024, 64), graph_seed=6)
    want_sp, _, want_ck = _batch_ref("ic", g, p, w, seed_off, seeds, trials, keys, first_trial=128)
    a = P.cnd_ic_simulate_batch(G, seed_off, torch.as_tensor(seeds, device="cuda"), trials, keys,
                                edge_checks=True, first_trial=128)
    torch.cuda.synchronize()
    assert np.array_equal(a.spread.cpu().numpy(), want_sp)
    assert a.edge_checks == want_ck


def test_batch_single_item_equals_plain_call(er0):
    g, G, p, w, seeds = er0
    a = P.cnd_lt_simulate_batch(G, [0, len(seeds)], seeds, [1000], [4], node_count=True, edge_checks=True,
                                level_counts_len=LC)
    b = sim("lt", G, seeds, 1000, 4)
    assert np.array_equal(a.spread, b.spread) and np.array_equal(a.node_count[0], b.node_count)
    assert a.edge_checks == b.edge_checks and np.array_equal(a.level_counts, b.level_counts)


def test_pull_direction_same_results(er0, ba, rmat14):
    """IC steps expanded by pulling over in-edges give the same trials, counts and steps."""
    for fx in (er0, ba, rmat14):
        g, G, p, w, seeds = fx
        b = ref("ic", g, seeds, 320, 6, p=p)
        for kw in ({"direction": "pull"}, {"direction": "auto", "pull_permille": 1},
                   {"direction": "auto", "pull_permille": 200}, {"direction": "pull", "word_bits": 64}):
            a = sim("ic", G, seeds, 320, 6, stats=2, **kw)
            assert_same(a, b)
            if kw.get("direction") == "pull":
                assert a.stats["pull_steps"] > 0
        # LT has no pull step: the option leaves it pushing
        bl = ref("lt", g, seeds, 128, 6, w=w)
        assert_same(sim("lt", G, seeds, 128, 6, direction="pull"), bl)


def test_pull_direction_batch_and_edge_cases(rmat14):
    g, G, p, w, _ = rmat14
    seed_off, seeds, trials, keys = I.batch_items(g.n, 9, 1, 30, (64, 200, 500), graph_seed=8)
    want_sp, want_nc, want_ck = _batch_ref("ic", g, p, w, seed_off, seeds, trials, keys)
    a = P.cnd_ic_simulate_batch(G, seed_off, seeds, trials, keys, node_count=True, edge_checks=True,
                                direction="pull")
    assert np.array_equal(a.spread, want_sp) and np.array_equal(a.node_count, want_nc) and a.edge_checks == want_ck
    src = np.array([0, 0, 0, 1, 2, 2, 3, 5, 5, 6, 7, 7])
    dst = np.array([1, 1, 2, 3, 2, 4, 5, 6, 7, 8, 8, 0])
    g2 = I.csr_from_edges(10, src, dst, sort=False)
    p2 = np.array([0.5, 0.5, 1.0, 0.0, 0.7, 1.0, 0.9, 0.3, 0.6, 1.0, 0.2, 0.4], dtype=np.float32)
    G2 = P.cnd_graph_create(g2.n, g2.row_ptr, g2.col, p2, None)
    for seeds2 in ([0], [9], [0, 0, 3, 3], list(range(10))):
        assert_same(sim("ic", G2, seeds2, 300, 5, direction="pull"), ref("ic", g2, seeds2, 300, 5, p=p2))


@pytest.mark.parametrize("model", ["ic", "lt"])
def test_graph_mode_same_results(ba, rmat14, model):
    """One CUDA-graph launch per call (device-side step loop) gives the host-loop results."""
    for fx in (ba, rmat14):
        g, G, p, w, seeds = fx
        b = ref(model, g, seeds, 700, 12, p=p, w=w)
        assert_same(sim(model, G, seeds, 700, 12, graph=1), b)
        assert_same(sim(model, G, seeds, 700, 12, graph=1, word_bits=192), b)  # several passes
        a = sim(model, G, seeds, 700, 12, graph=1, stats=2)
        assert a.stats["levels"] > 0 and a.stats["frontier_slots"] > 0
        bc = ref(model, g, seeds, 200, 12, p=p, w=w, max_levels=3)
        assert_same(sim(model, G, seeds, 200, 12, graph=1, max_levels=3), bc)
    g, G, p, w, seeds = rmat14
    b0 = ref(model, g, seeds, 256, 2, p=p, w=w, level_counts_len=0)
    a = sim(model, G, seeds, 256, 2, graph=1, defer_bits=16, defer_steps=2, level_counts_len=0)
    assert np.array_equal(a.spread, b0.spread) and np.array_equal(a.node_count, b0.node_count)
    if model == "ic":
        assert_same(sim("ic", G, seeds, 256, 2, graph=1, direction="pull"), ref("ic", g, seeds, 256, 2, p=p))


def test_graph_mode_batch(rmat14):
    g, G, p, w, _ = rmat14
    seed_off, seeds, trials, keys = I.batch_items(g.n, 17, 1, 40, (64, 256, 1000, 3), graph_seed=9)
    for model in ("ic", "lt"):
        f = P.cnd_ic_simulate_batch if model == "ic" else P.cnd_lt_simulate_batch
        want_sp, want_nc, want_ck = _batch_ref(model, g, p, w, seed_off, seeds, trials, keys)
        a = f(G, seed_off, seeds, trials, keys, node_count=True, edge_checks=True, graph=1, word_bits=256)
        assert np.array_equal(a.spread, want_sp) and np.array_equal(a.node_count, want_nc)
        assert a.edge_checks == want_ck


def test_autotune_keeps_results(ba, rmat14):
    """The autotuner only picks engine settings: results stay bit-exact."""
    g, G, p, w, seeds = ba
    best = P.cnd_autotune(G, "ic", seeds, 3000, 1)
    assert best["word_bits"] in (0, 1024, 4096) and best["chunk_edges"] in (0, 32, 512)
    assert best["graph"] in (0, 1) and best["sample_ms"] > 0
    b = ref("ic", g, seeds, 3000, 1, p=p, level_counts_len=0)
    for _ in range(2):  # tunes on the first call, cache hit on the second
        a = sim("ic", G, seeds, 3000, 1, autotune=1, level_counts_len=0)
        assert np.array_equal(a.spread, b.spread) and np.array_equal(a.node_count, b.node_count)
        assert a.edge_checks == b.edge_checks
    g, G, p, w, _ = rmat14
    seed_off, seeds2, trials, keys = I.batch_items(g.n, 12, 1, 30, (64, 300), graph_seed=10)
    best = P.cnd_autotune(G, "lt", seeds2, trials, keys, seed_off=seed_off)
    assert best["pull_permille"] == 0
    want_sp, want_nc, want_ck = _batch_ref("lt", g, p, w, seed_off, seeds2, trials, keys)
    a = P.cnd_lt_simulate_batch(G, seed_off, seeds2, trials, keys, edge_checks=True, autotune=1)
    assert np.array_equal(a.spread, want_sp) and a.edge_checks == want_ck


@pytest.mark.parametrize("graph", [0, 1])
def test_timeout_stops_the_call_and_leaves_the_context_usable(ba, graph):
    """Failure detection without a fault: a time limit far below the call's run time ends it with
    CND_ETIMEOUT (host watchdog per step, or the device loop's check of the GPU global timer), and
    the next call on the same graph still gives the oracle's results."""
    g, G, p, w, seeds = ba
    with pytest.raises(P.CndError) as ei:
        sim("lt", G, seeds, 10_000, 1, timeout_s=1e-4, graph=graph)
    assert ei.value.status == P.CND_ETIMEOUT
    assert "timed out" in P.cnd_last_error()
    assert_same(sim("lt", G, seeds, 640, 1, graph=graph), ref("lt", g, seeds, 640, 1, w=w))
