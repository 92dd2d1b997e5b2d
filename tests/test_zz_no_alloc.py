"""The allocation-free IC entry point against the regular one, through the C ABI.

cnd_ic_simulate_noalloc is for callers that cannot allocate device memory
while a simulation runs (a device whose memory another allocator has claimed,
or a loop that must not wait on the CUDA allocator).  It keeps its working
state in the library's static device scratch, which every call shares and
which keeps the previous call's contents.  So the test makes two calls in a
row on different inputs and checks that each one matches cnd_ic_simulate_ex
exactly (the results are integers: spreads and per-node counts are bit-exact).
This file is collected last so that a failure here leaves the other tests run.
"""
import numpy as np
import pytest

import paper_2404_17059_gb300 as P
from paper_2404_17059_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def test_noalloc_matches_regular_entry_point_twice():
    torch = pytest.importorskip("torch")
    g = I.erdos_renyi_m(1000, 10_000, graph_seed=1)
    p = I.ic_uniform(g, 0.1)
    G = P.cnd_graph_create(g.n, g.row_ptr, g.col, p, None)
    dev = torch.device("cuda", torch.cuda.current_device())
    cases = [(I.uniform_seeds(g.n, 10, 1), 1000, 1), (I.uniform_seeds(g.n, 3, 7), 333, 12345)]
    for seeds, T, rng in cases:
        s = torch.as_tensor(seeds, dtype=torch.int32, device=dev)
        spread = torch.full((T,), -7, dtype=torch.int32, device=dev)
        counts = torch.full((g.n,), -7, dtype=torch.int32, device=dev)
        assert P.cnd_ic_simulate_noalloc(G, s, T, rng, spread, counts) == P.CND_OK
        torch.cuda.synchronize()
        ref = P.cnd_ic_simulate_ex(G, seeds, T, rng)
        assert np.array_equal(spread.cpu().numpy(), ref.spread)
        assert np.array_equal(counts.cpu().numpy(), ref.node_count)


def test_noalloc_several_passes_match_regular_entry_point():
    """A graph large enough that the scratch holds only some words per pass (BA n=100,000: about a dozen
    64-trial words), so a call runs several passes: the per-pass re-upload of the word descriptors, the
    per-pass clear of the active sets, stamps that continue across passes and node counts summed over
    passes are all exercised; two calls in a row, the second with a ragged last word."""
    torch = pytest.importorskip("torch")
    g = I.barabasi_albert(100_000, 5, graph_seed=1)
    p = I.ic_weighted_cascade(g)
    G = P.cnd_graph_create(g.n, g.row_ptr, g.col, p, None)
    dev = torch.device("cuda", torch.cuda.current_device())
    seeds = I.top_degree_seeds(g, 50)
    for T, rng in ((4096, 3), (2500, 4)):
        s = torch.as_tensor(seeds, dtype=torch.int32, device=dev)
        spread = torch.full((T,), -7, dtype=torch.int32, device=dev)
        counts = torch.full((g.n,), -7, dtype=torch.int32, device=dev)
        assert P.cnd_ic_simulate_noalloc(G, s, T, rng, spread, counts) == P.CND_OK
        torch.cuda.synchronize()
        ref = P.cnd_ic_simulate_ex(G, seeds, T, rng, stats=P.CND_STATS_COUNT)
        assert ref.stats["passes"] == 1  # the regular call holds all its words in one pass
        assert np.array_equal(spread.cpu().numpy(), ref.spread)
        assert np.array_equal(counts.cpu().numpy(), ref.node_count)


def test_noalloc_rejects_graph_beyond_scratch():
    torch = pytest.importorskip("torch")
    g = I.rmat(20, 1 << 22, graph_seed=5)
    G = P.cnd_graph_create(g.n, g.row_ptr, g.col, I.ic_uniform(g, 0.01), None)
    s = torch.zeros(1, dtype=torch.int32, device="cuda")
    spread = torch.zeros(64, dtype=torch.int32, device="cuda")
    counts = torch.zeros(g.n, dtype=torch.int32, device="cuda")
    with pytest.raises(P.CndError) as ei:
        P.cnd_ic_simulate_noalloc(G, s, 64, 1, spread, counts)
    assert ei.value.status == P.CND_EINVAL
    assert "static scratch" in str(ei.value)
