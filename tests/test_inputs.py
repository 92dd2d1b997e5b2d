"""Synthetic workload generators: the structural properties the workloads rely on."""
import numpy as np
import pytest

from paper_2404_17059_gb300 import inputs as I


def _simple(g):
    src = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    assert not np.any(src == g.col)
    k = src.astype(np.int64) * g.n + g.col
    assert np.unique(k).size == k.size
    return src


def test_random_regular_is_simple_regular_and_symmetric():
    for n, d, seed in [(5000, 7, 1), (50, 3, 2), (11, 4, 3)]:
        g = I.random_regular(n, d, graph_seed=seed)
        assert g.m == n * d
        assert np.all(np.diff(g.row_ptr) == d) and np.all(g.in_degree() == d)
        src = _simple(g)
        fwd = set(zip(src.tolist(), g.col.tolist()))
        assert all((v, u) in fwd for u, v in fwd)
    a = I.random_regular(200, 5, graph_seed=9)
    b = I.random_regular(200, 5, graph_seed=9)
    assert np.array_equal(a.col, b.col)


def test_erdos_renyi_and_ba_shapes():
    g = I.erdos_renyi_m(1000, 10_000, graph_seed=1)
    assert g.m == 10_000
    _simple(g)
    b = I.barabasi_albert(2000, 5, graph_seed=1)
    assert b.m == 2 * (2000 - 5) * 5
    _simple(b)


def test_watts_strogatz_and_gnp():
    w = I.watts_strogatz(1000, 10, 0.05, graph_seed=2)
    assert w.m == 1000 * 10          # n k / 2 undirected edges, both directions stored
    src = _simple(w)
    fwd = set(zip(src.tolist(), w.col.tolist()))
    assert all((v, u) in fwd for u, v in fwd)
    g = I.erdos_renyi_gnp(2000, 0.002, graph_seed=1)
    src = _simple(g)
    assert abs(g.m / 2 - 0.002 * 2000 * 1999 / 2) < 5 * np.sqrt(0.002 * 2000 * 1999 / 2)


def test_edge_weight_models():
    g = I.erdos_renyi_m(500, 4000, graph_seed=3)
    tv = I.ic_trivalency(g, graph_seed=1)
    assert tv.dtype == np.float32 and set(np.unique(tv).tolist()) == {np.float32(0.1), np.float32(0.01),
                                                                      np.float32(0.001)}
    ur = I.ic_uniform_random(g, 1.0, graph_seed=1)
    assert ur.dtype == np.float32 and ur.min() >= 0 and ur.max() < 1
    wc = I.ic_weighted_cascade(g)
    indeg = g.in_degree()
    np.testing.assert_array_equal(wc, (np.float32(1.0) / indeg[g.col].astype(np.float32)))
    lw = I.lt_weighted_cascade(g)
    sums = np.bincount(g.col, weights=lw.astype(np.float64), minlength=g.n)
    assert np.all(sums <= 2**32 - 1)


def test_batch_items_shape():
    off, seeds, tr, keys = I.batch_items(10_000, 4096, 1, 100, (256, 1024, 4096), graph_seed=1)
    sizes = np.diff(off)
    assert sizes.min() >= 1 and sizes.max() <= 100 and set(np.unique(tr).tolist()) == {256, 1024, 4096}
    assert np.array_equal(keys, np.arange(1, 4097, dtype=np.uint64))
    for i in range(0, 4096, 512):
        s = seeds[off[i]:off[i + 1]]
        assert np.unique(s).size == s.size


def test_overlapping_hubs_structure():
    g = I.overlapping_hubs(graph_seed=3)
    assert g.n == 10 + 10 + 300 + 10 * 150 + 3000
    out = g.out_degree()
    shared = [set(g.col[g.row_ptr[h]:g.row_ptr[h + 1]].tolist()) & set(range(20, 320)) for h in range(10)]
    assert all(s == set(range(20, 320)) for s in shared)      # the redundant hubs reach the same 300 nodes
    for i, h in enumerate(range(10, 20)):                      # each small hub has 150 targets of its own
        assert set(range(320 + 150 * i, 470 + 150 * i)) <= set(g.col[g.row_ptr[h]:g.row_ptr[h + 1]].tolist())
    assert out[:10].min() > out[10:20].max() > out[20:].max()   # out-degree ranks the redundant hubs first
    p = I.hub_probabilities(g)
    src = g.src()
    assert np.all(p[src < 20] == np.float32(0.9)) and np.all(p[src >= 20] == np.float32(0.02))


def test_csr_file_roundtrip_and_digest(tmp_path):
    g = I.barabasi_albert(2000, 3, graph_seed=5)
    p = str(tmp_path / "ba.csr")
    d = I.save_csr(g, p)
    h = I.load_csr(p)
    assert d == g.digest() == h.digest() and h.n == g.n
    assert np.array_equal(h.row_ptr, g.row_ptr) and np.array_equal(h.col, g.col)
    raw = bytearray(open(p, "rb").read())
    raw[-1] ^= 1                                              # one flipped bit in col
    open(p, "wb").write(bytes(raw))
    with pytest.raises(ValueError, match="digest"):
        I.load_csr(p)
    open(p, "wb").write(bytes(raw[:-4]))                      # truncated
    with pytest.raises(ValueError, match="sizes"):
        I.load_csr(p)


def test_read_edge_list(tmp_path):
    p = tmp_path / "edges.txt"
    p.write_text("# a comment\n# FromNodeId\tToNodeId\n10 20\n20 30\n10 20\n30 30\n\n40 10\n")
    g, ids = I.read_edge_list(str(p))
    assert ids.tolist() == [10, 20, 30, 40] and g.n == 4
    assert sorted(zip(g.src().tolist(), g.col.tolist())) == [(0, 1), (1, 2), (3, 0)]
    u, ids_u = I.read_edge_list(str(p), undirected=True)
    assert sorted(zip(u.src().tolist(), u.col.tolist())) == [(0, 1), (0, 3), (1, 0), (1, 2), (2, 1), (3, 0)]
    p.write_text("1 2\n3\n")
    with pytest.raises(ValueError, match="malformed"):
        I.read_edge_list(str(p))
