"""C-ABI library checks that need no GPU: it loads, exports every declared
symbol, and rejects malformed input on the host before touching the device."""
import re
import os

import numpy as np
import pytest

import paper_2404_17059_gb300 as P
from paper_2404_17059_gb300 import binding, inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "cnd.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(cnd_[a-z0-9_]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    L = binding.load()
    decl = declared_symbols()
    assert "cnd_ic_simulate" in decl and "cnd_graph_create" in decl
    for name in decl:
        assert hasattr(L, name), name
    assert sorted(binding.EXPORTS) == decl


def test_opts_struct_layout():
    import ctypes
    o = P.cnd_sim_opts_init()
    assert ctypes.sizeof(o) == 104
    assert binding.cnd_sim_opts.timeout_s.offset == 64


def test_im_opts_layout_and_host_validation():
    import ctypes
    assert ctypes.sizeof(binding.cnd_im_opts) == 104
    assert binding.cnd_im_opts.sim.offset == 40 and binding.cnd_im_opts.reserved.offset == 72
    L = binding.load()
    o = binding.cnd_im_opts()
    L.cnd_im_opts_init(ctypes.byref(o))
    assert o.n_trials == 1024 and o.rng_seed == 1 and o.k == 0
    out = np.zeros(4, dtype=np.int32)
    # a NULL graph is rejected on the host, before any CUDA call
    assert L.cnd_ic_im_celf(None, ctypes.byref(o), out.ctypes.data, None) == P.CND_EINVAL
    assert "required" in P.cnd_last_error()


def test_surrogate_and_screen_abi_on_host():
    """Struct layouts, defaults, and NULL-handle rejection of the surrogate and screened-greedy entry points
    (all checked on the host, before any CUDA call)."""
    import ctypes
    L = binding.load()
    assert ctypes.sizeof(binding.cnd_sur_train_opts) == 112
    assert ctypes.sizeof(binding.cnd_screen_opts) == 56
    assert binding.cnd_screen_opts.sur_ms_out.offset == 16
    o = binding.cnd_sur_train_opts()
    L.cnd_sur_train_opts_init(ctypes.byref(o))
    assert (o.set_size_lo, o.set_size_hi, o.n_trials, o.batch_sets, o.sim_chunk) == (1, 50, 1024, 16, 256)
    assert abs(o.lr - 1e-3) < 1e-9 and o.n_pairs == 0
    buf = np.zeros(binding.CND_SUR_N_PARAMS, dtype=np.float32)
    out = ctypes.c_void_p()
    assert L.cnd_sur_create(None, buf.ctypes.data, ctypes.byref(out)) == P.CND_EINVAL and not out.value
    for name, args in (("cnd_sur_set_params", (None, buf.ctypes.data)), ("cnd_sur_get_params", (None, buf.ctypes.data)),
                       ("cnd_sur_forward", (None, None, 0, None, None)),
                       ("cnd_sur_loss_grad", (None, None, 0, buf.ctypes.data, None, None)),
                       ("cnd_sur_adam", (None, buf.ctypes.data, ctypes.c_float(1e-3))),
                       ("cnd_sur_scores", (None, None, 0, buf.ctypes.data)),
                       ("cnd_sur_onehop", (None, None, 0, buf.ctypes.data)),
                       ("cnd_sur_train", (None, ctypes.byref(o), None))):
        assert getattr(L, name)(*args) == P.CND_EINVAL, name
        assert "NULL" in P.cnd_last_error() or "required" in P.cnd_last_error(), name
    L.cnd_sur_destroy(None)  # NULL-safe
    io = binding.cnd_im_opts()
    L.cnd_im_opts_init(ctypes.byref(io))
    so = binding.cnd_screen_opts()
    seeds = np.zeros(4, dtype=np.int32)
    assert L.cnd_ic_im_screened(None, None, ctypes.byref(io), ctypes.byref(so), seeds.ctypes.data, None) == P.CND_EINVAL


def _graph():
    return I.erdos_renyi_m(50, 200, graph_seed=2)


def test_graph_validation_on_host():
    g = _graph()
    p = I.ic_uniform(g, 0.2)
    cases = []
    rp = g.row_ptr.copy(); rp[0] = 1; cases.append((rp, g.col, p, None, P.CND_EINVAL))
    rp = g.row_ptr.copy(); rp[5], rp[6] = rp[6], rp[5] - 1; cases.append((rp, g.col, p, None, P.CND_EINVAL))
    c = g.col.copy(); c[7] = g.n; cases.append((g.row_ptr, c, p, None, P.CND_EINVAL))
    c = g.col.copy(); c[7] = -1; cases.append((g.row_ptr, c, p, None, P.CND_EINVAL))
    for bad in (np.nan, -1e-9, 1.0000001, np.inf):
        q = p.copy(); q[3] = bad; cases.append((g.row_ptr, g.col, q, None, P.CND_EINVAL))
    w = np.full(g.m, 0x80000000, dtype=np.uint32)
    cases.append((g.row_ptr, g.col, None, w, P.CND_EOVERFLOW))
    for rp, c, q, w_, want in cases:
        with pytest.raises(P.CndError) as ei:
            P.cnd_graph_create(g.n, rp, c, q, w_)
        assert ei.value.status == want, P.cnd_last_error()


def test_lt_weights_wc_helper():
    g = I.barabasi_albert(300, 3, graph_seed=4)
    assert np.array_equal(P.cnd_lt_weights_wc(g.n, g.col), I.lt_weighted_cascade(g))
    w = P.cnd_lt_weights_wc(g.n, g.col).astype(np.uint64)
    assert np.all(np.bincount(g.col, weights=w, minlength=g.n) <= 0xFFFFFFFF)
    with pytest.raises(P.CndError):
        P.cnd_lt_weights_wc(g.n, np.array([0, g.n], dtype=np.int32))


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """No CPU fallback: without the compiled library the binding raises instead of computing."""
    monkeypatch.setattr(binding, "_lib", None)
    monkeypatch.setattr(binding._build, "LIB", str(tmp_path / "libcnd.so"))
    with pytest.raises(RuntimeError, match="not built"):
        binding.load(build_if_missing=False)


def test_measurement_probes_reject_bad_arguments_on_host():
    """The rate probes check their arguments on the host, before any CUDA call."""
    import ctypes
    L = binding.load()
    r, ms = ctypes.c_double(), ctypes.c_double()
    for region, op, iters in ((32, 0, 16), (1 << 20, 2, 16), (1 << 20, -1, 16), (1 << 20, 0, 0)):
        assert L.cnd_random_access_rate(region, op, iters, None, ctypes.byref(r), ctypes.byref(ms)) == P.CND_EINVAL
    assert L.cnd_random_access_rate(1 << 20, 0, 16, None, None, None) == P.CND_EINVAL
    assert "bad arguments" in P.cnd_last_error()
    assert L.cnd_philox_rate(0, None, ctypes.byref(r), None) == P.CND_EINVAL
