"""Thin ctypes binding of libcnd (include/cnd.h): argument marshalling only.

Every simulation step runs in the library's CUDA kernels.  Host numpy arrays
are passed as host pointers; torch CUDA tensors are passed as device pointers
(``device_ptrs = 1``) together with torch's current stream.  There is no CPU
fallback: if the library cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os
import threading

import numpy as np

from . import build as _build

CND_OK, CND_EINVAL, CND_ENOMEM, CND_ECUDA, CND_ELIMIT, CND_ETIMEOUT, CND_EOVERFLOW = 0, -1, -2, -3, -4, -5, -6
CND_DIR_AUTO, CND_DIR_PUSH, CND_DIR_PULL = 0, 1, 2
_DIRS = {"auto": CND_DIR_AUTO, "push": CND_DIR_PUSH, "pull": CND_DIR_PULL}

# every symbol include/cnd.h declares
EXPORTS = (
    "cnd_sim_opts_init", "cnd_graph_create", "cnd_graph_destroy", "cnd_graph_info", "cnd_ic_simulate",
    "cnd_lt_simulate", "cnd_ic_simulate_ex", "cnd_lt_simulate_ex", "cnd_lt_weights_wc",
    "cnd_philox4x32_10", "cnd_last_error", "cnd_ic_simulate_noalloc", "cnd_ic_simulate_batch",
    "cnd_lt_simulate_batch", "cnd_autotune", "cnd_im_opts_init", "cnd_ic_im_celf", "cnd_lt_im_celf",
    "cnd_sur_create", "cnd_sur_destroy", "cnd_sur_set_params", "cnd_sur_get_params", "cnd_sur_forward",
    "cnd_sur_loss_grad", "cnd_sur_adam", "cnd_sur_scores", "cnd_sur_train_opts_init", "cnd_sur_train",
    "cnd_ic_im_screened", "cnd_sur_onehop", "cnd_philox_rate", "cnd_random_access_rate",
)
CND_SUR_N_PARAMS = 18689


class CndError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"cnd status {status}: {msg}")
        self.status = status


CND_STATS_TIMING, CND_STATS_COUNT = 1, 2


class cnd_sim_stats(C.Structure):
    _fields_ = [
        ("flags", C.c_int32),
        ("passes", C.c_int32),
        ("word_bits", C.c_int32),
        ("levels", C.c_int32),
        ("launches", C.c_int64),
        ("expand_launches", C.c_int64),
        ("expand_ms", C.c_double),
        ("finalize_launches", C.c_int64),
        ("finalize_ms", C.c_double),
        ("frontier_slots", C.c_int64),
        ("work_items", C.c_int64),
        ("edges_scanned", C.c_int64),
        ("frontier_words", C.c_int64),
        ("word_checks", C.c_int64),
        ("draws", C.c_int64),
        ("updates", C.c_int64),
        ("pull_steps", C.c_int64),
        ("lt_counters", C.c_int32),
        ("pad0", C.c_int32),
        ("setup_ms", C.c_double),
        ("graph_reused", C.c_int32),
        ("pad1", C.c_int32),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class cnd_sim_opts(C.Structure):
    _fields_ = [
        ("first_trial", C.c_int64),
        ("max_levels", C.c_int32),
        ("direction", C.c_int32),
        ("word_bits", C.c_int32),
        ("device_ptrs", C.c_int32),
        ("stream", C.c_void_p),
        ("edge_checks_out", C.c_void_p),
        ("level_counts_out", C.c_void_p),
        ("level_counts_len", C.c_int32),
        ("pull_permille", C.c_int32),
        ("chunk_edges", C.c_int32),
        ("defer_bits", C.c_int32),
        ("timeout_s", C.c_double),
        ("stats", C.c_void_p),
        ("defer_steps", C.c_int32),
        ("graph", C.c_int32),
        ("autotune", C.c_int32),
        ("lt_accumulate", C.c_int32),
        ("reserved", C.c_int64 * 1),
    ]


_lock = threading.Lock()
_lib = None


class cnd_im_opts(C.Structure):
    _fields_ = [
        ("k", C.c_int32), ("eval_batch", C.c_int32), ("n_trials", C.c_int64), ("rng_seed", C.c_uint64),
        ("candidates", C.c_void_p), ("n_candidates", C.c_int32), ("max_items", C.c_int32),
        ("sim", C.c_void_p), ("stream", C.c_void_p), ("evaluations_out", C.c_void_p),
        ("edge_checks_out", C.c_void_p), ("reserved", C.c_int64 * 4),
    ]


class cnd_sur_train_opts(C.Structure):
    _fields_ = [
        ("first_pair", C.c_int64), ("n_pairs", C.c_int64), ("set_size_lo", C.c_int32), ("set_size_hi", C.c_int32),
        ("n_trials", C.c_int32), ("batch_sets", C.c_int32), ("sim_chunk", C.c_int32), ("lr", C.c_float),
        ("data_seed", C.c_uint64), ("rng_seed", C.c_uint64), ("stream", C.c_void_p), ("sim_ms_out", C.c_void_p),
        ("train_ms_out", C.c_void_p), ("hub_frac", C.c_float), ("pad", C.c_int32), ("reserved", C.c_int64 * 3),
    ]


class cnd_screen_opts(C.Structure):
    _fields_ = [("n_screen", C.c_int32), ("n_exact", C.c_int32), ("mode", C.c_int32), ("pad", C.c_int32),
                ("sur_ms_out", C.c_void_p), ("sim_ms_out", C.c_void_p), ("reserved", C.c_int64 * 3)]


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libcnd.so (building it with nvcc if it is missing)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path):
            if not build_if_missing:
                raise RuntimeError(f"libcnd not built: {path} is missing")
            _build.build()
        L = C.CDLL(path)
        vp, i32, i64, u64 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64
        L.cnd_sim_opts_init.argtypes = [vp]
        L.cnd_sim_opts_init.restype = None
        L.cnd_graph_create.argtypes = [i32, i32, vp, vp, vp, vp, C.POINTER(vp)]
        L.cnd_graph_create.restype = i32
        L.cnd_graph_destroy.argtypes = [vp]
        L.cnd_graph_destroy.restype = None
        L.cnd_graph_info.argtypes = [vp, vp, vp, vp, vp]
        L.cnd_graph_info.restype = i32
        for name in ("cnd_ic_simulate", "cnd_lt_simulate"):
            getattr(L, name).argtypes = [vp, vp, i32, i64, u64, vp, vp]
            getattr(L, name).restype = i32
        for name in ("cnd_ic_simulate_ex", "cnd_lt_simulate_ex"):
            getattr(L, name).argtypes = [vp, vp, i32, i64, u64, vp, vp, C.POINTER(cnd_sim_opts)]
            getattr(L, name).restype = i32
        for name in ("cnd_ic_simulate_batch", "cnd_lt_simulate_batch"):
            getattr(L, name).argtypes = [vp, i32, vp, vp, vp, vp, vp, vp, C.POINTER(cnd_sim_opts)]
            getattr(L, name).restype = i32
        L.cnd_autotune.argtypes = [vp, i32, i32, vp, vp, i32, vp, vp, C.POINTER(cnd_sim_opts),
                                   C.POINTER(cnd_sim_opts), C.POINTER(C.c_double)]
        L.cnd_autotune.restype = i32
        L.cnd_im_opts_init.argtypes = [vp]
        L.cnd_im_opts_init.restype = None
        for name in ("cnd_ic_im_celf", "cnd_lt_im_celf"):
            getattr(L, name).argtypes = [vp, C.POINTER(cnd_im_opts), vp, vp]
            getattr(L, name).restype = i32
        L.cnd_sur_create.argtypes = [vp, vp, C.POINTER(vp)]
        L.cnd_sur_create.restype = i32
        L.cnd_sur_destroy.argtypes = [vp]
        L.cnd_sur_destroy.restype = None
        for name in ("cnd_sur_set_params", "cnd_sur_get_params"):
            getattr(L, name).argtypes = [vp, vp]
            getattr(L, name).restype = i32
        L.cnd_sur_forward.argtypes = [vp, vp, i32, vp, vp]
        L.cnd_sur_forward.restype = i32
        L.cnd_sur_loss_grad.argtypes = [vp, vp, i32, vp, vp, vp]
        L.cnd_sur_loss_grad.restype = i32
        L.cnd_sur_adam.argtypes = [vp, vp, C.c_float]
        L.cnd_sur_adam.restype = i32
        for name in ("cnd_sur_scores", "cnd_sur_onehop"):
            getattr(L, name).argtypes = [vp, vp, i32, vp]
            getattr(L, name).restype = i32
        L.cnd_sur_train_opts_init.argtypes = [vp]
        L.cnd_sur_train_opts_init.restype = None
        L.cnd_sur_train.argtypes = [vp, C.POINTER(cnd_sur_train_opts), vp]
        L.cnd_sur_train.restype = i32
        L.cnd_ic_im_screened.argtypes = [vp, vp, C.POINTER(cnd_im_opts), C.POINTER(cnd_screen_opts), vp, vp]
        L.cnd_ic_im_screened.restype = i32
        L.cnd_lt_weights_wc.argtypes = [i32, i32, vp, vp]
        L.cnd_lt_weights_wc.restype = i32
        L.cnd_philox4x32_10.argtypes = [u64, vp, i64, vp]
        L.cnd_philox4x32_10.restype = i32
        L.cnd_philox_rate.argtypes = [i32, vp, C.POINTER(C.c_double), C.POINTER(C.c_double)]
        L.cnd_philox_rate.restype = i32
        L.cnd_random_access_rate.argtypes = [i64, i32, i32, vp, C.POINTER(C.c_double), C.POINTER(C.c_double)]
        L.cnd_random_access_rate.restype = i32
        L.cnd_ic_simulate_noalloc.argtypes = [vp, vp, i32, i64, u64, vp, vp, vp]
        L.cnd_ic_simulate_noalloc.restype = i32
        L.cnd_last_error.argtypes = []
        L.cnd_last_error.restype = C.c_char_p
        _lib = L
        return L


def cnd_last_error() -> str:
    return load().cnd_last_error().decode()


def _check(st: int, allow=()):
    if st < 0 and st not in allow:
        raise CndError(st, cnd_last_error())
    return st


def _np_ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _is_torch_cuda(x) -> bool:
    try:
        import torch
    except ImportError:  # pragma: no cover
        return False
    return isinstance(x, torch.Tensor) and x.is_cuda


def cnd_sim_opts_init() -> cnd_sim_opts:
    o = cnd_sim_opts()
    load().cnd_sim_opts_init(C.byref(o))
    return o


class CndGraph:
    """Owning handle of a cnd_graph (destroyed with the object)."""

    def __init__(self, handle, n, m, has_ic, has_lt):
        self.handle = handle
        self.n, self.m, self.has_ic, self.has_lt = n, m, has_ic, has_lt

    def __del__(self):
        h, self.handle = getattr(self, "handle", None), None
        if h and _lib is not None:
            _lib.cnd_graph_destroy(h)

    def close(self):
        self.__del__()


def cnd_graph_create(n, row_ptr, col, ic_prob=None, lt_weight_fx=None) -> CndGraph:
    L = load()
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    icp = None if ic_prob is None else np.ascontiguousarray(ic_prob, dtype=np.float32)
    ltw = None if lt_weight_fx is None else np.ascontiguousarray(lt_weight_fx, dtype=np.uint32)
    m = int(col.shape[0])
    out = C.c_void_p()
    _check(L.cnd_graph_create(int(n), m, _np_ptr(row_ptr), _np_ptr(col), _np_ptr(icp), _np_ptr(ltw), C.byref(out)))
    return CndGraph(out, int(n), m, icp is not None, ltw is not None)


def cnd_graph_destroy(g: CndGraph) -> None:
    g.close()


def cnd_graph_info(g: CndGraph):
    n, m, hi, hl = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
    _check(load().cnd_graph_info(g.handle, C.byref(n), C.byref(m), C.byref(hi), C.byref(hl)))
    return n.value, m.value, bool(hi.value), bool(hl.value)


@dataclasses.dataclass
class SimResult:
    status: int
    spread: object = None        # int32 [n_trials]
    node_count: object = None    # int32 [n]
    edge_checks: int | None = None
    level_counts: object = None  # int64 [level_counts_len]
    stats: dict | None = None    # cnd_sim_stats fields, when requested


def _simulate(fn_name, g: CndGraph, seeds, n_trials, rng_seed, *, ex, spread=True, node_count=True,
              first_trial=0, max_levels=0, direction="auto", word_bits=0, level_counts_len=0,
              edge_checks=False, pull_permille=0, chunk_edges=0, timeout_s=0.0, stream=None, stats=0,
              defer_bits=0, defer_steps=0, graph=0, autotune=0, lt_accumulate=0):
    L = load()
    n_trials = int(n_trials)
    dev = _is_torch_cuda(seeds)
    if dev:
        import torch
        seeds_t = seeds.to(torch.int32).contiguous()
        sp = torch.empty(n_trials, dtype=torch.int32, device=seeds.device) if spread else None
        nc = torch.empty(g.n, dtype=torch.int32, device=seeds.device) if node_count else None
        ec = torch.zeros(1, dtype=torch.int64, device=seeds.device) if edge_checks else None
        lc = torch.zeros(level_counts_len, dtype=torch.int64, device=seeds.device) if level_counts_len else None
        seeds_p = C.c_void_p(seeds_t.data_ptr()) if seeds_t.numel() else None
        n_seeds = seeds_t.numel()
        sp_p = C.c_void_p(sp.data_ptr()) if sp is not None and n_trials else None
        nc_p = C.c_void_p(nc.data_ptr()) if nc is not None else None
        ec_p = ec.data_ptr() if ec is not None else None
        lc_p = lc.data_ptr() if lc is not None else None
        strm = stream if stream is not None else torch.cuda.current_stream(seeds.device).cuda_stream
    else:
        seeds_a = np.ascontiguousarray(np.asarray(seeds, dtype=np.int32).ravel())
        sp = np.empty(n_trials, dtype=np.int32) if spread else None
        nc = np.empty(g.n, dtype=np.int32) if node_count else None
        ec = np.zeros(1, dtype=np.int64) if edge_checks else None
        lc = np.zeros(level_counts_len, dtype=np.int64) if level_counts_len else None
        seeds_p = _np_ptr(seeds_a) if seeds_a.size else None
        n_seeds = seeds_a.size
        sp_p = _np_ptr(sp) if sp is not None and n_trials else None
        nc_p = _np_ptr(nc)
        ec_p = ec.ctypes.data if ec is not None else None
        lc_p = lc.ctypes.data if lc is not None else None
        strm = stream
    if ex:
        o = cnd_sim_opts_init()
        o.first_trial = int(first_trial)
        o.max_levels = int(max_levels)
        o.direction = _DIRS[direction] if isinstance(direction, str) else int(direction)
        o.word_bits = int(word_bits)
        o.device_ptrs = 1 if dev else 0
        o.stream = strm
        o.edge_checks_out = ec_p
        o.level_counts_out = lc_p
        o.level_counts_len = int(level_counts_len)
        o.pull_permille = int(pull_permille)
        o.chunk_edges = int(chunk_edges)
        o.defer_bits = int(defer_bits)
        o.defer_steps = int(defer_steps)
        o.graph = int(graph)
        o.autotune = int(autotune)
        o.lt_accumulate = int(lt_accumulate)
        o.timeout_s = float(timeout_s)
        stt = None
        if stats:
            stt = cnd_sim_stats()
            stt.flags = int(stats)
            o.stats = C.cast(C.pointer(stt), C.c_void_p)
        st = getattr(L, fn_name)(g.handle, seeds_p, int(n_seeds), n_trials, C.c_uint64(rng_seed), sp_p, nc_p,
                                 C.byref(o))
    else:
        stt = None
        if dev:
            raise ValueError(f"{fn_name} takes host arrays; use the _ex form for device tensors")
        st = getattr(L, fn_name)(g.handle, seeds_p, int(n_seeds), n_trials, C.c_uint64(rng_seed), sp_p, nc_p)
    _check(st, allow=(CND_ELIMIT,))
    ecv = None
    if ec is not None:
        ecv = int(ec[0].item()) if dev else int(ec[0])
    return SimResult(st, sp, nc, ecv, lc, stt.as_dict() if stt is not None else None)


def cnd_ic_simulate(g, seeds, n_trials, rng_seed, *, spread=True, node_count=True) -> SimResult:
    return _simulate("cnd_ic_simulate", g, seeds, n_trials, rng_seed, ex=False, spread=spread, node_count=node_count)


def cnd_lt_simulate(g, seeds, n_trials, rng_seed, *, spread=True, node_count=True) -> SimResult:
    return _simulate("cnd_lt_simulate", g, seeds, n_trials, rng_seed, ex=False, spread=spread, node_count=node_count)


def cnd_ic_simulate_ex(g, seeds, n_trials, rng_seed, **kw) -> SimResult:
    return _simulate("cnd_ic_simulate_ex", g, seeds, n_trials, rng_seed, ex=True, **kw)


def cnd_lt_simulate_ex(g, seeds, n_trials, rng_seed, **kw) -> SimResult:
    return _simulate("cnd_lt_simulate_ex", g, seeds, n_trials, rng_seed, ex=True, **kw)


def cnd_lt_weights_wc(n, col) -> np.ndarray:
    col = np.ascontiguousarray(col, dtype=np.int32)
    w = np.empty(col.shape[0], dtype=np.uint32)
    _check(load().cnd_lt_weights_wc(int(n), int(col.shape[0]), _np_ptr(col), _np_ptr(w)))
    return w


def cnd_philox4x32_10(rng_seed, ctr) -> np.ndarray:
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    out = np.empty_like(ctr)
    _check(load().cnd_philox4x32_10(C.c_uint64(rng_seed), _np_ptr(ctr), int(ctr.shape[0]), _np_ptr(out)))
    return out


def cnd_philox_rate(iters=4096, stream=None):
    """Measured Philox4x32-10 blocks per second of the engine's generator on the current device
    (returns (blocks_per_s, launch_ms))."""
    r, ms = C.c_double(), C.c_double()
    _check(load().cnd_philox_rate(int(iters), stream, C.byref(r), C.byref(ms)))
    return r.value, ms.value


RANDOM_OPS = {"read": 0, "atomic": 1}


def cnd_random_access_rate(region_bytes, op="read", iters=256, stream=None):
    """Measured random 8-byte reads ("read") or atomic XORs with return ("atomic") per second over a
    device region of region_bytes (rounded down to a power of two); returns (ops_per_s, launch_ms)."""
    r, ms = C.c_double(), C.c_double()
    _check(load().cnd_random_access_rate(int(region_bytes), RANDOM_OPS[op], int(iters), stream, C.byref(r),
                                         C.byref(ms)))
    return r.value, ms.value


def cnd_ic_simulate_noalloc(g, seeds, n_trials, rng_seed, spread_out, node_count_out, stream=None) -> int:
    """IC simulation that allocates nothing: its working state is the library's
    fixed static device scratch (CND_NOALLOC_SCRATCH_BYTES).  For callers that
    cannot allocate device memory during the call.  `seeds`, `spread_out`
    (n_trials int32) and `node_count_out` (n int32) are CUDA tensors the caller
    owns; calls that overlap on the GPU race on the shared scratch."""
    import torch
    for name, t in (("seeds", seeds), ("spread_out", spread_out), ("node_count_out", node_count_out)):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.int32 and t.is_contiguous()):
            raise TypeError(f"{name} must be a contiguous int32 CUDA tensor")
    if spread_out.numel() < int(n_trials) or node_count_out.numel() < g.n:
        raise ValueError("output tensors are too small")
    strm = stream if stream is not None else torch.cuda.current_stream(seeds.device).cuda_stream
    st = load().cnd_ic_simulate_noalloc(
        g.handle, C.c_void_p(seeds.data_ptr()) if seeds.numel() else None, int(seeds.numel()), int(n_trials),
        C.c_uint64(rng_seed), C.c_void_p(spread_out.data_ptr()) if int(n_trials) else None,
        C.c_void_p(node_count_out.data_ptr()), strm)
    return _check(st)


def _simulate_batch(fn_name, g, seed_off, seeds, n_trials, rng_seed, *, spread=True, node_count=False,
                    edge_checks=False, level_counts_len=0, stream=None, stats=0, **kw):
    """Batch form: seed_off / n_trials / rng_seed are host arrays; seeds may be a CUDA tensor."""
    L = load()
    seed_off = np.ascontiguousarray(seed_off, dtype=np.int64)
    n_trials = np.ascontiguousarray(n_trials, dtype=np.int32)
    rng_seed = np.ascontiguousarray(rng_seed, dtype=np.uint64)
    n_items = int(n_trials.shape[0])
    total = int(n_trials.astype(np.int64).sum())
    dev = _is_torch_cuda(seeds)
    if dev:
        import torch
        seeds_t = seeds.to(torch.int32).contiguous()
        sp = torch.empty(total, dtype=torch.int32, device=seeds.device) if spread else None
        nc = torch.empty(n_items * g.n, dtype=torch.int32, device=seeds.device) if node_count else None
        ec = torch.zeros(1, dtype=torch.int64, device=seeds.device) if edge_checks else None
        lc = torch.zeros(level_counts_len, dtype=torch.int64, device=seeds.device) if level_counts_len else None
        ptr = lambda t: C.c_void_p(t.data_ptr()) if t is not None and t.numel() else None  # noqa: E731
        seeds_p, sp_p, nc_p = ptr(seeds_t), ptr(sp), ptr(nc)
        ec_p = ec.data_ptr() if ec is not None else None
        lc_p = lc.data_ptr() if lc is not None else None
        strm = stream if stream is not None else torch.cuda.current_stream(seeds.device).cuda_stream
    else:
        seeds_a = np.ascontiguousarray(np.asarray(seeds, dtype=np.int32).ravel())
        sp = np.empty(total, dtype=np.int32) if spread else None
        nc = np.empty(n_items * g.n, dtype=np.int32) if node_count else None
        ec = np.zeros(1, dtype=np.int64) if edge_checks else None
        lc = np.zeros(level_counts_len, dtype=np.int64) if level_counts_len else None
        seeds_p = _np_ptr(seeds_a) if seeds_a.size else None
        sp_p = _np_ptr(sp) if sp is not None and total else None
        nc_p = _np_ptr(nc)
        ec_p = ec.ctypes.data if ec is not None else None
        lc_p = lc.ctypes.data if lc is not None else None
        strm = stream
    o = cnd_sim_opts_init()
    o.device_ptrs = 1 if dev else 0
    o.stream = strm
    o.edge_checks_out = ec_p
    o.level_counts_out = lc_p
    o.level_counts_len = int(level_counts_len)
    for k, v in kw.items():
        setattr(o, k, _DIRS[v] if k == "direction" and isinstance(v, str) else int(v) if k != "timeout_s" else float(v))
    stt = None
    if stats:
        stt = cnd_sim_stats()
        stt.flags = int(stats)
        o.stats = C.cast(C.pointer(stt), C.c_void_p)
    st = getattr(L, fn_name)(g.handle, n_items, _np_ptr(seed_off), seeds_p, _np_ptr(n_trials), _np_ptr(rng_seed),
                             sp_p, nc_p, C.byref(o))
    _check(st, allow=(CND_ELIMIT,))
    ecv = None
    if ec is not None:
        ecv = int(ec[0].item()) if dev else int(ec[0])
    if nc is not None:
        nc = nc.reshape(n_items, g.n)
    return SimResult(st, sp, nc, ecv, lc, stt.as_dict() if stt is not None else None)


def cnd_ic_simulate_batch(g, seed_off, seeds, n_trials, rng_seed, **kw) -> SimResult:
    return _simulate_batch("cnd_ic_simulate_batch", g, seed_off, seeds, n_trials, rng_seed, **kw)


def cnd_lt_simulate_batch(g, seed_off, seeds, n_trials, rng_seed, **kw) -> SimResult:
    return _simulate_batch("cnd_lt_simulate_batch", g, seed_off, seeds, n_trials, rng_seed, **kw)


def cnd_autotune(g, model, seeds, n_trials, rng_seed, *, seed_off=None) -> dict:
    """Autotuner: the fastest engine settings for this work (host arrays).

    Single seed set: ``seeds``, ``n_trials`` and ``rng_seed`` are scalars / one
    array; batch: pass ``seed_off`` and per-item ``n_trials`` / ``rng_seed``."""
    L = load()
    mdl = {"ic": 0, "lt": 1}[model] if isinstance(model, str) else int(model)
    seeds = np.ascontiguousarray(np.asarray(seeds, dtype=np.int32).ravel())
    tr = np.ascontiguousarray(np.atleast_1d(np.asarray(n_trials, dtype=np.int32)))
    ks = np.ascontiguousarray(np.atleast_1d(np.asarray(rng_seed, dtype=np.uint64)))
    so = None if seed_off is None else np.ascontiguousarray(seed_off, dtype=np.int64)
    n_items = 0 if so is None else int(tr.shape[0])
    best = cnd_sim_opts()
    ms = C.c_double()
    base = cnd_sim_opts_init()
    _check(L.cnd_autotune(g.handle, mdl, n_items, _np_ptr(so), _np_ptr(seeds) if seeds.size else None,
                          int(seeds.size), _np_ptr(tr), _np_ptr(ks), C.byref(base), C.byref(best), C.byref(ms)))
    return {"word_bits": best.word_bits, "chunk_edges": best.chunk_edges, "pull_permille": best.pull_permille,
            "graph": best.graph, "sample_ms": ms.value}


@dataclasses.dataclass
class ImResult:
    seeds: np.ndarray        # int32 [k], in the order chosen
    f: np.ndarray            # int64 [k]: F(first j+1 seeds) = sum of spreads over the trials
    evaluations: int         # seed sets simulated
    edge_checks: int


def _im_opts(k, n_trials, rng_seed, candidates, eval_batch, max_items, first_trial, stream, sim_kw):
    L = load()
    o = cnd_im_opts()
    L.cnd_im_opts_init(C.byref(o))
    o.k = int(k)
    o.n_trials = int(n_trials)
    o.rng_seed = int(rng_seed)
    o.eval_batch = int(eval_batch)
    o.max_items = int(max_items)
    cand = None
    if candidates is not None:
        cand = np.ascontiguousarray(np.asarray(candidates, dtype=np.int32).ravel())
        o.candidates = _np_ptr(cand)
        o.n_candidates = int(cand.size)
    so = cnd_sim_opts_init()
    so.first_trial = int(first_trial)
    for key, val in sim_kw.items():
        setattr(so, key, int(val))
    o.sim = C.cast(C.pointer(so), C.c_void_p)
    o.stream = stream
    ev = C.c_int64()
    ec = C.c_int64()
    o.evaluations_out = C.cast(C.pointer(ev), C.c_void_p)
    o.edge_checks_out = C.cast(C.pointer(ec), C.c_void_p)
    return o, (cand, so, ev, ec)


def _im_celf(fn_name, g, k, n_trials, rng_seed, *, candidates=None, eval_batch=0, max_items=0, first_trial=0,
             stream=None, **sim_kw) -> ImResult:
    o, keep = _im_opts(k, n_trials, rng_seed, candidates, eval_batch, max_items, first_trial, stream, sim_kw)
    seeds = np.empty(int(k), dtype=np.int32)
    f = np.empty(int(k), dtype=np.int64)
    _check(getattr(load(), fn_name)(g.handle, C.byref(o), _np_ptr(seeds), _np_ptr(f)))
    return ImResult(seeds, f, keep[2].value, keep[3].value)


def cnd_ic_im_celf(g, k, n_trials, rng_seed, **kw) -> ImResult:
    """Lazy-greedy (CELF) IC influence maximisation; engine options (word_bits, chunk_edges,
    pull_permille, graph, autotune) pass through to the batched calls."""
    return _im_celf("cnd_ic_im_celf", g, k, n_trials, rng_seed, **kw)


def cnd_lt_im_celf(g, k, n_trials, rng_seed, **kw) -> ImResult:
    return _im_celf("cnd_lt_im_celf", g, k, n_trials, rng_seed, **kw)


# ----------------------------------------------------------------------------- learned surrogate
class CndSur:
    """A surrogate network bound to a graph (cnd_sur); freed with cnd_sur_destroy or on collection."""

    def __init__(self, handle, graph):
        self.handle = handle
        self.graph = graph  # keeps the graph alive

    def __del__(self):
        if getattr(self, "handle", None):
            try:
                load().cnd_sur_destroy(self.handle)
            except Exception:
                pass
            self.handle = None


def _seeds_arr(seeds):
    a = np.ascontiguousarray(np.asarray(seeds, dtype=np.int32).ravel())
    return a, (_np_ptr(a) if a.size else None)


def cnd_sur_create(g: CndGraph, params) -> CndSur:
    L = load()
    p = np.ascontiguousarray(np.asarray(params, dtype=np.float32).ravel())
    if p.size != CND_SUR_N_PARAMS:
        raise ValueError(f"need {CND_SUR_N_PARAMS} parameters")
    out = C.c_void_p()
    _check(L.cnd_sur_create(g.handle, _np_ptr(p), C.byref(out)))
    return CndSur(out, g)


def cnd_sur_destroy(s: CndSur) -> None:
    if s.handle:
        load().cnd_sur_destroy(s.handle)
        s.handle = None


def cnd_sur_set_params(s: CndSur, params) -> None:
    p = np.ascontiguousarray(np.asarray(params, dtype=np.float32).ravel())
    if p.size != CND_SUR_N_PARAMS:
        raise ValueError(f"need {CND_SUR_N_PARAMS} parameters")
    _check(load().cnd_sur_set_params(s.handle, _np_ptr(p)))


def cnd_sur_get_params(s: CndSur) -> np.ndarray:
    p = np.empty(CND_SUR_N_PARAMS, dtype=np.float32)
    _check(load().cnd_sur_get_params(s.handle, _np_ptr(p)))
    return p


def cnd_sur_forward(s: CndSur, seeds, *, yhat=True):
    """(yhat float32 [n] or None, predicted spread sum(yhat))."""
    sd, sp = _seeds_arr(seeds)
    y = np.empty(s.graph.n, dtype=np.float32) if yhat else None
    tot = C.c_double()
    _check(load().cnd_sur_forward(s.handle, sp, int(sd.size), _np_ptr(y), C.byref(tot)))
    return y, tot.value


def cnd_sur_loss_grad(s: CndSur, seeds, y):
    sd, sp = _seeds_arr(seeds)
    yy = np.ascontiguousarray(np.asarray(y, dtype=np.float32).ravel())
    if yy.size != s.graph.n:
        raise ValueError("one target per node")
    grad = np.empty(CND_SUR_N_PARAMS, dtype=np.float32)
    loss = C.c_double()
    _check(load().cnd_sur_loss_grad(s.handle, sp, int(sd.size), _np_ptr(yy), C.byref(loss), _np_ptr(grad)))
    return loss.value, grad


def cnd_sur_adam(s: CndSur, grad, lr: float) -> None:
    gg = np.ascontiguousarray(np.asarray(grad, dtype=np.float32).ravel())
    _check(load().cnd_sur_adam(s.handle, _np_ptr(gg), C.c_float(lr)))


def cnd_sur_scores(s: CndSur, seeds) -> np.ndarray:
    sd, sp = _seeds_arr(seeds)
    out = np.empty(s.graph.n, dtype=np.float32)
    _check(load().cnd_sur_scores(s.handle, sp, int(sd.size), _np_ptr(out)))
    return out


def cnd_sur_onehop(s: CndSur, seeds) -> np.ndarray:
    sd, sp = _seeds_arr(seeds)
    out = np.empty(s.graph.n, dtype=np.float32)
    _check(load().cnd_sur_onehop(s.handle, sp, int(sd.size), _np_ptr(out)))
    return out


def cnd_sur_train(s: CndSur, n_pairs, *, first_pair=0, set_size=(1, 50), n_trials=1024, batch_sets=16,
                  sim_chunk=256, lr=1e-3, data_seed=1, rng_seed=1, stream=None, hub_frac=0.0) -> dict:
    L = load()
    o = cnd_sur_train_opts()
    L.cnd_sur_train_opts_init(C.byref(o))
    o.first_pair, o.n_pairs = int(first_pair), int(n_pairs)
    o.set_size_lo, o.set_size_hi = int(set_size[0]), int(set_size[1])
    o.n_trials, o.batch_sets, o.sim_chunk, o.lr = int(n_trials), int(batch_sets), int(sim_chunk), float(lr)
    o.data_seed, o.rng_seed, o.stream = int(data_seed), int(rng_seed), stream
    o.hub_frac = float(hub_frac)
    sim_ms, train_ms = C.c_double(), C.c_double()
    o.sim_ms_out = C.cast(C.pointer(sim_ms), C.c_void_p)
    o.train_ms_out = C.cast(C.pointer(train_ms), C.c_void_p)
    B = int(batch_sets) if batch_sets > 0 else 16
    chunk = max(B, (int(sim_chunk) // B) * B) if sim_chunk > 0 else max(B, (256 // B) * B)
    steps = sum(-(-min(chunk, n_pairs - c) // B) for c in range(0, int(n_pairs), chunk))
    loss = np.zeros(max(steps, 1), dtype=np.float64)
    _check(L.cnd_sur_train(s.handle, C.byref(o), _np_ptr(loss)))
    return {"loss": loss[:steps], "sim_ms": sim_ms.value, "train_ms": train_ms.value}


SCREEN_MODES = {"gradient": 0, "onehop": 1, "degree": 2, "mixed": 3}


def cnd_ic_im_screened(g, sur, k, n_trials, rng_seed, *, n_screen=64, n_exact=4, mode="gradient", candidates=None,
                       max_items=0, first_trial=0, stream=None, **sim_kw):
    """Greedy IC influence maximisation with the surrogate as a screen; returns (ImResult, timings)."""
    o, keep = _im_opts(k, n_trials, rng_seed, candidates, 0, max_items, first_trial, stream, sim_kw)
    so = cnd_screen_opts()
    so.n_screen, so.n_exact = int(n_screen), int(n_exact)
    so.mode = SCREEN_MODES[mode] if isinstance(mode, str) else int(mode)
    sur_ms, sim_ms = C.c_double(), C.c_double()
    so.sur_ms_out = C.cast(C.pointer(sur_ms), C.c_void_p)
    so.sim_ms_out = C.cast(C.pointer(sim_ms), C.c_void_p)
    seeds = np.empty(int(k), dtype=np.int32)
    f = np.empty(int(k), dtype=np.int64)
    _check(load().cnd_ic_im_screened(g.handle, sur.handle if sur is not None else None, C.byref(o), C.byref(so),
                                     _np_ptr(seeds), _np_ptr(f)))
    return ImResult(seeds, f, keep[2].value, keep[3].value), {"sur_ms": sur_ms.value, "sim_ms": sim_ms.value}
