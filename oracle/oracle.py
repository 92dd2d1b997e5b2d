"""ctypes binding of the C oracle (``cnd_oracle.c``) -- test infrastructure only."""
from __future__ import annotations

import concurrent.futures as _cf
import ctypes as C
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cnd_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "liboracle.so")

OK, LIMIT, EINVAL, EOVERFLOW = 0, 1, -1, -2

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no vendor code, plain C99)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            p = C.c_void_p
            L.oracle_philox_many.argtypes = [p, C.c_int64, C.c_uint64, p]
            L.oracle_philox_many.restype = None
            L.oracle_ic_coin.argtypes = [C.c_uint64, C.c_int64, C.c_int64]
            L.oracle_ic_coin.restype = C.c_uint32
            L.oracle_lt_theta.argtypes = [C.c_uint64, C.c_int64, C.c_int64]
            L.oracle_lt_theta.restype = C.c_uint32
            L.oracle_ic_threshold.argtypes = [C.c_float]
            L.oracle_ic_threshold.restype = C.c_uint32
            L.oracle_simulate.argtypes = [C.c_int32, C.c_int32, C.c_int32, p, p, p, p, p, C.c_int32,
                                          C.c_int64, C.c_int64, C.c_uint64, C.c_int32,
                                          p, p, p, p, C.c_int32, p, p]
            L.oracle_simulate.restype = C.c_int32
            _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def philox(ctr: np.ndarray, rng_seed: int) -> np.ndarray:
    """Philox4x32-10 of each row of ``ctr`` (k x 4 uint32) under key rng_seed."""
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    out = np.empty_like(ctr)
    lib().oracle_philox_many(_ptr(ctr), ctr.shape[0], C.c_uint64(rng_seed), _ptr(out))
    return out


def ic_coin(rng_seed: int, trial: int, edge: int) -> int:
    return int(lib().oracle_ic_coin(rng_seed, trial, edge))


def lt_theta(rng_seed: int, trial: int, node: int) -> int:
    return int(lib().oracle_lt_theta(rng_seed, trial, node))


def ic_threshold(p) -> np.ndarray:
    p = np.asarray(p, dtype=np.float32).ravel()
    L = lib()
    return np.array([L.oracle_ic_threshold(float(x)) for x in p], dtype=np.uint32)


@dataclasses.dataclass
class OracleResult:
    status: int
    spread: np.ndarray
    node_count: np.ndarray
    edge_checks: int
    level_counts: np.ndarray
    active: np.ndarray | None = None
    level: np.ndarray | None = None


def simulate(model: str, graph, seeds, n_trials: int, rng_seed: int, *, ic_prob=None, lt_weight=None,
             first_trial: int = 0, mode: str = "bfs", max_levels: int = 0, level_counts_len: int = 64,
             want_sets: bool = False) -> OracleResult:
    """Run trials first_trial .. first_trial+n_trials-1 of the IC or LT model on one thread."""
    mdl = {"ic": 0, "lt": 1}[model]
    md = {"bfs": 0, "sweep": 1}[mode]
    n = int(graph.n)
    row_ptr = np.ascontiguousarray(graph.row_ptr, dtype=np.int32)
    col = np.ascontiguousarray(graph.col, dtype=np.int32)
    seeds = np.ascontiguousarray(np.asarray(seeds, dtype=np.int32).ravel())
    icp = None if ic_prob is None else np.ascontiguousarray(ic_prob, dtype=np.float32)
    ltw = None if lt_weight is None else np.ascontiguousarray(lt_weight, dtype=np.uint32)
    spread = np.zeros(n_trials, dtype=np.int32)
    counts = np.zeros(n, dtype=np.int32)
    checks = np.zeros(1, dtype=np.int64)
    lcount = np.zeros(max(level_counts_len, 0), dtype=np.int64)
    active = np.zeros((n_trials, n), dtype=np.uint8) if want_sets else None
    level = np.zeros((n_trials, n), dtype=np.int32) if want_sets else None
    st = lib().oracle_simulate(mdl, md, n, _ptr(row_ptr), _ptr(col), _ptr(icp), _ptr(ltw),
                               _ptr(seeds) if seeds.size else None, int(seeds.size),
                               int(first_trial), int(n_trials), C.c_uint64(rng_seed), int(max_levels),
                               _ptr(spread), _ptr(counts), _ptr(checks), _ptr(lcount) if lcount.size else None,
                               int(lcount.size), _ptr(active), _ptr(level))
    return OracleResult(int(st), spread, counts, int(checks[0]), lcount, active, level)


def simulate_threads(model: str, graph, seeds, n_trials: int, rng_seed: int, *, threads: int | None = None,
                     first_trial: int = 0, **kw) -> OracleResult:
    """Same trials split into contiguous ranges run on host threads (ctypes releases the GIL).

    Each trial's computation is unchanged; per-node counts, edge checks and
    level counts are summed over ranges, spreads concatenated.
    """
    if threads is None:
        threads = len(os.sched_getaffinity(0))
    threads = max(1, min(threads, n_trials)) if n_trials > 0 else 1
    bounds = np.linspace(0, n_trials, threads + 1).astype(np.int64)
    jobs = [(int(bounds[i]), int(bounds[i + 1] - bounds[i])) for i in range(threads)]
    lib()
    with _cf.ThreadPoolExecutor(max_workers=threads) as ex:
        parts = list(ex.map(lambda j: simulate(model, graph, seeds, j[1], rng_seed,
                                               first_trial=first_trial + j[0], **kw), jobs))
    st = min(p.status for p in parts) if any(p.status < 0 for p in parts) else max(p.status for p in parts)
    return OracleResult(
        st,
        np.concatenate([p.spread for p in parts]),
        np.sum([p.node_count for p in parts], axis=0).astype(np.int32),
        int(sum(p.edge_checks for p in parts)),
        np.sum([p.level_counts for p in parts], axis=0),
    )
