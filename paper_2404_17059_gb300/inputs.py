"""Seeded synthetic workload generators (graphs, edge probabilities, weights, seed sets).

This module is shared by the CPU oracle's tests and by the GPU path's tests and
benchmark.  It holds none of the diffusion method's arithmetic: it only builds
the inputs a caller hands to ``cnd_graph_create`` / ``cnd_*_simulate`` -- a CSR
graph, a per-edge IC probability (fp32), a per-edge LT weight (uint32 fixed
point), and seed sets.  Every generator is a pure function of its integer
``graph_seed`` (numpy ``Philox`` bit generator), so both sides see the same
bytes.

Workload shapes follow the paper's benchmark section (Sec. 4, "Benchmarks"):
undirected edges become two directed edges, and the edge-weight models are
trivalency (TV), uniformly random (UR) and weighted cascade (WC,
p(u,v) = 1/in-degree(v)).  The LT weight for WC is the fixed-point value
floor((2^32 - 1) / in-degree(v)), so the in-weights of a node sum to at most
2^32 - 1 (Sec. 2, "Diffusion Models": the in-weights of a node sum to at most 1).
"""
from __future__ import annotations

import dataclasses
import hashlib
import os

import numpy as np

__all__ = [
    "Graph", "csr_from_edges", "erdos_renyi_m", "barabasi_albert", "rmat",
    "random_regular", "watts_strogatz", "path_graph", "out_star", "in_star",
    "ic_uniform", "ic_weighted_cascade", "ic_uniform_random", "ic_trivalency",
    "lt_weighted_cascade", "lt_random", "top_degree_seeds", "uniform_seeds", "batch_items",
    "save_csr", "load_csr", "read_edge_list",
]

LT_ONE = 0xFFFFFFFF  # largest total in-weight a node may carry (fixed point "1")


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(int(seed)))


@dataclasses.dataclass
class Graph:
    """Directed graph in CSR form: out-neighbours of u are col[row_ptr[u]:row_ptr[u+1]]."""
    n: int
    row_ptr: np.ndarray  # int32 [n+1]
    col: np.ndarray      # int32 [m]
    name: str = ""

    @property
    def m(self) -> int:
        return int(self.col.shape[0])

    def out_degree(self) -> np.ndarray:
        return np.diff(self.row_ptr.astype(np.int64)).astype(np.int64)

    def in_degree(self) -> np.ndarray:
        return np.bincount(self.col, minlength=self.n).astype(np.int64)

    def src(self) -> np.ndarray:
        """Source node of every edge, in CSR edge order."""
        return np.repeat(np.arange(self.n, dtype=np.int32), self.out_degree())

    def digest(self) -> str:
        h = hashlib.sha256()
        h.update(np.int64(self.n).tobytes())
        h.update(np.ascontiguousarray(self.row_ptr).tobytes())
        h.update(np.ascontiguousarray(self.col).tobytes())
        return h.hexdigest()[:16]


def csr_from_edges(n: int, src: np.ndarray, dst: np.ndarray, name: str = "",
                   sort: bool = True) -> Graph:
    """CSR from an edge list.  With ``sort`` the edges of a row are ordered by target."""
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    if sort:
        order = np.lexsort((dst, src))
    else:
        order = np.argsort(src, kind="stable")
    src = src[order]
    dst = dst[order]
    counts = np.bincount(src, minlength=n)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    if row_ptr[-1] > np.iinfo(np.int32).max:
        raise ValueError("edge count exceeds int32")
    return Graph(n=n, row_ptr=row_ptr.astype(np.int32), col=dst.astype(np.int32), name=name)


def erdos_renyi_m(n: int, m: int, graph_seed: int = 1) -> Graph:
    """Directed G(n, m): m distinct edges with uniform endpoints and no self-loops.

    Duplicates and self-loops are dropped and redrawn until exactly m distinct
    edges remain (first occurrence kept, in draw order).
    """
    if m > n * (n - 1):
        raise ValueError("too many edges")
    rng = _rng(graph_seed)
    chosen = np.empty(0, dtype=np.int64)
    seen: set = set()
    out = []
    while len(out) < m:
        need = m - len(out)
        s = rng.integers(0, n, size=2 * need + 16, dtype=np.int64)
        d = rng.integers(0, n, size=2 * need + 16, dtype=np.int64)
        for a, b in zip(s.tolist(), d.tolist()):
            if a == b:
                continue
            k = a * n + b
            if k in seen:
                continue
            seen.add(k)
            out.append(k)
            if len(out) == m:
                break
    chosen = np.array(out, dtype=np.int64)
    return csr_from_edges(n, chosen // n, chosen % n, name=f"er_n{n}_m{m}")


def erdos_renyi_gnp(n: int, p: float, graph_seed: int = 1) -> Graph:
    """Undirected G(n, p) (every pair independently with probability p), both directions stored."""
    rng = _rng(graph_seed)
    iu, ju = np.triu_indices(n, k=1)
    keep = rng.random(iu.size) < p
    u = iu[keep].astype(np.int64)
    v = ju[keep].astype(np.int64)
    return csr_from_edges(n, np.concatenate([u, v]), np.concatenate([v, u]), name=f"gnp_n{n}_p{p}")


def barabasi_albert(n: int, m_attach: int, graph_seed: int = 1) -> Graph:
    """Barabasi-Albert preferential attachment, each undirected edge stored both ways.

    Nodes 0..m_attach-1 start unconnected; node m_attach links to all of them;
    every later node links to m_attach distinct earlier nodes drawn with
    probability proportional to degree (uniform draws from the list of edge
    endpoints).  Undirected edges: (n - m_attach) * m_attach.
    """
    if not (1 <= m_attach < n):
        raise ValueError("need 1 <= m_attach < n")
    rng = _rng(graph_seed)
    n_und = (n - m_attach) * m_attach
    ends = np.empty(2 * n_und, dtype=np.int64)  # endpoint multiset, grows as edges are added
    e_src = np.empty(n_und, dtype=np.int64)
    e_dst = np.empty(n_und, dtype=np.int64)
    filled = 0
    targets = list(range(m_attach))
    pool = rng.integers(0, 1 << 62, size=1 << 16, dtype=np.int64)
    pi = 0
    for v in range(m_attach, n):
        base = filled
        for t in targets:
            e_src[filled] = v
            e_dst[filled] = t
            ends[2 * filled] = v
            ends[2 * filled + 1] = t
            filled += 1
        if v + 1 == n:
            break
        size = 2 * filled
        picked: list = []
        while len(picked) < m_attach:
            if pi == pool.size:
                pool = rng.integers(0, 1 << 62, size=1 << 16, dtype=np.int64)
                pi = 0
            cand = int(ends[int(pool[pi]) % size])
            pi += 1
            if cand not in picked:
                picked.append(cand)
        targets = picked
        del base
    src = np.concatenate([e_src, e_dst])
    dst = np.concatenate([e_dst, e_src])
    return csr_from_edges(n, src, dst, name=f"ba_n{n}_m{m_attach}")


_GEN_LIB = None


def _genlib():
    """ctypes handle of the C R-MAT generator (gen/rmat_gen.c), built with gcc on first use."""
    global _GEN_LIB
    if _GEN_LIB is None:
        import ctypes as C
        import subprocess
        here = os.path.dirname(os.path.abspath(__file__))
        src = os.path.join(here, "gen", "rmat_gen.c")
        out = os.path.join(here, "_build", "librmatgen.so")
        os.makedirs(os.path.dirname(out), exist_ok=True)
        if not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
            tmp = out + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O3", "-std=c99", "-fPIC", "-shared", "-pthread", "-o", tmp, src])
            os.replace(tmp, out)
        L = C.CDLL(out)
        L.rmat_keys.argtypes = [C.c_int, C.c_int64, C.c_int, C.c_int, C.c_int, C.c_uint64, C.c_int, C.c_void_p]
        L.rmat_keys.restype = None
        L.sort_unique_u64.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_int, C.c_int]
        L.sort_unique_u64.restype = C.c_int64
        _GEN_LIB = L
    return _GEN_LIB


def rmat(scale: int, n_samples: int, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         graph_seed: int = 1, threads: int | None = None) -> Graph:
    """R-MAT graph on n = 2^scale nodes from ``n_samples`` edge samples.

    Each sample descends ``scale`` levels of the adjacency matrix, choosing the
    quadrant (a: top-left, b: top-right, c: bottom-left, d: bottom-right) with
    the given probabilities, taken in units of 1/100.  Draws come from a
    counter-based stream per sample (gen/rmat_gen.c), so the graph depends only
    on (scale, n_samples, probabilities, graph_seed).  Self-loops and duplicate
    edges are dropped, so m <= n_samples; rows are sorted by target.
    """
    if scale < 1 or scale > 30:
        raise ValueError("scale must be in 1..30")
    n = 1 << scale
    pa, pb, pc = int(round(a * 100)), int(round(b * 100)), int(round(c * 100))
    if min(pa, pb, pc) < 0 or pa + pb + pc > 100:
        raise ValueError("bad quadrant probabilities")
    threads = threads or len(os.sched_getaffinity(0))
    L = _genlib()
    keys = np.empty(n_samples, dtype=np.uint64)
    tmp = np.empty(n_samples, dtype=np.uint64)
    L.rmat_keys(scale, n_samples, pa, pb, pc, int(graph_seed), threads, keys.ctypes.data)
    m = L.sort_unique_u64(keys.ctypes.data, tmp.ctypes.data, n_samples, 64, threads)
    del tmp
    if m < 0:
        raise MemoryError("R-MAT sort")
    keys = keys[:m]
    src = (keys >> np.uint64(32)).astype(np.int64)
    counts = np.bincount(src, minlength=n)
    del src
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    if row_ptr[-1] > np.iinfo(np.int32).max:
        raise ValueError("edge count exceeds int32")
    col = (keys & np.uint64(0xFFFFFFFF)).astype(np.int32)
    return Graph(n=n, row_ptr=row_ptr.astype(np.int32), col=col, name=f"rmat_s{scale}_{n_samples}")


def random_regular(n: int, d: int, graph_seed: int = 1, max_tries: int = 100) -> Graph:
    """Random d-regular simple undirected graph, both directions stored (n*d directed edges).

    Sequential stub pairing in the manner of Steger and Wormald (1999): two
    random open stubs are joined when that makes neither a self-loop nor a
    repeated edge; when no such pair is left the attempt restarts.  (Plain
    pairing with rejection of the whole graph succeeds with probability about
    exp(-(d^2 - 1) / 4), hopeless beyond d = 4.)
    """
    if (n * d) % 2 or d >= n:
        raise ValueError("need n*d even and d < n")
    rng = _rng(graph_seed)
    for _ in range(max_tries):
        stubs = np.repeat(np.arange(n, dtype=np.int64), d)
        rng.shuffle(stubs)
        open_ = list(stubs)
        adj = [set() for _ in range(n)]
        src, dst = [], []
        stuck = False
        while open_ and not stuck:
            for _attempt in range(64):
                i, j = rng.integers(0, len(open_), size=2)
                u, v = open_[i], open_[j]
                if i != j and u != v and v not in adj[u]:
                    break
            else:
                ok = [(i, j) for i in range(len(open_)) for j in range(i + 1, len(open_))
                      if open_[i] != open_[j] and open_[j] not in adj[open_[i]]]
                if not ok:
                    stuck = True
                    break
                i, j = ok[int(rng.integers(0, len(ok)))]
                u, v = open_[i], open_[j]
            adj[u].add(v)
            adj[v].add(u)
            src.append(u)
            dst.append(v)
            for k in sorted((int(i), int(j)), reverse=True):
                open_[k] = open_[-1]
                open_.pop()
        if not stuck:
            s_ = np.asarray(src, dtype=np.int64)
            t_ = np.asarray(dst, dtype=np.int64)
            return csr_from_edges(n, np.concatenate([s_, t_]), np.concatenate([t_, s_]), name=f"rr_n{n}_d{d}")
    raise RuntimeError("stub pairing kept getting stuck")


def watts_strogatz(n: int, k: int, p: float, graph_seed: int = 1) -> Graph:
    """Watts-Strogatz small world (ring lattice with k/2 neighbours each side, rewiring p), both directions stored."""
    rng = _rng(graph_seed)
    half = k // 2
    edges = set()
    for u in range(n):
        for j in range(1, half + 1):
            v = (u + j) % n
            edges.add((min(u, v), max(u, v)))
    edge_list = sorted(edges)
    adj = {e for e in edge_list}
    out = []
    for (u, v) in edge_list:
        if rng.random() < p:
            for _ in range(64):
                w = int(rng.integers(0, n))
                e = (min(u, w), max(u, w))
                if w != u and e not in adj:
                    adj.discard((u, v))
                    adj.add(e)
                    u, v = e
                    break
        out.append((u, v))
    arr = np.array(sorted(adj), dtype=np.int64)
    src = np.concatenate([arr[:, 0], arr[:, 1]])
    dst = np.concatenate([arr[:, 1], arr[:, 0]])
    return csr_from_edges(n, src, dst, name=f"ws_n{n}_k{k}")


def overlapping_hubs(n_shared_hubs: int = 10, shared: int = 300, n_own_hubs: int = 10, own: int = 150,
                     n_background: int = 3000, background_deg: int = 3, graph_seed: int = 1) -> Graph:
    """Hubs with redundant reach: n_shared_hubs hubs all point to the same `shared` nodes, n_own_hubs
    smaller hubs each point to `own` nodes of their own, and background nodes carry random edges.
    Out-degree ranks the redundant hubs first, though after one of them the others add little."""
    rng = _rng(graph_seed)
    hubs_a = np.arange(n_shared_hubs)
    hubs_b = np.arange(n_shared_hubs, n_shared_hubs + n_own_hubs)
    base = n_shared_hubs + n_own_hubs
    shared_nodes = np.arange(base, base + shared)
    own0 = base + shared
    n = own0 + n_own_hubs * own + n_background
    src, dst = [], []
    for h in hubs_a:
        src.append(np.full(shared, h))
        dst.append(shared_nodes)
    for i, h in enumerate(hubs_b):
        src.append(np.full(own, h))
        dst.append(np.arange(own0 + i * own, own0 + (i + 1) * own))
    bg = np.repeat(np.arange(n), background_deg)
    tg = rng.integers(0, n, size=bg.size)
    keep = bg != tg
    src.append(bg[keep])
    dst.append(tg[keep])
    s_ = np.concatenate(src).astype(np.int64)
    d_ = np.concatenate(dst).astype(np.int64)
    k = np.unique(s_ * n + d_)
    return csr_from_edges(n, k // n, k % n, name=f"hubs_{n_shared_hubs}x{shared}_{n_own_hubs}x{own}")


def hub_probabilities(g: Graph, p_hub: float = 0.9, p_background: float = 0.02, n_hubs: int = 20) -> np.ndarray:
    """IC probabilities for overlapping_hubs: p_hub on the hubs' edges, p_background elsewhere."""
    src = g.src()
    return np.where(src < n_hubs, np.float32(p_hub), np.float32(p_background)).astype(np.float32)


def path_graph(length: int) -> Graph:
    """Directed path 0 -> 1 -> ... -> length (length edges)."""
    n = length + 1
    src = np.arange(length, dtype=np.int64)
    return csr_from_edges(n, src, src + 1, name=f"path{length}")


def out_star(k: int) -> Graph:
    """Centre 0 with edges 0 -> 1..k."""
    return csr_from_edges(k + 1, np.zeros(k, dtype=np.int64), np.arange(1, k + 1), name=f"ostar{k}")


def in_star(k: int) -> Graph:
    """Leaves 1..k with edges leaf -> 0."""
    return csr_from_edges(k + 1, np.arange(1, k + 1), np.zeros(k, dtype=np.int64), name=f"istar{k}")


# ---------------------------------------------------------------- edge weights
def ic_uniform(g: Graph, p: float) -> np.ndarray:
    return np.full(g.m, np.float32(p), dtype=np.float32)


def ic_weighted_cascade(g: Graph) -> np.ndarray:
    """p(u,v) = 1/in-degree(v), one IEEE fp32 division per edge."""
    indeg = g.in_degree().astype(np.float32)
    return (np.float32(1.0) / indeg[g.col]).astype(np.float32)


def ic_uniform_random(g: Graph, hi: float = 1.0, graph_seed: int = 1) -> np.ndarray:
    """p ~ U[0, hi) in fp32 per edge (UR model; hi=0.1 for the batched R-MAT workload)."""
    rng = _rng(graph_seed + 0x5EED)
    return (rng.random(g.m, dtype=np.float32) * np.float32(hi)).astype(np.float32)


def ic_trivalency(g: Graph, graph_seed: int = 1) -> np.ndarray:
    """p drawn uniformly from {0.1, 0.01, 0.001} per edge (TV model)."""
    rng = _rng(graph_seed + 0x7EED)
    vals = np.array([0.1, 0.01, 0.001], dtype=np.float32)
    return vals[rng.integers(0, 3, size=g.m)]


def lt_weighted_cascade(g: Graph) -> np.ndarray:
    """LT weight of (u,v) = floor((2^32-1)/in-degree(v)) as uint32 (in-weights sum <= 2^32-1)."""
    indeg = g.in_degree()
    w = np.zeros(g.n, dtype=np.uint64)
    nz = indeg > 0
    w[nz] = np.uint64(LT_ONE) // indeg[nz].astype(np.uint64)
    return w[g.col].astype(np.uint32)


def lt_random(g: Graph, total: float = 1.0, graph_seed: int = 1) -> np.ndarray:
    """LT weights that differ between a node's in-edges: raw U[0.1, 1) per edge, scaled so that each
    node's in-weights sum to at most total * (2^32-1) (floored, uint32)."""
    rng = _rng(graph_seed + 0x17EED)
    raw = rng.uniform(0.1, 1.0, size=g.m)
    tot = np.zeros(g.n)
    np.add.at(tot, g.col, raw)
    w = np.floor(raw / tot[g.col] * (float(total) * LT_ONE)).astype(np.uint64)
    return np.minimum(w, LT_ONE).astype(np.uint32)


# ---------------------------------------------------------------- seed sets
def top_degree_seeds(g: Graph, k: int) -> np.ndarray:
    """k nodes of largest out-degree, ties broken by lower node id."""
    deg = g.out_degree()
    order = np.lexsort((np.arange(g.n), -deg))
    return order[:k].astype(np.int32)


def uniform_seeds(n: int, k: int, rng_or_seed) -> np.ndarray:
    """k distinct nodes drawn uniformly (order of first draw kept)."""
    rng = rng_or_seed if isinstance(rng_or_seed, np.random.Generator) else _rng(rng_or_seed)
    if k > n:
        raise ValueError("k > n")
    out: list = []
    seen: set = set()
    while len(out) < k:
        for x in rng.integers(0, n, size=2 * (k - len(out)) + 4).tolist():
            if x not in seen:
                seen.add(x)
                out.append(x)
                if len(out) == k:
                    break
    return np.array(out, dtype=np.int32)


def batch_items(n: int, n_items: int, size_lo: int, size_hi: int, trial_choices,
                graph_seed: int = 1):
    """Batched-simulation items: (seed_off[n_items+1] int64, seeds int32, n_trials int32, rng_seed uint64).

    Seed-set sizes are uniform on {size_lo..size_hi}; each set holds distinct
    uniform nodes; trial counts are uniform over ``trial_choices``; item i uses
    rng_seed i+1.
    """
    rng = _rng(graph_seed + 0xBA7C)
    sizes = rng.integers(size_lo, size_hi + 1, size=n_items)
    trials = np.asarray(trial_choices, dtype=np.int32)[rng.integers(0, len(trial_choices), size=n_items)]
    seed_off = np.zeros(n_items + 1, dtype=np.int64)
    np.cumsum(sizes, out=seed_off[1:])
    seeds = np.concatenate([uniform_seeds(n, int(s), rng) for s in sizes]) if n_items else np.zeros(0, np.int32)
    rng_seeds = np.arange(1, n_items + 1, dtype=np.uint64)
    return seed_off, seeds.astype(np.int32), trials.astype(np.int32), rng_seeds


# ----------------------------------------------------------------------------- graph files
_CSR_MAGIC = b"CNDCSR01"


def save_csr(g: Graph, path: str) -> str:
    """Write ``g`` as a binary CSR file and return its digest (``Graph.digest``).

    Layout (little-endian): 8-byte magic ``CNDCSR01``, n and m as int64, the
    16 ASCII hex digits of the digest, row_ptr (int32, n + 1), col (int32, m).
    """
    d = g.digest()
    with open(path, "wb") as f:
        f.write(_CSR_MAGIC)
        f.write(np.array([g.n, g.m], dtype="<i8").tobytes())
        f.write(d.encode("ascii"))
        f.write(np.ascontiguousarray(g.row_ptr, dtype="<i4").tobytes())
        f.write(np.ascontiguousarray(g.col, dtype="<i4").tobytes())
    return d


def load_csr(path: str) -> Graph:
    """Read a file written by ``save_csr``; ValueError if its magic, sizes or digest do not match."""
    with open(path, "rb") as f:
        raw = f.read()
    head = len(_CSR_MAGIC) + 16 + 16
    if len(raw) < head or raw[:len(_CSR_MAGIC)] != _CSR_MAGIC:
        raise ValueError(f"{path}: not a CSR graph file")
    n, m = (int(x) for x in np.frombuffer(raw, dtype="<i8", count=2, offset=len(_CSR_MAGIC)))
    want = raw[len(_CSR_MAGIC) + 16:head].decode("ascii")
    if n < 1 or m < 0 or len(raw) != head + 4 * (n + 1) + 4 * m:
        raise ValueError(f"{path}: sizes do not match the header")
    row_ptr = np.frombuffer(raw, dtype="<i4", count=n + 1, offset=head).astype(np.int32)
    col = np.frombuffer(raw, dtype="<i4", count=m, offset=head + 4 * (n + 1)).astype(np.int32)
    g = Graph(n=n, row_ptr=row_ptr, col=col, name=os.path.basename(path))
    if g.digest() != want:
        raise ValueError(f"{path}: digest mismatch (file {want}, contents {g.digest()})")
    return g


def read_edge_list(path: str, undirected: bool = False, comments: str = "#"):
    """Graph from a whitespace-separated edge-list text file: one ``u v`` pair of integer ids per
    line, lines starting with ``comments`` ignored (the format SNAP distributes its networks in).

    Ids are relabelled 0..n-1 in increasing order of the original id; self-loops and repeated
    edges are dropped; with ``undirected`` every edge is stored in both directions (as the
    paper's benchmarks treat undirected networks, Sec. 4).  Returns (graph, ids) with ids[i]
    the original id of node i.
    """
    pairs = []
    with open(path) as f:
        for line in f:
            t = line.strip()
            if not t or t.startswith(comments):
                continue
            a = t.split()
            if len(a) < 2:
                raise ValueError(f"{path}: malformed line {line!r}")
            pairs.append((int(a[0]), int(a[1])))
    e = np.asarray(pairs, dtype=np.int64).reshape(-1, 2)
    ids, inv = np.unique(e.ravel(), return_inverse=True)
    inv = inv.reshape(-1, 2)
    src, dst = inv[:, 0], inv[:, 1]
    if undirected:
        src, dst = np.concatenate([src, dst]), np.concatenate([dst, src])
    keep = src != dst
    n = max(int(ids.size), 1)
    k = np.unique(src[keep] * n + dst[keep])
    return csr_from_edges(n, k // n, k % n, name=os.path.basename(path)), ids


# ----------------------------------------------------------------------------- surrogate inputs
SURROGATE_SHAPES = (  # parameter layout of the surrogate network: (name, rows, cols), fp32, row-major
    ("Ws1", 64, 16), ("Wn1", 64, 16), ("b1", 64, 1), ("Ws2", 64, 64), ("Wn2", 64, 64), ("b2", 64, 1),
    ("Ws3", 64, 64), ("Wn3", 64, 64), ("b3", 64, 1), ("wo", 64, 1), ("bo", 1, 1),
)
SURROGATE_N_PARAMS = sum(r * c for _, r, c in SURROGATE_SHAPES)


def surrogate_init(graph_seed: int = 1) -> np.ndarray:
    """Initial surrogate parameters: uniform on +-1/sqrt(fan_in) (fan-in of a layer counts both of
    its inputs), drawn from numpy's Philox generator; fp32, flat, in SURROGATE_SHAPES order."""
    rng = _rng(graph_seed + 0x5122)
    fan_in = {"Ws1": 32, "Wn1": 32, "b1": 32, "Ws2": 128, "Wn2": 128, "b2": 128, "Ws3": 128, "Wn3": 128,
              "b3": 128, "wo": 64, "bo": 64}
    parts = [rng.uniform(-1.0, 1.0, size=r * c) / np.sqrt(fan_in[name]) for name, r, c in SURROGATE_SHAPES]
    return np.concatenate(parts).astype(np.float32)


def surrogate_pairs(n: int, n_sets: int, size_lo: int = 1, size_hi: int = 50, graph_seed: int = 1):
    """Training seed sets: sizes U{size_lo..size_hi}, distinct uniform nodes; returns (seed_off, seeds)."""
    rng = _rng(graph_seed + 0x7A15)
    sizes = rng.integers(size_lo, size_hi + 1, size=n_sets)
    off = np.zeros(n_sets + 1, dtype=np.int64)
    np.cumsum(sizes, out=off[1:])
    seeds = np.empty(int(off[-1]), dtype=np.int32)
    for i in range(n_sets):
        seeds[off[i]:off[i + 1]] = rng.choice(n, size=int(sizes[i]), replace=False)
    return off, seeds
