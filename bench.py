#!/usr/bin/env python
"""Throughput of Monte Carlo IC / LT simulation on GB300 (one JSON line).

A step is one pass of the whole path over one batch of synthetic input (graph
ingest happens once, before the timed region):

  rmat24 (default)  the large configuration: R-MAT scale 24, edge factor 16 (2^28
                    samples, deduplicated: 263,430,501 edges); IC with p = 0.01
                    and LT with weighted-cascade weights; 100 highest-degree
                    seeds; 100,000 trials per model.  A step is one IC call and
                    one LT call on 1,024 trials each (--trials, --lt-trials),
                    each a contiguous range of trial ids; the
                    ranges rotate through the 100,000 from step to step
                    (first_trial), so every step does full trials and no work
                    is skipped.  --scale changes the scale (ncu captures).
  ba100k            Barabasi-Albert n=100,000, 5 attachments, undirected edges
                    stored both ways (999,950 directed edges); weighted-cascade
                    IC probabilities (fp32) and LT weights (uint32 fixed point);
                    the 50 highest-degree nodes as seeds; one IC and one LT
                    simulation of 10,000 trials each.
  rmat20batch       R-MAT scale 20, 2^24 samples (16,084,954 edges), p ~ U[0,0.1)
                    per edge; one batched IC call over the first K of 4,096 seed
                    sets (|S| ~ U{1..100}, trials from {256, 1024, 4096}).
  er1k              directed ER n=1,000, m=10,000, p=0.1, 10 seeds, 1,000 trials.
  surrogate         the learned screen: R-MAT scale 17 (2^21 samples deduplicated),
                    weighted-cascade IC; the network is trained on --pairs seed
                    sets (|S| ~ U{1..50}, 1,024 exact trials each, generated on
                    the fly by the simulator), then greedy k=50 with the
                    surrogate as a screen is timed against MC CELF (1,024
                    common trials); both seed sets are scored with 10,000
                    exact trials.  metric: CELF time / screened-greedy time.
  surrogate24       surrogate inference over the large graph: R-MAT scale 24 (edge factor 16,
                    --scale to change), IC p = 0.01, one forward pass per candidate seed set
                    for 1,000 sets of 100 distinct uniform nodes (--items sets); metric:
                    sets/s, with the forward's algorithmic bytes against the HBM peak.
  rmat20batch_full  all 4,096 seed sets of the batched workload in one call (one CUDA graph),
                    after one warm-up call on 8 of them; about 150 s on one GB300.
  table1            the paper's run-time table scenario: IC, 1,000 runs from 100 uniform seeds on
                    an undirected G(n=2000, p=0.002) and a Watts-Strogatz (n=10000, k=10,
                    p=0.007) graph (edges both ways), trivalency / uniform [0,1] / weighted-
                    cascade probabilities; GPU time per 1,000 runs next to the oracle on one
                    host thread (the paper's measurements are single-threaded).
  celf_rr7          influence maximisation: CELF with k=10 on a random 7-regular
                    graph, n=5,000 (35,000 directed edges), IC with trivalency and
                    weighted-cascade probabilities, 1,000 common trials per
                    evaluation (--trials); a step is one CELF run per model.
                    metric: seconds per CELF run (lower is better), next to the
                    oracle's CELF on the host cores.

value        = edge checks per second over the whole job (all ranks), device-
               resident inputs, CUDA-event time of each step, L2 flushed
               between steps outside the step events.
e2e          = the same metric through the host-pointer C-ABI calls (seeds copied
               in, spreads / counts / edge checks copied out).
roofline     = the dominant expansion kernel: algorithmic bytes it must move
               (counted by the kernels) / its CUDA-event time.
cpu_baseline = the CPU oracle on a bounded sample of the same workload, on all
               host cores.
--impl reference times the CPU oracle alone, each step a bounded sample.
Multi-GPU (torchrun): every rank simulates its own trials (single workloads:
its own trial range; batches: its own seed sets) -- weak scaling, no collective
on the data path.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2404_17059_gb300 import inputs as I  # noqa: E402

METRIC = "IC/LT edge checks/sec and trials/sec at 1 GB300 (% of HBM peak); surrogate vs MC greedy speedup"
UNIT = "edge_checks/s"
FALLBACK_HBM_GBS = 6800.0


# ----------------------------------------------------------------------------- workloads
class Workload:
    """A graph, its per-model edge data, seeds and the calls of one step.

    trials: {"ic": T, "lt": T} trials per model per step.  total: the configuration's trial count per
    model; when it exceeds a step's trials, step i simulates the contiguous range of trial ids
    [r T, (r + 1) T) with r = (i * world + rank) mod floor(total / T), so that successive steps (and
    ranks) rotate through the configuration's trials via first_trial."""

    def __init__(self, name, desc, g, models, seeds=None, trials=None, rng_seed=1, batch=None, cpu=None, total=0,
                 ref=None):
        self.name, self.desc, self.g = name, desc, g
        self.models = models          # {"ic": p or None, "lt": w or None}
        self.seeds, self.rng_seed = seeds, rng_seed
        self.trials = dict(trials or {})
        self.total = total
        self.batch = batch            # (seed_off, seeds, trials, keys) or None
        self.cpu = cpu or {}          # CPU-oracle sample sizes (the cpu_baseline of our arm)
        self.ref = ref or self.cpu    # the reference arm's sample per step

    def create(self, P):
        return P.cnd_graph_create(self.g.n, self.g.row_ptr, self.g.col, self.models.get("ic"),
                                  self.models.get("lt"))

    def rank_batch(self, rank):
        seed_off, seeds, trials, keys = self.batch
        k = len(trials)
        return seed_off, seeds, trials, keys, k

    def first_trial(self, model, step, rank, world):
        T = self.trials[model]
        span = ((T + 63) // 64) * 64
        if self.total <= T:
            return rank * span  # every step simulates the whole configuration; ranks take their own ids
        return ((step * world + rank) % (self.total // span)) * span

    def calls(self, P, G, seeds_arg, rank, stats=0, graph=0, step=0, world=1):
        """One step: a list of (model, SimResult)."""
        out = []
        if self.batch is None:
            for model in ("ic", "lt"):
                if self.models.get(model) is None:
                    continue
                f = P.cnd_ic_simulate_ex if model == "ic" else P.cnd_lt_simulate_ex
                out.append((model, f(G, seeds_arg, self.trials[model], self.rng_seed,
                                     first_trial=self.first_trial(model, step, rank, world), edge_checks=True,
                                     stats=stats, graph=graph)))
        else:
            seed_off, _, trials, keys = self.batch
            out.append(("ic", P.cnd_ic_simulate_batch(G, seed_off, seeds_arg, trials, keys, edge_checks=True,
                                                      stats=stats, graph=graph)))
        return out

    def host_seeds(self):
        return self.seeds if self.batch is None else self.batch[1]

    def trials_per_step(self):
        if self.batch is None:
            return sum(self.trials[m] for m in ("ic", "lt") if self.models.get(m) is not None)
        return int(np.asarray(self.batch[2], dtype=np.int64).sum())

    def io_bytes(self):
        """Bytes copied in / out per step by the host-pointer calls."""
        if self.batch is None:
            ms = [m for m in ("ic", "lt") if self.models.get(m) is not None]
            return len(ms) * self.seeds.size * 4, sum(self.trials[m] * 4 + self.g.n * 4 + 8 for m in ms)
        return self.batch[1].size * 4, self.trials_per_step() * 4 + 8


def select_models(wl: Workload, models: str) -> Workload:
    keep = {m.strip() for m in models.split(",") if m.strip()}
    if not keep <= {"ic", "lt"} or not keep:
        raise SystemExit("--models takes ic, lt or ic,lt")
    if wl.batch is None:
        wl.models = {m: (d if m in keep else None) for m, d in wl.models.items()}
    return wl


RMAT24_TRIALS = {"ic": 1024, "lt": 1024}  # trials per model per step of the R-MAT workload (of 100,000)


def make_workload(name: str, trials: int = 0, items: int = 0, lt_trials: int = 0, scale: int = 24) -> Workload:
    if name == "ba100k":
        g = I.barabasi_albert(100_000, 5, graph_seed=1)
        T = {"ic": trials or 10_000, "lt": lt_trials or trials or 10_000}
        return Workload(
            name, f"BA n=100000 m_attach=5 symmetrised ({g.m} directed edges), weighted-cascade IC (fp32 "
                  f"p=1/indeg) and LT (uint32 floor((2^32-1)/indeg)), 50 top-degree seeds, {T['ic']} IC and "
                  f"{T['lt']} LT trials per step, rng_seed=1",
            g, {"ic": I.ic_weighted_cascade(g), "lt": I.lt_weighted_cascade(g)}, seeds=I.top_degree_seeds(g, 50),
            trials=T, cpu={"ic": 2048, "lt": 1536}, total=10_000, ref={"ic": 384, "lt": 256})
    if name == "er1k":
        g = I.erdos_renyi_m(1000, 10_000, graph_seed=1)
        T = {"ic": trials or 1000, "lt": lt_trials or trials or 1000}
        return Workload(
            name, f"directed ER n=1000 m=10000, IC p=0.1, LT weighted cascade, 10 uniform seeds, {T['ic']} IC and "
                  f"{T['lt']} LT trials per step",
            g, {"ic": I.ic_uniform(g, 0.1), "lt": I.lt_weighted_cascade(g)}, seeds=I.uniform_seeds(g.n, 10, 1),
            trials=T, cpu={"ic": 1000, "lt": 1000}, total=1000)
    if name == "rmat24":
        g = I.rmat(scale, 16 << scale, graph_seed=1)
        T = {"ic": trials or RMAT24_TRIALS["ic"], "lt": lt_trials or RMAT24_TRIALS["lt"]}
        return Workload(
            name, f"R-MAT scale {scale} edge factor 16 (a,b,c,d=.57,.19,.19,.05; {g.m} directed edges after dedup), "
                  f"IC p=0.01 and LT weighted cascade, 100 top-degree seeds, 100000 trials per model, rng_seed=1; "
                  f"each step simulates a contiguous range of {T['ic']} IC and {T['lt']} LT trial ids, the ranges "
                  f"rotating through the 100000 via first_trial",
            g, {"ic": I.ic_uniform(g, 0.01), "lt": I.lt_weighted_cascade(g)}, seeds=I.top_degree_seeds(g, 100),
            trials=T, cpu={"ic": 16, "lt": 16}, total=100_000, ref={"ic": 8, "lt": 8})
    if name == "rmat20batch":
        g = I.rmat(20, 1 << 24, graph_seed=1)
        so, seeds, tr, keys = I.batch_items(g.n, 4096, 1, 100, (256, 1024, 4096), graph_seed=1)
        k = items or 64
        batch = (so[:k + 1], seeds[:so[k]], tr[:k], keys[:k])
        return Workload(
            name, f"R-MAT scale 20 ({g.m} directed edges), IC p~U[0,0.1) fp32 per edge, batched: the first {k} of "
                  "4096 seed sets (|S|~U{1..100}, trials from {256,1024,4096}, rng_seed i+1) in one call",
            g, {"ic": I.ic_uniform_random(g, 0.1, graph_seed=1)}, batch=batch, cpu={"items": 2, "trials": 16})
    raise SystemExit(f"unknown workload {name}")


# ----------------------------------------------------------------------------- helpers
def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


ENGINE_SOURCES = ("cnd_common.cuh", "cnd_sim.cu")  # the expansion kernels the traffic figures cover


def source_hash() -> str:
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2404_17059_gb300", "csrc")
    for fn in ENGINE_SOURCES:
        with open(os.path.join(d, fn), "rb") as f:
            h.update(fn.encode())
            h.update(f.read())
    return h.hexdigest()[:12]


def ncu_traffic(kernel: str, workload: str, word_checks_per_launch: float):
    """DRAM bytes per launch, from the committed ncu summary's bytes per word check.

    The summary is taken on a trial sample of the same workload (ncu replays
    each launch, so the sample keeps the device memory it saves small) and is
    scaled by the word checks a launch of this run performs.  None unless it
    was taken on the current sources.
    """
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    cur = source_hash()
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line.startswith("{"):
                continue
            rec = json.loads(line)
            if rec.get("kernel") == kernel and rec.get("workload") == workload and rec.get("src") == cur:
                return rec["dram_bytes_per_word_check"] * word_checks_per_launch
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        if not self.lines:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def oracle_sample(wl: Workload, first: int = 0):
    """The oracle, as it stands, on a bounded sample of the workload over all host cores.

    Returns (edge checks, trials, seconds, description)."""
    import oracle
    cores = len(os.sched_getaffinity(0))
    checks = trials = 0
    parts = []
    t0 = time.perf_counter()
    if wl.batch is None:
        # the models' trials share one pool of host threads, one trial per job, so that the cores stay busy
        # across both models (a large-graph trial is the unit of work here: tens of seconds on one core)
        import concurrent.futures as cf
        jobs = []
        for model in ("ic", "lt"):
            data = wl.models.get(model)
            if data is None:
                continue
            n = wl.cpu[model]
            kw = {"ic_prob": data} if model == "ic" else {"lt_weight": data}
            jobs += [(model, first + j, kw) for j in range(n)]
            trials += n
            parts.append(f"{model.upper()} trials {first}..{first + n - 1}")
        oracle.lib()
        with cf.ThreadPoolExecutor(max_workers=max(1, min(cores, len(jobs)))) as ex:
            res = list(ex.map(lambda j: oracle.simulate(j[0], wl.g, wl.seeds, 1, wl.rng_seed, first_trial=j[1],
                                                        level_counts_len=0, **j[2]), jobs))
        checks = sum(r.edge_checks for r in res)
    else:
        seed_off, seeds, tr, keys = wl.batch
        for i in range(wl.cpu["items"]):
            n = min(int(tr[i]), wl.cpu["trials"])
            r = oracle.simulate_threads("ic", wl.g, seeds[seed_off[i]:seed_off[i + 1]], n, int(keys[i]),
                                        threads=cores, level_counts_len=0, first_trial=first, ic_prob=wl.models["ic"])
            checks += r.edge_checks
            trials += n
        parts.append(f"{wl.cpu['trials']} trials of each of the first {wl.cpu['items']} seed sets")
    dt = time.perf_counter() - t0
    return checks, trials, dt, ", ".join(parts) + f" on {cores} threads", cores


def cpu_baseline(wl: Workload):
    checks, trials, dt, desc, cores = oracle_sample(wl)
    return {"value": checks / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{desc}: {checks} edge checks in {dt:.2f} s wall", "trials_per_s": trials / dt}


# ----------------------------------------------------------------------------- reference arm
def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    wl = select_models(make_workload(args.workload, args.trials, args.items, args.lt_trials, args.scale),
                       args.models)
    wl.cpu = dict(wl.ref)
    if args.ref_trials:
        for m, n in zip(("ic", "lt"), args.ref_trials):
            if m in wl.cpu:
                wl.cpu[m] = n
    times, checks, cores, desc = [], 0, 1, ""
    for i in range(args.warmup + args.steps):
        c, _, dt, desc, cores = oracle_sample(wl, first=64 * i)
        if i >= args.warmup:
            times.append(dt)
            checks += c
    total = sum(times)
    value = checks / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": wl.desc, "name": wl.name, "graph_sha256": wl.g.digest(), "sample_per_step": desc},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"each step: {desc}"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- CELF
CELF_K = 10


def celf_models(trials):
    g = I.random_regular(5000, 7, graph_seed=1)
    return g, {"tv": I.ic_trivalency(g, graph_seed=1), "wc": I.ic_weighted_cascade(g)}, trials or 1000


def run_celf(args):
    """CELF (k=10) on the random 7-regular graph: GPU batch engine vs the oracle's CELF."""
    import torch
    import paper_2404_17059_gb300 as P
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    g, probs, T = celf_models(args.trials)
    res = {}
    for name, p in probs.items():
        G = P.cnd_graph_create(g.n, g.row_ptr, g.col, p, None)
        for _ in range(args.warmup):
            r = P.cnd_ic_im_celf(G, CELF_K, T, 1, graph=1)
        times = []
        for _ in range(args.steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = P.cnd_ic_im_celf(G, CELF_K, T, 1, graph=1)
            times.append(time.perf_counter() - t0)
        res[name] = {"s_per_run": statistics.median(times), "runs_s": times, "seeds": r.seeds.tolist(),
                     "sigma": (r.f / T).tolist(), "evaluations": r.evaluations, "edge_checks": r.edge_checks}
        P.cnd_graph_destroy(G)
    cpu = None
    if not args.no_cpu_baseline and rank == 0:
        from oracle import im
        cores = len(os.sched_getaffinity(0))
        cpu = {}
        for name, p in probs.items():
            t0 = time.perf_counter()
            s_, f_, ev = im.celf("ic", g, CELF_K, T, 1, threads=cores, ic_prob=p)
            dt = time.perf_counter() - t0
            same = s_.tolist() == res[name]["seeds"] and (f_ / T).tolist() == res[name]["sigma"]
            cpu[name] = {"s_per_run": dt, "evaluations": ev, "same_seeds_and_sigma": same}
        cpu = {"value": sum(v["s_per_run"] for v in cpu.values()), "unit": "s", "cores": cores, "kind": "oracle",
               "sample": f"the full CELF (k={CELF_K}, {T} trials) per model on {cores} threads", "models": cpu}
    if rank != 0:
        return 0
    total = sum(v["s_per_run"] for v in res.values())
    line = {"metric": f"CELF k={CELF_K} wall-clock seconds (TV + WC IC)", "value": total, "unit": "s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total,
            "higher_is_better": False, "scaling": "replicas only", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic",
            "config": {"workload": f"random 7-regular n=5000 (35000 directed edges), IC trivalency and weighted "
                                   f"cascade, CELF k={CELF_K}, {T} common trials per evaluation, rng_seed=1",
                       "name": "celf_rr7", "timing": "host wall clock around each CELF call (device work synced)"},
            "models": res, "cpu_baseline": cpu,
            "paper_context": "CyNetDiff (Cython, one CPU core, trial count unstated): 2 s TV, 10 s WC for CELF k=10"}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- surrogate
def run_surrogate(args):
    import torch
    import paper_2404_17059_gb300 as P
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if rank != 0:
        return 0
    k, T, score_T, score_key = args.k, 1024, 10_000, 7777
    g = I.rmat(17, 1 << 21, graph_seed=1)
    p = I.ic_weighted_cascade(g)
    G = P.cnd_graph_create(g.n, g.row_ptr, g.col, p, None)
    # held-out sets and their exact per-node frequencies
    ho_off, ho_seeds = I.surrogate_pairs(g.n, 64, 1, 50, graph_seed=99)
    ho_keys = np.arange(1_000_000, 1_000_064, dtype=np.uint64)
    ho = P.cnd_ic_simulate_batch(G, ho_off, ho_seeds, np.full(64, T, dtype=np.int32), ho_keys, node_count=True)
    freq = ho.node_count.reshape(64, g.n).astype(np.float64) / T

    def quality(sur):
        err, mse = [], []
        for i in range(64):
            yh, tot = P.cnd_sur_forward(sur, ho_seeds[ho_off[i]:ho_off[i + 1]])
            mc = freq[i].sum()
            err.append(abs(tot - mc) / mc)
            mse.append(float(np.mean((yh - freq[i]) ** 2)))
        return {"spread_rel_err_mean": float(np.mean(err)), "spread_rel_err_max": float(np.max(err)),
                "node_mse": float(np.mean(mse))}

    init = I.surrogate_init(1)
    sur = P.cnd_sur_create(G, init)
    untrained = P.cnd_sur_create(G, init)
    q0 = quality(sur)
    # forward throughput: aggregation gathers (layers 2, 3: 128 B rows over m in-edges, 8 B edge records)
    # and dense layers (read [h | a] 256 B, write h 128 B per node; layer 1 reads 64 B)
    fseeds = ho_seeds[ho_off[0]:ho_off[1]]
    for _ in range(3):
        P.cnd_sur_forward(sur, fseeds, yhat=False)
    t0 = time.perf_counter()
    for _ in range(50):
        P.cnd_sur_forward(sur, fseeds, yhat=False)
    fwd_s = (time.perf_counter() - t0) / 50
    fwd_bytes = 2 * g.m * (128 + 8 + 0) + 2 * g.n * 128 + g.n * (64 + 128) + 2 * g.n * (256 + 128)
    peak, _ = measured_peak()
    fwd = {"ms": fwd_s * 1e3, "alg_bytes": fwd_bytes, "achieved_gbs": fwd_bytes / fwd_s / 1e9,
           "frac_of_hbm": fwd_bytes / fwd_s / 1e9 / peak,
           "note": "host wall time of cnd_sur_forward (seed upload and result copy included)"}
    t0 = time.perf_counter()
    tr = P.cnd_sur_train(sur, args.pairs, n_trials=T, batch_sets=16, sim_chunk=256, lr=1e-3, data_seed=1, rng_seed=1,
                         hub_frac=args.hub_frac)
    train_s = time.perf_counter() - t0
    q1 = quality(sur)
    print(f"trained {args.pairs} pairs in {train_s:.1f} s; held-out before {q0} after {q1}", file=sys.stderr,
          flush=True)

    def mc_spread(seeds):
        r = P.cnd_ic_simulate_ex(G, seeds, score_T, score_key, node_count=False)
        return float(r.spread.astype(np.float64).mean())

    runs = {}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rc = P.cnd_ic_im_celf(G, k, T, 1, graph=1)
    runs["mc_celf"] = {"s": time.perf_counter() - t0, "seeds": rc.seeds.tolist(), "evaluations": rc.evaluations,
                       "edge_checks": rc.edge_checks}
    print(f"mc_celf: {runs['mc_celf']['s']:.2f} s", file=sys.stderr, flush=True)
    variants = (("screened_trained", sur, args.screen_mode), ("screened_trained_onehop_no_rerank", sur, "onehop"),
                ("screened_trained_gradient", sur, "gradient"), ("screened_trained_mixed", sur, "mixed"),
                ("screened_trained_onehop", sur, "onehop"), ("screened_untrained", untrained, args.screen_mode),
                ("screened_degree_no_network", None, "degree"))
    for name, model, mode in variants:
        no_rerank = name.endswith("no_rerank") or mode in ("mixed", "degree")
        if name != "screened_trained" and not no_rerank and mode == args.screen_mode and model is sur:
            continue
        t0 = time.perf_counter()
        rs, tm = P.cnd_ic_im_screened(G, model, k, T, 1, n_screen=args.exact if no_rerank else args.screen,
                                      n_exact=args.exact, mode=mode, graph=1)
        runs[name] = {"s": time.perf_counter() - t0, "mode": mode, "seeds": rs.seeds.tolist(),
                      "evaluations": rs.evaluations, "edge_checks": rs.edge_checks, **tm}
        print(f"{name}: {runs[name]['s']:.2f} s", file=sys.stderr, flush=True)
    for v in runs.values():
        v["scored_spread"] = mc_spread(v["seeds"])
    base = runs["mc_celf"]
    for name in runs:
        if name == "mc_celf":
            continue
        runs[name]["spread_vs_celf"] = runs[name]["scored_spread"] / base["scored_spread"]
        runs[name]["speedup_vs_celf"] = base["s"] / runs[name]["s"]
    hubs = surrogate_hubs(P)
    line = {"metric": "surrogate vs MC greedy speedup", "value": runs["screened_trained"]["speedup_vs_celf"],
            "unit": "x", "n_gpus": 1, "steps": 1, "warmup": 0, "ms_per_step": 1e3 * runs["screened_trained"]["s"],
            "higher_is_better": True, "scaling": "replicas only", "vs_baseline": None, "dtype": "bf16+u64",
            "data": "synthetic",
            "config": {"workload": f"R-MAT scale 17 ({g.m} directed edges), WC IC; surrogate trained on "
                                   f"{args.pairs} pairs (|S|~U{{1..50}}, {T} trials); greedy k={k} screened "
                                   f"({args.screen} by the {args.screen_mode} score, then by predicted spread, "
                                   f"{args.exact} simulated per round) vs MC CELF, "
                                   f"{T} common trials; scored with {score_T} trials (key {score_key})",
                       "name": "surrogate"},
            "spread_vs_celf": runs["screened_trained"]["spread_vs_celf"],
            "training": {"pairs": args.pairs, "s": train_s, "sim_ms": tr["sim_ms"], "train_ms": tr["train_ms"],
                         "loss_first": float(tr["loss"][:8].mean()), "loss_last": float(tr["loss"][-8:].mean())},
            "speedup_including_training": base["s"] / (runs["screened_trained"]["s"] + train_s),
            "heldout_untrained": q0, "heldout_trained": q1, "forward": fwd, "runs": runs, "overlapping_hubs": hubs}
    print(json.dumps(line), flush=True)
    return 0


def surrogate_hubs(P):
    """The screen on a graph whose highest-degree nodes reach the same nodes (inputs.overlapping_hubs): greedy
    k=8 with 2 (mixed) or 4 (gradient) simulated candidates per round, trained on hub-including seed sets vs
    the untrained network vs out-degree (no network) vs MC CELF; spreads scored with 4,096 exact trials."""
    g = I.overlapping_hubs(graph_seed=1)
    G = P.cnd_graph_create(g.n, g.row_ptr, g.col, I.hub_probabilities(g), None)
    init = I.surrogate_init(1)

    def scored(seeds):
        r = P.cnd_ic_simulate_ex(G, np.asarray(seeds, dtype=np.int32), 4096, 99, node_count=False)
        return float(r.spread.astype(np.float64).mean())

    K, T = 8, 512
    t0 = time.perf_counter()
    celf = P.cnd_ic_im_celf(G, K, T, 1)
    out = {"celf": {"spread": scored(celf.seeds), "evaluations": celf.evaluations, "s": time.perf_counter() - t0,
                    "seeds": celf.seeds.tolist()}}
    trained = P.cnd_sur_create(G, init)
    t0 = time.perf_counter()
    P.cnd_sur_train(trained, 32768, set_size=(1, 20), n_trials=256, batch_sets=16, lr=3e-3, hub_frac=0.5)
    out["train_s"] = time.perf_counter() - t0
    for nex, mode in ((2, "mixed"), (4, "gradient")):
        for name, model, md in (("trained", trained, mode), ("untrained", P.cnd_sur_create(G, init), mode),
                                ("degree_no_network", None, "degree")):
            t0 = time.perf_counter()
            r, _ = P.cnd_ic_im_screened(G, model, K, T, 1, n_screen=nex, n_exact=nex, mode=md)
            sp = scored(r.seeds)
            out[f"{name}_{md}_{nex}"] = {"spread": sp, "vs_celf": sp / out["celf"]["spread"],
                                         "evaluations": r.evaluations, "s": time.perf_counter() - t0,
                                         "seeds": r.seeds.tolist()}
    return out


def run_table1(args):
    """The paper's Table 1 scenario on the GPU and on one host thread (oracle)."""
    import torch
    import oracle
    import paper_2404_17059_gb300 as P
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if rank != 0:
        return 0
    graphs = {"erdos_renyi": I.erdos_renyi_gnp(2000, 0.002, graph_seed=1),
              "watts_strogatz": I.watts_strogatz(10_000, 10, 0.007, graph_seed=1)}
    cases = []
    for gname, g in graphs.items():
        models = {"TV": I.ic_trivalency(g, graph_seed=1), "UR": I.ic_uniform_random(g, 1.0, graph_seed=1),
                  "WC": I.ic_weighted_cascade(g)}
        seeds = I.uniform_seeds(g.n, 100, 1)
        sd = torch.as_tensor(seeds, device="cuda")
        for mname, p in models.items():
            G = P.cnd_graph_create(g.n, g.row_ptr, g.col, p, None)
            for _ in range(max(3, args.warmup)):  # same arguments as the timed calls (first-use costs)
                P.cnd_ic_simulate_ex(G, sd, 1000, 1, graph=1, edge_checks=True)
            torch.cuda.synchronize()
            reps = max(1, args.steps)
            t0 = time.perf_counter()
            for _ in range(reps):
                r = P.cnd_ic_simulate_ex(G, sd, 1000, 1, graph=1, edge_checks=True)
            torch.cuda.synchronize()
            gpu_ms = (time.perf_counter() - t0) / reps * 1e3
            t0 = time.perf_counter()
            ro = oracle.simulate("ic", g, seeds, 1000, 1, ic_prob=p, level_counts_len=0)
            cpu_ms = (time.perf_counter() - t0) * 1e3
            same = bool(np.array_equal(r.spread.cpu().numpy(), ro.spread))
            cases.append({"graph": gname, "n": g.n, "m": g.m, "ewm": mname, "gpu_ms_per_1000_runs": gpu_ms,
                          "oracle_1_thread_ms": cpu_ms, "speedup": cpu_ms / gpu_ms, "mean_spread": float(ro.spread.mean()),
                          "edge_checks": r.edge_checks, "same_spreads": same})
            P.cnd_graph_destroy(G)
    geo = float(np.exp(np.mean([np.log(c["speedup"]) for c in cases])))
    line = {"metric": "paper run-time table scenario: speedup over the oracle on one host thread (geometric mean)",
            "value": geo, "unit": "x", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": float(np.mean([c["gpu_ms_per_1000_runs"] for c in cases])), "higher_is_better": True,
            "scaling": "replicas only", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": "IC, 1,000 runs, 100 uniform seeds; G(2000, 0.002) and WS(10000, 10, 0.007), "
                                   "undirected edges both ways; TV / UR[0,1] / WC", "name": "table1",
                       "timing": "host wall clock around each call (one CUDA-graph launch), device-resident seeds"},
            "cases": cases,
            "paper_context": "CyNetDiff (Cython, one core) ran 11x / 9x faster than pure Python and 194-327x faster "
                             "than NDlib on these graphs; no absolute times are printed"}
    print(json.dumps(line), flush=True)
    return 0


def run_batch_full(args):
    """The whole batched workload (4,096 seed sets, 7.3 M trials) in one call."""
    import torch
    import paper_2404_17059_gb300 as P
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if rank != 0:
        return 0
    g = I.rmat(20, 1 << 24, graph_seed=1)
    G = P.cnd_graph_create(g.n, g.row_ptr, g.col, I.ic_uniform_random(g, 0.1, graph_seed=1), None)
    so, seeds, tr, keys = I.batch_items(g.n, 4096, 1, 100, (256, 1024, 4096), graph_seed=1)
    sd = torch.as_tensor(seeds, device="cuda")
    P.cnd_ic_simulate_batch(G, so[:9], sd[:so[8]], tr[:8], keys[:8], graph=1, edge_checks=True)  # first-use costs
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r = P.cnd_ic_simulate_batch(G, so, sd, tr, keys, graph=1, edge_checks=True)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    line = {"metric": METRIC, "value": r.edge_checks / dt, "unit": UNIT, "n_gpus": 1, "steps": 1, "warmup": 1,
            "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "replicas only", "vs_baseline": None,
            "dtype": "u64", "data": "synthetic",
            "config": {"workload": f"R-MAT scale 20 ({g.m} directed edges), IC p~U[0,0.1) fp32 per edge; all 4096 "
                                   "seed sets (|S|~U{1..100}, trials from {256,1024,4096}, rng_seed i+1) in one call",
                       "name": "rmat20batch_full", "timing": "host wall clock around the call (one CUDA graph)"},
            "trials_per_s": float(tr.sum()) / dt, "edge_checks": r.edge_checks, "trials": int(tr.sum()),
            "words": int(((tr.astype(np.int64) + 63) // 64).sum()),
            "mean_spread": float(r.spread.to(torch.float64).mean().item())}
    print(json.dumps(line), flush=True)
    return 0


def run_surrogate24(args):
    """Surrogate forward passes over R-MAT-24 (n = 16.8 M nodes, 263 M edges)."""
    import torch
    import paper_2404_17059_gb300 as P
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if rank != 0:
        return 0
    n_sets = args.items or 1000
    g = I.rmat(args.scale, 16 << args.scale, graph_seed=1)
    G = P.cnd_graph_create(g.n, g.row_ptr, g.col, I.ic_uniform(g, 0.01), None)
    sur = P.cnd_sur_create(G, I.surrogate_init(1))
    off, seeds = I.surrogate_pairs(g.n, n_sets, 100, 100, graph_seed=24)
    for i in range(3):
        P.cnd_sur_forward(sur, seeds[off[i]:off[i + 1]], yhat=False)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    spreads = [P.cnd_sur_forward(sur, seeds[off[i]:off[i + 1]], yhat=False)[1] for i in range(n_sets)]
    dt = time.perf_counter() - t0
    per = dt / n_sets
    fwd_bytes = 2 * g.m * (128 + 8) + 2 * g.n * 128 + g.n * (64 + 128) + 2 * g.n * (256 + 128)
    peak, kind = measured_peak()
    line = {"metric": "surrogate inference: seed sets scored per second", "value": n_sets / dt, "unit": "sets/s",
            "n_gpus": 1, "steps": n_sets, "warmup": 3, "ms_per_step": per * 1e3, "higher_is_better": True,
            "scaling": "replicas only", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": f"R-MAT scale {args.scale} edge factor 16 ({g.m} directed edges), IC p=0.01; one "
                                   f"surrogate forward per seed set of 100 distinct uniform nodes, {n_sets} sets",
                       "name": "surrogate24", "timing": "host wall clock of each cnd_sur_forward (seed upload, "
                                                         "all kernels and the spread copy)"},
            "roofline": {"bound": "hbm", "achieved": fwd_bytes / per / 1e9, "peak": peak, "unit": "GB/s",
                         "frac": fwd_bytes / per / 1e9 / peak, "traffic": None,
                         "alg_bytes_per_forward": fwd_bytes,
                         "peak_source": f"{kind} (MEASURED_PEAKS.json hbm_gbs)" if kind == "measured" else "fallback"},
            "predicted_spread_mean": float(np.mean(spreads))}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- our arm
def kernel_name(model, s):
    """The expansion kernel a counted call ran: k_push<0> (IC), k_push<1> (LT, per-trial in-weight
    sums) or k_push<2> (LT, counting form)."""
    if model == "ic":
        return "k_push<0>"
    return "k_push<2>" if s.get("lt_counters") else "k_push<1>"


def alg_bytes(model, s):
    """Bytes the expansion kernel must move, from its own work counters: 8 per work item (row_ptr pair),
    8 per frontier word loaded, 8 per edge read ({col, thr}), 8 per word check (the target's word) and
    16 per IC word update (vis and next read-modify-write), 8 per LT accumulator add (4-byte read-modify-
    write) or 16 per counter-plane update of the LT counting form (8-byte read-modify-write)."""
    base = 8 * s["work_items"] + 8 * s["frontier_words"] + 8 * s["edges_scanned"] + 8 * s["word_checks"]
    if model == "ic":
        return base + 16 * s["updates"]
    return base + (16 if s.get("lt_counters") else 8) * s["updates"]


TRAFFIC_RMAT_SCALE = 21  # the R-MAT workload's DRAM traffic is captured at this scale (small enough for ncu)


def traffic_key(wl, args):
    """Workload key of the ncu traffic records: the R-MAT workload's figures per word check come from the
    scale-21 capture, scaled to the run's word checks (at scale 24 L2 holds a smaller share of the state,
    so the scaled figure is a lower bound)."""
    return f"rmat{TRAFFIC_RMAT_SCALE}" if wl.name == "rmat24" else wl.name


def hbm_bound_rate(peak_gbs, edge_checks, alg_b):
    """Edge checks per second of an expansion that moved only its algorithmic bytes at the HBM peak."""
    return peak_gbs * 1e9 * edge_checks / alg_b if alg_b > 0 else None


def run_ours(args):
    import torch
    import paper_2404_17059_gb300 as P
    from paper_2404_17059_gb300.binding import CND_STATS_COUNT, CND_STATS_TIMING, CndError

    rank, world, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (the engine has no CPU path)")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)

    wl = select_models(make_workload(args.workload, args.trials, args.items, args.lt_trials, args.scale),
                       args.models)
    if wl.batch is not None and world > 1:
        # each rank its own seed sets: a disjoint slice of the 4096-item list
        g = wl.g
        so, seeds, tr, keys = I.batch_items(g.n, 4096, 1, 100, (256, 1024, 4096), graph_seed=1)
        k = len(wl.batch[2])
        a, b = rank * k, (rank + 1) * k
        wl.batch = (so[a:b + 1] - so[a], seeds[so[a]:so[b]], tr[a:b], keys[a:b])
    G = wl.create(P)
    seeds_d = torch.as_tensor(wl.host_seeds(), device=dev)
    if args.profile_calls:
        out = {m: r.stats for m, r in wl.calls(P, G, seeds_d, rank, stats=CND_STATS_COUNT, world=world)}
        torch.cuda.synchronize()
        print(json.dumps({"profile_calls": out, "workload": wl.name, "trials": wl.trials, "src": source_hash()}))
        return 0
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    # step indices: 0 the counted call, then warm-up, timed, graph-mode and end-to-end steps, so that
    # single-seed-set workloads rotate through their trial ranges (Workload.first_trial)
    step = 0
    counted = dict(wl.calls(P, G, seeds_d, rank, stats=CND_STATS_COUNT, step=step, world=world))  # work counts
    for _ in range(args.warmup):
        step += 1
        wl.calls(P, G, seeds_d, rank, step=step, world=world)
    torch.cuda.synchronize()

    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    checks = launches = 0
    exp_ms, exp_n, fin_ms, set_ms, mchecks = {}, {}, {}, {}, {}
    wall0 = time.perf_counter()
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            step += 1
            flush.zero_()  # L2 flush (256 MiB write) outside the timed events
            ev[i][0].record(stream)
            res = wl.calls(P, G, seeds_d, rank, stats=CND_STATS_TIMING, step=step, world=world)
            ev[i][1].record(stream)
            for model, r in res:
                checks += r.edge_checks
                launches += r.stats["launches"]
                exp_ms[model] = exp_ms.get(model, 0.0) + r.stats["expand_ms"]
                exp_n[model] = exp_n.get(model, 0) + r.stats["expand_launches"]
                fin_ms[model] = fin_ms.get(model, 0.0) + r.stats["finalize_ms"]
                set_ms[model] = set_ms.get(model, 0.0) + r.stats["setup_ms"]
                mchecks[model] = mchecks.get(model, 0) + r.edge_checks
        torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if dist:
        dist.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)
    checks_all = float(checks)
    if dist:
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
        c = torch.tensor([checks_all], dtype=torch.float64, device=dev)
        dist.all_reduce(c)
        checks_all = float(c.item())
    value = checks_all / (total_ms / 1e3)
    trials_per_s = world * wl.trials_per_step() * args.steps / (total_ms / 1e3)

    # ---- a few more steps as one CUDA-graph launch per call (device-side step loop; no per-kernel events)
    ng = max(1, args.graph_steps)
    ev_g = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(ng)]
    g_checks = 0
    for i in range(ng):
        step += 1
        flush.zero_()
        ev_g[i][0].record(stream)
        g_checks += sum(r.edge_checks for _, r in wl.calls(P, G, seeds_d, rank, graph=1, step=step, world=world))
        ev_g[i][1].record(stream)
    torch.cuda.synchronize()
    graph_ms = sum(a.elapsed_time(b) for a, b in ev_g)

    # ---- end to end through the host-pointer API (seeds in, spreads / counts / edge checks out)
    seeds_h = wl.host_seeds()
    ne = max(1, args.e2e_steps)
    torch.cuda.synchronize()
    e2e_checks = 0
    t0 = time.perf_counter()
    for i in range(ne):
        step += 1
        e2e_checks += sum(r.edge_checks for _, r in wl.calls(P, G, seeds_h, rank, step=step, world=world))
    e2e_s = time.perf_counter() - t0
    h2d, d2h = wl.io_bytes()

    if dist:
        dist.destroy_process_group()
    if rank != 0:
        return 0

    # ---- roofline of the dominant expansion kernel: algorithmic bytes per edge check counted by the
    # kernels in the counted call, times the timed steps' edge checks, over the timed expansion time
    peak, peak_kind = measured_peak()
    kern = {}
    for model, r in counted.items():
        cs = r.stats
        name = kernel_name(model, cs)
        b_per_check = alg_bytes(model, cs) / max(1, r.edge_checks)
        tb = b_per_check * mchecks[model]  # algorithmic bytes of the timed steps
        n_l = max(1, exp_n[model])
        kern[model] = {"kernel": name, "launches_per_step": n_l / args.steps, "avg_launch_ms": exp_ms[model] / n_l,
                       "alg_bytes_per_launch": tb / n_l, "alg_bytes_per_edge_check": b_per_check,
                       "achieved_gbs": tb / (exp_ms[model] * 1e-3) / 1e9 if exp_ms[model] > 0 else None,
                       "expand_ms_per_step": exp_ms[model] / args.steps,
                       "edge_checks_per_step": mchecks[model] / args.steps,
                       "edge_checks_per_s_expand": mchecks[model] / (exp_ms[model] * 1e-3)
                       if exp_ms[model] > 0 else None,
                       "hbm_bound_edge_checks_per_s": hbm_bound_rate(peak, r.edge_checks, alg_bytes(model, cs)),
                       "finalize_ms_per_step": fin_ms[model] / args.steps,
                       "setup_ms_per_step": set_ms[model] / args.steps,
                       "lt_counters": cs.get("lt_counters", 0) if model == "lt" else None,
                       "passes": cs["passes"], "word_bits": cs["word_bits"], "levels": cs["levels"],
                       "counted_call": {"edge_checks": r.edge_checks,
                                        **{k: cs[k] for k in ("frontier_slots", "work_items", "edges_scanned",
                                                              "frontier_words", "word_checks", "draws", "updates")}}}
    dom = max(kern, key=lambda k: kern[k]["expand_ms_per_step"])
    K = kern[dom]
    ach = K["achieved_gbs"] or 0.0
    cc = K["counted_call"]
    wc_per_launch = cc["word_checks"] / max(1, cc["edge_checks"]) * K["edge_checks_per_step"] / K["launches_per_step"]
    roof = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
            "traffic": ncu_traffic(K["kernel"], traffic_key(wl, args), wc_per_launch), "kernel": K["kernel"],
            "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs, burst copy)" if peak_kind == "measured"
            else "fallback"}
    # the IC push draws Philox-4x32-10 blocks for its coins: where its draws outweigh its bytes it is
    # bound by integer arithmetic, and its roofline is the Philox rate, measured here on this device
    # with the engine's own generator (cnd_philox_rate)
    alu = None
    if "ic" in kern:
        KI = kern["ic"]
        pk, pk_ms = P.cnd_philox_rate(4096)
        pk_g = pk / 1e9
        draws_per_check = KI["counted_call"]["draws"] / max(1, KI["counted_call"]["edge_checks"])
        draws_s = draws_per_check * mchecks["ic"] / max(1e-9, exp_ms["ic"] * 1e-3)
        alu = {"bound": "alu", "achieved": draws_s / 1e9, "peak": pk_g, "unit": "G Philox/s",
               "frac": draws_s / 1e9 / pk_g, "kernel": KI["kernel"],
               "peak_source": f"measured: cnd_philox_rate on this device ({pk_ms:.1f} ms launch; "
                              f"{torch.cuda.get_device_properties(dev).multi_processor_count} SMs)",
               "draws_per_word_check": KI["counted_call"]["draws"] / max(1, KI["counted_call"]["word_checks"])}
        if dom == "ic" and alu["frac"] > roof["frac"]:
            roof, alu = dict(alu, traffic=roof["traffic"], hbm_view={k: roof[k] for k in ("achieved", "peak",
                                                                                     "unit", "frac")}), roof

    # the LT counting push is a stream of scattered 8-byte reads (the target's word of vis) and atomics
    # (counter-plane toggles): its ceiling is the device's rate of such accesses, measured here for
    # uniformly random words of an L2-resident region (32 MiB) and of a DRAM-resident one (4 GiB)
    rnd = None
    if "lt" in kern and kern["lt"]["kernel"] == "k_push<2>" and exp_ms["lt"] > 0:
        KL = kern["lt"]
        cl = KL["counted_call"]
        per_s = mchecks["lt"] / max(1, cl["edge_checks"]) / (exp_ms["lt"] * 1e-3)
        reads, atomics = cl["word_checks"] * per_s / 1e9, cl["updates"] * per_s / 1e9
        try:
            rates = {f"{where}_{op}": P.cnd_random_access_rate(nbytes, op)[0] / 1e9
                     for where, nbytes in (("l2", 32 << 20), ("dram", 4 << 30)) for op in ("read", "atomic")}
        except CndError as e:  # e.g. no room for the 4 GiB region next to a large workload
            rnd = {"kernel": KL["kernel"], "error": str(e)}
        else:
            rnd = {"kernel": KL["kernel"], "unit": "G ops/s", "reads": reads, "atomics": atomics, "measured": rates,
                   "l2_time_frac": reads / rates["l2_read"] + atomics / rates["l2_atomic"],
                   "dram_time_frac": reads / rates["dram_read"] + atomics / rates["dram_atomic"],
                   "note": "reads = word checks, atomics = counter-plane toggles (activations not counted) per "
                           "second of the kernel; *_time_frac = the share of the kernel's time the same accesses "
                           "take at the measured uniformly random rates (cnd_random_access_rate): L2-resident is "
                           "the ceiling, DRAM-resident the floor"}

    cpu = None if args.no_cpu_baseline else cpu_baseline(wl)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": wl.desc, "name": wl.name, "graph_nodes": wl.g.n, "graph_edges": wl.g.m,
                   "graph_sha256": wl.g.digest(), "trials_per_step_per_rank": wl.trials_per_step(),
                   "trials_per_model_per_step": wl.trials, "parallelism": f"trial-sharded x{world}",
                   "call_mode": "host step loop (the default), CUDA events around each expansion launch",
                   "l2": "flushed between timed steps (256 MiB write, outside the step events)"},
        "trials_per_s": trials_per_s,
        "graph_mode": {"steps": ng, "ms_per_step": graph_ms / ng, "value": g_checks * world / (graph_ms / 1e3),
                       "note": "further steps (their own trial ranges), one CUDA-graph launch per call (opts.graph=1)"},
        "edge_checks_per_step": checks_all / args.steps,
        "clocks": clk.summary(),
        "e2e": {"value": world * e2e_checks / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "steps": ne},
        "gpu_launches": launches,
        "roofline": roof,
        "roofline_other": alu,
        "random_access": rnd,
        "kernels": kern,
        "cpu_baseline": cpu,
        "wall_s_timed_region": wall,
        "step_ms": step_ms,
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="rmat24",
                    choices=["ba100k", "rmat24", "rmat20batch", "er1k", "celf_rr7", "surrogate", "surrogate24",
                             "table1", "rmat20batch_full"])
    ap.add_argument("--scale", type=int, default=24, help="rmat24 / surrogate24: R-MAT scale (edge factor 16)")
    ap.add_argument("--models", default="ic,lt", help="single-seed-set workloads: models to run (ic, lt or both)")
    ap.add_argument("--pairs", type=int, default=200_000, help="surrogate: training pairs")
    ap.add_argument("--k", type=int, default=50, help="surrogate: seeds to choose")
    ap.add_argument("--screen", type=int, default=64, help="surrogate: candidates kept by the gradient score")
    ap.add_argument("--exact", type=int, default=8, help="surrogate: candidates simulated per round")
    ap.add_argument("--screen-mode", default="mixed", choices=["gradient", "onehop", "mixed"],
                    help="surrogate: first score of the screen")
    ap.add_argument("--hub-frac", type=float, default=0.5,
                    help="surrogate: share of each training set's seeds drawn in proportion to out-degree")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--trials", type=int, default=0, help="override the workload's (IC) trials per step")
    ap.add_argument("--lt-trials", type=int, default=0, help="override the workload's LT trials per step")
    ap.add_argument("--graph-steps", type=int, default=3, help="extra steps timed in CUDA-graph mode")
    ap.add_argument("--e2e-steps", type=int, default=3, help="extra steps timed end to end through host pointers")
    ap.add_argument("--items", type=int, default=0, help="rmat20batch: seed sets per step (default 64)")
    ap.add_argument("--profile-calls", action="store_true",
                    help="run one counted step only (for ncu captures of its launches)")
    ap.add_argument("--ref-trials", type=int, nargs=2, default=None,
                    help="IC and LT trials per reference step (single-seed-set workloads; default: the "
                         "workload's reference sample, 8 + 8 on R-MAT scale 24: one trial per host thread)")
    args = ap.parse_args()
    if args.warmup < 3:
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "celf_rr7":
        return run_celf(args)
    if args.workload == "surrogate":
        return run_surrogate(args)
    if args.workload == "surrogate24":
        return run_surrogate24(args)
    if args.workload == "table1":
        return run_table1(args)
    if args.workload == "rmat20batch_full":
        return run_batch_full(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
