#!/usr/bin/env python
"""Throughput of Monte Carlo IC + LT simulation on GB300 (one JSON line).

A step is one pass of the whole path over one batch: an IC simulation and an
LT simulation of the same workload (graph ingest happens once, before the
timed region).  Default workload: Barabasi-Albert n=100,000 with 5
attachments, undirected edges stored both ways (999,950 directed edges);
weighted-cascade IC probabilities (fp32) and LT weights (uint32 fixed point);
the 50 highest-degree nodes as seeds; 10,000 trials of each model.

value  = edge checks per second over the whole job (IC + LT, all ranks),
         device-resident inputs, CUDA-event time of each step, L2 flushed
         between steps.
e2e    = the same metric through the host-pointer C-ABI calls (seeds copied
         in, spreads / counts / edge checks copied out inside the timed region).
roofline = the dominant expansion kernel: algorithmic bytes it must move
         (counted by the kernels themselves) / its CUDA-event time.
cpu_baseline = the CPU oracle on a bounded sample of the same workload, on
         all host cores.

--impl reference times the CPU oracle alone (each step a bounded sample).
Multi-GPU (torchrun): every rank simulates its own trial range of the same
workload (weak scaling, no collective on the data path).
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
def make_workload(name: str):
    if name == "ba100k":
        g = I.barabasi_albert(100_000, 5, graph_seed=1)
        return dict(
            name=name, g=g, p=I.ic_weighted_cascade(g), w=I.lt_weighted_cascade(g),
            seeds=I.top_degree_seeds(g, 50), trials=10_000, rng_seed=1,
            desc=(f"BA n=100000 m_attach=5 symmetrised ({g.m} directed edges), weighted-cascade IC (fp32 p=1/indeg) "
                  "and LT (uint32 floor((2^32-1)/indeg)), 50 top-degree seeds, 10000 trials per model, rng_seed=1"),
            cpu_trials=(2048, 1536))
    if name == "er1k":
        g = I.erdos_renyi_m(1000, 10_000, graph_seed=1)
        return dict(
            name=name, g=g, p=I.ic_uniform(g, 0.1), w=I.lt_weighted_cascade(g),
            seeds=I.uniform_seeds(g.n, 10, 1), trials=1000, rng_seed=1,
            desc="directed ER n=1000 m=10000, IC p=0.1, LT weighted cascade, 10 uniform seeds, 1000 trials per model",
            cpu_trials=(1000, 1000))
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


def source_hash() -> str:
    h = hashlib.sha256()
    for fn in sorted(os.listdir(os.path.join(ROOT, "paper_2404_17059_gb300", "csrc"))):
        with open(os.path.join(ROOT, "paper_2404_17059_gb300", "csrc", fn), "rb") as f:
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


def cpu_baseline(wl, rank):
    """The oracle, as it stands, on a bounded sample of the workload's trials over all host cores."""
    import oracle
    cores = len(os.sched_getaffinity(0))
    n_ic, n_lt = wl["cpu_trials"]
    t0 = time.perf_counter()
    a = oracle.simulate_threads("ic", wl["g"], wl["seeds"], n_ic, wl["rng_seed"], ic_prob=wl["p"], threads=cores,
                                level_counts_len=0)
    b = oracle.simulate_threads("lt", wl["g"], wl["seeds"], n_lt, wl["rng_seed"], lt_weight=wl["w"],
                                threads=cores, level_counts_len=0)
    dt = time.perf_counter() - t0
    checks = a.edge_checks + b.edge_checks
    return {"value": checks / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"trials 0..{n_ic - 1} (IC) and 0..{n_lt - 1} (LT) of the same workload, {checks} edge checks "
                      f"in {dt:.2f} s wall on {cores} threads",
            "trials_per_s": (n_ic + n_lt) / dt}


# ----------------------------------------------------------------------------- reference arm
def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    wl = make_workload(args.workload)
    cores = len(os.sched_getaffinity(0))
    n_ic, n_lt = args.ref_trials
    times, checks = [], 0
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        a = oracle.simulate_threads("ic", wl["g"], wl["seeds"], n_ic, wl["rng_seed"], ic_prob=wl["p"],
                                    threads=cores, level_counts_len=0, first_trial=64 * i)
        b = oracle.simulate_threads("lt", wl["g"], wl["seeds"], n_lt, wl["rng_seed"], lt_weight=wl["w"],
                                    threads=cores, level_counts_len=0, first_trial=64 * i)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
            checks += a.edge_checks + b.edge_checks
    total = sum(times)
    value = checks / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": wl["desc"], "sample_per_step": f"{n_ic} IC + {n_lt} LT trials"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{n_ic} IC + {n_lt} LT trials per step over {cores} threads"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- our arm
def run_ours(args):
    import torch
    import paper_2404_17059_gb300 as P
    from paper_2404_17059_gb300.binding import CND_STATS_COUNT, CND_STATS_TIMING

    rank, world, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (the engine has no CPU path)")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)

    wl = make_workload(args.workload)
    if args.trials:
        wl["trials"] = args.trials
    g, T = wl["g"], wl["trials"]
    G = P.cnd_graph_create(g.n, g.row_ptr, g.col, wl["p"], wl["w"])
    if args.profile_calls:
        # one IC and one LT call with kernel-counted work (for ncu captures of those launches)
        seeds_d = torch.as_tensor(wl["seeds"], device=dev)
        out = {}
        for model, f in (("ic", P.cnd_ic_simulate_ex), ("lt", P.cnd_lt_simulate_ex)):
            r = f(G, seeds_d, T, wl["rng_seed"], edge_checks=True, stats=CND_STATS_COUNT)
            out[model] = r.stats
        torch.cuda.synchronize()
        print(json.dumps({"profile_calls": out, "workload": wl["name"], "trials": T, "src": source_hash()}))
        return 0
    seeds_d = torch.as_tensor(wl["seeds"], device=dev)
    first = rank * (((T + 63) // 64) * 64)  # each rank its own trial range
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def step(stats=0):
        r_ic = P.cnd_ic_simulate_ex(G, seeds_d, T, wl["rng_seed"], first_trial=first, edge_checks=True,
                                    stats=stats)
        r_lt = P.cnd_lt_simulate_ex(G, seeds_d, T, wl["rng_seed"], first_trial=first, edge_checks=True,
                                    stats=stats)
        return r_ic, r_lt

    # work counts for the roofline (untimed)
    c_ic, c_lt = step(stats=CND_STATS_COUNT)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    checks = 0
    launches = 0
    exp_ms = {"ic": 0.0, "lt": 0.0}
    exp_n = {"ic": 0, "lt": 0}
    fin_ms = {"ic": 0.0, "lt": 0.0}
    wall0 = time.perf_counter()
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            flush.zero_()  # L2 flush (256 MiB write) outside the timed events
            ev[i][0].record(stream)
            r_ic, r_lt = step(stats=CND_STATS_TIMING)
            ev[i][1].record(stream)
            checks += r_ic.edge_checks + r_lt.edge_checks
            for k, r in (("ic", r_ic), ("lt", r_lt)):
                launches += r.stats["launches"]
                exp_ms[k] += r.stats["expand_ms"]
                exp_n[k] += r.stats["expand_launches"]
                fin_ms[k] += r.stats["finalize_ms"]
        torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if dist:
        dist.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)
    if dist:
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
        c = torch.tensor([checks], dtype=torch.float64, device=dev)
        dist.all_reduce(c)
        checks_all = float(c.item())
    else:
        checks_all = float(checks)
    value = checks_all / (total_ms / 1e3)
    trials_per_s = world * 2 * T * args.steps / (total_ms / 1e3)

    # ---- end to end through the host-pointer API
    seeds_h = wl["seeds"]
    torch.cuda.synchronize()
    e2e_checks = 0
    t0 = time.perf_counter()
    for i in range(args.steps):
        a = P.cnd_ic_simulate_ex(G, seeds_h, T, wl["rng_seed"], first_trial=first, edge_checks=True)
        b = P.cnd_lt_simulate_ex(G, seeds_h, T, wl["rng_seed"], first_trial=first, edge_checks=True)
        e2e_checks += a.edge_checks + b.edge_checks
    e2e_s = time.perf_counter() - t0
    h2d = 2 * seeds_h.size * 4
    d2h = 2 * (T * 4 + g.n * 4 + 8)

    if dist:
        dist.destroy_process_group()
    if rank != 0:
        return 0

    # ---- roofline of the dominant expansion kernel (algorithmic bytes counted by the kernels)
    def alg_bytes(model, s):
        base = 8 * s["work_items"] + 8 * s["frontier_words"] + 8 * s["edges_scanned"] + 8 * s["word_checks"]
        return base + (16 if model == "ic" else 8) * s["updates"]

    peak, peak_kind = measured_peak()
    kern = {}
    for model, cs in (("ic", c_ic.stats), ("lt", c_lt.stats)):
        n_l = max(1, cs["expand_launches"])
        bpl = alg_bytes(model, cs) / n_l
        avg_ms = exp_ms[model] / max(1, exp_n[model])
        kern[model] = {"kernel": "k_push<0>" if model == "ic" else "k_push<1>", "launches_per_step": n_l,
                       "avg_launch_ms": avg_ms, "alg_bytes_per_launch": bpl,
                       "achieved_gbs": bpl / (avg_ms * 1e-3) / 1e9 if avg_ms > 0 else None,
                       "expand_ms_per_step": exp_ms[model] / args.steps,
                       "finalize_ms_per_step": fin_ms[model] / args.steps,
                       "counts": {k: cs[k] for k in ("frontier_slots", "work_items", "edges_scanned",
                                                     "frontier_words", "word_checks", "draws", "updates")}}
    dom = max(kern, key=lambda k: kern[k]["expand_ms_per_step"])
    K = kern[dom]
    ach = K["achieved_gbs"] or 0.0
    wc_per_launch = K["counts"]["word_checks"] / max(1, K["launches_per_step"])
    roof = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
            "traffic": ncu_traffic(K["kernel"], wl["name"], wc_per_launch), "kernel": K["kernel"],
            "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else "fallback"}

    cpu = None if args.no_cpu_baseline else cpu_baseline(wl, rank)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": wl["desc"], "name": wl["name"], "graph_nodes": g.n, "graph_edges": g.m,
                   "trials_per_model_per_rank": T, "parallelism": f"trial-sharded x{world}",
                   "l2": "flushed between timed steps (256 MiB write, outside the step events)",
                   "word_bits": c_ic.stats["word_bits"]},
        "trials_per_s": trials_per_s,
        "edge_checks_per_step": checks_all / args.steps,
        "clocks": clk.summary(),
        "e2e": {"value": world * e2e_checks / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "roofline": roof,
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
    ap.add_argument("--workload", default="ba100k", choices=["ba100k", "er1k"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--trials", type=int, default=0, help="override the workload's trials per model")
    ap.add_argument("--profile-calls", action="store_true",
                    help="run one counted IC and one counted LT call only (for ncu captures)")
    ap.add_argument("--ref-trials", type=int, nargs=2, default=(384, 256),
                    help="IC and LT trials per reference step")
    args = ap.parse_args()
    if args.warmup < 3:
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
