"""Worker for the world-size-2 gloo tests of the trial-sharded mode (spawned processes)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


class _OracleRun:
    """simulate() callable backed by the CPU oracle (test-only), matching the binding's keywords."""

    def __init__(self, model, ic_prob=None, lt_weight=None):
        self.model, self.ic_prob, self.lt_weight = model, ic_prob, lt_weight

    def __call__(self, graph, seeds, count, rng_seed, *, first_trial, level_counts_len, edge_checks):
        import oracle
        return oracle.simulate(self.model, graph, seeds, count, rng_seed, ic_prob=self.ic_prob,
                               lt_weight=self.lt_weight, first_trial=first_trial,
                               level_counts_len=level_counts_len)


def run(rank, world, port, backend_path, out_dir, case):
    import numpy as np
    import torch.distributed as dist
    from paper_2404_17059_gb300 import inputs as I
    from paper_2404_17059_gb300 import shard
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        g = I.erdos_renyi_m(400, 3000, graph_seed=3)
        seeds = I.uniform_seeds(g.n, 5, 4)
        n_trials = case["n_trials"]
        model = case["model"]
        kw = {}
        if backend_path == "oracle":
            sim = _OracleRun(model, ic_prob=I.ic_uniform(g, 0.12) if model == "ic" else None,
                             lt_weight=I.lt_weighted_cascade(g) if model == "lt" else None)
        else:
            from paper_2404_17059_gb300 import binding as B
            gd = B.cnd_graph_create(g.n, g.row_ptr, g.col, ic_prob=I.ic_uniform(g, 0.12),
                                    lt_weight_fx=I.lt_weighted_cascade(g))
            sim = None
            g = gd
        r = shard.simulate_sharded(model, g, seeds, n_trials, case["rng_seed"], simulate=sim,
                                   level_counts_len=32, **kw)
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"), spread=r.spread, node_count=r.node_count,
                 edge_checks=r.edge_checks, level_counts=r.level_counts, first=r.first_trial, count=r.n_local)
    finally:
        dist.destroy_process_group()
