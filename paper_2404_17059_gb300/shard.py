"""Trial-sharded multi-process mode: one process per GPU, one contiguous trial range each.

Trials are independent and each is a pure function of (rng_seed, trial index)
(Sec. 2: every trial is its own run of the diffusion process), so a job of T
trials splits into per-rank ranges [first, first + count) passed as
``first_trial``.  Concatenating the ranks' spreads in rank order and summing
their per-node counts, edge checks and per-step counts gives exactly the
single-process result.  The only exchange is that host-side sum and
concatenation, done over a CPU (gloo) process group: no device collective
is on the data path.
"""
from __future__ import annotations

import dataclasses

import numpy as np

WORD = 64  # trials per bit-parallel word: ranges start on word boundaries


def trial_shard(n_trials: int, rank: int, world: int, align: int = WORD) -> tuple[int, int]:
    """(first_trial, count) of ``rank``'s contiguous share of ``n_trials`` trials.

    Shares are whole multiples of ``align`` trials except the last non-empty
    one, and differ by at most ``align`` trials; trailing ranks may get none.
    """
    if n_trials < 0 or world < 1 or not 0 <= rank < world or align < 1:
        raise ValueError("trial_shard: need n_trials >= 0, world >= 1, 0 <= rank < world, align >= 1")
    units = -(-n_trials // align)
    lo = units * rank // world
    hi = units * (rank + 1) // world
    first = min(lo * align, n_trials)
    return first, min(hi * align, n_trials) - first


@dataclasses.dataclass
class ShardedResult:
    spread: np.ndarray        # int32 [n_trials], all ranks' trials in order
    node_count: np.ndarray    # int64 [n], summed over ranks
    edge_checks: int
    level_counts: np.ndarray | None
    first_trial: int          # this rank's range
    n_local: int


_GLOO = {}


def _cpu_group(group):
    """The gloo group the exchange runs on: ``group`` itself when it is gloo."""
    import torch.distributed as dist
    if dist.get_backend(group) == "gloo":
        return group
    key = id(group)
    if key not in _GLOO:
        ranks = None if group is None else dist.get_process_group_ranks(group)
        _GLOO[key] = dist.new_group(ranks=ranks, backend="gloo")
    return _GLOO[key]


def exchange(spread_local, node_count_local, edge_checks_local: int, level_counts_local=None, *, group=None):
    """Concatenate spreads in rank order and sum counts over the ranks of ``group`` (host side)."""
    import torch
    import torch.distributed as dist
    grp = _cpu_group(group)
    world = dist.get_world_size(grp)
    sp = torch.as_tensor(np.asarray(spread_local, dtype=np.int32).ravel())
    lens = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(lens, torch.tensor([sp.numel()], dtype=torch.int64), group=grp)
    width = max(int(x.item()) for x in lens)
    padded = torch.zeros(width, dtype=torch.int32)
    padded[:sp.numel()] = sp
    parts = [torch.zeros(width, dtype=torch.int32) for _ in range(world)]
    dist.all_gather(parts, padded, group=grp)
    spread = torch.cat([p[:int(n.item())] for p, n in zip(parts, lens)]).numpy()
    nc = torch.as_tensor(np.asarray(node_count_local, dtype=np.int64).ravel()).clone()
    dist.all_reduce(nc, group=grp)
    ec = torch.tensor([int(edge_checks_local)], dtype=torch.int64)
    dist.all_reduce(ec, group=grp)
    lc = None
    if level_counts_local is not None:
        lc_t = torch.as_tensor(np.asarray(level_counts_local, dtype=np.int64).ravel()).clone()
        dist.all_reduce(lc_t, group=grp)
        lc = lc_t.numpy()
    return spread, nc.numpy(), int(ec.item()), lc


def simulate_sharded(model: str, graph, seeds, n_trials: int, rng_seed: int, *, group=None, simulate=None,
                     level_counts_len: int = 0, **kw) -> ShardedResult:
    """Run this rank's share of ``n_trials`` trials and exchange the results with the other ranks.

    ``simulate(graph, seeds, count, rng_seed, first_trial=, level_counts_len=, **kw)`` runs
    the local share and returns an object with ``spread``, ``node_count``,
    ``edge_checks`` and ``level_counts``; by default it is ``cnd_ic_simulate_ex`` or
    ``cnd_lt_simulate_ex`` of this package (host arrays in and out).
    """
    import torch.distributed as dist
    rank = dist.get_rank(group)
    world = dist.get_world_size(group)
    first, count = trial_shard(int(n_trials), rank, world)
    if simulate is None:
        from . import binding
        simulate = {"ic": binding.cnd_ic_simulate_ex, "lt": binding.cnd_lt_simulate_ex}[model]
    r = simulate(graph, seeds, count, rng_seed, first_trial=first, level_counts_len=level_counts_len,
                 edge_checks=True, **kw)
    lc = r.level_counts if level_counts_len else None
    spread, nc, ec, lc = exchange(r.spread, r.node_count, r.edge_checks, lc, group=group)
    return ShardedResult(spread, nc, ec, lc, first, count)
