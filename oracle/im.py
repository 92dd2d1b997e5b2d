"""Lazy-greedy (CELF) influence maximisation on the CPU oracle -- TEST INFRASTRUCTURE ONLY.

Sec. 2 "Influence Maximization": choose |S| = k maximising sigma(S); the paper
applies CELF (Leskovec et al. 2007) in Sec. 4.  sigma is estimated with common
random numbers: every set X is scored by the exact integer
F(X) = sum of the spreads of trials first_trial .. first_trial + n_trials - 1
under one key.  The lazy rule, which fixes the result:
  round 0   gain(v) = F({v}) for every candidate;
  round j   entries ordered by (gain descending, node id ascending); while the
            first entry was last evaluated before round j, re-evaluate the
            stale entries that precede the first fresh one (at most
            eval_batch, in order): gain(v) = F(S + v) - F(S); once the first
            entry is fresh, choose it and add its gain to F(S).
``greedy`` is the plain greedy algorithm (every candidate re-scored every
round), the textbook definition CELF must reproduce when F is submodular.
"""
from __future__ import annotations

import concurrent.futures as _cf
import heapq
import os

import numpy as np

from .oracle import lib, simulate


def _score_sets(model, graph, sets, n_trials, rng_seed, first_trial, threads, kw):
    """F(X) for each X in sets: one single-threaded oracle run per set, sets spread over threads."""
    lib()

    def one(X):
        r = simulate(model, graph, np.asarray(X, dtype=np.int32), n_trials, rng_seed, first_trial=first_trial,
                     level_counts_len=0, **kw)
        return int(r.spread.astype(np.int64).sum())

    if threads <= 1 or len(sets) <= 1:
        return [one(X) for X in sets]
    with _cf.ThreadPoolExecutor(max_workers=threads) as ex:
        return list(ex.map(one, sets))


def celf(model: str, graph, k: int, n_trials: int, rng_seed: int, *, candidates=None, eval_batch: int = 64,
         first_trial: int = 0, threads: int | None = None, **kw):
    """Returns (seeds, F) with F[j] = F(first j+1 seeds), and the number of sets scored."""
    threads = len(os.sched_getaffinity(0)) if threads is None else threads
    cand = list(range(graph.n)) if candidates is None else [int(v) for v in candidates]
    if not 1 <= k <= len(cand):
        raise ValueError("k must be in 1 .. number of candidates")
    args = (model, graph)
    S: list[int] = []
    gains = _score_sets(*args, [[v] for v in cand], n_trials, rng_seed, first_trial, threads, kw)
    evals = len(cand)
    heap = [(-g, v, 0) for g, v in zip(gains, cand)]
    heapq.heapify(heap)
    fS = 0
    seeds, F = [], []
    for j in range(k):
        while heap[0][2] != j:
            stale = []
            while heap and heap[0][2] != j and len(stale) < eval_batch:
                stale.append(heapq.heappop(heap)[1])
            vals = _score_sets(*args, [S + [v] for v in stale], n_trials, rng_seed, first_trial, threads, kw)
            evals += len(stale)
            for v, f in zip(stale, vals):
                heapq.heappush(heap, (-(f - fS), v, j))
        g, v, _ = heapq.heappop(heap)
        S.append(v)
        fS += -g
        seeds.append(v)
        F.append(fS)
    return np.array(seeds, dtype=np.int32), np.array(F, dtype=np.int64), evals


def greedy(model: str, graph, k: int, n_trials: int, rng_seed: int, *, candidates=None, first_trial: int = 0,
           threads: int | None = None, **kw):
    """Plain greedy: each round scores S + v for every remaining candidate; max gain, lowest id on ties."""
    threads = len(os.sched_getaffinity(0)) if threads is None else threads
    cand = list(range(graph.n)) if candidates is None else [int(v) for v in candidates]
    S: list[int] = []
    F = []
    for _ in range(k):
        rest = [v for v in cand if v not in S]
        vals = _score_sets(model, graph, [S + [v] for v in rest], n_trials, rng_seed, first_trial, threads, kw)
        best = max(range(len(rest)), key=lambda i: (vals[i], -rest[i]))
        S.append(rest[best])
        F.append(vals[best])
    return np.array(S, dtype=np.int32), np.array(F, dtype=np.int64)
