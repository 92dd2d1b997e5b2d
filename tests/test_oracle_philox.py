"""Pins of the oracle's random numbers and of its IC probability -> threshold map.

* Philox4x32-10 against an independent library implementation (triton's
  ``tl.philox`` run on the CPU by triton's interpreter).
* The counter layout of IC coins and LT thresholds (trial group, lane, domain,
  high counter word) against that same library routine.
* Uniformity of the coins (chi-square).
* The threshold map floor(p * 2^32) against exact rational arithmetic.
"""
import fractions
import os
import subprocess
import sys
import tempfile

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
SEEDS = np.array([0, 1, 2, 0xDEADBEEF, 0x123456789ABCDEF0, (1 << 64) - 1, 1 << 63], dtype=np.uint64)


def _triton_philox(ctr: np.ndarray, seeds: np.ndarray) -> np.ndarray:
    pytest.importorskip("triton")
    with tempfile.TemporaryDirectory() as d:
        inp = os.path.join(d, "in.npz")
        outp = os.path.join(d, "out.npz")
        np.savez(inp, ctr=ctr.astype(np.uint32), seeds=seeds.astype(np.uint64))
        env = dict(os.environ, TRITON_INTERPRET="1")
        subprocess.check_call([sys.executable, os.path.join(HERE, "_triton_philox.py"), inp, outp], env=env)
        return np.load(outp)["out"]


@pytest.fixture(scope="module")
def triton_cases():
    rng = np.random.default_rng(7)
    ctr = rng.integers(0, 1 << 32, size=(256, 4), dtype=np.uint64).astype(np.uint32)
    ctr[0] = 0
    ctr[1] = 0xFFFFFFFF
    ctr[2] = [1, 0, 0, 0]
    ctr[3] = [0, 0, 1, 0]
    ref = _triton_philox(ctr, SEEDS)
    return ctr, ref


def test_philox_matches_library(triton_cases):
    ctr, ref = triton_cases
    for i, s in enumerate(SEEDS.tolist()):
        got = oracle.philox(ctr, s)
        assert np.array_equal(got, ref[i]), f"seed {s:#x}"


def test_coin_and_theta_counter_layout(triton_cases):
    # Build the counters for (trial, index, domain) the way the definition says and let the
    # library compute them; the oracle's coin/theta must pick lane t & 3 of that block.
    rng = np.random.default_rng(11)
    trials = np.concatenate([np.arange(16), rng.integers(0, 1 << 40, size=48)]).astype(np.int64)
    trials[-4:] = [(1 << 34) + 3, (1 << 34) + 4, (1 << 36) + 1, (1 << 40) - 1]
    index = rng.integers(0, 1 << 31, size=trials.size).astype(np.int64)
    rows = []
    for dom in (0, 1):
        for t, e in zip(trials.tolist(), index.tolist()):
            g = t >> 2
            rows.append([e & 0xFFFFFFFF, g & 0xFFFFFFFF, dom, g >> 32])
    rows = np.array(rows, dtype=np.uint64)
    k = 1
    while k < len(rows):
        k *= 2
    pad = np.zeros((k, 4), dtype=np.uint64)
    pad[: len(rows)] = rows
    seeds = np.array([1, 0xFEEDFACECAFEBEEF], dtype=np.uint64)
    ref = _triton_philox(pad.astype(np.uint32), seeds)
    for si, s in enumerate(seeds.tolist()):
        for j, (t, e) in enumerate(zip(trials.tolist(), index.tolist())):
            assert oracle.ic_coin(s, t, e) == ref[si, j, t & 3]
            assert oracle.lt_theta(s, t, e) == ref[si, trials.size + j, t & 3]


def test_coin_uniformity_chi2():
    from scipy import stats
    n_edges, n_trials = 64, 4096
    ctr = np.zeros((n_edges * n_trials // 4, 4), dtype=np.uint32)
    ctr[:, 0] = np.repeat(np.arange(n_edges), n_trials // 4)
    ctr[:, 1] = np.tile(np.arange(n_trials // 4), n_edges)
    u = oracle.philox(ctr, 1).ravel()
    bins = np.bincount((u >> 24).astype(np.int64), minlength=256)
    chi2 = ((bins - u.size / 256) ** 2 / (u.size / 256)).sum()
    p = stats.chi2.sf(chi2, 255)
    assert 1e-6 < p < 1 - 1e-6, (chi2, p)
    # every output bit is balanced
    bits = ((u[:, None] >> np.arange(32, dtype=np.uint32)) & 1).mean(axis=0)
    assert np.all(np.abs(bits - 0.5) < 5 * 0.5 / np.sqrt(u.size))


def _exact_thr(p: np.float32) -> int:
    if p == np.float32(1.0):
        return 0xFFFFFFFF
    return int(fractions.Fraction(float(p)) * (1 << 32))  # int() floors a non-negative Fraction


def test_threshold_exact():
    rng = np.random.default_rng(3)
    ps = list(rng.random(2000, dtype=np.float32))
    ps += [np.float32(0.0), np.float32(1.0), np.float32(0.5), np.float32(0.1), np.float32(0.01),
           np.float32(1e-3), np.nextafter(np.float32(1.0), np.float32(0.0)),
           np.float32(np.finfo(np.float32).tiny), np.float32(1.4e-45), np.float32(2.0 ** -32),
           np.float32(2.0 ** -33), np.float32(3 * 2.0 ** -33)]
    ps = np.array(ps, dtype=np.float32)
    got = oracle.ic_threshold(ps)
    want = np.array([_exact_thr(p) for p in ps], dtype=np.uint64)
    assert np.array_equal(got.astype(np.uint64), want)
    below_one = ps < np.float32(1.0)
    assert np.all(got[below_one] < 0xFFFFFFFF)
    assert got[ps == np.float32(0.0)][0] == 0
