"""The measurement probes behind the bench's rooflines: the Philox rate and the
rates of random 8-byte reads and atomics, in and out of L2."""
import pytest

import paper_2404_17059_gb300 as P

pytestmark = pytest.mark.gpu


def test_random_access_rates_are_ordered():
    r = {(where, op): P.cnd_random_access_rate(nbytes, op, iters=64)[0]
         for where, nbytes in (("l2", 32 << 20), ("dram", 1 << 30)) for op in ("read", "atomic")}
    print({f"{w}_{o}": v / 1e9 for (w, o), v in r.items()})
    assert all(v > 1e9 for v in r.values())
    # a region inside L2 serves random accesses faster than one in DRAM
    assert r[("l2", "read")] > r[("dram", "read")] and r[("l2", "atomic")] > r[("dram", "atomic")]


def test_philox_rate_is_positive():
    rate, ms = P.cnd_philox_rate(64)
    assert rate > 1e9 and ms > 0
