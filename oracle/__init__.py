"""CPU oracle for IC/LT Monte Carlo simulation -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The product library (``paper_2404_17059_gb300``)
never imports it and shares no code with it; see ``cnd_oracle.c`` for what is
computed and the readings of the paper it follows.

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
(library Philox, closed forms, brute-force enumeration, exact invariants).
"""
from .oracle import (  # noqa: F401
    build, lib, philox, ic_coin, lt_theta, ic_threshold, simulate, simulate_threads,
    OracleResult, OK, LIMIT, EINVAL, EOVERFLOW,
)
from . import im  # noqa: F401  (lazy-greedy influence maximisation on the oracle)
