"""Host logic of bench.py: the algorithmic-byte count of the expansion kernels, the traffic lookup keyed
by the engine sources, model selection and the rotation of trial ranges over steps (no GPU needed)."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_alg_bytes_per_term():
    base = {"work_items": 1, "frontier_words": 0, "edges_scanned": 0, "word_checks": 0, "updates": 0}
    assert bench.alg_bytes("ic", base) == 8
    for key in ("frontier_words", "edges_scanned", "word_checks"):
        s = dict(base, work_items=0, **{key: 1})
        assert bench.alg_bytes("ic", s) == 8 and bench.alg_bytes("lt", s) == 8
    s = dict(base, work_items=0, updates=1)
    assert bench.alg_bytes("ic", s) == 16   # vis and nxt read-modify-write
    assert bench.alg_bytes("lt", s) == 8    # one 4-byte accumulator read and write
    assert bench.alg_bytes("lt", dict(s, lt_counters=1)) == 16  # one 8-byte counter plane read and write


def test_kernel_names():
    assert bench.kernel_name("ic", {}) == "k_push<0>"
    assert bench.kernel_name("lt", {"lt_counters": 0}) == "k_push<1>"
    assert bench.kernel_name("lt", {"lt_counters": 1}) == "k_push<2>"


def test_trial_ranges_rotate_through_the_configuration():
    wl = bench.Workload("x", "", None, {"ic": 1, "lt": 1}, trials={"ic": 2048, "lt": 1000}, total=100_000)
    k_ic = 100_000 // 2048
    firsts = [wl.first_trial("ic", s, 0, 1) for s in range(2 * k_ic)]
    assert firsts[:k_ic] == [2048 * i for i in range(k_ic)] and firsts[k_ic:] == firsts[:k_ic]
    assert all(f + 2048 <= 100_000 for f in firsts)
    # LT ranges are 64-aligned (1000 trials span 1024 ids) and stay inside the configuration too
    lt = [wl.first_trial("lt", s, 0, 1) for s in range(200)]
    assert all(f % 64 == 0 and f + 1000 <= 100_000 for f in lt) and len(set(lt)) == 100_000 // 1024
    # ranks take disjoint ranges within a step
    assert len({wl.first_trial("ic", 3, r, 4) for r in range(4)}) == 4
    # a workload whose steps cover the whole configuration: every step the same ids, ranks their own
    whole = bench.Workload("y", "", None, {"ic": 1}, trials={"ic": 1000}, total=1000)
    assert [whole.first_trial("ic", s, 0, 1) for s in range(3)] == [0, 0, 0]
    assert whole.first_trial("ic", 0, 2, 4) == 2 * 1024


def test_traffic_lookup_needs_the_current_sources(tmp_path, monkeypatch):
    cur = bench.source_hash()
    assert len(cur) == 12
    prof = tmp_path / "profiles"
    prof.mkdir()
    lines = ["# comment", json.dumps({"kernel": "k_push<1>", "workload": "ba100k", "src": cur,
                                      "dram_bytes_per_word_check": 100.0}),
             json.dumps({"kernel": "k_push<0>", "workload": "ba100k", "src": "000000000000",
                         "dram_bytes_per_word_check": 10.0})]
    (prof / "traffic.txt").write_text("\n".join(lines) + "\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "source_hash", lambda: cur)
    assert bench.ncu_traffic("k_push<1>", "ba100k", 3.0) == 300.0
    assert bench.ncu_traffic("k_push<0>", "ba100k", 3.0) is None   # taken on other sources
    assert bench.ncu_traffic("k_push<1>", "rmat24", 3.0) is None


def test_committed_traffic_matches_the_engine():
    """The committed traffic figures of the default workload's expansion kernels were taken on the current
    engine sources (a smaller R-MAT of the same generator, scale 21, keeps the capture small)."""
    assert bench.ncu_traffic("k_push<0>", "rmat21", 1.0) is not None
    assert bench.ncu_traffic("k_push<2>", "rmat21", 1.0) is not None


def test_select_models():
    wl = bench.make_workload("er1k")
    assert set(m for m, d in wl.models.items() if d is not None) == {"ic", "lt"}
    wl = bench.select_models(bench.make_workload("er1k"), "lt")
    assert wl.models["ic"] is None and wl.models["lt"] is not None
    assert wl.trials_per_step() == 1000
    with pytest.raises(SystemExit):
        bench.select_models(bench.make_workload("er1k"), "xx")


def test_hbm_bound_rate():
    # 1e9 edge checks moving 21.8e9 algorithmic bytes at 6,663.9 GB/s: 21.8e9 / 6663.9e9 s
    assert bench.hbm_bound_rate(6663.9, 1e9, 21.8e9) == pytest.approx(1e9 / (21.8e9 / 6663.9e9))
    assert bench.hbm_bound_rate(6663.9, 1e9, 0) is None


def test_reference_arm_json_contract():
    """`bench.py --impl reference` (the oracle, CPU only) prints one JSON line with the contract's keys."""
    import subprocess
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "er1k",
                          "--steps", "1", "--warmup", "3"], capture_output=True, text=True, timeout=600, check=True)
    lines = [ln for ln in out.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 1 and d["warmup"] == 3 and d["value"] > 0
    assert d["config"]["workload"] and d["config"]["graph_sha256"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
