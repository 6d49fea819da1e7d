"""Host-side parts of the benchmark that need no GPU: the oracle baselines
(one core and all cores) and the configuration line (CPU only)."""

import synth


def test_cpu_baselines_on_tiny():
    import bench

    t = synth.make_graph("tiny")
    qs = synth.make_queries("tiny", t)
    sample = bench.reference_sample("tiny", qs)
    one = bench.cpu_baseline(t, sample, budget_s=30.0, workload="tiny")
    assert one["value"] > 0 and one["cores"] == 1 and one["kind"] == "oracle"
    assert one["attempted"] == len(sample) and one["nproc"] >= 1
    assert one["sample"].startswith("tiny:")
    allc = bench.cpu_baseline_all_cores(t, qs[: one["attempted"]], max_procs=2)
    assert "error" not in allc, allc
    assert allc["value"] > 0 and allc["cores"] == min(2, len(qs))
    assert f"{len(qs)} queries" in allc["sample"]


def test_workload_config_names_the_workload():
    import bench

    c = bench.workload_config("medium", 40, 10_000_000, 1)
    assert c["queries_per_step"] == 40 and c["triples"] == 10_000_000
    assert "medium" in c["workload"] and "flushed" in c["l2"]
    c = bench.workload_config("large", 20, 300_000_000, 1)
    assert "large" in c["workload"] and "3x10^8" in c["workload"]


def test_reference_sample_leaves_out_queries_above_the_row_cap():
    import bench

    class Q:
        def __init__(self, name, bound):
            self.name, self.bound = name, bound

    qs = [Q("a", 10), Q("b", 1e9), Q("c", None), Q("d", bench.ORACLE_ROW_CAP)]
    s = bench.reference_sample("large", qs)
    assert [q.name for q in s] == ["a", "c", "d"] and s.skipped == ["b"]


def test_reference_arm_prints_one_contract_line():
    """`bench.py --impl reference` (the oracle, host cores) prints one JSON
    line with the contract's keys, the arm's own e2e and cpu_baseline."""
    import json
    import os
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--workload", "tiny",
                        "--steps", "3", "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=root)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "e2e", "cpu_baseline", "impl"):
        assert k in d, k
    assert d["impl"] == "reference" and d["metric"] == "queries/s" and d["steps"] == 3 and d["warmup"] == 3
    assert d["value"] > 0 and d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert "tiny" in d["config"]["workload"] and "reference_sample" in d["config"]
