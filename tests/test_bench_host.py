"""Host-side parts of the benchmark that need no GPU: the oracle baselines
(one core and all cores) and the configuration line (CPU only)."""

import synth


def test_cpu_baselines_on_tiny():
    import bench

    t = synth.make_graph("tiny")
    qs = synth.make_queries("tiny", t)
    one = bench.cpu_baseline(t, qs, budget_s=30.0)
    assert one["value"] > 0 and one["cores"] == 1 and one["kind"] == "oracle"
    assert one["attempted"] == len(qs) and one["nproc"] >= 1
    allc = bench.cpu_baseline_all_cores(t, qs[: one["attempted"]], max_procs=2)
    assert "error" not in allc, allc
    assert allc["value"] > 0 and allc["cores"] == min(2, len(qs))
    assert f"{len(qs)} queries" in allc["sample"]


def test_workload_config_names_the_workload():
    import bench

    c = bench.workload_config(40, 10_000_000, 1)
    assert c["queries_per_step"] == 40 and c["triples"] == 10_000_000
    assert "medium" in c["workload"] and "flushed" in c["l2"]
