"""Benchmark of the SM-based BGP join on one B300 (or N replicas).

A step is one pass of the whole hot path over one workload: gsmat_load of
the device-resident triples (sort, dedupe, CSR/CSC, predicate index)
followed by every BGP of the workload (plan, joins, canonical sort), each
result left on the device.  The headline workload is the largest
configuration, large (4x10^7 entities, 256 predicates, 3x10^8 distinct int32
triples; 20 anchored BGPs of 4-8 patterns); the medium one (10^7 triples,
40 BGPs) is reported beside it.  The metric is queries/s of whole steps;
result rows/s, per-query p50/p99 latency, an end-to-end figure with host
buffers and the dominant kernel family's HBM roofline come with it, then
the batched mix, the planners, the front end, row shards and the served
arrivals.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload large|medium]
                    [--impl gsmat|reference]

--impl reference times the CPU oracle (the plain nested-loop join over the
raw triple list; the paper publishes no code) on the host cores, on the
same sample of the workload as the cpu_baseline field.
Multi-GPU (torchrun): every rank runs the same workload on its own GPU
(independent replicas, no collective on the data path); value = all ranks'
queries / max rank time.
"""

from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "queries/s"
L2_FLUSH_BYTES = 256 << 20


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _workload(name):
    import synth

    t0 = time.time()
    triples = synth.make_graph(name)
    queries = synth.make_large_queries(triples) if name == "large" else synth.make_queries(name, triples)
    return triples, queries, time.time() - t0


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks/throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": []}
        try:
            rows = [l.strip().split(",") for l in open(self.path) if l.strip()]
            os.unlink(self.path)
        except Exception:
            return out
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except Exception:
                continue
            for name, val in zip(names, r[5:9]):
                if val.lower() in ("active", "1"):
                    reasons.add(name)
        if sm:
            out["sm_mhz"] = float(np.median(sm))
            out["sm_max_mhz"] = float(max(mx))
            out["samples"] = len(sm)
        out["reasons"] = sorted(reasons)
        return out


def reduce_over_ranks(my_ms: float, my_rows: int, device: str = "cpu"):
    """Max of the ranks' timed milliseconds and sum of their result rows
    (replicas: every rank runs the whole workload; the slowest rank sets the
    job's time).  Identity when torch.distributed is not initialised."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(my_ms), int(my_rows)
    t = torch.tensor([float(my_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    r = torch.tensor([int(my_rows)], dtype=torch.int64, device=device)
    dist.all_reduce(r, op=dist.ReduceOp.SUM)
    return float(t.item()), int(r.item())


def job_value(world_size: int, steps: int, queries_per_step: int, total_ms: float) -> float:
    """Whole-job queries/s: all ranks' queries over the slowest rank's time."""
    return world_size * steps * queries_per_step / (total_ms / 1e3)


def _flush_l2(torch, buf):
    buf.add_(1)


def plain_leg(args, gs, torch, name, triples, queries, stream, ws, local, steps, warmup):
    """The plain path on one workload: `warmup` untimed steps, then `steps`
    timed steps (gsmat_load of the device-resident triples + every BGP,
    sorted results left on the device), each bracketed by CUDA events on the
    launching stream with L2 flushed (256 MB write) before it; per-query
    device latency; per-kernel-family event times; the library's launch
    count; then the same steps end to end through the public API with host
    buffers (pinned triples in, every result copied to pinned host memory)."""
    nq = len(queries)
    d_tri = torch.from_numpy(np.array(triples, copy=True)).cuda()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    marsh = [gs.Store.marshal(q) for q in queries]  # BGPs converted to the C layout once
    # tile shapes: tuned once on this workload (untimed), set on every step's store
    S0 = gs.Store(d_tri, stream=stream)
    t0 = time.perf_counter()
    tiles = S0.tiles() if args.no_tune else S0.tune(queries, stream=stream)
    tune_s = time.perf_counter() - t0
    S0.free()

    n_streams = max(1, int(getattr(args, "query_streams", 1)))
    qstreams = [torch.cuda.Stream() for _ in range(n_streams)] if n_streams > 1 else []

    def step(lat=None):
        S = gs.Store(d_tri, stream=stream)
        S.set_tiles(**tiles)
        tabs = []
        rows = 0
        if n_streams == 1:
            for q in marsh:
                if lat is not None:
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                T = S.query_raw(q, stream=stream)
                if lat is not None:
                    e1.record(stream)
                    lat.append((e0, e1))
                rows += T.rows
                tabs.append(T)
        else:
            # the step's queries are independent: host threads, each with
            # its own stream, take them in workload order as they free up
            # (one thread's host round trips overlap another's kernels)
            import threading

            built = torch.cuda.Event()
            built.record(stream)
            nxt = [0]
            lock = threading.Lock()

            def worker(st):
                torch.cuda.set_device(st.device)  # a new thread starts on device 0
                st.wait_event(built)
                out = []
                while True:
                    with lock:
                        qi = nxt[0]
                        nxt[0] += 1
                    if qi >= len(marsh):
                        return out
                    e0 = e1 = None
                    if lat is not None:
                        e0 = torch.cuda.Event(enable_timing=True)
                        e1 = torch.cuda.Event(enable_timing=True)
                        e0.record(st)
                    T = S.query_raw(marsh[qi], stream=st)
                    if lat is not None:
                        e1.record(st)
                    out.append((T, e0, e1))

            res = [None] * n_streams
            ths = [threading.Thread(target=lambda w=w: res.__setitem__(w, worker(qstreams[w])))
                   for w in range(n_streams)]
            for th in ths:
                th.start()
            for th in ths:
                th.join()
            for st in qstreams:
                stream.wait_stream(st)
            for part in res:
                for T, e0, e1 in part:
                    rows += T.rows
                    tabs.append(T)
                    if lat is not None:
                        lat.append((e0, e1))
        for T in tabs:
            T.free()
        S.free()
        return rows

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            import torch.distributed as dist

            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(warmup):
        step()
    barrier()
    gs.profile_read(reset=True)
    gs.profile_enable(True)
    step_ms = []
    lat = []
    rows_total = 0
    with ClockSampler(local) as clk:
        barrier()
        lc0 = gs.launch_count()
        for _ in range(steps):
            _flush_l2(torch, flush)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            rows_total += step(lat=lat)
            b.record(stream)
            b.synchronize()
            step_ms.append(a.elapsed_time(b))
        lc1 = gs.launch_count()
        barrier()
    gs.profile_enable(False)
    prof = gs.profile_read(reset=True)
    del flush
    my_ms = float(sum(step_ms))
    total_ms, _ = reduce_over_ranks(my_ms, rows_total, device="cuda")
    q_lat = np.array([e0.elapsed_time(e1) for (e0, e1) in lat])

    # end to end: H2D of the triples inside gsmat_load, D2H of every result
    # table into pinned host memory on a second stream while the next query
    # computes; the step ends when the last copy has landed
    h_tri = torch.from_numpy(np.array(triples, copy=True)).pin_memory()
    e2e_ms = []
    d2h = 0
    host_out = {}  # pinned result buffers, allocated in the first (untimed) pass
    copy_stream = torch.cuda.Stream()
    for it in range(1 + max(1, min(steps, 3))):
        barrier()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        S = gs.Store(h_tri.numpy(), stream=stream)
        S.set_tiles(**tiles)
        d2h = 0
        held = []
        for qi, q in enumerate(marsh):
            T = S.query_raw(q, stream=stream)  # returns with `stream` synchronised
            rows, cols = T.shape
            if qi not in host_out or host_out[qi].numel() < rows * cols:
                host_out[qi] = torch.empty(max(1, rows * cols), dtype=torch.int32).pin_memory()
            T.copy_to(host_out[qi], stream=copy_stream, sync=False)
            d2h += rows * cols * 4
            held.append(T)
        copy_stream.synchronize()
        for T in held:
            T.free()
        S.free()
        b.record(stream)
        b.synchronize()
        if it > 0:
            e2e_ms.append(a.elapsed_time(b))
    del host_out, h_tri
    launches = int(lc1 - lc0)
    return {
        "name": name,
        "value": job_value(ws, steps, nq, total_ms),
        "total_ms": total_ms,
        "steps": steps,
        "step_ms": step_ms,
        "rows_total": rows_total,
        "q_lat": q_lat,
        "prof": prof,
        "launches": launches,
        "clocks": clk.summary(),
        "e2e": {"value": round(nq / (float(np.median(e2e_ms)) / 1e3), 2), "unit": "queries/s",
                "h2d_bytes_per_step": int(np.asarray(triples).nbytes), "d2h_bytes_per_step": int(d2h),
                "ms_per_step": round(float(np.median(e2e_ms)), 3)},
        "d_tri": d_tri,
        "tiles": dict(tiles, tune_s=round(tune_s, 2)),
        "nq": nq,
        "n_triples": int(np.asarray(triples).shape[0]),
    }


# DRAM bytes / algorithmic bytes per launch, measured with ncu
# (dram__bytes_read.sum + dram__bytes_write.sum over a family's kernels
# against the library's algorithmic bytes for the same calls); the profiles
# named give the captures.
TRAFFIC_RATIO = {
    # profiles/reorder_sort_q14_traffic.md: the 62 M-row reorder of the medium
    # chain query q14, 10965.3 MB of DRAM traffic against 10917.8 MB algorithmic
    "reorder_sort": (10965.3 / 10917.8, "profiles/reorder_sort_q14_traffic.md (one call: medium q14)"),
    # profiles/radix_sort_keys60_traffic.md: a 2^28-key, 60-bit keys-only sort
    # (the store build's shape), 37.52 GB of DRAM traffic against 34.36 GB
    "radix_sort_u64": (37.52 / 34.36, "profiles/radix_sort_keys60_traffic.md (one call: 2^28 keys, 60 bits)"),
    # profiles/product_fixed_star4_traffic.md: a 40.96 M-row product of four
    # constant rows, 592.4 MB of DRAM traffic against 819.2 MB algorithmic
    "product": (592.4 / 819.2, "profiles/product_fixed_star4_traffic.md (one call: 40.96 M-row star)"),
}


def roofline(prof, ws, peak, peak_kind, exclude=("store_build",)):
    """The dominant kernel family by event time (pipelines that bracket
    several families, such as the whole store build, are reported in
    `kernels` but are not a kernel): algorithmic bytes per launch over the
    average launch time, against the measured HBM copy bandwidth."""
    cands = [(k, v) for k, v in prof.items() if k not in exclude and v["total_ms"] > 0]
    if not cands:
        return None
    name, p = max(cands, key=lambda kv: kv[1]["total_ms"])
    achieved = p["algo_bytes"] / 1e9 / (p["total_ms"] / 1e3)
    per_launch_algo = p["algo_bytes"] / max(1, p["launches"])
    per_launch_ms = p["total_ms"] / max(1, p["launches"])
    ratio = TRAFFIC_RATIO.get(name)
    traffic = round(per_launch_algo * ratio[0]) if ratio else None
    return {"kernel": name, "bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "traffic": traffic,
            "traffic_source": ratio[1] if ratio else "no ncu capture of this family on the current build",
            "dram_GBps": round(traffic / 1e9 / (per_launch_ms / 1e3), 1) if traffic and per_launch_ms > 0 else None,
            "per_launch_ms": round(per_launch_ms, 4), "launches": int(p["launches"]),
            "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else peak_kind}


def kernel_table(prof):
    return {k: {"launches": v["launches"], "total_ms": round(v["total_ms"], 3),
                "GBps": round(v["algo_bytes"] / 1e9 / (v["total_ms"] / 1e3), 1) if v["total_ms"] else None}
            for k, v in sorted(prof.items(), key=lambda kv: -kv[1]["total_ms"])}


def leg_summary(leg, peak, peak_kind, ws):
    """The JSON fields of one workload's plain path."""
    q = leg["q_lat"]
    return {
        "value": round(leg["value"], 2),
        "unit": "queries/s",
        "ms_per_step": round(leg["total_ms"] / leg["steps"], 3),
        "result_rows_per_s": round(ws * leg["rows_total"] / (leg["total_ms"] / 1e3), 1),
        "result_rows_per_step": int(leg["rows_total"] / max(1, leg["steps"])),
        "latency_ms": {"p50": round(float(np.percentile(q, 50)), 4), "p99": round(float(np.percentile(q, 99)), 4),
                       "note": "per-query device time inside the timed steps (store resident)"},
        "e2e": leg["e2e"],
        "gpu_launches": leg["launches"],
        "roofline": roofline(leg["prof"], ws, peak, peak_kind),
        "kernels": kernel_table(leg["prof"]),
        "clocks": leg["clocks"],
        "tiles": leg["tiles"],
    }


def run_gsmat(args):
    import torch

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_1807_07691_b300 as gs

    stream = torch.cuda.current_stream()
    peak, peak_kind = _peaks()
    head_name = args.workload
    triples, queries, gen_s = _workload(head_name)
    head = plain_leg(args, gs, torch, head_name, triples, queries, stream, ws, local, args.steps, args.warmup)

    # the medium workload: a second plain-path line, and the graph of the
    # batched, planner, front-end and shard legs
    if head_name == "medium":
        m_tri, m_queries, m_gen_s, medium = triples, queries, gen_s, None
        d_med = head["d_tri"]
    else:
        m_tri, m_queries, m_gen_s = _workload("medium")
        medium = None
        if not args.no_medium and head_name == "large":
            medium = plain_leg(args, gs, torch, "medium", m_tri, m_queries, stream, ws, local, args.steps, args.warmup)
            d_med = medium["d_tri"]
        else:
            d_med = torch.from_numpy(np.array(m_tri, copy=True)).cuda()

    batched = served = planner = bq = None
    if not args.no_batched:
        batched, bq, tuned = run_batched(args, gs, torch, d_med, stream)
        if not args.no_planner:
            planner = run_planner(args, gs, torch, d_med, stream, m_queries, bq, tuned)
    frontend = None
    if not args.no_frontend:
        frontend = run_frontend(args, gs, torch, d_med, stream, m_tri, m_queries)
    shards = None
    if not args.no_shards:
        shards = run_shards(args, gs, torch, d_med, stream, m_queries)
    if not args.no_served and rank == 0:
        if args.served_graph == "large":
            served = run_served_large(args, gs, torch, stream,
                                      d_tri=head["d_tri"] if head_name == "large" else None,
                                      triples=triples if head_name == "large" else None)
        elif bq is not None:  # the medium graph's batched mix
            served = run_served(args, gs, torch, d_med, stream, bq)

    if rank != 0:
        if ws > 1:
            import torch.distributed as dist

            dist.destroy_process_group()
        return None

    hs = leg_summary(head, peak, peak_kind, ws)
    out = {
        "metric": METRIC,
        "value": hs["value"],
        "unit": "queries/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": hs["ms_per_step"],
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "int32",
        "data": "synthetic",
        "config": _add_streams(workload_config(head_name, head["nq"], head["n_triples"], ws), args.query_streams),
        "result_rows_per_s": hs["result_rows_per_s"],
        "result_rows_per_step": hs["result_rows_per_step"],
        "latency_ms": hs["latency_ms"],
        "e2e": hs["e2e"],
        "gpu_launches": hs["gpu_launches"],
        "roofline": hs["roofline"],
        "kernels": hs["kernels"],
        "clocks": hs["clocks"],
        "tiles": hs["tiles"],
        "generation_s": round(gen_s, 1),
    }
    if medium is not None:
        ms_ = leg_summary(medium, peak, peak_kind, ws)
        ms_["config"] = _add_streams(workload_config("medium", medium["nq"], medium["n_triples"], ws), args.query_streams)
        out["medium"] = ms_
    if batched is not None:
        out["batched"] = batched
    if planner is not None:
        out["planner"] = planner
    if frontend is not None:
        out["frontend"] = frontend
    if shards is not None:
        out["row_shards"] = shards
    if served is not None:
        out["served"] = served
    if not args.no_cpu_baseline:
        sample = reference_sample(head_name, queries)
        out["cpu_baseline"] = cpu_baseline(triples, sample, budget_s=args.cpu_budget, workload=head_name,
                                           n_total=len(queries))
        if head_name == "medium" or medium is not None:
            m_sample = reference_sample("medium", m_queries)
            one_m = cpu_baseline(m_tri, m_sample, budget_s=args.cpu_budget, workload="medium", n_total=len(m_queries))
            out["cpu_baseline_all_cores"] = cpu_baseline_all_cores(m_tri, m_sample[:one_m["attempted"]])
            out["cpu_baseline_all_cores"]["workload"] = "medium"
            if head_name != "medium":
                out["medium"]["cpu_baseline"] = one_m
    if ws > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return out


def run_batched(args, gs, torch, d_tri, stream):
    """The batched mix (medium graph, 4096 BGPs of 2-8 patterns, star:chain:
    snowflake:cycle = 4:3:2:1): the plain path one query at a time against
    one prepared batch (persistent kernel, CUDA graph), each timed with CUDA
    events after a warm-up pass; results are bit-identical (tested)."""
    import synth

    t0 = time.time()
    bq = synth.make_batched_queries(args.batched_n)
    gen_s = time.time() - t0
    S = gs.Store(d_tri, stream=stream)

    bmarsh = [gs.Store.marshal(q) for q in bq]

    def plain_pass():
        rows = 0
        for q in bmarsh:
            T = S.query_raw(q, stream=stream)
            rows += T.rows
            T.free()
        return rows

    plain_pass()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    rows_plain = plain_pass()
    b.record(stream)
    b.synchronize()
    plain_ms = a.elapsed_time(b)

    tuned = gs.batch_autotune(S, bq[:512], stream=stream)
    t_prep = time.perf_counter()
    B = gs.Batch(S, bq, config=tuned, stream=stream)
    prep_ms = 1e3 * (time.perf_counter() - t_prep)
    B.execute(stream)
    torch.cuda.synchronize()
    runs = []
    for _ in range(max(3, args.steps)):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        B.execute(stream)
        b.record(stream)
        b.synchronize()
        runs.append(a.elapsed_time(b))
    st = B.stats()
    rows_batch = sum(B.result(i)[0] for i in range(len(bq)))
    assert rows_batch == rows_plain, (rows_batch, rows_plain)
    # every result equal to the plain path's (compared on the device)
    mismatched = 0
    for i, q in enumerate(bmarsh):
        T = S.query_raw(q, stream=stream)
        a = torch.from_numpy(B.to_numpy(i))
        b = torch.from_numpy(T.to_numpy())
        mismatched += int(a.shape != b.shape or not torch.equal(a, b))
        T.free()
    batch_ms = float(np.median(runs))
    out = {
        "workload": f"{len(bq)} BGPs, 2-8 patterns, star:chain:snowflake:cycle 4:3:2:1, medium graph",
        "queries_per_s": round(len(bq) / (batch_ms / 1e3), 1),
        "queries_per_s_with_prepare": round(len(bq) / ((batch_ms + prep_ms) / 1e3), 1),
        "plain_queries_per_s": round(len(bq) / (plain_ms / 1e3), 1),
        "speedup_vs_plain": round(plain_ms / batch_ms, 2),
        "speedup_vs_plain_with_prepare": round(plain_ms / (batch_ms + prep_ms), 2),
        "results_equal_to_plain": len(bq) - mismatched,
        "batch_ms": round(batch_ms, 3),
        "plain_ms": round(plain_ms, 3),
        "prepare_ms": round(prep_ms, 2),
        "intersect_steps": st["n_intersect"],
        "kernel_ms": round(st["kernel_ms"], 3),
        "reorder_ms": round(st["reorder_ms"], 3),
        "in_kernel": st["n_in_kernel"],
        "reordered": st["n_reordered"],
        "fallback": st["n_fallback"],
        "result_rows": int(rows_batch),
        "tuned": {"block": tuned["block"], "ctas_per_sm": tuned["ctas_per_sm"], "expand_slots": tuned["expand_slots"]},
        "generation_s": round(gen_s, 1),
    }
    B.free()
    S.free()
    return out, bq, tuned


def run_planner(args, gs, torch, d_tri, stream, queries, bq, tuned):
    """Alg. 1 against the cost-based variant (GSMAT_PLAN_COST): the medium
    workload one query at a time with the store resident (three passes each,
    the median), and the batched mix as one prepared batch; per variant the
    device time, the intermediate rows the plans produce and the planner's
    estimated cost."""
    S = gs.Store(d_tri, stream=stream)
    marsh = [gs.Store.marshal(q) for q in queries]

    def plain(flags):
        ms, inter, est, orders = [], 0, 0.0, []
        for rep in range(4):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            tabs = [S.query_raw(q, flags=flags, stream=stream) for q in marsh]
            b.record(stream)
            b.synchronize()
            if rep:
                ms.append(a.elapsed_time(b))
            if rep == 1:
                for T in tabs:
                    st = T.stats()
                    inter += sum(r for r in st["rows"] if r > 0)
                    est += st["est_cost"]
                    orders.append(st["order"])
            for T in tabs:
                T.free()
        return float(np.median(ms)), inter, est, orders

    g_ms, g_inter, g_est, g_orders = plain(gs.SORTED)
    c_ms, c_inter, c_est, c_orders = plain(gs.PLAN_COST)
    nq = len(queries)

    def batched(plan_cost):
        cfg = dict(tuned, plan_cost=plan_cost)
        t0 = time.perf_counter()
        B = gs.Batch(S, bq, config=cfg, stream=stream)
        prep = 1e3 * (time.perf_counter() - t0)
        B.execute(stream)
        runs = []
        for _ in range(max(3, args.steps)):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            B.execute(stream)
            b.record(stream)
            b.synchronize()
            runs.append(a.elapsed_time(b))
        rows = sum(B.result(i)[0] for i in range(len(bq)))
        B.free()
        return float(np.median(runs)), prep, rows

    bg_ms, bg_prep, bg_rows = batched(0)
    bc_ms, bc_prep, bc_rows = batched(1)
    assert bg_rows == bc_rows, (bg_rows, bc_rows)
    S.free()
    return {
        "workload": f"medium, {nq} BGPs one at a time (store resident); batched mix of {len(bq)} BGPs",
        "plain": {"alg1_queries_per_s": round(nq / (g_ms / 1e3), 1), "cost_queries_per_s": round(nq / (c_ms / 1e3), 1),
                  "plans_changed": sum(a != b for a, b in zip(g_orders, c_orders)),
                  "alg1_intermediate_rows": int(g_inter), "cost_intermediate_rows": int(c_inter),
                  "alg1_est_cost": g_est, "cost_est_cost": c_est},
        "batched": {"alg1_queries_per_s": round(len(bq) / (bg_ms / 1e3), 1),
                    "cost_queries_per_s": round(len(bq) / (bc_ms / 1e3), 1),
                    "alg1_prepare_ms": round(bg_prep, 2), "cost_prepare_ms": round(bc_prep, 2)},
    }


def run_frontend(args, gs, torch, d_tri, stream, triples, queries):
    """The user-facing path on the medium workload: dictionary encoding of
    10^6 of its triples written as IRI text (host), reading the 40 BGPs
    written as SPARQL text (host, through the Python binding), and device
    projection with DISTINCT of their results onto one variable -- the
    leading one (rows already sorted: one compaction) and the last one
    (stable radix reorder, then the compaction)."""
    sample = np.asarray(triples[:1_000_000])
    text = "\n".join(f"<http://x.org/e{s}> <http://x.org/p{p}> <http://x.org/e{o}> ." for s, p, o in sample.tolist())
    t0 = time.perf_counter()
    d = gs.Dictionary()
    d.add_text(text)
    enc_s = time.perf_counter() - t0
    n_pred, n_terms = d.size()
    d.free()

    def as_text(q):
        def term(x, isv):
            return f"?v{x}" if isv else str(x)
        body = " . ".join(f"{term(s, sv)} {p} {term(o, ov)}" for (s, p, o, sv, ov) in q.patterns)
        return f"SELECT * WHERE {{ {body} }}"

    texts = [as_text(q) for q in queries]
    t0 = time.perf_counter()
    for _ in range(10):
        for t in texts:
            gs.Sparql(t)
    parse_us = 1e6 * (time.perf_counter() - t0) / (10 * len(texts))

    S = gs.Store(d_tri, stream=stream)
    marsh = [gs.Store.marshal(q) for q in queries]
    res = {}
    for which in ("leading", "last"):
        ms, rows_in, rows_out, algo = 0.0, 0, 0, 0.0
        for rep in range(2):
            for q, m in zip(queries, marsh):
                T = S.query_raw(m, stream=stream)
                v = 0 if which == "leading" else q.n_vars - 1
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                P = T.project([v], True, stream=stream)
                b.record(stream)
                b.synchronize()
                if rep:
                    ms += a.elapsed_time(b)
                    rows_in += T.rows
                    rows_out += P.rows
                    algo += 4.0 * T.rows + 4.0 * P.rows
                P.free()
                T.free()
        res[which] = {"ms": round(ms, 3), "rows_in": int(rows_in), "rows_out": int(rows_out),
                      "GBps": round(algo / 1e9 / (ms / 1e3), 1) if ms > 0 else None}
    S.free()
    return {
        "workload": "medium: 10^6 triples as IRI text; its 40 BGPs as SPARQL text; DISTINCT of one variable of each result",
        "encode_triples_per_s": round(len(sample) / enc_s, 1),
        "encode_terms": {"predicates": n_pred, "subjects_objects": n_terms},
        "sparql_parse_us": round(parse_us, 2),
        "distinct_leading": res["leading"],
        "distinct_last": res["last"],
    }


def run_shards(args, gs, torch, d_tri, stream, queries, n_shards=2):
    """Row sharding of the medium queries, shards one after another on this
    GPU (as each of n_shards GPUs would run one), then the device merge of
    the sorted shards; against the unsharded query.  Rows are checked equal."""
    S = gs.Store(d_tri, stream=stream)

    def timed(fn):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        r = fn()
        b.record(stream)
        b.synchronize()
        return r, a.elapsed_time(b)

    whole_ms = shard_ms = merge_ms = 0.0
    max_shard_ms = 0.0
    rows = 0
    for rep in range(2):
        for q in queries:
            T, t_whole = timed(lambda: S.query(q, stream=stream))
            parts, t_parts = [], []
            for k in range(n_shards):
                P, t = timed(lambda: S.query_shard(q, k, n_shards, stream=stream))
                parts.append(P)
                t_parts.append(t)
            M, t_merge = timed(lambda: gs.merge_tables(parts, stream=stream))
            assert M.rows == T.rows
            if rep:
                whole_ms += t_whole
                shard_ms += sum(t_parts)
                max_shard_ms += max(t_parts)
                merge_ms += t_merge
                rows += T.rows
            for x in parts + [M, T]:
                x.free()
    S.free()
    return {"workload": f"medium, 40 BGPs, {n_shards} row shards run one after another on one GPU",
            "whole_ms": round(whole_ms, 3), "shards_ms": round(shard_ms, 3),
            "slowest_shard_ms": round(max_shard_ms, 3), "merge_ms": round(merge_ms, 3), "result_rows": int(rows)}


def _spin_until(t):
    while True:
        d = t - time.perf_counter()
        if d <= 0:
            return
        if d > 2e-4:
            time.sleep(d - 1e-4)


def run_served(args, gs, torch, d_tri, stream, bq, workload=None):
    """Open-loop Poisson arrivals drawn from the batched mix, served by
    continuous batching (gsmat_server) and, for comparison, by the plain
    path one query at a time (FIFO).  Latency = completion - arrival."""
    S = gs.Store(d_tri, stream=stream)
    marsh = [gs.Server.marshal(q) for q in bq]
    marsh_plain = [gs.Store.marshal(q) for q in bq]
    rng = np.random.default_rng(7691 + 4)
    out = {"workload": workload or f"Poisson arrivals over {len(bq)} batched-mix BGPs (medium graph, resident store)",
           "seconds_per_rate": args.served_seconds, "rates": []}
    for rate in args.served_rates:
        n = max(1, int(rate * args.served_seconds))
        arrivals = np.cumsum(rng.exponential(1.0 / rate, size=n))
        pick = rng.integers(len(bq), size=n)
        # continuous batching
        srv = gs.Server(S, max_batch=args.served_max_batch, slots=args.served_slots)
        t0 = time.perf_counter() + 0.02
        tickets = np.empty(n, dtype=np.int64)
        sub = np.empty(n)
        for i in range(n):
            _spin_until(t0 + arrivals[i])
            sub[i] = time.perf_counter()
            tickets[i] = srv.submit_raw(marsh[pick[i]])
        lat = np.empty(n)
        for i in range(n):
            srv.wait(int(tickets[i]))
            lat[i] = srv.result(int(tickets[i]))[2] / 1e3  # ms from submit
        done = sub + lat / 1e3
        lat_arr = (done - (t0 + arrivals)) * 1e3  # from the scheduled arrival
        st = srv.stats()
        srv.close()
        served = {"p50_ms": round(float(np.percentile(lat_arr, 50)), 3),
                  "p99_ms": round(float(np.percentile(lat_arr, 99)), 3),
                  "queries_per_s": round(n / (done.max() - t0), 1),
                  "batches": int(st["batches"]), "fallbacks": int(st["fallbacks"])}
        # plain path, one query at a time
        t0 = time.perf_counter() + 0.02
        lat_p = np.empty(n)
        last = t0
        for i in range(n):
            _spin_until(t0 + arrivals[i])
            T = S.query_raw(marsh_plain[pick[i]], stream=stream)
            T.free()
            last = time.perf_counter()
            lat_p[i] = (last - (t0 + arrivals[i])) * 1e3
        plain = {"p50_ms": round(float(np.percentile(lat_p, 50)), 3),
                 "p99_ms": round(float(np.percentile(lat_p, 99)), 3),
                 "queries_per_s": round(n / (last - t0), 1)}
        out["rates"].append({"offered_qps": rate, "requests": n, "served": served, "plain": plain})
    S.free()
    return out


# The oracle's sample of a workload: the queries, in workload order, whose
# generator size bound (an upper bound on every connected sub-pattern's rows;
# exact for the large stars and chains) is at most this many rows.  The
# others would keep a host core busy for minutes each.
ORACLE_ROW_CAP = 30_000_000


def reference_sample(name, queries):
    """(sample, skipped names): the queries the oracle runs for `name`."""
    keep, skipped = [], []
    for q in queries:
        b = getattr(q, "bound", None)
        if b is not None and b > ORACLE_ROW_CAP:
            skipped.append(q.name)
        else:
            keep.append(q)
    return keep if not skipped else _Sample(keep, skipped)


class _Sample(list):
    """A list of queries that remembers which ones were left out."""

    def __init__(self, keep, skipped):
        super().__init__(keep)
        self.skipped = list(skipped)


def _run_oracle(ix, q):
    """Runs one query on the oracle; False if it passed the guard limit."""
    import oracle

    try:
        ix.query(q, row_limit=4 * ORACLE_ROW_CAP)
        return True
    except oracle.OracleError:
        return False


def cpu_baseline(triples, sample, budget_s=20.0, workload="medium", n_total=None):
    """The oracle as it stands, single-threaded, on a bounded sample: its
    index build, then the sample's queries in workload order until the
    budget is spent; value = queries finished / their time (an aborted
    query's time counts too)."""
    import oracle

    t0 = time.perf_counter()
    ix = oracle.OracleIndex(triples)
    t_index = time.perf_counter() - t0
    done = 0
    t_q = 0.0
    aborted = []
    for q in sample:
        if t_q > budget_s:
            break
        a = time.perf_counter()
        ok = _run_oracle(ix, q)
        t_q += time.perf_counter() - a
        if ok:
            done += 1
        else:
            aborted.append(q.name)
    value = done / t_q if t_q > 0 else None
    left_out = getattr(sample, "skipped", [])
    n_total = len(sample) + len(left_out) if n_total is None else n_total
    return {"value": round(value, 3) if value else None, "unit": "queries/s", "cores": 1, "kind": "oracle",
            "cpu_model": _cpu_model(), "nproc": os.cpu_count(), "attempted": done + len(aborted),
            "sample": f"{workload}: oracle index build ({t_index:.1f} s, not in value), then {done + len(aborted)} of "
                      f"the {n_total} queries in workload order ({t_q:.2f} s); left out (generator bound above "
                      f"{ORACLE_ROW_CAP:.0e} rows): {len(left_out)} {left_out}; aborted past "
                      f"{4 * ORACLE_ROW_CAP:.0e} rows: {aborted}"}


def _cpu_model() -> str:
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def _oracle_worker(path, queries, barrier, results, row_limit):
    """One process of the all-cores oracle run: its own index over the
    triples, then its share of the queries, one at a time."""
    import oracle

    try:
        ix = oracle.OracleIndex(np.load(path))
    except Exception:
        barrier.abort()
        raise
    barrier.wait(timeout=600)
    t0 = time.perf_counter()
    done = 0
    for q in queries:
        try:
            ix.query(q, row_limit=row_limit)
            done += 1
        except oracle.OracleError:
            pass
    results.put((done, time.perf_counter() - t0))


def cpu_baseline_all_cores(triples, queries, max_procs=32):
    """The same oracle on the same queries, spread over the host's cores:
    one spawned process per core (at most one per query and max_procs),
    each with its own index, taking every W-th query; the time runs from the
    moment every index is built to the last query's end."""
    import multiprocessing as mp
    import shutil
    import tempfile

    ctx = mp.get_context("spawn")  # never fork a process that holds a CUDA context
    W = max(1, min(os.cpu_count() or 1, len(queries), max_procs))
    tmp = tempfile.mkdtemp(prefix="oracle_")
    path = os.path.join(tmp, "triples.npy")
    np.save(path, np.ascontiguousarray(triples))
    barrier = ctx.Barrier(W + 1)
    results = ctx.Queue()
    procs = [ctx.Process(target=_oracle_worker, args=(path, queries[w::W], barrier, results, 30_000_000))
             for w in range(W)]
    out = None
    try:
        for p in procs:
            p.start()
        barrier.wait(timeout=600)
        t0 = time.perf_counter()
        got = [results.get(timeout=600) for _ in range(W)]
        wall = time.perf_counter() - t0
        done = sum(g[0] for g in got)
        out = {"value": round(done / wall, 3), "unit": "queries/s", "cores": W, "kind": "oracle",
               "cpu_model": _cpu_model(), "nproc": os.cpu_count(),
               "sample": f"the {len(queries)} queries of the one-core sample over {W} processes, each with its own "
                         f"index ({done} finished under the row limit); {wall:.1f} s from all indexes built to the "
                         f"last query done"}
    except Exception as e:  # a worker failed or the wait ran out
        out = {"value": None, "unit": "queries/s", "cores": W, "kind": "oracle", "error": repr(e)[:200]}
    finally:
        for p in procs:
            p.join(timeout=30)
            if p.is_alive():
                p.terminate()
                p.join(timeout=10)
        shutil.rmtree(tmp, ignore_errors=True)
    return out


WORKLOAD_TEXT = {
    "tiny": "plain SM-join, tiny: 10^4 entities, 8 predicates, 10^5 int32 triples, 10 BGPs of 2-3 patterns",
    "large": "plain SM-join, large: 4x10^7 entities, 256 predicates, 3x10^8 int32 triples, 20 anchored BGPs of "
             "4-8 patterns (stars, chains, snowflakes; results up to 5x10^8 rows)",
    "medium": "plain SM-join, medium: 10^6 entities, 64 predicates, 10^7 int32 triples, 40 BGPs of 3-6 patterns "
              "(stars, chains, snowflakes, one 4-cycle)",
}


def workload_config(name, nq, n_triples, ws):
    """The `config` of a plain-path line (the reference arm adds which
    queries of it the oracle ran)."""
    return {
        "workload": f"{WORKLOAD_TEXT[name]}; step = gsmat_load + {nq} queries (sorted results kept on device)",
        "queries_per_step": nq,
        "triples": n_triples,
        "l2": "flushed between timed steps (256 MB write); the inputs are far larger than L2",
        "parallelism": f"replicas x{ws}",
    }


def _add_streams(cfg, n_streams):
    cfg["query_streams"] = n_streams
    return cfg


def run_reference(args):
    """The reference arm: the oracle (the paper publishes no code) on the
    host cores, each step the same sample of the workload that cpu_baseline
    uses, with the index built once before the steps."""
    ws, rank, local = _dist()
    if rank != 0:
        return None
    triples, queries, _ = _workload(args.workload)
    import oracle

    sample = reference_sample(args.workload, queries)
    left_out = getattr(sample, "skipped", [])
    t0 = time.perf_counter()
    ix = oracle.OracleIndex(triples)
    t_index = time.perf_counter() - t0
    times = []
    aborted = set()
    for i in range(args.warmup + args.steps):
        a = time.perf_counter()
        n = 0
        for q in sample:
            if _run_oracle(ix, q):
                n += 1
            else:
                aborted.add(q.name)
        dt = time.perf_counter() - a
        if i >= args.warmup:
            times.append((n, dt))
    n_tot = sum(n for n, _ in times)
    t_tot = sum(dt for _, dt in times)
    value = n_tot / t_tot if t_tot > 0 else 0.0
    cfg = workload_config(args.workload, len(queries), int(triples.shape[0]), ws)
    cfg["reference_sample"] = (f"{len(sample)} of {len(queries)} queries per step, workload order; left out "
                               f"(generator bound above {ORACLE_ROW_CAP:.0e} rows): {left_out}; oracle index prebuilt "
                               f"({t_index:.1f} s), no store load in the step")
    return {
        "impl": "reference",
        "metric": METRIC,
        "value": round(value, 3),
        "unit": "queries/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(1e3 * t_tot / max(1, args.steps), 3),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "int32",
        "data": "synthetic",
        "config": cfg,
        "cpu_baseline": {"value": round(value, 3), "unit": "queries/s", "cores": 1, "kind": "oracle",
                         "sample": f"each step: {cfg['reference_sample']}; aborted past {4 * ORACLE_ROW_CAP:.0e} "
                                   f"rows: {sorted(aborted)}"},
        "e2e": {"value": round(value, 3), "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def run_served_large(args, gs, torch, stream, d_tri=None, triples=None):
    """The served measurement over the large graph (3x10^8 triples resident
    on the device) with its own anchored 2-8-pattern mix."""
    import synth

    t0 = time.time()
    tri = synth.make_graph("large") if triples is None else triples
    qs = synth.make_large_served_queries(tri, n_queries=args.served_large_n)
    gen_s = time.time() - t0
    own = d_tri is None
    if own:
        d_tri = torch.from_numpy(np.array(tri, copy=True)).cuda()
    out = run_served(args, gs, torch, d_tri, stream, qs,
                     workload=f"Poisson arrivals over {len(qs)} anchored BGPs of 2-8 patterns, star:chain:snowflake "
                              "4:3:2 (large graph, 3x10^8 triples, resident store, 120 GiB admission budget)")
    out["generation_s"] = round(gen_s, 1)
    if own:
        del d_tri
        torch.cuda.empty_cache()
    return out


def run_micro(args):
    """One library primitive on a synthetic input larger than L2, timed with
    CUDA events (for kernel-level measurements and ncu captures)."""
    import torch

    import paper_1807_07691_b300 as gs

    torch.cuda.set_device(0)
    g = torch.Generator(device="cuda").manual_seed(7)
    n = args.n
    out = {"micro": args.micro, "n": n}
    if args.micro == "sort":
        src = torch.randint(0, 1 << min(args.bits, 62), (n,), device="cuda", dtype=torch.int64, generator=g)
        keys = src.clone()
        vals = None if args.keys_only else torch.arange(n, device="cuda", dtype=torch.int32)
        ms = []
        for it in range(args.warmup + args.steps):
            keys.copy_(src)
            if vals is not None:
                vals.copy_(torch.arange(n, device="cuda", dtype=torch.int32))
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            gs.radix_sort_u64(keys, vals, 0, args.bits)
            b.record()
            b.synchronize()
            if it >= args.warmup:
                ms.append(a.elapsed_time(b))
        passes = (args.bits + 7) // 8
        algo = n * (8.0 if args.keys_only else 12.0) * 2 * passes
        t = float(np.median(ms))
        out.update({"bits": args.bits, "passes": passes, "ms": round(t, 4),
                    "algo_GBps": round(algo / 1e9 / (t / 1e3), 1), "Mkeys_per_s": round(n / 1e3 / t, 1)})
        assert bool((keys[1:] >= keys[:-1]).all())
    elif args.micro == "scan":
        x = torch.randint(0, 1000, (n,), device="cuda", dtype=torch.int32, generator=g)
        o = torch.empty(n + 1, device="cuda", dtype=torch.int64)
        ms = []
        for it in range(args.warmup + args.steps):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            gs.exclusive_scan_i32(x, o)
            b.record()
            b.synchronize()
            if it >= args.warmup:
                ms.append(a.elapsed_time(b))
        t = float(np.median(ms))
        out.update({"ms": round(t, 4), "algo_GBps": round(n * 12.0 / 1e9 / (t / 1e3), 1)})
    elif args.micro == "rows":
        # the canonical reorder on its own: n rows of V random columns of
        # `row_bits`-bit values, stably sorted by the first key_cols
        V, m, bits = args.cols, args.key_cols, args.row_bits
        cols = [torch.randint(0, 1 << bits, (n,), device="cuda", dtype=torch.int32, generator=g) for _ in range(V)]
        outc = [c.new_empty(n) for c in cols]
        ms = []
        gs.profile_read(reset=True)
        for it in range(args.warmup + args.steps):
            if it == args.warmup:
                gs.profile_read(reset=True)
                gs.profile_enable(True)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            gs.sort_rows(cols, m, bits, out=outc, flags=args.sort_flags)
            b.record()
            b.synchronize()
            if it >= args.warmup:
                ms.append(a.elapsed_time(b))
        gs.profile_enable(False)
        prof = gs.profile_read(reset=True).get("reorder_sort")
        undecided = torch.ones(n - 1, dtype=torch.bool, device="cuda")
        for c in range(m):
            x, y = outc[c][:-1], outc[c][1:]
            assert not bool((undecided & (y < x)).any())
            undecided &= y == x
        t = float(np.median(ms))
        out.update({"cols": V, "key_cols": m, "row_bits": bits, "ms": round(t, 4),
                    "algo_GBps": round(prof["algo_bytes"] / 1e9 / (prof["total_ms"] / 1e3), 1) if prof else None,
                    "algo_bytes_per_row": round(prof["algo_bytes"] / prof["items"], 2) if prof else None,
                    "Mrows_per_s": round(n / 1e3 / t, 1)})
    elif args.micro == "product":
        # a star around one constant: `cols` predicates with rows of length
        # L = round(n^(1/cols)), so the result is a product of about n rows
        # (written by the product step, no reorder)
        V = args.cols
        L = max(2, int(round(n ** (1.0 / V))))
        c = 5
        tri = []
        for p in range(V):
            objs = np.arange(L, dtype=np.int64) * 7 + p  # distinct, ascending
            tri.append(np.stack([np.full(L, c), np.full(L, 100 + p), objs], axis=1))
        tri = np.concatenate(tri).astype(np.int32)
        S = gs.Store(torch.from_numpy(tri).cuda())
        # variables numbered against the plan's order of equal-length rows
        pats = [(c, 100 + p, V - 1 - p, False, True) for p in range(V)]
        ms = []
        gs.profile_read(reset=True)
        rows = 0
        for it in range(args.warmup + args.steps):
            if it == args.warmup:
                gs.profile_read(reset=True)
                gs.profile_enable(True)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            T = S.query(pats, V)
            b.record()
            b.synchronize()
            rows = T.rows
            T.free()
            if it >= args.warmup:
                ms.append(a.elapsed_time(b))
        gs.profile_enable(False)
        prof = gs.profile_read(reset=True).get("product")
        t = float(np.median(ms))
        out.update({"cols": V, "row_len": L, "rows": rows, "query_ms": round(t, 4),
                    "product_ms_per_launch": round(prof["total_ms"] / prof["launches"], 4) if prof else None,
                    "algo_GBps": round(prof["algo_bytes"] / 1e9 / (prof["total_ms"] / 1e3), 1) if prof else None})
    elif args.micro == "query":
        triples, queries, _ = _workload(args.workload)
        S = gs.Store(torch.from_numpy(np.array(triples, copy=True)).cuda())
        q = queries[args.query_index]
        ms = []
        rows = 0
        for it in range(args.warmup + args.steps):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            T = S.query(q)
            b.record()
            b.synchronize()
            rows = T.rows
            T.free()
            if it >= args.warmup:
                ms.append(a.elapsed_time(b))
        out.update({"query": q.name, "rows": rows, "ms": round(float(np.median(ms)), 4)})
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--query-index", type=int, default=14)
    ap.add_argument("--micro", choices=["sort", "scan", "rows", "product", "query"], default=None,
                    help="time one primitive on a synthetic input instead of the workload")
    ap.add_argument("--n", type=int, default=1 << 25)
    ap.add_argument("--bits", type=int, default=40)
    ap.add_argument("--keys-only", action="store_true", help="--micro sort: no payload")
    ap.add_argument("--cols", type=int, default=4, help="--micro rows: columns")
    ap.add_argument("--key-cols", type=int, default=2, help="--micro rows: leading sort columns")
    ap.add_argument("--row-bits", type=int, default=20, help="--micro rows: bits per value")
    ap.add_argument("--sort-flags", type=int, default=0, help="--micro rows: 1 carry, 2 gather (0: by size)")
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gsmat", choices=["gsmat", "reference"])
    ap.add_argument("--workload", default="large", choices=["large", "medium", "tiny"],
                    help="the headline plain-path workload (large: the largest configuration)")
    ap.add_argument("--no-medium", action="store_true", help="skip the medium plain-path line")
    ap.add_argument("--no-tune", action="store_true", help="plain-path steps: default tile shapes (no tuning pass)")
    ap.add_argument("--query-streams", type=int, default=1,
                    help="plain-path steps: host threads (each with its own stream) running the step's queries")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--batched-n", type=int, default=4096)
    ap.add_argument("--no-planner", action="store_true", help="skip Alg. 1 vs the cost-based planner")
    ap.add_argument("--no-frontend", action="store_true", help="skip the dictionary / SPARQL / DISTINCT leg")
    ap.add_argument("--no-shards", action="store_true", help="skip the row-sharding leg")
    ap.add_argument("--no-served", action="store_true")
    ap.add_argument("--served-seconds", type=float, default=30.0)
    ap.add_argument("--served-rates", type=float, nargs="+", default=[1000, 5000, 20000])
    ap.add_argument("--served-max-batch", type=int, default=1024)
    ap.add_argument("--served-slots", type=int, default=4)
    ap.add_argument("--served-graph", choices=["medium", "large"], default="large",
                    help="large: an anchored mix over the resident large graph; medium: the batched mix")
    ap.add_argument("--served-large-n", type=int, default=1024)
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    args = ap.parse_args()
    if args.micro:
        out = run_micro(args)
    else:
        out = run_reference(args) if args.impl == "reference" else run_gsmat(args)
    if out is not None:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
