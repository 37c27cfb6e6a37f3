"""Benchmark of the Graphical Join hot path on GB300.

One step = the whole path over one synthetic instance of the workload:
factor construction of every relation, the summary (upward and downward
sum-product passes, offsets), and desummarisation of every result row into
device columns, chunk by chunk.  Inputs are resident in HBM before the timed
region.  Those of the default workload are larger than L2, so nothing is
flushed between steps; when a workload's inputs fit in L2, a buffer twice the
L2 is written before every timed step and that time is taken out.

Default workload: 5-table chain R_i(K_{i-1}, K_i), 10^7 rows per table,
int32 keys Zipf(s=1.1) over a domain of 10^6 (independently permuted per
table and column), one int64 payload per table; desummarised in 2^28-row
chunks.

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle
instead, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "result tuples materialised/s"
UNIT = "tuples/s"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gj", choices=["gj", "reference"])
    p.add_argument("--workload", default="chain5_zipf",
                   choices=["chain5_zipf", "chain3_uniform", "star_poisson", "triangle", "square",
                            "batch", "serve", "reuse", "sensitivity"])
    p.add_argument("--rates", default="100,200,500,1000,2000,5000,10000",
                   help="serve workload: offered arrival rates (queries/s)")
    p.add_argument("--serve-seconds", type=float, default=2.0)
    p.add_argument("--slots", type=int, default=16)
    p.add_argument("--pool", type=int, default=512, help="serve workload: distinct small queries")
    p.add_argument("--serve-engine", default="native", choices=["native", "python"])
    p.add_argument("--serve-chunk-log2", type=int, default=20,
                   help="serve workload: rows per streamed chunk, log2")
    p.add_argument("--serve-max-rows", type=int, default=1 << 24,
                   help="serve workload: result rows streamed per request, in 2^20-row chunks "
                        "(0: the whole result)")
    p.add_argument("--queries", type=int, default=4096, help="batch workload: queries")
    p.add_argument("--rows", type=int, default=10**7)
    p.add_argument("--fact-rows", type=int, default=10**8, help="star_poisson workload: fact rows")
    p.add_argument("--domain", type=int, default=10**6)
    p.add_argument("--zipf", type=float, default=1.1)
    p.add_argument("--drop-attrs", default="",
                   help="comma-separated attribute ids projected away early (Section 3.7); "
                        "each must be held by one relation, e.g. 0,5 for the 5-chain's ends")
    p.add_argument("--chunk-log2", type=int, default=28)
    p.add_argument("--emit-rpt", type=int, default=4, choices=[2, 4, 8],
                   help="result rows per thread of the emit kernel")
    p.add_argument("--e2e-chunk-log2", type=int, default=24)
    p.add_argument("--e2e-steps", type=int, default=1)
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-sample-rows", type=int, default=None,
                   help="root rows kept for the oracle sample (default per workload)")
    return p.parse_args()


def workload_name(a):
    if a.workload == "chain3_uniform":
        return ("chain3_uniform: R1(A,B) R2(B,C) R3(C,D), 10^4 rows/table, int32 keys, A,D "
                "uniform over [0,10^4), B,C uniform over [0,1000), int32 payload/table, "
                f"desummarised in 2^{a.chunk_log2}-row chunks" + drop_note(a))
    if a.workload == "triangle":
        return ("triangle: cyclic R(A,B) S(B,C) T(C,A), 10^6 rows/table, int32 keys uniform over "
                "[0,1000), int64 payload/table, one-cluster junction tree, "
                f"desummarised in 2^{a.chunk_log2}-row chunks")
    if a.workload == "square":
        return ("square: cyclic R0(A,B) R1(B,C) R2(C,D) R3(D,A), 10^5 rows/table, int32 keys "
                "uniform over [0,1000), int64 payload/table, "
                f"desummarised in 2^{a.chunk_log2}-row chunks")
    if a.workload == "star_poisson":
        return (f"star_poisson: fact F(K1..K4,P) {a.fact_rows} rows, K_j uniform over [0,10^6), joined to "
                "4 dimensions D_j(K_j,P_j) with Poisson(2) copies of every key, int64 payloads, "
                f"desummarised in 2^{a.chunk_log2}-row chunks")
    return (f"chain5_zipf: 5-table chain R_i(K_i-1,K_i), {a.rows} rows/table, int32 keys "
            f"Zipf({a.zipf}) over [0,{a.domain}), int64 payload/table, "
            f"desummarised in 2^{a.chunk_log2}-row chunks" + drop_note(a))


def drop_list(a):
    return [int(x) for x in a.drop_attrs.split(",") if x.strip()]


def drop_note(a):
    d = drop_list(a)
    return f"; attributes {d} projected away early (Section 3.7)" if d else ""


def make_query(a, rank):
    from paper_2206_10435_gb300 import datagen as G
    if a.workload == "chain3_uniform":
        return G.chain3_uniform(seed=G.SEED_BASE + 0 + 1000 * rank)
    if a.workload == "star_poisson":
        return G.star_poisson(seed=G.SEED_BASE + 2 + 1000 * rank, fact_rows=a.fact_rows)
    if a.workload == "triangle":
        return G.triangle_query(G.SEED_BASE + 5 + 1000 * rank, [10**6] * 3, domain=1000)
    if a.workload == "square":
        return G.cyclic_query(G.SEED_BASE + 7 + 1000 * rank, "square", [10**5] * 4, domain=1000)
    return G.chain5_zipf(seed=G.SEED_BASE + 1 + 1000 * rank, rows=a.rows, domain=a.domain,
                         s=a.zipf)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (FileNotFoundError, OSError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        return self.summarize(self.lines)

    @staticmethod
    def summarize(lines):
        """Median SM clock under load, the maximum SM clock, and every
        slowdown reason seen active, from the sampled CSV lines (lines that
        are not a full sample are skipped)."""
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                mhz, max_mhz = float(f[1]), float(f[2])
            except ValueError:
                continue
            sm.append(mhz)
            smax = max_mhz
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


EMIT_PROFILE = os.path.join(ROOT, "profiles", "k_emit_chain5_zipf.md")
EMIT_SOURCE = os.path.join(ROOT, "paper_2206_10435_gb300", "csrc", "gj_emit.cu")


def emit_traffic_per_row():
    """DRAM bytes (read + write) per result row of the emit kernel, from the
    committed ncu summary, or None if the kernel source changed since that
    capture (its sha256 no longer matches)."""
    import hashlib
    try:
        text = open(EMIT_PROFILE).read()
        src = hashlib.sha256(open(EMIT_SOURCE, "rb").read()).hexdigest()
    except OSError:
        return None, "no ncu summary"
    fields = {}
    for line in text.splitlines():
        if ":" in line and line.startswith("- "):
            k, v = line[2:].split(":", 1)
            fields[k.strip()] = v.strip().strip("`")
    if fields.get("kernel_source_sha256") != src:
        return None, "kernel changed since the ncu capture"
    try:
        return float(fields["dram_bytes_per_row"]), "ncu capture, scaled by rows per launch"
    except (KeyError, ValueError):
        return None, "no traffic in the ncu summary"


def cpu_baseline(a, q_full, sample_rows, drop=(), min_seconds=0.0):
    """The oracle, as it stands, on a bounded sample: the same tables with
    the root restricted to its first `sample_rows` rows (a sub-join of the
    workload); cascade of hash joins + canonical sort + column materialisation
    on one host core.  The sample is joined again until `min_seconds` of CPU
    work have been timed (at least once)."""
    from oracle import oracle as O
    from paper_2206_10435_gb300 import datagen as G
    O.build()
    R1 = q_full.relations[0]
    sub = G.Relation(R1.name, R1.attrs, [k[:sample_rows].copy() for k in R1.keys],
                     [p[:sample_rows].copy() for p in R1.payloads])
    qs = G.Query("sample", [sub] + q_full.relations[1:], q_full.attr_names)
    dt, n, reps = 0.0, 0, 0
    while reps == 0 or dt < min_seconds:
        t0 = time.perf_counter()
        j = O.join(qs, max_tuples=400_000_000, drop=drop)
        cols = O.columns(qs, j.rowids, drop)
        dt += time.perf_counter() - t0
        n += int(j.rowids.shape[0])
        reps += 1
        del cols, j
    return {"value": n / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": sample_note(R1, sample_rows) +
                      f": {n // reps} result tuples per join, {reps} join(s) in {dt:.2f} s",
            "seconds": dt, "tuples": n}


def sample_note(R1, sample_rows):
    return (f"root relation cut to its first {min(sample_rows, R1.n_rows)} of {R1.n_rows} rows, "
            f"other tables whole (hash-join cascade + canonical sort + columns)")


def run_reference(a, rank, world):
    """The oracle on the same bounded sample as the cpu_baseline leg of the
    GPU arm: one join of the sample per step."""
    if rank != 0:
        return
    q = make_query(a, 0)
    for _ in range(a.warmup):
        cpu_baseline(a, q, a.cpu_sample_rows, drop_list(a))
    secs, tuples = 0.0, 0
    for _ in range(a.steps):
        r = cpu_baseline(a, q, a.cpu_sample_rows, drop_list(a))
        secs += r["seconds"]
        tuples += r["tuples"]
    value = tuples / secs
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus, "steps": a.steps,
           "warmup": a.warmup, "ms_per_step": 1000 * secs / a.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
           "impl": "reference",
           "config": {"workload": workload_name(a),
                      "input_bytes": int(sum(sum(x.nbytes for x in R.keys + R.payloads) for R in q.relations)),
                      "l2": "not applicable: the oracle runs on the host",
                      "parallelism": "one host process (the oracle, one core)"},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                            "sample": sample_note(q.relations[0], a.cpu_sample_rows) +
                                      ", one join per step"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def reduce_over_ranks(dist, elapsed_ms: float, rows: int, device):
    """Whole-job figures of a weak-scaling run: the slowest rank's time and
    the rows of all ranks (each rank joins its own instance, so there is no
    data-path collective; this is the only communication).  dist is
    torch.distributed or None; device is where the backend wants tensors."""
    if dist is None:
        return elapsed_ms, rows
    import torch
    t = torch.tensor([elapsed_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    r = torch.tensor([rows], dtype=torch.int64, device=device)
    dist.all_reduce(r)
    return float(t.item()), int(r.item())


DEFAULT_SAMPLE = {"chain5_zipf": 5000, "chain3_uniform": 10**4, "star_poisson": 250000, "triangle": 2500,
                  "square": 500,
                  "batch": 0, "serve": 0, "reuse": 0, "sensitivity": 0}


def main():
    a = parse()
    if a.cpu_sample_rows is None:
        a.cpu_sample_rows = DEFAULT_SAMPLE[a.workload]
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if a.impl == "reference":
        return run_reference(a, rank, world)
    if a.workload == "batch":
        return run_batch(a, rank, world, local)
    if a.workload == "serve":
        return run_serve(a, rank, world, local)
    if a.workload == "reuse":
        return run_reuse(a, rank, world, local)
    if a.workload == "sensitivity":
        return run_sensitivity(a, rank, world, local)

    import numpy as np
    import torch
    from paper_2206_10435_gb300 import gj

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    from paper_2206_10435_gb300 import partition as P
    # every rank builds the same instance (factors and summary replicated);
    # each desummarises its own equal, contiguous share of the result rows
    q = make_query(a, 0)
    rels = []
    for R in q.relations:
        rels.append(([torch.from_numpy(k).to(dev) for k in R.keys],
                     [torch.from_numpy(p).to(dev) for p in R.payloads], R.attrs))
    in_bytes = sum(sum(t.numel() * t.element_size() for t in ks + ps) for ks, ps, _ in rels)
    flush_buf, l2_note = l2_plan(torch, dev, in_bytes)
    stream = torch.cuda.Stream(dev)
    ctx = gj.Context(local, stream)
    ctx.set_option(gj.GJ_OPT_EMIT_ROWS_PER_THREAD, a.emit_rpt)
    CH = 1 << a.chunk_log2
    out_bufs = None
    phase = {"build_ms": 0.0, "summary_ms": 0.0, "desum_ms": 0.0}
    groups = []

    def step(record=False):
        nonlocal out_bufs, groups
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)] if record else None
        if record:
            ev[0].record(stream)
        ids = [ctx.load_relation(ks, attrs, ps) for ks, ps, attrs in rels]
        qq = ctx.query(ids, drop_attrs=drop_list(a))   # factor construction
        groups = list(qq.n_groups)
        if record:
            ev[1].record(stream)
        total = qq.summarize()                    # upward + downward passes
        if record:
            ev[2].record(stream)
        lo, hi = P.row_range(total, rank, world)
        if out_bufs is None:
            out_bufs = qq.alloc_columns(max(1, min(CH, hi - lo)))
        for r0, n in P.windows(lo, hi, CH):
            qq.desummarize(r0, n, out=out_bufs)
        if record:
            ev[3].record(stream)
        qq.close()
        for i in ids:
            ctx.release_relation(i)
        return total, ev

    with torch.cuda.stream(stream):
        total = 0
        for _ in range(a.warmup):
            total, _ = step()
        torch.cuda.synchronize()
        ctx.profile(True)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        clocks = ClockSampler(local)
        clocks.start()
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_start.record(stream)
        evs, flush_evs = [], []
        for k in range(a.steps):
            if flush_buf is not None:
                # inputs that fit in L2: evict them before every timed step
                # (writing a buffer twice the L2); this time is taken out
                fe = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
                fe[0].record(stream)
                flush_buf.fill_(k & 0xff)
                fe[1].record(stream)
                flush_evs.append(fe)
            total, ev = step(record=True)
            evs.append(ev)
        t_end.record(stream)
        torch.cuda.synchronize()
        clk = clocks.stop()
        prof = ctx.profile(False)
        elapsed_ms = t_start.elapsed_time(t_end) - sum(f[0].elapsed_time(f[1]) for f in flush_evs)
        for ev in evs:
            phase["build_ms"] += ev[0].elapsed_time(ev[1]) / a.steps
            phase["summary_ms"] += ev[1].elapsed_time(ev[2]) / a.steps
            phase["desum_ms"] += ev[2].elapsed_time(ev[3]) / a.steps
    lo, hi = P.row_range(total, rank, world)
    rows_local = (hi - lo) * a.steps
    t_max, rows_all = reduce_over_ranks(dist, elapsed_ms, rows_local, dev)
    value = rows_all / (t_max / 1000.0)

    # end to end through the C ABI with host buffers: H2D of the relations
    # from pinned memory, the whole path, D2H of every result chunk
    e2e = None
    if not a.no_e2e:
        e2e = run_e2e(a, q, ctx, stream, dev, total, dist, rank, world)

    peak, peak_kind = measured_peaks()
    achieved = (prof["emit_bytes"] / (prof["emit_ms"] * 1e6)) if prof["emit_ms"] else None
    tpr, tnote = emit_traffic_per_row() if a.workload == "chain5_zipf" and not drop_list(a) else (None, "captured for chain5_zipf (all columns) only")
    rows_per_launch = prof["emit_rows"] / max(prof["emit_launches"], 1)
    traffic = tpr * rows_per_launch if tpr is not None else None
    roofline = {"bound": "hbm", "kernel": f"k_emit<K={len(q.relations)},RPT={a.emit_rpt}> (desummarise emit)",
                "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                "traffic_note": tnote,
                "peak_kind": f"{peak_kind} hbm_gbs (burst copy)",
                "bytes_per_launch": prof["emit_bytes"] / max(prof["emit_launches"], 1),
                "avg_launch_ms": prof["emit_ms"] / max(prof["emit_launches"], 1),
                "expand_ms_per_step": prof["expand_ms"] / a.steps,
                "emit_ms_per_step": prof["emit_ms"] / a.steps}
    # the other phases against the same roofline, with the algorithmic bytes
    # of the hot-path definitions: factor build reads every key column and
    # payload once, writes the row order, the payloads in group order and per
    # group its keys and start; the summary reads per group its keys and
    # count and writes w, mult and off (8 B each)
    build_b = summ_b = 0
    for (ks, ps, _), G in zip(rels, groups):
        n = ks[0].numel() if ks else 0
        k = len(ks)
        w = sum(t.element_size() for t in ps)
        build_b += n * (4 * k + 4 + 2 * w) + G * (4 * k + 4)
        summ_b += G * (4 * k + 4 + 24)
    phase_rooflines = {}
    for name, b, ms in (("factor_build", build_b, phase["build_ms"]),
                        ("summary", summ_b, phase["summary_ms"])):
        if name == "summary" and a.workload in ("triangle", "square"):
            # a cyclic join's summary is its maxclique potential (segment
            # intersections for the 3-cycle, group-wise joins otherwise),
            # not a pass over groups
            phase_rooflines[name] = {"algorithmic_bytes": None, "ms": ms, "achieved": None,
                                     "unit": "GB/s", "frac": None,
                                     "note": "maxclique potential: no per-group byte count"}
            continue
        gbs = b / (ms * 1e6) if ms else None
        phase_rooflines[name] = {"algorithmic_bytes": b, "ms": ms, "achieved": gbs, "unit": "GB/s",
                                 "frac": gbs / peak if gbs else None}
    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        cpu = cpu_baseline(a, q, a.cpu_sample_rows, drop_list(a), min_seconds=10.0)
        cpu.pop("seconds")
        cpu.pop("tuples")
    if rank == 0:
        row_bytes = int(prof["emit_bytes"] // max(prof["emit_rows"], 1))
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
               "steps": a.steps, "warmup": a.warmup, "ms_per_step": t_max / a.steps,
               "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
               "dtype": "int64", "data": "synthetic",
               "config": {"workload": workload_name(a), "join_size": total,
                          "result_row_bytes": row_bytes, "input_bytes": in_bytes,
                          "l2": l2_note,
                          "parallelism": (f"{world} rank(s), one per GPU: factors and summary "
                                          "built on every rank, the result rows split into "
                                          "equal contiguous ranges, one per rank")},
               "summary_build_ms": phase["build_ms"] + phase["summary_ms"],
               "phases_ms": phase,
               "phase_rooflines": phase_rooflines,
               "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
               "gpu_launches": int(prof["launches"]), "clocks": clk}
        print(json.dumps(out), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()


def run_batch(a, rank, world, local):
    """Batched summaries of --queries independent chain joins (3-6 tables,
    rows log-uniform 1e3-1e6, domains log-uniform 1e2-1e5, Zipf s in
    [0, 1.5]): one query at a time through the plain API, versus the batched
    path (cold: planning + graph capture + one launch; warm: graph replay),
    with identical totals required."""
    import numpy as np
    import torch
    from paper_2206_10435_gb300 import autotune, datagen as G, gj
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    t = time.perf_counter()
    queries = G.batch_queries_torch(seed=G.SEED_BASE + 3 + 1000 * rank, n_queries=a.queries,
                                    device=dev)
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t
    n_rows = sum(int(k[0].shape[0]) for q in queries for _, k in q)
    stream = torch.cuda.Stream(dev)
    ctx = gj.Context(local, stream)
    with torch.cuda.stream(stream):
        # plain: one query at a time (factors + summary), every query once
        def plain_pass():
            out = []
            for q in queries:
                ids = [ctx.load_relation(keys, attrs) for attrs, keys in q]
                qq = ctx.query(ids)
                try:
                    out.append(qq.summarize())
                except gj.GJError as e:
                    if e.status != gj.GJ_ERR_OVERFLOW:
                        raise
                    out.append(gj.SAT)
                qq.close()
                for i in ids:
                    ctx.release_relation(i)
            return out
        plain_pass() if a.warmup > 0 else None
        torch.cuda.synchronize()
        t = time.perf_counter()
        plain_totals = plain_pass()
        torch.cuda.synchronize()
        plain_s = time.perf_counter() - t
        ids = [[ctx.load_relation(keys, attrs) for attrs, keys in q] for q in queries]
        # batched, cold: planning + capture + one launch
        torch.cuda.synchronize()
        t = time.perf_counter()
        b = gj.Batch(ctx, ids)
        b.run(use_graph=True)
        stream.synchronize()
        cold_s = time.perf_counter() - t
        tuned = autotune.tune_batch(b)
        for _ in range(max(a.warmup, 1)):
            b.run(use_graph=True)
        stream.synchronize()
        ctx.profile(True)
        clocks = ClockSampler(local)
        clocks.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(a.steps):
            b.run(use_graph=True)
        e1.record(stream)
        e1.synchronize()
        clk = clocks.stop()
        prof = ctx.profile(False)
        warm_ms = e0.elapsed_time(e1) / a.steps
        batched = [int(x) for x in b.totals.cpu().numpy().view(np.uint64)]
    same = batched == [int(x) for x in plain_totals]
    # the global query list is the ranks' sets in rank order: totals of all
    # of them, gathered in query order (the slowest rank's time counts)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    from paper_2206_10435_gb300 import partition as P
    all_totals = P.gather_in_order(dist, np.array(batched, dtype=np.uint64), a.queries * world,
                                   rank, world, dev)
    warm_ms = P.max_over_ranks(dist, warm_ms, dev)
    plain_s = P.max_over_ranks(dist, plain_s, dev)
    cold_s = P.max_over_ranks(dist, cold_s, dev)
    same = P.max_over_ranks(dist, 0.0 if same else 1.0, dev) == 0.0
    out = {"metric": "queries summarised/s (batched, one CUDA-graph launch)",
           "value": a.queries * world / (warm_ms / 1000.0), "unit": "queries/s", "n_gpus": world,
           "steps": a.steps, "warmup": a.warmup, "ms_per_step": warm_ms,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
           "data": "synthetic",
           "config": {"workload": (f"batch: {a.queries} chain joins of 3-6 tables, rows/table "
                                   "log-uniform 1e3-1e6, domains log-uniform 1e2-1e5, Zipf s "
                                   "uniform in [0,1.5], int32 keys; totals per query"),
                      "rows": n_rows, "relations": b.n_relations, "levels": b.levels,
                      "key_bits": b.key_bits, "generation_s": gen_s,
                      "l2": "inputs larger than L2 (no flush)",
                      "parallelism": (f"{world} rank(s): each summarises its own {a.queries} "
                                      "queries (one block of the global query list); totals "
                                      "gathered in query order")},
           "plain_qps": a.queries * world / plain_s, "plain_s": plain_s,
           "batched_cold_qps": a.queries * world / cold_s, "batched_cold_s": cold_s,
           "speedup_warm_vs_plain": plain_s / (warm_ms / 1000.0),
           "speedup_cold_vs_plain": plain_s / cold_s,
           "identical_totals": same,
           "overflowed_queries": int(np.sum(all_totals == np.uint64(gj.SAT))),
           "autotune": tuned, "gpu_launches": int(prof["launches"]), "clocks": clk}
    if rank == 0:
        print(json.dumps(out), flush=True)
    b.close()
    ctx.close()
    if dist:
        dist.destroy_process_group()
    if not same:
        sys.exit(1)


def run_serve(a, rank, world, local):
    """Poisson streams of queries drawn from the batch distribution plus 1%
    4-table chains of 10^7 rows (Zipf 1.1 over 10^6), served with relations
    and factors resident, under a 150 GB HBM budget, each answered with its
    summary and its result rows (up to --serve-max-rows) streamed in 2^20-row
    chunks."""
    import numpy as np
    import torch
    from paper_2206_10435_gb300 import datagen as G, gj
    from paper_2206_10435_gb300.serve import GJEngine, Server, latency_stats, poisson_arrivals, run_stream
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    small = G.batch_queries_torch(seed=G.SEED_BASE + 4 + 1000 * rank, n_queries=a.pool, device=dev)
    large = [G.chain_zipf_torch(G.SEED_BASE + 5 + 1000 * rank + i, device=dev) for i in range(4)]
    ctx = gj.Context(local, torch.cuda.Stream(dev))
    t = time.perf_counter()
    small_ids = [[ctx.load_relation(k, attrs) for attrs, k in q] for q in small]
    large_ids = [[ctx.load_relation(k, attrs) for attrs, k in q] for q in large]
    for q in small_ids + large_ids:       # factors built once, then resident
        ctx.query(q).close()
    torch.cuda.synchronize()
    warm_s = time.perf_counter() - t
    rates = [float(x) for x in a.rates.split(",")]
    rng = np.random.default_rng(G.SEED_BASE + 6)
    sweep = []
    clocks = ClockSampler(local)
    clocks.start()
    from paper_2206_10435_gb300.serve import native_latency_stats
    n_warm = max(a.warmup, 3)
    for w in range(n_warm + len(rates)):
        warm = w < n_warm   # untimed streams of 100 requests at the first rate
        rate = rates[0] if warm else rates[w - n_warm]
        n = 100 if warm else int(min(max(rate * a.serve_seconds, 100), 20000))
        picks = [large_ids[int(rng.integers(0, len(large_ids)))] if rng.random() < 0.01
                 else small_ids[int(rng.integers(0, len(small_ids)))] for _ in range(n)]
        offsets = poisson_arrivals(rate, n, seed=int(rate) + (1000 + w if warm else 0))
        if a.serve_engine == "native":
            srv = gj.NativeServer(ctx, n_slots=a.slots, hbm_budget=150 * 10**9,
                                  chunk_rows=1 << a.serve_chunk_log2, max_rows=a.serve_max_rows)
            res, sst = srv.run(picks, offsets)
            srv.close()
            st = native_latency_stats(res)
            st.update({"offered_qps": rate, "requests": n, "peak_in_flight": sst["peak_in_flight"],
                       "peak_admitted_gb": sst["peak_admitted_bytes"] / 1e9})
        else:
            eng = GJEngine(ctx, a.slots, chunk_rows=1 << a.serve_chunk_log2, max_rows=a.serve_max_rows)
            srv = Server(eng, n_slots=a.slots, hbm_budget=150 * 10**9)
            reqs = run_stream(srv, picks, offsets)
            st = latency_stats(reqs)
            st.update({"offered_qps": rate, "requests": n, "peak_in_flight": srv.peak_in_flight,
                       "peak_admitted_gb": srv.peak_used / 1e9})
        if not warm:
            sweep.append(st)
    clk = clocks.stop()
    # every rank serves its own stream at each offered rate (weak scaling):
    # the job's served rate at a step is the sum over ranks; the latencies
    # reported are the worst rank's
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        q = torch.tensor([s.get("qps") or 0.0 for s in sweep], dtype=torch.float64, device=dev)
        dist.all_reduce(q)
        lat_keys = ["p50_first_chunk_ms", "p99_first_chunk_ms", "p50_last_chunk_ms", "p99_last_chunk_ms"]
        lat = torch.tensor([[s.get(k) or 0.0 for k in lat_keys] for s in sweep], dtype=torch.float64, device=dev)
        dist.all_reduce(lat, op=dist.ReduceOp.MAX)
        for i, s in enumerate(sweep):
            s["qps_all_ranks"] = float(q[i].item())
            s["offered_qps_all_ranks"] = s["offered_qps"] * world
            for j, k in enumerate(lat_keys):
                s[k + "_worst_rank"] = float(lat[i, j].item())
        best = max(s["qps_all_ranks"] for s in sweep)
        dist.destroy_process_group()
    else:
        best = max((s.get("qps") or 0) for s in sweep)
    out = {"metric": "served queries/s (continuous admission, resident factors)",
           "value": best, "unit": "queries/s", "n_gpus": world, "steps": len(rates),
           "warmup": n_warm, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "int64", "data": "synthetic",
           "config": {"workload": (f"serve: Poisson arrivals at {a.rates} q/s, {a.serve_seconds}s "
                                   f"each; {a.pool} queries of the batch distribution + 1% "
                                   "4-table chains of 1e7 rows (Zipf 1.1 over 1e6); summary + "
                                   f"the result's first {a.serve_max_rows or 'all'} rows streamed "
                                   f"in 2^{a.serve_chunk_log2}-row chunks per request; 150 GB HBM budget"),
                      "slots": a.slots, "engine": a.serve_engine, "factor_build_s": warm_s,
                      "parallelism": (f"{world} rank(s), one per GPU, each serving its own stream at "
                                      "every offered rate; served q/s summed over ranks"),
                      "l2": "not flushed: the requests of a stream share L2, as in service"},
           "sweep": sweep, "clocks": clk}
    if rank == 0:
        print(json.dumps(out), flush=True)
    ctx.close()


def run_reuse(a, rank, world, local):
    """Compute-and-reuse on the 5-chain Zipf workload: summarise, store the
    summary in a file, load it back into a query that has none of the
    original relations, and desummarise every result row from it."""
    import tempfile
    import torch
    from paper_2206_10435_gb300 import datagen as G, gj
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    q = G.chain5_zipf(seed=G.SEED_BASE + 1 + 1000 * rank, rows=a.rows, domain=a.domain, s=a.zipf)
    stream = torch.cuda.Stream(dev)
    ctx = gj.Context(local, stream)
    CH = 1 << a.chunk_log2
    path = os.path.join(tempfile.gettempdir(), f"gj_summary_{os.getpid()}.gjs")
    with torch.cuda.stream(stream):
        ids = gj.load_query(ctx, q)
        qq = ctx.query(ids)
        total = qq.summarize()
        row_bytes = sum(qq.col_width)
        t = time.perf_counter()
        nbytes = qq.save(path)
        save_s = time.perf_counter() - t
        qq.close()
        for r in ids:
            ctx.release_relation(r)
        torch.cuda.synchronize()
        bufs = None
        load_s = desum_s = 0.0
        for it in range(a.warmup + a.steps):
            t = time.perf_counter()
            lq = gj.Query.load(ctx, path)
            torch.cuda.synchronize()
            dt_load = time.perf_counter() - t
            if bufs is None:
                bufs = lq.alloc_columns(min(CH, total))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for r0 in range(0, total, CH):
                lq.desummarize(r0, CH, out=bufs)
            e1.record(stream)
            e1.synchronize()
            if it >= a.warmup:
                load_s += dt_load / a.steps
                desum_s += e0.elapsed_time(e1) / 1000.0 / a.steps
            lq.close()
    os.remove(path)
    out = {"metric": "result tuples/s, loading a stored summary and desummarising",
           "value": total / (load_s + desum_s), "unit": "tuples/s", "n_gpus": world, "steps": a.steps,
           "warmup": a.warmup, "ms_per_step": 1000 * (load_s + desum_s), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
           "config": {"workload": workload_name(a) + "; summary stored in a local file and loaded back",
                      "join_size": total,
                      "l2": (f"the loaded summary ({nbytes / 1e6:.0f} MB on file) is larger than L2 (no flush)"
                             if nbytes > (128 << 20) else
                             f"the loaded summary ({nbytes / 1e6:.1f} MB on file) may sit in L2: each step loads it anew")},
           "summary_bytes": nbytes, "result_bytes": total * row_bytes,
           "result_to_summary_ratio": total * row_bytes / nbytes,
           "save_s": save_s, "load_s": load_s, "desummarise_s": desum_s,
           "note": "the file was just written, so the load reads from the page cache"}
    if rank == 0:
        print(json.dumps(out), flush=True)
    ctx.close()


def l2_plan(torch, dev, in_bytes):
    """Timing hygiene for inputs of in_bytes: None and a note when they are
    larger than L2 (nothing to flush); otherwise a buffer twice the L2 to
    write before every timed step (outside the timed time) and a note."""
    l2 = int(getattr(torch.cuda.get_device_properties(dev), "L2_cache_size", 0) or (128 << 20))
    if in_bytes > l2:
        return None, "inputs larger than L2 (no flush)"
    return (torch.empty(2 * l2, dtype=torch.uint8, device=dev),
            f"inputs ({in_bytes / 1e6:.1f} MB) fit in L2 ({l2 / 1e6:.0f} MB): a {2 * l2 / 1e6:.0f} MB "
            "buffer is written before every timed step, outside the timed time")


def time_query(ctx, q, stream, chunk, steps, warmup):
    """Device time of the whole path on one query (factors, summary, every
    result row), averaged over `steps` after `warmup` runs."""
    import torch
    from paper_2206_10435_gb300 import gj
    dev = torch.device("cuda", ctx.device)
    rels = [([torch.from_numpy(k).to(dev) for k in R.keys],
             [torch.from_numpy(p).to(dev) for p in R.payloads], R.attrs) for R in q.relations]
    in_bytes = sum(sum(t.numel() * t.element_size() for t in ks + ps) for ks, ps, _ in rels)
    flush_buf, note = l2_plan(torch, dev, in_bytes)
    bufs = None
    out = {}
    with torch.cuda.stream(stream):
        for it in range(warmup + steps):
            if flush_buf is not None:
                flush_buf.fill_(it & 0xff)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            ev[0].record(stream)
            ids = [ctx.load_relation(ks, attrs, ps) for ks, ps, attrs in rels]
            qq = ctx.query(ids)
            total = qq.summarize()
            ev[1].record(stream)
            if bufs is None:
                bufs = qq.alloc_columns(min(chunk, total))
            for r0 in range(0, total, chunk):
                qq.desummarize(r0, chunk, out=bufs)
            ev[2].record(stream)
            ev[2].synchronize()
            groups = sum(qq.n_groups)
            qq.close()
            for i in ids:
                ctx.release_relation(i)
            if it >= warmup:
                out.setdefault("summary_ms", 0.0)
                out.setdefault("total_ms", 0.0)
                out["summary_ms"] += ev[0].elapsed_time(ev[1]) / steps
                out["total_ms"] += ev[0].elapsed_time(ev[2]) / steps
    out.update({"join_size": total, "groups": groups, "rows": q.n_rows_total,
                "tuples_per_s": total / (out["total_ms"] / 1000.0), "l2": note})
    return out


def run_sensitivity(a, rank, world, local):
    """Section 4.2: the same chain with every tuple duplicated (result
    redundancy x 2^k) and with one more hop (more unneeded intermediate
    results).  GJ's summary cost follows the input, its desummarisation the
    result size, so neither form should change the rate of result rows."""
    import torch
    from paper_2206_10435_gb300 import datagen as G, gj
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream(torch.device("cuda", local))
    ctx = gj.Context(local, stream)
    base = G.chain_sensitivity(rows=a.rows, domain=a.domain, s=a.zipf, hops=3)
    variants = {"base_3hop": base, "dup_3hop": G.duplicate_rows(base),
                "extra_hop_4hop": G.chain_sensitivity(rows=a.rows, domain=a.domain, s=a.zipf, hops=4)}
    res = {name: time_query(ctx, q, stream, 1 << a.chunk_log2, a.steps, a.warmup)
           for name, q in variants.items()}
    out = {"metric": "result tuples materialised/s per variant (sensitivity, Section 4.2)",
           "value": res["base_3hop"]["tuples_per_s"], "unit": "tuples/s", "n_gpus": world,
           "steps": a.steps, "warmup": a.warmup, "ms_per_step": res["base_3hop"]["total_ms"],
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
           "data": "synthetic",
           "config": {"workload": (f"sensitivity: chain R_i(K_i-1,K_i), {a.rows} rows/table, Zipf("
                                   f"{a.zipf}) over [0,{a.domain}), int64 payloads; base 3 tables, "
                                   "every tuple duplicated, one extra hop"),
                      "l2": res["base_3hop"]["l2"]},
           "variants": res}
    if rank == 0:
        print(json.dumps(out), flush=True)
    ctx.close()


def run_e2e(a, q, ctx, stream, dev, total, dist, rank=0, world=1):
    import torch
    from paper_2206_10435_gb300 import gj, partition as P
    host = []
    h2d = 0
    for R in q.relations:
        ks = [torch.from_numpy(k).pin_memory() for k in R.keys]
        ps = [torch.from_numpy(p).pin_memory() for p in R.payloads]
        h2d += sum(t.numel() * t.element_size() for t in ks + ps)
        host.append((ks, ps, R.attrs))
    CH = 1 << a.e2e_chunk_log2
    d2h = 0
    with torch.cuda.stream(stream):
        ids0 = [ctx.load_relation(ks, attrs, ps, flags=gj.GJ_REL_HOST) for ks, ps, attrs in host]
        qq0 = ctx.query(ids0, drop_attrs=drop_list(a))
        qq0.summarize()
        # result chunks go straight into pinned host columns: the emit kernel
        # stores them over the host link (no device staging buffer, no copy)
        hbuf = [torch.empty(CH, dtype=torch.int32 if w == 4 else torch.int64, pin_memory=True)
                for w in qq0.col_width]
        qq0.close()
        for i in ids0:
            ctx.release_relation(i)
        row_bytes = sum(t.element_size() for t in hbuf)

        def one():
            ids = [ctx.load_relation(ks, attrs, ps, flags=gj.GJ_REL_HOST) for ks, ps, attrs in host]
            qq = ctx.query(ids, drop_attrs=drop_list(a))
            tot = qq.summarize()
            lo, hi = P.row_range(tot, rank, world)
            for r0, n in P.windows(lo, hi, CH):
                qq.desummarize(r0, n, out=hbuf)
            stream.synchronize()
            qq.close()
            for i in ids:
                ctx.release_relation(i)
            return tot

        one()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(a.e2e_steps):
            tot = one()
        torch.cuda.synchronize()
        dt = P.max_over_ranks(dist, time.perf_counter() - t0, dev)
    lo, hi = P.row_range(tot, rank, world)
    d2h = (hi - lo) * row_bytes
    return {"value": tot * a.e2e_steps / dt, "unit": UNIT, "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "steps": a.e2e_steps,
            "chunk_rows": CH, "note": "relations H2D from pinned host memory; every result chunk "
                                      "written by the emit kernel straight into pinned host "
                                      "memory over the host link; all inside the timed region"}


if __name__ == "__main__":
    main()
