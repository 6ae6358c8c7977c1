#!/usr/bin/env python
"""Benchmark of the tensor-path join + sort on one GB300 (or N replicas).

Workload (one step): the foreign-key join of R = 10^8 unique int64 keys (a
seeded random permutation of [0, 10^8), ids = positions) with S = 4x10^8 int64
foreign keys drawn Zipf(s) over R's keys, for s = 0, 0.8 and 1.2 (three joins,
each producing 4x10^8 (r_id, s_id) pairs sorted by key), plus ORDER BY key of
a 10^8-row int64 relation (a fresh copy of R).  Inputs are generated on the
device before timing and are far larger than L2 (129 MB), so no flush is
needed between steps.

Metric: join+sort input tuples per second = (3 (n_r + n_s) + n_sort) / step
time, step time = the sum of the CUDA-event times of the four library calls on
the launching stream (the untimed restore of the sort input is excluded).

`--impl reference` times the CPU oracle instead (bounded sample per step).
Under torchrun (N > 1) every rank runs an independent replica ("replicas only":
no data-path collective); the value is the sum over ranks' units / max time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "join+sort input tuples/s"
UNIT = "tuples/s"
N_R = 100_000_000
N_S = 400_000_000
N_SORT = 100_000_000


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="tj", choices=["tj", "reference"])
    ap.add_argument("--zipf", default="0,0.8,1.2")
    ap.add_argument("--budget-mb", type=float, default=256.0,
                    help="mem_budget_bytes of each join in MiB (0 = unbounded)")
    ap.add_argument("--scale", type=float, default=1.0, help="shrink the workload (debug only)")
    ap.add_argument("--e2e-steps", type=int, default=4)
    ap.add_argument("--e2e-buffers", type=int, default=2,
                    help="device buffers per input and result in the end-to-end pipeline")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the learned / batched / serving measurements")
    ap.add_argument("--serving-seconds", type=float, default=60.0,
                    help="seconds of Poisson arrivals per serving rate (at most)")
    ap.add_argument("--serving-requests", type=int, default=2000,
                    help="requests per serving rate (at most)")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# distributed plumbing (replicas)
# ---------------------------------------------------------------------------
def dist_setup():
    import torch
    import torch.distributed as dist

    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist

        dist.barrier()


def allreduce_max(x: float, ws: int) -> float:
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist

    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 8:
                continue
            try:
                sm.append(float(p[0]))
                mx.append(float(p[1]))
            except ValueError:
                continue
            for n, v in zip(names, p[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# workload
# ---------------------------------------------------------------------------
def make_workload(zipfs, scale, seed_base):
    import torch

    from paper_2602_21237_gb300 import datagen

    n_r = max(1000, int(N_R * scale))
    n_s = max(1000, int(N_S * scale))
    n_sort = max(1000, int(N_SORT * scale))
    rels = []
    kr = ir = None
    for i, s in enumerate(zipfs):
        r_k, r_i, s_k, s_i = datagen.fk_zipf(n_r, n_s, s, seed_base + 1, device="cuda")
        if kr is None:
            kr, ir = r_k, r_i
        else:
            # same R for every s (same seed), keep one copy
            del r_k, r_i
        rels.append((s, s_k, s_i))
    sort_src_k = kr.clone()
    sort_src_i = ir.clone()
    torch.cuda.synchronize()
    return n_r, n_s, n_sort, kr, ir, rels, sort_src_k[:n_sort], sort_src_i[:n_sort]


def roofline_traffic(kernel: str):
    """Bytes per algorithmic byte from the committed ncu summary of `kernel`,
    valid only while the kernel's source is unchanged since the capture."""
    import hashlib

    path = os.path.join(ROOT, "profiles", "roofline_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        ent = d[kernel]
        src = os.path.join(ROOT, ent["source"])
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        if h != ent["source_sha"]:
            return None
        return float(ent["dram_bytes_per_alg_byte"])
    except (OSError, KeyError, ValueError):
        return None


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# CPU oracle (bounded sample of the same workload)
# ---------------------------------------------------------------------------
def cpu_sample(kr, ir, rels, sort_k, sort_i, frac=1.0 / 64):
    """Host copies of a key-range slice of the workload: R rows with key below
    frac * n_r, the S rows (middle s) in that range, and frac of the sort input."""
    import torch

    n_r = kr.numel()
    lim = int(n_r * frac)
    m = kr < lim
    r_k, r_i = kr[m].cpu().numpy(), ir[m].cpu().numpy()
    s, s_k, s_i = rels[len(rels) // 2]
    ms = s_k < lim
    sk, si = s_k[ms].cpu().numpy(), s_i[ms].cpu().numpy()
    ns = int(sort_k.numel() * frac)
    return (r_k, r_i, sk, si, sort_k[:ns].cpu().numpy(), sort_i[:ns].cpu().numpy(), s, frac)


def time_oracle(sample, reps=1):
    import oracle

    r_k, r_i, sk, si, so_k, so_i, s, frac = sample
    oracle.build()
    t0 = time.perf_counter()
    for _ in range(reps):
        n = oracle.join_inner(r_k, r_i, sk, si, count_only=False).shape[0]
        oracle.sort(so_k, so_i)
    dt = (time.perf_counter() - t0) / reps
    tuples = len(r_k) + len(sk) + len(so_k)
    return tuples / dt, dt, tuples, n


def host_cores():
    try:
        n = len(os.sched_getaffinity(0))
    except AttributeError:
        n = os.cpu_count() or 1
    model = ""
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith(("model name", "cpu part", "processor name")):
                    model = ln.split(":", 1)[1].strip()
                    if ln.lower().startswith("model name"):
                        break
    except OSError:
        pass
    return n, model


def time_oracle_threads(sample, threads):
    """The same oracle on `threads` host threads: both relations and the sort
    input are split into `threads` key ranges (splitters from R's keys), each
    thread runs the unchanged oracle on its ranges (the C calls release the
    GIL), and the parts are concatenated in key order, which is the
    single-threaded result exactly.  Partitioning and concatenation are timed."""
    import concurrent.futures as cf

    import numpy as np

    import oracle

    r_k, r_i, sk, si, so_k, so_i, s, frac = sample
    oracle.build()
    oracle._load()
    t0 = time.perf_counter()
    q = np.quantile(r_k[:: max(1, len(r_k) // 65536)], np.arange(1, threads) / threads)
    split = np.unique(q.astype(r_k.dtype))
    qs = np.quantile(so_k[:: max(1, len(so_k) // 65536)], np.arange(1, threads) / threads)
    split_s = np.unique(qs.astype(so_k.dtype))

    def rng(keys, sp, t):
        lo = sp[t - 1] if t > 0 else None
        hi = sp[t] if t < len(sp) else None
        m = np.ones(len(keys), dtype=bool)
        if lo is not None:
            m &= keys >= lo
        if hi is not None:
            m &= keys < hi
        return m

    def join_part(t):
        mr, ms = rng(r_k, split, t), rng(sk, split, t)
        return oracle.join_inner(r_k[mr], r_i[mr], sk[ms], si[ms])

    def sort_part(t):
        m = rng(so_k, split_s, t)
        return oracle.sort(so_k[m], so_i[m])

    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        jp = list(ex.map(join_part, range(len(split) + 1)))
        sp = list(ex.map(sort_part, range(len(split_s) + 1)))
    pairs = np.concatenate(jp)
    sorted_k = np.concatenate([a for a, _ in sp])
    sorted_i = np.concatenate([b for _, b in sp])
    dt = time.perf_counter() - t0
    tuples = len(r_k) + len(sk) + len(so_k)
    return tuples / dt, dt, pairs, (sorted_k, sorted_i)


def cpu_baseline_line(sample, reps=3):
    """The oracle on this host's cores (T threads) and on one core, median of
    `reps` runs each; the T-thread result is checked against one core's."""
    import numpy as np

    import oracle

    cores, model = host_cores()
    one = sorted(time_oracle(sample)[1] for _ in range(reps))[reps // 2]
    runs = [time_oracle_threads(sample, cores) for _ in range(reps)]
    dt = sorted(r[1] for r in runs)[reps // 2]
    r_k, r_i, sk, si, so_k, so_i, s, frac = sample
    ok = np.array_equal(runs[0][2], oracle.join_inner(r_k, r_i, sk, si))
    ek, ei = oracle.sort(so_k, so_i)
    ok = ok and np.array_equal(runs[0][3][0], ek) and np.array_equal(runs[0][3][1], ei)
    tuples = sample_tuples(sample)
    desc = (f"key range [0, {frac:g} n_r) of the workload: {len(r_k)} R rows, {len(sk)} S rows "
            f"(Zipf s={s}), sort of {len(so_k)} rows; {cores} threads (key-range parts, "
            f"result equal to one thread's: {bool(ok)}) {dt:.3f} s, one thread {one:.2f} s, "
            f"median of {reps}; host CPU: {model or 'unknown'}")
    return {"value": tuples / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": desc, "single_thread": {"value": tuples / one, "cores": 1},
            "cpu_model": model, "threads_match_single": bool(ok)}


# ---------------------------------------------------------------------------
def run_reference(args, ws, rank):
    """The CPU oracle, as it stands, on a bounded sample per step."""
    if rank != 0:
        return
    import torch

    zipfs = [float(x) for x in args.zipf.split(",")]
    _, _, _, kr, ir, rels, sk, si = make_workload(zipfs, args.scale, 20260221)
    sample = cpu_sample(kr, ir, rels, sk, si)
    del kr, ir, rels, sk, si
    torch.cuda.empty_cache()
    cores, model = host_cores()
    for _ in range(args.warmup):
        time_oracle_threads(sample, cores)
    times = []
    for _ in range(args.steps):
        times.append(time_oracle_threads(sample, cores)[1])
    dt = statistics.mean(times)
    value = sample_tuples(sample) / dt
    desc = (f"key range [0, {sample[7]:g} n_r) of the workload: {len(sample[0])} R rows, "
            f"{len(sample[2])} S rows (Zipf s={sample[6]}), sort of {len(sample[4])} rows; "
            f"the oracle on {cores} threads over key-range parts; host CPU: {model or 'unknown'}")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": workload_config(args, zipfs),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def sample_tuples(sample):
    return len(sample[0]) + len(sample[2]) + len(sample[4])


def workload_config(args, zipfs):
    return {"workload": "fk_join_1e8x4e8_int64_zipf_plus_sort_1e8",
            "n_r": int(N_R * args.scale), "n_s": int(N_S * args.scale),
            "n_sort": int(N_SORT * args.scale), "zipf_s": zipfs,
            "mem_budget_bytes": int(args.budget_mb * (1 << 20)),
            "key_dtype": "int64", "l2_flush": "inputs larger than L2 (>= 1.6 GB per array)"}


# ---------------------------------------------------------------------------
def run_tj(args, ws, rank, local):
    import torch

    from paper_2602_21237_gb300 import api

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    zipfs = [float(x) for x in args.zipf.split(",")]
    budget = int(args.budget_mb * (1 << 20))
    n_r, n_s, n_sort, kr, ir, rels, sort_src_k, sort_src_i = make_workload(
        zipfs, args.scale, 20260221)
    out = torch.empty((n_s, 2), dtype=torch.int64, device=dev)
    sk = torch.empty_like(sort_src_k)
    si = torch.empty_like(sort_src_i)
    stream = torch.cuda.current_stream()
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    join_st = {}

    def step(timed):
        rec = {}
        for s, s_k, s_i in rels:
            a, b = ev(), ev()
            a.record(stream)
            res = api.join_inner(kr, ir, s_k, s_i, mem_budget_bytes=budget, out=out,
                                 stream=stream)
            b.record(stream)
            rec[f"join_s{s}"] = (a, b, res.shape[0])
            if not timed:
                join_st[s] = api.stats()
        sk.copy_(sort_src_k)
        si.copy_(sort_src_i)
        a, b = ev(), ev()
        a.record(stream)
        api.sort(sk, si, stream=stream)
        b.record(stream)
        rec["sort"] = (a, b, n_sort)
        return rec

    for _ in range(args.warmup):
        step(False)
    torch.cuda.synchronize()
    st0 = {f"s{s}": {k: join_st[s][k] for k in ("groups", "lanes", "partitions", "heavy_keys",
                                                  "scratch_peak", "staging_bytes",
                                                  "route_regions", "balance")}
           for s in join_st}
    for s in join_st:
        d = st0[f"s{s}"]
        # scratch (bounded by the budget) + the routed batches (held apart)
        d["device_footprint_bytes"] = d["scratch_peak"] + d["staging_bytes"]
        d["mem_budget_bytes"] = budget

    api.trace_reset()
    api.trace_enable(True)
    per_op = {}
    barrier(ws)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        w0 = time.perf_counter()
        recs = [step(True) for _ in range(args.steps)]
        torch.cuda.synchronize()
        wall = time.perf_counter() - w0
    barrier(ws)
    api.trace_enable(False)
    trace = api.trace_table()
    step_ms = []
    for rec in recs:
        tot = 0.0
        for k, (a, b, n) in rec.items():
            ms = a.elapsed_time(b)
            per_op.setdefault(k, []).append(ms)
            tot += ms
        step_ms.append(tot)
    for s, _, _ in rels:
        assert recs[-1][f"join_s{s}"][2] == n_s, "FK join must return one pair per S row"
    ms_step = statistics.mean(step_ms)
    ms_step_max = allreduce_max(ms_step, ws)
    tuples_step = len(rels) * (n_r + n_s) + n_sort
    value = tuples_step * ws / (ms_step_max / 1e3)

    def pct(xs, q):
        xs = sorted(xs)
        return xs[min(len(xs) - 1, int(round(q * (len(xs) - 1))))]

    ops = {}
    for k, xs in per_op.items():
        n_in = (n_r + n_s) if k.startswith("join") else n_sort
        ops[k] = {"mean_ms": statistics.mean(xs), "p50_ms": pct(xs, 0.5), "p99_ms": pct(xs, 0.99),
                  "tuples_per_s": n_in / (statistics.mean(xs) / 1e3)}
    peak, peak_kind = measured_peaks()
    roof = None
    launches = sum(v["launches"] for v in trace.values())
    # k_onesweep dominates the step.  The groups of a budgeted join alternate
    # between two streams and are traced per group ("group/lanes": sort passes
    # and join), since their launches overlap: the kernel's figure comes from
    # its launches that ran alone (the route passes, tj_sort's passes and the
    # learned router's sample sorts), the whole step's from all traced bytes
    # over the step time.
    solo = [trace[k] for k in ("route", "onesweep") if k in trace]
    if solo:
        by = sum(d["bytes"] for d in solo)
        ms = sum(d["ms"] for d in solo)
        n_l = sum(d["launches"] for d in solo)
        ach = by / (ms / 1e3) / 1e9
        # DRAM bytes per algorithmic byte of each kind of launch (ncu)
        ratios = {k: roofline_traffic(k) for k in ("route", "onesweep") if k in trace}
        traffic = (sum(trace[k]["bytes"] * r for k, r in ratios.items()) / n_l
                   if all(r is not None for r in ratios.values()) else None)
        per_launch_alg = by / n_l
        step_bytes = sum(v["bytes"] for v in trace.values()) / len(step_ms)
        step_ach = step_bytes / (ms_step / 1e3) / 1e9
        roof = {"bound": "hbm",
                "kernel": "k_onesweep (launches that ran alone: route passes, tj_sort, the "
                          "router's sample sorts)",
                "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                "peak_kind": f"{peak_kind} hbm_gbs (copy, burst)",
                "traffic": traffic,
                "alg_bytes_per_launch": per_launch_alg, "launches": n_l,
                "share_of_traced_ms": ms / sum(v["ms"] for v in trace.values()),
                "step": {"alg_bytes": step_bytes, "achieved": step_ach,
                         "frac": step_ach / peak,
                         "what": "algorithmic bytes of every traced kernel of one step / "
                                 "the step's time (overlapped lanes included)"}}
        # the bytes no implementation can avoid: every input row read once and
        # every result written once (keys and ids of 8 bytes, pairs of 16)
        comp = len(rels) * ((n_r + n_s) * 16 + n_s * 16) + n_sort * 32
        comp_ach = comp / (ms_step / 1e3) / 1e9
        roof["compulsory"] = {"bytes": comp, "achieved": comp_ach, "frac": comp_ach / peak,
                              "what": "inputs read once and results written once per step "
                                      "(keys, ids, pairs) / the step's time"}
        # the partitioned join's algorithmic bytes by the hash-partition model:
        # one partition pass (read + write of key and id), build read of R,
        # probe read of S, table writes at load 0.5, one 32-byte sector per
        # probe, the pairs written once (w = 16 bytes of key + id per row)
        wrow = 16
        jb = (2 * (n_r + n_s) * wrow + n_r * wrow + n_s * wrow + 2 * n_r * wrow + 32 * n_s
              + n_s * wrow)
        roof["join"] = {
            "alg_bytes_per_join": jb,
            "what": "2 (n_r + n_s) w + n_r w + n_s w + 2 n_r w + 32 n_s + |J| 2 w_id "
                    "(w = 16 B, |J| = n_s) / the join call's time",
            "per_zipf": {}}
        for s, _, _ in rels:
            ms_j = statistics.mean(per_op[f"join_s{s}"])
            a = jb / (ms_j / 1e3) / 1e9
            roof["join"]["per_zipf"][f"s{s}"] = {"ms": ms_j, "achieved": a, "frac": a / peak}
    kernels = {k: {"launches": v["launches"], "ms": v["ms"],
                   "gbs": v["bytes"] / (v["ms"] / 1e3) / 1e9 if v["ms"] > 0 else None}
               for k, v in trace.items()}

    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, kr, ir, rels, sort_src_k, sort_src_i, budget, n_r, n_s, n_sort,
                      ws)
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        sample = cpu_sample(kr, ir, rels, sort_src_k, sort_src_i)
        cpu = cpu_baseline_line(sample)
    extras = None
    if rank == 0 and ws == 1 and not args.no_extras:
        del kr, ir, rels, sort_src_k, sort_src_i, out, sk, si
        torch.cuda.empty_cache()
        extras = {"small_int32_1e6": extra_small(),
                  "learned_vs_radix": extra_learned(args.scale),
                  "batched_vs_one_at_a_time": extra_batched(args.scale),
                  "path_selection_fk_join": extra_paths(args.scale),
                  "regime_shift": extra_regime(args.scale),
                  "late_materialisation": extra_payload(args.scale),
                  "sort_single_vs_multi_key": extra_sort_multi(args.scale),
                  "serving": extra_serving(args.scale, args.serving_seconds,
                                           args.serving_requests)}
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step_max,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "int64", "data": "synthetic", "config": workload_config(args, zipfs),
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
                "clocks": clk.summary(), "gpu_launches": launches,
                "wall_ms_per_step": wall * 1e3 / args.steps, "ops": ops, "kernels": kernels,
                "join_stats": st0, "parallelism": f"replicas{ws}", "extras": extras}
        print(json.dumps(line), flush=True)


def _events_ms(fn, reps=3, warm=1):
    import torch

    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        r = fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps, r


def extra_small():
    """R and S of 10^6 rows each, int32 keys uniform in [0, 2^20), ids =
    positions: join (about 9.5e5 pairs) and sort of R, latency per call."""
    import torch

    from paper_2602_21237_gb300 import api, datagen

    kr, ir, ks, is_ = datagen.uniform_pair(10**6, 10**6, 0, 1 << 20, 20260221,
                                           torch.int32, device="cuda")
    out = torch.empty((2 * 10**6, 2), dtype=torch.int32, device="cuda")
    ms_join, r = _events_ms(lambda: api.join_inner(kr, ir, ks, is_, out=out), reps=20, warm=3)
    sk, si = kr.clone(), ir.clone()

    def srt():
        sk.copy_(kr)
        si.copy_(ir)
        return api.sort(sk, si)

    ms_copy, _ = _events_ms(lambda: (sk.copy_(kr), si.copy_(ir)), reps=20, warm=3)
    ms_sort, _ = _events_ms(srt, reps=20, warm=3)
    ms_sort = max(0.0, ms_sort - ms_copy)
    return {"workload": "uniform_int32_1e6x1e6_keys_2^20", "pairs": int(r.shape[0]),
            "join_us": 1e3 * ms_join, "join_tuples_per_s": 2e6 / (ms_join / 1e3),
            "sort_us": 1e3 * ms_sort, "sort_keys_per_s": 1e6 / (ms_sort / 1e3)}


def extra_paths(scale):
    """Execution-time path selection (paper Sec. 3.3) against the forced
    paths (Sec. 5.4) on the benchmark's FK join at Zipf 0.8 (R = 10^8, S =
    4x10^8 int64), without a budget and under the 256 MiB one: the single
    pass, the partitioned join with equal-width, PLA and MLP batches, and
    router AUTO's choice."""
    import torch

    from paper_2602_21237_gb300 import api, datagen

    n_r, n_s = max(1000, int(10**8 * scale)), max(4000, int(4 * 10**8 * scale))
    kr, ir, ks, is_ = datagen.fk_zipf(n_r, n_s, 0.8, 20260221 + 1, device="cuda")
    out = torch.empty((n_s, 2), dtype=torch.int64, device="cuda")
    res = {"workload": "fk_join_1e8x4e8_zipf0.8_int64"}
    for label, budget in (("unbounded", 0), ("budget_256MiB", 256 << 20)):
        row = {}
        for name in ("single", "radix", "pla", "mlp", "auto"):
            try:
                ms, r = _events_ms(lambda: api.join_inner(kr, ir, ks, is_, out=out, router=name,
                                                          mem_budget_bytes=budget), reps=3, warm=1)
            except api.TjError as e:
                row[name] = {"status": f"{e.name}: {e.detail}"}
                continue
            assert r.shape[0] == n_s
            st = api.stats()
            row[name] = {"ms": ms, "tuples_per_s": (n_r + n_s) / (ms / 1e3),
                         "path": "single_pass" if st["partitions"] == 0 else
                         ("radix (judge) for " if st["learned"] >= 100 else "") +
                         {2: "radix", 3: "pla", 4: "mlp"}.get(st["learned"] % 100, "?"),
                         "fused_batches": st["fused_batches"], "groups": st["groups"]}
        best = min(v["ms"] for v in row.values() if "ms" in v)
        row["auto_over_best_forced"] = row["auto"]["ms"] / best if "ms" in row["auto"] else None
        res[label] = row
    del kr, ir, ks, is_, out
    torch.cuda.empty_cache()
    return res


def extra_regime(scale, budget_mb=256):
    """Time against size at a fixed device budget: FK joins (R = N/5 unique
    int64 keys, S = 4N/5 Zipf(0.8) foreign keys) for N from 1.25e6 to 3.2e8,
    under a 256 MiB budget and unbounded.  The paper's relational path pays a
    spill term once N outgrows its working memory (Sec. 6); here every size
    stays within the budget, so the cost per tuple should not jump."""
    import torch

    from paper_2602_21237_gb300 import api, datagen

    rows = []
    for n in (1_250_000, 5_000_000, 20_000_000, 80_000_000, 320_000_000):
        n = max(1000, int(n * scale))
        n_r, n_s = n // 5, n - n // 5
        kr, ir, ks, is_ = datagen.fk_zipf(n_r, n_s, 0.8, 20260231, device="cuda")
        out = torch.empty((n_s, 2), dtype=torch.int64, device="cuda")
        row = {"n": n, "n_r": n_r, "n_s": n_s}
        for name, budget in (("budget", budget_mb << 20), ("unbounded", 0)):
            ms, r = _events_ms(lambda: api.join_inner(kr, ir, ks, is_, out=out,
                                                      mem_budget_bytes=budget), reps=3, warm=2)
            assert r.shape[0] == n_s
            st = api.stats()
            row[name] = {"ms": ms, "ns_per_tuple": 1e6 * ms / n, "tuples_per_s": n / (ms / 1e3),
                         "groups": st["groups"], "lanes": st["lanes"],
                         "scratch_peak_bytes": st["scratch_peak"]}
        rows.append(row)
        del kr, ir, ks, is_, out
        torch.cuda.empty_cache()
    return {"workload": "fk_zipf0.8_int64_R=N/5_S=4N/5", "mem_budget_bytes": budget_mb << 20,
            "sizes": rows}


def extra_payload(scale):
    """Late materialisation (paper Sec. 3.1, Sec. 3.2): the C1 join at Zipf 0.8
    (R = 10^8, S = 4x10^8 int64 keys, 256 MiB budget), then two int64 payload
    columns of R and two of S gathered through its 4x10^8 (r_id, s_id) pairs."""
    import torch

    from paper_2602_21237_gb300 import api, datagen

    n_r, n_s = max(1000, int(10**8 * scale)), max(4000, int(4 * 10**8 * scale))
    kr, ir, ks, is_ = datagen.fk_zipf(n_r, n_s, 0.8, 20260232, device="cuda")
    pairs = api.join_inner(kr, ir, ks, is_, mem_budget_bytes=256 << 20)
    del kr, ks
    g = torch.Generator(device="cuda").manual_seed(7)
    rc = [torch.randint(0, 1 << 62, (n_r,), generator=g, device="cuda") for _ in range(2)]
    sc = [torch.randint(0, 1 << 62, (n_s,), generator=g, device="cuda") for _ in range(2)]
    ms, (ro, so) = _events_ms(lambda: api.gather_pairs(pairs, rc, sc), reps=3, warm=1)
    n = pairs.shape[0]
    alg = n * (16 + 4 * 16)  # pair read + per column 8 B read and 8 B written
    res = {"workload": "fk_join_1e8x4e8_zipf0.8_int64 + 2 R and 2 S int64 payload columns",
           "pairs": int(n), "gather_ms": ms, "pairs_per_s": n / (ms / 1e3),
           "alg_bytes": alg, "alg_gbs": alg / (ms / 1e3) / 1e9,
           "note": "the payload reads are at data-dependent rows: one 32-byte sector per "
                   "8-byte element unless neighbouring pairs share it"}
    del pairs, rc, sc, ro, so, ir, is_
    torch.cuda.empty_cache()
    return res


def extra_sort_multi(scale):
    """Single-key versus multi-attribute sort keys (paper Sec. 3.2 and Sec. 5.3,
    Fig. 5) and forced versus selected paths (Sec. 5.4): int64 columns k0 in
    [0, 2^20), k1 in [0, 2^30), k2 in [0, 2^10), ids = positions; ORDER BY k1
    alone, by (k0, k1) and by (k0, k1, k2), each multi-key order sorted per
    column, folded into one key, and on the path tj_sort_multi selects.  At
    10^8 rows and at the paper's 10^6."""
    import torch

    from paper_2602_21237_gb300 import api

    res = {}
    for n in (max(1000, int(10**8 * scale)), 10**6):
        g = torch.Generator(device="cuda").manual_seed(11)
        k0 = torch.randint(0, 1 << 20, (n,), generator=g, device="cuda")
        k1 = torch.randint(0, 1 << 30, (n,), generator=g, device="cuda")
        k2 = torch.randint(0, 1 << 10, (n,), generator=g, device="cuda")
        ids = torch.arange(n, device="cuda")
        w = [torch.empty_like(k0) for _ in range(4)]

        def load(srcs):
            for d, x in zip(w, list(srcs) + [ids]):
                d.copy_(x)

        def timed(srcs, fn):
            ms_copy, _ = _events_ms(lambda: load(srcs), reps=3, warm=1)
            ms, _ = _events_ms(lambda: (load(srcs), fn()), reps=3, warm=1)
            return max(0.0, ms - ms_copy)

        row = {"rows": n, "single_key_ms": timed([k1], lambda: api.sort(w[0], w[1]))}
        for name, cols in (("two_keys", [k0, k1]), ("three_keys", [k0, k1, k2])):
            m = len(cols)
            for path in ("per_column", "packed", "auto"):
                row[f"{name}_{path}_ms"] = timed(
                    cols, lambda p=path, m=m: api.sort_multi(w[:m], w[m], path=p))
            row[f"{name}_auto_packed"] = bool(api.stats()["packed_keys"])
        res[f"n={n}"] = row
        del k0, k1, k2, ids, w
        torch.cuda.empty_cache()
    return {"workload": "int64 k0 in [0,2^20), k1 in [0,2^30), k2 in [0,2^10), ids = positions",
            "sizes": res}


def extra_learned(scale):
    """Learned partitioning (PLA, MLP) versus equal-width radix ranges on the
    log-normal mixture workload: 2^28 int64 keys per side, 1024 batches."""
    import torch

    from paper_2602_21237_gb300 import api, datagen

    n = max(1 << 16, int((1 << 28) * scale))
    kr, ir = datagen.lognormal_mix(n, 20260223, device="cuda")
    ks, is_ = datagen.lognormal_mix(n, 20260233, device="cuda")
    out = torch.empty((2 * n, 2), dtype=torch.int64, device="cuda")
    res = {"workload": f"lognormal_mix_2^{n.bit_length() - 1}_per_side_int64", "partitions": 1024}
    pairs = None
    for name, cfg in (("single_pass", dict(router="single")),
                      ("radix", dict(router="radix", partitions=1024)),
                      ("pla", dict(router="pla", partitions=1024)),
                      ("mlp", dict(router="mlp", partitions=1024))):
        ms, r = _events_ms(lambda: api.join_inner(kr, ir, ks, is_, out=out, **cfg))
        st = api.stats()
        if pairs is None:
            pairs = r.shape[0]
        assert r.shape[0] == pairs
        res[name] = {"ms": ms, "tuples_per_s": 2 * n / (ms / 1e3),
                     "balance_max_over_mean": st["balance"] if name != "single_pass" else None,
                     "radix_passes": st["radix_passes"]}
    res["pairs"] = pairs
    res["radix_balance_estimated_from_sample"] = api.stats()["radix_balance"]
    # under a device-memory budget the batches must each fit it: equal-width
    # ranges of this skewed CDF put ~40% of the rows in one batch
    budget = 1 << 30
    under = {"mem_budget_bytes": budget}
    for name in ("radix", "pla", "mlp"):
        try:
            ms, r = _events_ms(lambda: api.join_inner(kr, ir, ks, is_, out=out, router=name,
                                                      partitions=1024, mem_budget_bytes=budget))
            assert r.shape[0] == pairs
            st = api.stats()
            under[name] = {"ms": ms, "tuples_per_s": 2 * n / (ms / 1e3), "groups": st["groups"],
                           "balance_max_over_mean": st["balance"],
                           "scratch_peak_bytes": st["scratch_peak"]}
        except api.TjError as e:
            under[name] = {"status": f"{e.name}: {e.detail}"}
    # the path selected at execution time (Sec. 3.3) against the forced ones
    # (Sec. 5.4): unbounded, and under the 1 GB budget
    for label, budget_b in (("auto_unbounded", 0), ("auto_under_1GB_budget", budget)):
        ms, r = _events_ms(lambda: api.join_inner(kr, ir, ks, is_, out=out, router="auto",
                                                  partitions=1024, mem_budget_bytes=budget_b))
        assert r.shape[0] == pairs
        st = api.stats()
        res[label] = {"ms": ms, "tuples_per_s": 2 * n / (ms / 1e3),
                      "path": "single_pass" if st["partitions"] == 0 else
                      ("radix (judge) for " if st["learned"] >= 100 else "") +
                      {2: "radix", 3: "pla", 4: "mlp"}.get(st["learned"] % 100, "?"),
                      "groups": st["groups"]}
    res["under_1GB_budget"] = under
    del kr, ir, ks, is_, out
    torch.cuda.empty_cache()
    return res


def extra_batched(scale):
    """4096 joins, |R|, |S| log-uniform in [1e3, 1e6], int32 keys uniform over
    [0, 2|R|): one batched call (autotuned, one CUDA graph) versus one call per
    join."""
    import time as _t

    import torch

    from paper_2602_21237_gb300 import api, datagen

    hi = max(2e3, 1e6 * scale)
    r_off, s_off, kr, ir, ks, is_ = datagen.batch_jobs(4096, 1e3, hi, 20260224, device="cuda")
    out = torch.empty((max(1, s_off[-1] * 2), 2), dtype=torch.int32, device="cuda")
    reps = 3

    def timed():
        api.join_batch(r_off, s_off, kr, ir, ks, is_, out=out)  # warm
        torch.cuda.synchronize()
        t0 = _t.perf_counter()
        for _ in range(reps):
            p, _o = api.join_batch(r_off, s_off, kr, ir, ks, is_, out=out)
        torch.cuda.synchronize()
        return (_t.perf_counter() - t0) / reps, p, api.stats()

    # the default digit width and tile (forced, before any tuning in this
    # process), then the autotuner's choice (selected, Sec. 5.4)
    td, pd, sd = timed()
    api.join_batch(r_off, s_off, kr, ir, ks, is_, out=out, autotune=True)
    torch.cuda.synchronize()
    tb, p, st = timed()
    assert pd.shape[0] == p.shape[0]
    t0 = _t.perf_counter()
    tot = 0
    for j in range(4096):
        a, b, c, d = r_off[j], r_off[j + 1], s_off[j], s_off[j + 1]
        tot += api.join_inner(kr[a:b], ir[a:b], ks[c:d], is_[c:d], out=out[tot:]).shape[0]
    torch.cuda.synchronize()
    t1 = _t.perf_counter() - t0
    rows = r_off[-1] + s_off[-1]
    assert tot == p.shape[0]
    res = {"jobs": 4096, "rows": rows, "pairs": tot,
           "batched": {"ms": tb * 1e3, "tuples_per_s": rows / tb, "tile_rows": st["tile_rows"],
                       "digit_cap": st["digit_cap"], "radix_passes": st["radix_passes"],
                       "config": "autotuned (selected)"},
           "batched_default": {"ms": td * 1e3, "tuples_per_s": rows / td,
                               "tile_rows": sd["tile_rows"], "digit_cap": sd["digit_cap"],
                               "radix_passes": sd["radix_passes"],
                               "config": "default digit width and tile (forced)"},
           "one_at_a_time": {"ms": t1 * 1e3, "tuples_per_s": rows / t1}}
    del kr, ir, ks, is_, out
    torch.cuda.empty_cache()
    return res


def extra_serving(scale, seconds=60.0, max_requests=2000,
                  rates=(10.0, 30.0, 100.0, 300.0, 1000.0, 3000.0, 10000.0), budget_gb=64,
                  workers=8):
    """Serving (the P50/P99 framing of the paper's Sec. 5.2 and Sec. 6): Poisson
    arrivals of foreign-key join requests at each rate, 2000 requests or 60 s
    of arrivals per rate, admitted against a 64 GB device budget.  |R| and |S|
    are log-uniform in [1e4, 1e8]: R takes one of nine log-spaced sizes (the
    first |R| keys of one random permutation of [0, 1e8), so R keys are
    unique), S is a slice of a pool of Zipf(1.0) draws over that R's keys
    (so |J| = |S|), int64 keys and ids."""
    import math

    import torch

    from paper_2602_21237_gb300 import api, datagen

    top = max(20_000, int(1e8 * scale))
    g = torch.Generator(device="cuda").manual_seed(20260225)
    kr = torch.randperm(top, generator=g, device="cuda", dtype=torch.int64)  # R pool
    ir = torch.arange(top, device="cuda", dtype=torch.int64)
    classes = sorted({max(10_000, min(top, int(round(10 ** (4 + 0.5 * i))))) for i in range(9)})
    pools = {}
    for c in classes:  # Zipf(1.0) over R[:c], through an independent permutation
        perm = torch.randperm(c, generator=g, device="cuda", dtype=torch.int64)
        ranks = datagen.zipf_ranks(top, c, 1.0, g, "cuda")
        pools[c] = kr[:c][perm[ranks]]
        del perm, ranks
    # the workers' own streams do not wait for this one: inputs complete first
    torch.cuda.synchronize()
    srv = api.Server(mem_budget_bytes=int(budget_gb * (1 << 30)), workers=workers)
    out = []
    for i, lam in enumerate(rates):
        n_req = int(min(max_requests, max(20, lam * seconds)))
        nr = datagen.log_uniform_sizes(n_req, 1e4, top, 20260300 + i)
        ns = datagen.log_uniform_sizes(n_req, 1e4, top, 20260400 + i)
        gh = torch.Generator().manual_seed(20260500 + i)
        reqs = []
        for a, b in zip(nr, ns):
            # the class nearest |R| in log scale
            c = min(classes, key=lambda x: abs(math.log(x) - math.log(a)))
            off = int(torch.randint(0, top - b + 1, (1,), generator=gh))
            reqs.append(api.Server.join_request(kr[:c], ir[:c], pools[c][off:off + b],
                                                ir[off:off + b], None, b))
        arr = datagen.poisson_arrivals(lam, n_req, 20260600 + i)
        srv.reset_stats()
        tickets = srv.replay(reqs, arr)
        res = [srv.wait(t) for t in tickets]
        rep = srv.report()
        assert all(r["status"] == 0 for r in res), res[:3]
        # foreign keys: every S row has exactly one partner
        assert all(r["out_count"] == q.n_s for r, q in zip(res, reqs))
        out.append({"rate_per_s": lam, "requests": n_req, "completed": rep["completed"],
                    "p50_ms": rep["p50_ms"], "p99_ms": rep["p99_ms"], "max_ms": rep["max_ms"],
                    "mean_ms": rep["mean_ms"], "arrival_span_s": float(arr[-1]),
                    "throughput_tuples_per_s": rep["tuples"] / max(rep["makespan_s"], 1e-9),
                    "peak_inflight": rep["peak_inflight"], "bypasses": rep["bypasses"],
                    "peak_reserved_gb": rep["peak_reserved"] / 2**30})
        del reqs
    srv.close()
    del kr, ir, pools
    torch.cuda.empty_cache()
    return {"budget_gb": budget_gb, "workers": workers,
            "sizes": f"|R| in 9 log-spaced sizes of [1e4, {top:.0e}] (log-uniform draws "
                     f"rounded), |S| log-uniform in [1e4, {top:.0e}]",
            "keys": "int64, R unique, S Zipf(1.0) over the request's R keys (|J| = |S|)",
            "per_rate": f"min({max_requests} requests, {seconds:g} s of arrivals)",
            "rates": out}


def run_e2e(args, kr, ir, rels, sort_src_k, sort_src_i, budget, n_r, n_s, n_sort, ws):
    """Same metric through the public API with host buffers: every step copies
    its inputs from pinned host memory and reads every result back.  The steps
    are pipelined the way a caller streaming batches would: copies in on one
    stream, the library calls on another, copies out on a third, with two (or
    --e2e-buffers) device buffers for R, S, the pairs and the sort input, so the next job's
    inputs arrive while the current job runs and each result leaves while the
    next one runs.  The timed region covers K whole steps, from the first copy
    in to the last copy out."""
    import torch

    from paper_2602_21237_gb300 import api

    dev = kr.device
    pin = lambda t: t.cpu().pin_memory()  # noqa: E731
    h_kr, h_ir = pin(kr), pin(ir)
    h_s = [(s, pin(a), pin(b)) for s, a, b in rels]
    h_sk, h_si = pin(sort_src_k), pin(sort_src_i)
    h_out = torch.empty((n_s, 2), dtype=torch.int64).pin_memory()
    h_sorted_k = torch.empty_like(h_sk).pin_memory()
    h_sorted_i = torch.empty_like(h_si).pin_memory()
    nb = max(2, int(getattr(args, "e2e_buffers", 2)))  # device buffers per input and result
    many = lambda f: [f() for _ in range(nb)]  # noqa: E731
    d_kr, d_ir = many(lambda: torch.empty_like(kr)), many(lambda: torch.empty_like(ir))
    d_sk = many(lambda: torch.empty((n_s,), dtype=torch.int64, device=dev))
    d_si = many(lambda: torch.empty((n_s,), dtype=torch.int64, device=dev))
    d_out = many(lambda: torch.empty((n_s, 2), dtype=torch.int64, device=dev))
    d_ok, d_oi = many(lambda: torch.empty_like(sort_src_k)), many(lambda: torch.empty_like(sort_src_i))
    s_in, s_run, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    ev = lambda: torch.cuda.Event()  # noqa: E731
    nj = len(h_s)
    bytes_in = 2 * kr.numel() * 8 + sum(2 * a.numel() * 8 for _, a, _ in h_s) + \
        2 * h_sk.numel() * 8

    def run(steps):
        """K steps; returns the D2H bytes of one step (the pairs counts)."""
        done_s = {}    # join item -> event: its S and pair buffers are free again
        done_out = {}  # join item -> event: its pairs have been read out
        done_r = {}    # step -> event: its R buffer is free again
        done_sort = {}
        d2h = 0
        items = [(k, j) for k in range(steps) for j in range(nj)]

        def copy_in(i):
            k, j = items[i]
            _, a, b = h_s[j]
            with torch.cuda.stream(s_in):
                if i >= nb:
                    s_in.wait_event(done_s[i - nb])
                d_sk[i % nb].copy_(a, non_blocking=True)
                d_si[i % nb].copy_(b, non_blocking=True)
                e = ev()
                e.record(s_in)
            return e

        def copy_in_r(k):
            with torch.cuda.stream(s_in):
                if k >= nb:
                    s_in.wait_event(done_r[k - nb])
                d_kr[k % nb].copy_(h_kr, non_blocking=True)
                d_ir[k % nb].copy_(h_ir, non_blocking=True)
                e = ev()
                e.record(s_in)
            return e

        def copy_in_sort(k):
            with torch.cuda.stream(s_in):
                if k >= nb:
                    s_in.wait_event(done_sort_read[k - nb])  # read out, free again
                d_ok[k % nb].copy_(h_sk, non_blocking=True)
                d_oi[k % nb].copy_(h_si, non_blocking=True)
                e = ev()
                e.record(s_in)
            return e

        done_sort_read = {}
        in_r = {0: copy_in_r(0)}
        in_s = {}
        for i0 in range(min(nb, len(items))):
            in_s[i0] = copy_in(i0)
        in_sort = {}
        for i, (k, j) in enumerate(items):
            s_run.wait_event(in_r[k])
            s_run.wait_event(in_s[i])
            if i >= nb:
                s_run.wait_event(done_out[i - nb])  # its pair buffer has been read out
            res = api.join_inner(d_kr[k % nb], d_ir[k % nb], d_sk[i % nb], d_si[i % nb],
                                 mem_budget_bytes=budget, out=d_out[i % nb], stream=s_run)
            done_s[i] = ev()
            done_s[i].record(s_run)
            with torch.cuda.stream(s_out):
                s_out.wait_event(done_s[i])
                h_out[: res.shape[0]].copy_(res, non_blocking=True)
                done_out[i] = ev()
                done_out[i].record(s_out)
            if k == 0:
                d2h += res.numel() * 8
            # inputs queued in the order they are needed: S two jobs ahead; after
            # a step's first join, its sort input and the next step's R
            if i + nb < len(items):
                in_s[i + nb] = copy_in(i + nb)
            if j == 0:
                in_sort[k] = copy_in_sort(k)
                if k + 1 < steps:
                    in_r[k + 1] = copy_in_r(k + 1)
            if j == nj - 1:
                s_run.wait_event(in_sort[k])
                api.sort(d_ok[k % nb], d_oi[k % nb], stream=s_run)
                done_sort[k] = ev()
                done_sort[k].record(s_run)
                done_r[k] = done_sort[k]  # the step's joins are done before its sort
                with torch.cuda.stream(s_out):
                    s_out.wait_event(done_sort[k])
                    h_sorted_k.copy_(d_ok[k % nb], non_blocking=True)
                    h_sorted_i.copy_(d_oi[k % nb], non_blocking=True)
                    done_sort_read[k] = ev()
                    done_sort_read[k].record(s_out)
                if k == 0:
                    d2h += 2 * d_ok[0].numel() * 8
        torch.cuda.synchronize()
        return d2h

    run(1)
    barrier(ws)
    t0 = time.perf_counter()
    d2h = run(args.e2e_steps)
    dt = (time.perf_counter() - t0) / args.e2e_steps
    dt = allreduce_max(dt, ws)
    tuples_step = len(rels) * (n_r + n_s) + n_sort
    return {"value": tuples_step * ws / dt, "unit": UNIT, "h2d_bytes_per_step": bytes_in,
            "d2h_bytes_per_step": d2h, "ms_per_step": dt * 1e3, "steps": args.e2e_steps,
            "pipelining": f"copies in, library calls and copies out on three streams, {nb} "
                          "device buffers per input and result; K steps back to back"}


def main():
    args = parse()
    ws, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, ws, rank)
    else:
        run_tj(args, ws, rank, local)
    if ws > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
