#!/usr/bin/env python
"""Throughput benchmark of the GB300 count-and-emit frequency sort.

Workload (one "step"): the single-array dispatch sweep at N = 3e7 int64 keys:
K in {4, 8, 9, 200, 4096, 1.3e5, 6.7e5, 1.5e7, 3e7} with uniform and Zipf(1.1)
frequencies over K values drawn uniformly from the 64-bit range, plus one
spill-trigger column (strided sample positions hold a 64-value set, every
other key distinct): 19 columns, 5.7e8 keys, every column sorted once through
the C ABI (cafs_sort) per step.  Inputs are resident in HBM before the timed
region; each column (240 MB) is larger than L2, so no flush is needed.

Printed JSON line (rank 0): value = whole-job Gkeys/s; roofline = the
pipeline kernel's achieved bytes (one read + one write of every column, the
sort's minimum traffic) per CUDA-event second against the measured HBM copy
bandwidth, with the DRAM traffic of the committed ncu summary when it was
taken on the current kernel sources; e2e = the same metric through the
request server (cafs_server_run_trace) with pinned host buffers, copies
inside the timed region, copies and sorting of different columns overlapped
(the blocking one-column-at-a-time cafs_sort_host figure beside it);
cpu_baseline = the CPU oracle on a bounded sample of the same columns.

Three more legs (rank 0; --no-argsort / --no-batched / --no-served skip them):
  argsort: cafs_argsort (sorted keys plus the stable permutation) on four
    sweep columns, checked against and timed beside torch.sort(stable=True),
    two sweep columns' bits sorted as uint64 and float64 keys, and five
    input profiles (runs of equal keys, one group per key, nearly sorted);
  batched: 4096 int64 columns (N log-uniform [1e3, 1e6], K log-uniform
    [2, min(N/4, 5e4)], Zipf 1.1) and 64 mixed int32/int64 columns (N 1e3..3e7,
    K 2..N, 4 spill-trigger columns): one recorded batched launch (default
    and autotuned knobs) against one cafs_sort per column;
  served: open-loop Poisson traces at 1e3, 1e4, 1e5 requests/s (int64, N
    log-uniform [1e3, 3e6], K log-uniform [2, 1e5], Zipf 1.1) against the
    request server with an 8 GB budget and against serial cafs_sort_host;
    p50/p99 latency and keys/s.

``--impl reference`` times the CPU oracle instead (the only "reference" this
method has: the paper ships no code), on the same metric and columns.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gkeys/s and % HBM roofline at N=3e7 over K; batched vs per-array; p99 latency"
SWEEP_K = [4, 8, 9, 200, 4096, 130_000, 670_000, 15_000_000, 30_000_000]


def sweep_specs(n: int):
    specs = []
    for dist in ("uniform", "zipf"):
        for k in SWEEP_K:
            specs.append({"name": f"{dist}_K{k}", "K": k, "dist": dist})
    specs.append({"name": "spill_trigger", "K": None, "dist": "spill"})
    return specs


def make_column(spec, n, seed):
    from paper_2605_25040_gb300 import datagen as G
    if spec["dist"] == "spill":
        return G.spill_trigger(n, np.int64, seed=seed)
    return G.column(n, min(spec["K"], n), spec["dist"], np.int64, seed=seed)


def make_column_device(spec, n, seed, device):
    """The same column as make_column, generated in device memory."""
    from paper_2605_25040_gb300 import datagen as G
    if spec["dist"] == "spill":
        return G.spill_trigger_torch(n, np.int64, seed=seed, device=device)
    return G.column_torch(n, min(spec["K"], n), spec["dist"], np.int64, seed=seed, device=device)


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def traffic_record(kernel: str):
    """DRAM bytes per launch from the committed ncu summary of ``kernel``, or
    None when the kernel's sources changed since that capture."""
    import glob
    import re
    from paper_2605_25040_gb300 import build as B
    try:
        current = B.kernel_source_hash(kernel)
    except Exception:
        return None
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        for line in open(path):
            m = re.match(r"traffic-record: (\{.*\})\s*$", line)
            if not m:
                continue
            rec = json.loads(m.group(1))
            if rec.get("kernel") == kernel and rec.get("source_sha256") == current:
                rec["profile"] = os.path.relpath(path, ROOT)
                return rec
    return None


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int, period_ms: int = 50):
        self.index = index
        self.period_ms = period_ms
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", f"-lms={self.period_ms}"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(columns, budget_s: float = 12.0) -> dict:
    """The CPU oracle (frequency_sort) as it stands on a bounded sample: the
    given columns in turn, repeated until about ``budget_s`` of CPU work."""
    from oracle import cafs_oracle as O
    keys, t, runs = 0, 0.0, 0
    while t < budget_s:
        name, x = columns[runs % len(columns)]
        t0 = time.perf_counter()
        O.frequency_sort(x)
        t += time.perf_counter() - t0
        keys += x.size
        runs += 1
    names = ", ".join(n for n, _ in columns)
    return {"value": keys / t / 1e9, "unit": "Gkeys/s", "cores": 1, "kind": "oracle",
            "sample": f"{runs} sorts of N={columns[0][1].size} sweep columns taken in turn from ({names}), "
                      f"{t:.1f} s of numpy count-then-emit (single-threaded)",
            **host_cpu()}


def host_cpu() -> dict:
    """The host the CPU legs ran on: logical CPUs and the model name."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() in ("Model name", "Model"):
                model = line.split(":", 1)[1].strip()
                if line.startswith("Model name"):
                    break
    except Exception:
        pass
    if not model:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith(("model name", "cpu part")):
                    model = line.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    import platform
    return {"nproc": os.cpu_count(), "cpu_model": model, "machine": platform.machine()}


def _time_ms(torch, fn, warmup=2, reps=5):
    """Median CUDA-event time of fn() on the current stream (ms)."""
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return statistics.median(ts), min(ts)


def _batched_case(torch, cafs, keys, workload, tune=True):
    """One recorded batched launch (CUDA graph) vs one cafs_sort per column;
    the launch with default knobs and with the autotuner's knobs."""
    import collections
    from paper_2605_25040_gb300 import autotune
    outs = [torch.empty_like(k) for k in keys]
    ref = [torch.empty_like(k) for k in keys]
    total = sum(k.numel() for k in keys)
    nbytes = sum(k.numel() * k.element_size() for k in keys)

    def per_array():
        for k, o in zip(keys, ref):
            cafs.sort(k, o)

    per_ms, per_min = _time_ms(torch, per_array)
    tuned = None
    default_ms = None
    if tune:
        tuned = autotune.tuned(keys, outs, reps=3, rounds=2)
        default_plan = cafs.BatchPlan(keys, outs)
        default_ms, _ = _time_ms(torch, default_plan.launch)
        default_plan.close()
    plan = cafs.BatchPlan(keys, outs, tuning=tuned["tuning"] if tuned else None)
    l0 = cafs.kernel_launch_count()
    plan_ms, plan_min = _time_ms(torch, plan.launch)
    launches_per_batch = (cafs.kernel_launch_count() - l0) / 7.0
    reps = plan.reports()
    plan.close()
    same = all(torch.equal(a, b) for a, b in zip(outs, ref))
    sorted_ok = all(torch.equal(o, torch.sort(k).values) for k, o in zip(keys, outs))
    peak, _ = load_peaks()
    return {
        "workload": workload, "columns": len(keys), "keys": total,
        "batched_graph": {"ms": plan_ms, "min_ms": plan_min, "gkeys_s": total / plan_ms / 1e6,
                          "frac_hbm": 2 * nbytes / (plan_ms / 1e3) / 1e9 / peak,
                          "kernel_launches": launches_per_batch},
        "per_array": {"ms": per_ms, "min_ms": per_min, "gkeys_s": total / per_ms / 1e6,
                      "kernel_launches": len(keys)},
        "default_knobs_ms": default_ms,
        "tuning": ({"knobs": tuned["tuning"], "cached": tuned["cached"], "trials": tuned["trials"],
                    "tuner_default_ms": tuned["default_ms"], "tuner_best_ms": tuned["ms"]}
                   if tuned else None),
        "speedup": per_ms / plan_ms,
        "verified_vs_torch_sort": bool(same and sorted_ok),
        "paths": dict(collections.Counter(cafs.path_name(r["path"]) for r in reps)),
        "timing": "CUDA events on the current stream, median of 5 after 2 warm-ups; inputs larger than L2",
    }


def bench_argsort(torch, cafs, dev_in, names, peak, want=("uniform_K4", "uniform_K200", "zipf_K4096",
                                                        "uniform_K30000000")):
    """cafs_argsort (sorted keys + stable permutation) on some sweep columns,
    checked against torch's stable sort; torch.sort(stable=True) timed beside."""
    res = {"timing": "CUDA events on the current stream, median of 5 after 2 warm-ups; inputs larger than L2",
           "algorithmic_bytes_per_key": 20, "columns": []}
    ok_all = True
    for name, x in zip(names, dev_in):
        if name not in want:
            continue
        out = torch.empty_like(x)
        perm = torch.empty(x.numel(), dtype=torch.int32, device=x.device)
        ms, ms_min = _time_ms(torch, lambda: cafs.argsort(x, out, perm))
        ref = torch.sort(x, stable=True)
        ok = bool(torch.equal(ref.values, out)) and bool(torch.equal(ref.indices, perm.long() & 0xFFFFFFFF))
        ok_all &= ok
        del ref
        t_ms, _ = _time_ms(torch, lambda: torch.sort(x, stable=True))
        _, _, r = cafs.argsort(x, out, perm, report=True)
        n = x.numel()
        res["columns"].append({"column": name, "path": cafs.path_name(r["path"]), "ms": round(ms, 4),
                               "gkeys_s": round(n / (ms / 1e3) / 1e9, 2),
                               "frac_hbm": round(20 * n / (ms / 1e3) / 1e9 / peak, 4),
                               "torch_sort_stable_ms": round(t_ms, 4)})
        del out, perm
    res["verified_vs_torch_sort_stable"] = ok_all
    torch.cuda.empty_cache()
    return res


def bench_key_types(torch, cafs, dev_in, names, col_ms, want=("uniform_K200", "uniform_K30000000")):
    """The same sweep columns' bits sorted as uint64 and as float64 keys
    (order-preserving map, signed sort, map back), checked against torch's
    signed sort of the mapped bits and timed beside the int64 sort."""
    res = {"timing": "CUDA events on the current stream, median of 5 after 2 warm-ups; inputs larger than L2",
           "columns": []}
    ok_all = True
    sign = torch.tensor(-(1 << 63), dtype=torch.int64, device="cuda")
    for i, (name, x) in enumerate(zip(names, dev_in)):
        if name not in want:
            continue
        out = torch.empty_like(x)
        row = {"column": name, "int64_ms": round(col_ms[i], 4)}
        for kt in ("uint64", "float64"):
            ms, _ = _time_ms(torch, lambda: cafs.sort(x, out, key_type=kt))
            mapped = x ^ sign if kt == "uint64" else torch.where(x < 0, x ^ ~sign, x)
            ref = torch.sort(mapped).values
            ref = ref ^ sign if kt == "uint64" else torch.where(ref < 0, ref ^ ~sign, ref)
            ok_all &= bool(torch.equal(ref, out))
            del mapped, ref
            row[kt + "_ms"] = round(ms, 4)
            row[kt + "_gkeys_s"] = round(x.numel() / (ms / 1e3) / 1e9, 2)
        res["columns"].append(row)
        del out
    res["verified_vs_torch_sort_of_mapped_bits"] = ok_all
    torch.cuda.empty_cache()
    return res


def bench_profiles(torch, cafs, n, peak):
    """Input profiles at N = 3e7 int64: runs of equal keys, one group per key,
    a nearly sorted column; checked against torch.sort."""
    from paper_2605_25040_gb300 import datagen as G
    cases = [("runs_mean64_zipf_K4096", lambda: G.runs_column(n, 4096, 64.0, "zipf", np.int64, seed=1)),
             ("runs_mean4_K200", lambda: G.runs_column(n, 200, 4.0, "uniform", np.int64, seed=2)),
             ("grouped_K200", lambda: G.grouped_column(n, 200, np.int64, seed=3)),
             ("grouped_K100000", lambda: G.grouped_column(n, 100_000, np.int64, seed=4)),
             ("almost_sorted_K200_swaps3000", lambda: G.almost_sorted(n, 200, 3000, np.int64, seed=5))]
    res = {"timing": "CUDA events on the current stream, median of 5 after 2 warm-ups; inputs larger than L2",
           "columns": []}
    ok_all = True
    for name, make in cases:
        x = torch.from_numpy(make()).cuda()
        out = torch.empty_like(x)
        ms, _ = _time_ms(torch, lambda: cafs.sort(x, out))
        _, rep = cafs.sort_ex(x, out)
        ok_all &= bool(torch.equal(torch.sort(x).values, out))
        res["columns"].append({"column": name, "path": cafs.path_name(rep["path"]), "ms": round(ms, 4),
                               "gkeys_s": round(n / (ms / 1e3) / 1e9, 2),
                               "frac_hbm": round(16 * n / (ms / 1e3) / 1e9 / peak, 4)})
        del x, out
    res["verified_vs_torch_sort"] = ok_all
    torch.cuda.empty_cache()
    return res


MID_K = [10_000, 30_000, 100_000]


def bench_mid_k(torch, cafs, n, peak):
    """The hash-count path between one CTA's shared table and K = 1e5 (the
    paper's operating range, Sec. 7.1): N = 3e7 int64, K in {1e4, 3e4, 1e5}
    with uniform and Zipf(1.1) frequencies; per column the branch, the phase
    split from the device timeline and the fraction of the HBM roofline."""
    from paper_2605_25040_gb300 import datagen as G
    res = {"timing": "CUDA events on the current stream, median of 5 after 2 warm-ups; inputs larger than L2",
           "algorithmic_bytes_per_key": 16, "columns": []}
    ok_all = True
    for dist, base in (("uniform", 1000), ("zipf", 2000)):
        for k in MID_K:
            x = G.column_torch(n, k, dist, np.int64, seed=base + k, device="cuda")
            out = torch.empty_like(x)
            ms, ms_min = _time_ms(torch, lambda: cafs.sort(x, out))
            _, rep = cafs.sort_ex(x, out)
            ok_all &= bool(torch.equal(torch.sort(x).values, out))
            tl = rep["timeline_ns"]
            phases, prev = {}, tl[0]
            for idx, nm in ((1, "sample"), (2, "monotone"), (3, "count"), (4, "pairs"),
                            (5, "finish")):
                if tl[idx]:
                    phases[nm] = round((tl[idx] - prev) / 1e3, 1)
                    prev = tl[idx]
            res["columns"].append({"column": f"{dist}_K{k}", "path": cafs.path_name(rep["path"]),
                                   "k_hat": rep["est"]["k_hat"], "k_distinct": rep["k_distinct"],
                                   "ms": round(ms, 4), "min_ms": round(ms_min, 4), "phases_us": phases,
                                   "gkeys_s": round(n / (ms / 1e3) / 1e9, 2),
                                   "frac_hbm": round(16 * n / (ms / 1e3) / 1e9 / peak, 4)})
            del x, out
    res["verified_vs_torch_sort"] = ok_all
    torch.cuda.empty_cache()
    return res


def hash_count_summary(sweep, mid_k, specs, bytes_per_col, peak):
    """The count-and-emit columns (tiny or main branch) with K <= 1e5 of the
    sweep and of the mid-K leg: their combined and worst fraction of the
    HBM roofline (the target range of the hash-count path)."""
    cols = []
    for row, spec in zip(sweep, specs):
        if spec["K"] is not None and spec["K"] <= 100_000 and row["path"] in ("tiny", "main", "tiny_miss_main"):
            cols.append((row["column"], row["ms"]))
    for row in (mid_k or {}).get("columns", []):
        if row["path"] in ("tiny", "main", "tiny_miss_main"):
            cols.append(("mid_" + row["column"], row["ms"]))
    if not cols:
        return None
    tot_ms = sum(ms for _, ms in cols)
    ach = bytes_per_col * len(cols) / (tot_ms / 1e3) / 1e9
    worst = max(cols, key=lambda c: c[1])
    return {"achieved": ach, "frac": ach / peak, "columns": [c for c, _ in cols],
            "worst_column": worst[0], "worst_frac": bytes_per_col / (worst[1] / 1e3) / 1e9 / peak}


def host_link(torch, nbytes=1 << 30, reps=5):
    """Pinned host <-> device copy bandwidth (GB/s), one cudaMemcpyAsync per
    buffer, CUDA events on the current stream: the ceiling of every figure
    that moves keys through host memory."""
    h = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    d = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    out = {}
    for name, fn in (("h2d_gbs", lambda: d.copy_(h, non_blocking=True)),
                     ("d2h_gbs", lambda: h.copy_(d, non_blocking=True))):
        ms, _ = _time_ms(torch, fn, warmup=2, reps=reps)
        out[name] = round(nbytes / (ms / 1e3) / 1e9, 1)
    # Both directions at once on two streams, as a pipeline of columns moves
    # them (one column's copy in beside another's copy out).
    h2 = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    d2 = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()

    def duplex():
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(s_in):
            d.copy_(h, non_blocking=True)
        with torch.cuda.stream(s_out):
            h2.copy_(d2, non_blocking=True)
        torch.cuda.synchronize()
        return time.perf_counter() - t0

    for _ in range(2):
        duplex()
    dt = float(np.median([duplex() for _ in range(reps)]))
    out["duplex_gbs_each_way"] = round(nbytes / dt / 1e9, 1)
    out["bytes_per_copy"] = nbytes
    out["method"] = ("pinned torch tensors, one copy per direction, median of 5 after 2 warm-ups; duplex: "
                     "one copy each way at once on two streams, host clock around both")
    del h, d, h2, d2
    torch.cuda.empty_cache()
    return out


def bench_batched(torch, cafs):
    from paper_2605_25040_gb300 import datagen as G
    res = {}
    specs = G.batch_specs(4096, seed=3)
    keys = [G.batch_column_torch(n, k, i, 3, device="cuda") for i, (n, k) in enumerate(specs)]
    res["batch_4096"] = _batched_case(
        torch, cafs, keys, "4096 int64 columns, N log-uniform [1e3, 1e6], K log-uniform [2, min(N/4, 5e4)], Zipf 1.1")
    del keys
    mspecs = G.mixed_specs()
    keys = [G.mixed_column_torch(n, k, t, kind, i, 0, device="cuda") for i, (n, k, t, kind) in enumerate(mspecs)]
    res["mixed_64"] = _batched_case(
        torch, cafs, keys, "64 columns alternating int32/int64, N log-spaced 1e3..3e7, K log-spaced 2..N "
                           "(K = N included), 4 spill-trigger columns")
    del keys
    torch.cuda.empty_cache()
    return res


def bench_served(torch, cafs, rates=(1e3, 1e4, 1e5), budget=8 << 30, pool_size=256):
    """Open-loop Poisson traces against the request server and the serial baseline."""
    from paper_2605_25040_gb300 import datagen as G
    specs = G.batch_specs(pool_size, seed=5, n_lo=1e3, n_hi=3e6, k_cap=1e5)
    dev = [G.batch_column_torch(n, k, i, 5, device="cuda") for i, (n, k) in enumerate(specs)]
    pin_in = [t.cpu().pin_memory() for t in dev]
    pin_out = [torch.empty_like(t).pin_memory() for t in pin_in]
    pool = [(a.numpy(), b.numpy()) for a, b in zip(pin_in, pin_out)]
    srv = cafs.Server(budget)
    out = {"budget_bytes": budget, "request_pool": f"{pool_size} int64 columns, N log-uniform [1e3, 3e6], "
                                                   "K log-uniform [2, 1e5], Zipf 1.1 (pinned host buffers)",
           "latency": "arrival (scheduled) to sorted keys in host memory", "rates": []}
    try:
        # untimed warm-up: every pool column once, so that the server's arena,
        # workspaces and plans exist before the first measured trace
        srv.run_trace(pool, np.arange(pool_size) * 1e-4)
        cafs.serial_run_trace(pool, np.arange(pool_size) * 1e-4)
        for rate in rates:
            nreq = int(min(20000, max(2000, rate)))
            gaps = G.exponential_gaps(rate, nreq, seed=int(rate))
            arrivals = np.cumsum(gaps) - gaps[0]
            pick = [(i * 7919) % pool_size for i in range(nreq)]
            pairs = [pool[j] for j in pick]
            keys = sum(pool[j][0].size for j in pick)
            lat, el = srv.run_trace(pairs, arrivals)
            st = srv.stats()
            lat_s, el_s = cafs.serial_run_trace(pairs, arrivals)
            out["rates"].append({
                "rate_req_s": rate, "requests": nreq, "keys": keys,
                "server": {"gkeys_s": keys / el / 1e9, "p50_us": float(np.percentile(lat, 50)),
                           "p99_us": float(np.percentile(lat, 99)), "elapsed_s": el},
                "serial": {"gkeys_s": keys / el_s / 1e9, "p50_us": float(np.percentile(lat_s, 50)),
                           "p99_us": float(np.percentile(lat_s, 99)), "elapsed_s": el_s},
            })
        out["server_stats"] = srv.stats()
    finally:
        srv.close()
    ok = True
    for t, (_, o) in zip(dev, pool):
        ok &= bool(torch.equal(torch.from_numpy(o).cuda(), torch.sort(t).values))
    out["verified_vs_torch_sort"] = ok
    return out


def sweep_config(n: int, ncol: int, world: int) -> dict:
    """The workload description both arms print."""
    return {"workload": f"dispatch sweep: N={n} int64, K in {SWEEP_K} x (uniform, zipf s=1.1) "
                        "+ spill-trigger column; one sort per column",
            "columns": ncol, "keys_per_step": n * ncol,
            "l2": "inputs larger than L2 (240 MB per column), no flush",
            "parallelism": f"replicas x{world}"}


def replica_throughput(elapsed_ms: float, keys_per_rank: int, dist=None, device="cpu"):
    """Whole-job figures of N independent replicas: the slowest rank's time
    (all-reduce MAX of one scalar, no data-path collective) and every rank's
    keys over it.  Returns (max elapsed ms, Gkeys/s)."""
    world = 1
    if dist is not None:
        import torch
        tt = torch.tensor([elapsed_ms], dtype=torch.float64, device=device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        elapsed_ms = float(tt.item())
        world = dist.get_world_size()
    return elapsed_ms, keys_per_rank * world / (elapsed_ms / 1e3) / 1e9


def run_reference(args, rank, world):
    """--impl reference: the CPU oracle on the host cores, bounded per step."""
    n = args.n
    specs = sweep_specs(n)
    if rank != 0:
        return 0
    cols = [(s["name"], make_column(s, n, seed=i)) for i, s in enumerate(specs)]
    from oracle import cafs_oracle as O
    per_step = max(1, min(len(cols), args.ref_cols_per_step))
    times, keys = [], 0
    for step in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        nk = 0
        for j in range(per_step):
            name, x = cols[(step * per_step + j) % len(cols)]
            O.frequency_sort(x)
            nk += x.size
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            times.append(dt)
            keys += nk
    total = sum(times)
    value = keys / total / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": "Gkeys/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "impl": "reference",
        "config": sweep_config(n, len(cols), world),
        "cpu_baseline": {"value": value, "unit": "Gkeys/s", "cores": 1, "kind": "oracle",
                         "sample": f"each step sorts {per_step} of the {len(cols)} sweep columns (full N), "
                                   "taken in turn; value = their keys / their CPU time", **host_cpu()},
        "e2e": {"value": value, "unit": "Gkeys/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["cafs", "reference"], default="cafs")
    ap.add_argument("--n", type=int, default=30_000_000)
    ap.add_argument("--ref-cols-per-step", type=int, default=2)
    ap.add_argument("--no-verify", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-form measurement")
    ap.add_argument("--no-served", action="store_true", help="skip the served-form measurement")
    ap.add_argument("--no-mid-k", action="store_true", help="skip the mid-K (1e4..1e5) hash-count leg")
    ap.add_argument("--no-argsort", action="store_true",
                    help="skip the argsort, key-type and input-profile measurements")
    ap.add_argument("--columns", default="",
                    help="comma-separated subset of sweep columns (e.g. uniform_K200); default all")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2605_25040_gb300 import cafs

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    n = args.n
    specs = sweep_specs(n)
    seeds = {s["name"]: i for i, s in enumerate(specs)}
    if args.columns:
        keep = set(args.columns.split(","))
        specs = [s for s in specs if s["name"] in keep]
        if not specs:
            raise SystemExit(f"no sweep column matches {args.columns}")
    names = [s["name"] for s in specs]
    dev_in = [make_column_device(s, n, seeds[s["name"]], "cuda") for s in specs]
    dev_out = [torch.empty_like(t) for t in dev_in]
    stream = torch.cuda.current_stream()

    def step(col_events=None):
        for i, (a, b) in enumerate(zip(dev_in, dev_out)):
            if col_events is not None:
                col_events[i][0].record(stream)
            cafs.sort(a, b, stream=stream)
            if col_events is not None:
                col_events[i][1].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    ncol = len(dev_in)
    events = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(ncol)] for _ in range(args.steps)]
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local_rank)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)  # let the sampler start
    launches0 = cafs.kernel_launch_count()
    t_start.record(stream)
    for s in range(args.steps):
        step(events[s])
    t_end.record(stream)
    torch.cuda.synchronize()
    launches = cafs.kernel_launch_count() - launches0
    if dist:
        dist.barrier()
    clk = clocks.stop()
    elapsed_ms, value = replica_throughput(t_start.elapsed_time(t_end), n * ncol * args.steps, dist, "cuda")

    # per-column device times (mean over timed steps)
    col_ms = [statistics.mean(events[s][i][0].elapsed_time(events[s][i][1]) for s in range(args.steps))
              for i in range(ncol)]
    peak, peak_kind = load_peaks()
    bytes_per_col = 2 * 8 * n
    achieved = bytes_per_col * ncol / (sum(col_ms) / 1e3) / 1e9
    main_idx = [i for i, s in enumerate(specs) if s["K"] is not None and s["K"] <= 100_000]
    main_ms = sum(col_ms[i] for i in main_idx)
    main_ach = bytes_per_col * len(main_idx) / (main_ms / 1e3) / 1e9 if main_idx else 0.0

    # branch taken per column + verification against torch.sort on the device
    sweep = []
    verified = True
    for i, name in enumerate(names):
        out, rep = cafs.sort_ex(dev_in[i], dev_out[i])
        if not args.no_verify:
            ref = torch.sort(dev_in[i]).values
            ok = bool(torch.equal(ref, out))
            verified &= ok
        tl = rep["timeline_ns"]
        phases = {}
        prev = tl[0]
        for idx, nm in ((1, "sample"), (2, "monotone"), (3, "count"), (4, "pairs"),
                        (5, "finish")):
            if tl[idx]:
                phases[nm] = round((tl[idx] - prev) / 1e3, 1)
                prev = tl[idx]
        sweep.append({"column": name, "path": cafs.path_name(rep["path"]), "k_hat": rep["est"]["k_hat"],
                      "k_distinct": rep["k_distinct"], "ms": round(col_ms[i], 4), "phases_us": phases,
                      "gkeys_s": round(n / (col_ms[i] / 1e3) / 1e9, 2),
                      "frac_hbm": round(bytes_per_col / (col_ms[i] / 1e3) / 1e9 / peak, 4)})

    e2e = None
    if not args.no_e2e:
        pin_in = [t.cpu().pin_memory() for t in dev_in]
        pin_out = [torch.empty_like(t).pin_memory() for t in pin_in]
        for a, b in zip(pin_in, pin_out):  # warm-up (allocates the io buffer)
            cafs.sort_host_ptr(a.data_ptr(), a.numel(), torch.int64, b.data_ptr(), stream=stream)
        torch.cuda.synchronize()
        e2e_steps = max(1, min(3, args.steps))
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            for a, b in zip(pin_in, pin_out):
                cafs.sort_host_ptr(a.data_ptr(), a.numel(), torch.int64, b.data_ptr(), stream=stream)
        torch.cuda.synchronize()
        dt_blocking = time.perf_counter() - t0
        bi = sum(t.numel() * 8 for t in pin_in)
        if not args.no_verify:
            verified &= bool(np.array_equal(pin_out[0].numpy(), np.sort(pin_in[0].numpy())))
        # The same columns through the request server: host-to-device copies,
        # sorting and device-to-host copies of different columns overlap.
        pairs = [(a.numpy(), b.numpy()) for a, b in zip(pin_in, pin_out)] * e2e_steps
        srv = cafs.Server(16 << 30, {"max_request_keys": n, "max_batch_columns": 1, "max_inflight": 4})
        try:
            srv.run_trace(pairs[:ncol], np.zeros(ncol))          # warm-up
            for b_ in pin_out:
                b_.zero_()
            lat, dt = srv.run_trace(pairs, np.zeros(len(pairs)))
        finally:
            srv.close()
        if not args.no_verify:
            verified &= all(bool(np.array_equal(b_.numpy(), np.sort(a.numpy()))) for a, b_ in
                            list(zip(pin_in, pin_out))[:3])
        e2e = {"value": n * ncol * e2e_steps * world / dt / 1e9, "unit": "Gkeys/s",
               "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bi,
               "api": "cafs_server_run_trace (pinned host buffers; copies in, sorting and copies out "
                      "of different columns overlap)",
               "blocking_per_column": {"value": n * ncol * e2e_steps * world / dt_blocking / 1e9,
                                       "api": "cafs_sort_host, one column at a time"}}

    mid_k = link = None
    if rank == 0 and not args.no_mid_k and n == 30_000_000:
        mid_k = bench_mid_k(torch, cafs, n, peak)
    if rank == 0 and not args.no_e2e:
        link = host_link(torch)
        if e2e is not None:
            e2e["host_link"] = link
            # each key crosses the link twice (in and out); the copies of one
            # column overlap the other direction's, so the slower direction
            # with both directions busy bounds the overlapped figure
            e2e["host_link_ceiling_gkeys_s"] = round(
                min(link["h2d_gbs"], link["d2h_gbs"], link["duplex_gbs_each_way"]) / 8, 2)

    argsort = key_types = profiles = None
    if rank == 0 and not args.no_argsort:
        argsort = bench_argsort(torch, cafs, dev_in, names, peak)
        key_types = bench_key_types(torch, cafs, dev_in, names, col_ms)
        if n == 30_000_000:
            profiles = bench_profiles(torch, cafs, n, peak)

    batched = served = None
    if rank == 0 and not args.no_batched:
        del dev_out
        torch.cuda.empty_cache()
        batched = bench_batched(torch, cafs)
    if rank == 0 and not args.no_served:
        served = bench_served(torch, cafs)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        want = ("uniform_K200", "zipf_K4096", "uniform_K4096", "uniform_K4")
        pick = [(nm, dev_in[i].cpu().numpy()) for i, nm in enumerate(names) if nm in want]
        cpu = cpu_baseline(pick or [(names[0], dev_in[0].cpu().numpy())])

    traffic = traffic_record("pipeline_kernel") if n == 30_000_000 and ncol == 19 else None
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "Gkeys/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": elapsed_ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "int64",
        "data": "synthetic",
        "config": dict(sweep_config(n, ncol, world), verified_vs_torch_sort=verified),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak,
                     "traffic": traffic["mean_dram_bytes_per_launch"] if traffic else None,
                     "traffic_source": traffic["profile"] if traffic else
                     "null: pipeline_kernel sources changed since the last ncu capture",
                     "peak_kind": peak_kind,
                     "kernel": "pipeline_kernel (whole sort, one cooperative launch per column)",
                     "algorithmic_bytes_per_launch": bytes_per_col,
                     "main_path_K_le_1e5": {"achieved": main_ach, "frac": main_ach / peak,
                                            "traffic": traffic["main_path_mean_dram_bytes_per_launch"]
                                            if traffic else None,
                                            "columns": [specs[i]["name"] for i in main_idx]},
                     "hash_count_K_le_1e5": hash_count_summary(sweep, mid_k, specs, bytes_per_col, peak)},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clk,
        "sweep": sweep,
        "mid_k": mid_k,
        "host_link": link,
        "batched": batched,
        "served": served,
        "argsort": argsort,
        "key_types": key_types,
        "profiles": profiles,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
