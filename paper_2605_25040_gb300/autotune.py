"""Autotuner of the batched kernel's knobs, with an on-disk cache.

The knobs never change a result (tests check that); they trade speed:
``emit_tile_vec`` is the emit tile in 16-byte vectors (items per thread =
emit_tile_vec / 1024), ``local_slots_max`` and ``replicas_max`` size the
per-CTA shared hash table (its capacity and counter replicas),
``grid_min_n`` / ``defer_min_n`` / ``cta_table_slots`` decide which columns
the whole grid sorts, and ``ctas`` is the number of CTAs of the launch.  Two
choices are not run-time knobs and so are not searched: the threads per CTA
(1024) and the split of the 226 KB of shared memory between the bulk-copy
ring (124 KB) and the count tables are compile-time constants of the kernel
(one CTA per SM; 512-thread CTAs and smaller rings measured slower for the
count phase).

Search: coordinate descent from the defaults -- one knob at a time over its
candidate values, keeping the fastest, two rounds.  Every measurement is a
native call (``cafs_batch_autotune``: recorded plan, CUDA events, median of
``reps`` launches).  The winner is cached per (GPU name, workload signature)
in a JSON file.
"""

from __future__ import annotations

import json
import math
import os

from . import cafs

SPACE = {
    "emit_tile_vec": [1024, 2048, 4096, 8192],
    "local_slots_max": [2048, 4096, 8192],
    "replicas_max": [8, 16, 32],
    "grid_min_n": [0, 1 << 19, 1 << 20, 1 << 21, 1 << 22],
    "defer_min_n": [0, 1 << 16, 1 << 18, 1 << 20],
    "cta_table_slots": [0, 1 << 14, 1 << 16, 1 << 18],
    "ctas": [0, 114, 76],
}

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "cafs_gb300", "autotune.json")


def workload_signature(keys_list) -> str:
    """Columns, dtype mix and the log2 spread of their lengths."""
    import torch
    n = [k.numel() for k in keys_list]
    i32 = sum(1 for k in keys_list if k.dtype == torch.int32)
    lo = int(math.log2(max(1, min(n)))) if n else 0
    hi = int(math.log2(max(1, max(n)))) if n else 0
    tot = int(math.log2(max(1, sum(n))))
    return f"cols={len(n)}:i32={i32}:log2n=[{lo},{hi}]:log2sum={tot}"


def _device_name() -> str:
    import torch
    return torch.cuda.get_device_name(torch.cuda.current_device())


def tune(keys_list, outs=None, reps: int = 3, rounds: int = 2, space: dict | None = None,
         log=None) -> dict:
    """Coordinate descent over ``space``; returns {"tuning", "ms", "default_ms", "trials"}."""
    import torch
    space = space or SPACE
    if outs is None:
        outs = [torch.empty_like(k) for k in keys_list]
    current = {}
    default_ms = cafs.time_tunings(keys_list, outs, [current], reps)[0]
    best_ms = default_ms
    trials = 1
    for _ in range(rounds):
        changed = False
        for knob, values in space.items():
            cands = []
            for v in values:
                t = dict(current)
                t[knob] = v
                cands.append(t)
            ms = cafs.time_tunings(keys_list, outs, cands, reps)
            trials += len(cands)
            i = min(range(len(ms)), key=ms.__getitem__)
            if log:
                log(f"{knob}: " + ", ".join(f"{v}={m:.3f}ms" for v, m in zip(values, ms)))
            if ms[i] < best_ms * 0.99:
                best_ms = ms[i]
                current = cands[i]
                changed = True
        if not changed:
            break
    return {"tuning": current, "ms": best_ms, "default_ms": default_ms, "trials": trials}


def tuned(keys_list, outs=None, cache_path: str = DEFAULT_CACHE, retune: bool = False, **kw) -> dict:
    """The cached tuning for this GPU and workload signature (tuning on a miss)."""
    key = f"{_device_name()}|{workload_signature(keys_list)}"
    cache = {}
    if os.path.exists(cache_path):
        try:
            with open(cache_path) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
    if not retune and key in cache:
        hit = dict(cache[key])
        hit["cached"] = True
        return hit
    res = tune(keys_list, outs, **kw)
    cache[key] = res
    os.makedirs(os.path.dirname(cache_path) or ".", exist_ok=True)
    tmp = cache_path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, cache_path)
    res = dict(res)
    res["cached"] = False
    return res
