"""Seeded synthetic key columns shared by the tests and the benchmark.

This module draws random numbers and nothing else: it contains none of the
sorting method's arithmetic, so both the CUDA path and the CPU oracle can be
fed from it without sharing any of the method's code.

All randomness comes from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used as a counter-based
generator: draw i of stream ``seed`` is ``mix(seed + (i + 1) * GAMMA)``.

Workload shapes follow the paper's evaluation (Sec. 6.1): a palette of K
distinct values, each element picked from it.  The paper's own palette is an
arithmetic progression ``a + b*i`` with ``a`` and an odd ``b`` derived from
seed ``42 + N + K`` through a SplitMix-style mixer whose exact form it does not
give; ``paper_palette`` implements it with SplitMix64, so the paper's datasets
are reproduced in shape but not bit for bit.  The other generators add what
the benchmark configurations ask for: values drawn uniformly from the full
64-bit range, Zipf(s) frequencies, a column whose strided sample positions hold
a small set while every other element is distinct, and sorted columns.
"""

from __future__ import annotations

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK64 = (1 << 64) - 1


def _u64(x: int) -> np.uint64:
    return np.uint64(int(x) & _MASK64)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Draws offset..offset+count-1 of SplitMix64 stream ``seed`` as uint64."""
    with np.errstate(over="ignore"):
        idx = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = _u64(seed) + idx * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def _uniform_index(r: np.ndarray, k: int) -> np.ndarray:
    """Maps uint64 draws to [0, k) by the multiply-high of their top 32 bits."""
    hi = (r >> np.uint64(32)).astype(np.uint64)
    with np.errstate(over="ignore"):
        return ((hi * np.uint64(k)) >> np.uint64(32)).astype(np.int64)


def _unit_float(r: np.ndarray) -> np.ndarray:
    """Maps uint64 draws to doubles in [0, 1) from their top 53 bits."""
    return (r >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


def _mix32(x: np.ndarray) -> np.ndarray:
    """A bijection on 32-bit words (xorshift-multiply finaliser, 'lowbias32')."""
    x = x.astype(np.uint32, copy=True)
    with np.errstate(over="ignore"):
        x ^= x >> np.uint32(16)
        x *= np.uint32(0x7FEB352D)
        x ^= x >> np.uint32(15)
        x *= np.uint32(0x846CA68B)
        x ^= x >> np.uint32(16)
    return x


def distinct_values(k: int, seed: int, dtype=np.int64, start: int = 0) -> np.ndarray:
    """K distinct values spread over the dtype's full range, in random order.

    Draws ``start .. start+k-1`` of a bijective counter mix: SplitMix64 for
    64-bit keys (its counter step is odd and its finaliser is a bijection, so
    distinct counters give distinct values) and a 32-bit bijective mix of
    ``seed + counter`` for 32-bit keys.  Two calls with the same seed and
    disjoint ``start`` ranges therefore never share a value.
    """
    if dtype == np.int64:
        return splitmix64(seed, k, offset=start).view(np.int64)
    if k + start > (1 << 32):
        raise ValueError("at most 2^32 distinct 32-bit values")
    ctr = (np.arange(start, start + k, dtype=np.uint64) + np.uint64(seed & 0xFFFFFFFF)) & np.uint64(0xFFFFFFFF)
    return _mix32(ctr).view(np.int32)


def shuffle(values: np.ndarray, seed: int) -> np.ndarray:
    """Seeded permutation (sort by SplitMix64 draws; ties broken by index)."""
    r = splitmix64(seed ^ 0x5DEECE66D, values.size)
    return values[np.argsort(r, kind="stable")]


def zipf_ranks(n: int, k: int, s: float, seed: int) -> np.ndarray:
    """N ranks in [0, K) with P(rank=j) proportional to 1/(j+1)^s.

    Inverse-CDF sampling on the cumulative table of the normalised weights.
    """
    w = 1.0 / np.power(np.arange(1, k + 1, dtype=np.float64), s)
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    u = _unit_float(splitmix64(seed, n))
    idx = np.searchsorted(cdf, u, side="right")
    return np.minimum(idx, k - 1).astype(np.int64)


def uniform_ranks(n: int, k: int, seed: int) -> np.ndarray:
    return _uniform_index(splitmix64(seed, n), k)


def column(n: int, k: int, dist: str = "uniform", dtype=np.int64, seed: int = 0,
           s: float = 1.1) -> np.ndarray:
    """N keys over a palette of K distinct values uniform in the dtype range.

    ``dist`` is "uniform" (every palette value equally likely) or "zipf"
    (frequency of the j-th most frequent value proportional to 1/j^s; the
    palette is shuffled so frequency does not follow key order).  When K >= N
    the column is a permutation of N distinct values (K = N, all distinct).
    """
    base = 42 + n + k
    if k >= n:
        return distinct_values(n, base ^ seed, dtype)
    pal = distinct_values(k, base ^ seed, dtype)
    if dist == "uniform":
        ranks = uniform_ranks(n, k, base * 31 + seed)
    elif dist == "zipf":
        ranks = zipf_ranks(n, k, s, base * 31 + seed)
    else:
        raise ValueError(dist)
    return pal[ranks].astype(dtype, copy=False)


def paper_palette(n: int, k: int, dtype=np.int64) -> np.ndarray:
    """Sec. 6.1 workload: palette a + b*i (b odd), uniform picks, seed 42+N+K."""
    seed = 42 + n + k
    r = splitmix64(seed, 2)
    info = np.iinfo(dtype)
    bits = 64 if dtype == np.int64 else 32
    a = int(r[0]) & ((1 << bits) - 1)
    b = (int(r[1]) & ((1 << bits) - 1)) | 1
    i = np.arange(k, dtype=object)
    vals = [((a + b * int(j)) & ((1 << bits) - 1)) for j in i]
    vals = np.array([v - (1 << bits) if v > info.max else v for v in vals], dtype=dtype)
    ranks = uniform_ranks(n, k, seed + 1)
    return vals[ranks]


def spill_trigger(n: int, dtype=np.int64, seed: int = 0, small_set: int = 64) -> np.ndarray:
    """Column whose strided sample positions hold ``small_set`` values only.

    The 1024 sample positions i*stride (stride = max(1, N // 1024)) receive a
    shuffled multiset of ``small_set`` values, each repeated 1024/small_set
    times; every other element is a fresh distinct random value not in that
    set.  A sampler therefore sees a low-cardinality column while the true
    number of distinct keys is about N.
    """
    stride = max(1, n // 1024)
    npos = min(1024, n)
    pos = np.arange(npos, dtype=np.int64) * stride
    small = distinct_values(small_set, 1000 + seed, dtype)
    reps = -(-npos // small_set)
    sample_vals = shuffle(np.tile(small, reps)[:npos], 2000 + seed)
    rest = distinct_values(n - npos, 1000 + seed, dtype, start=small_set)
    out = np.empty(n, dtype=dtype)
    mask = np.ones(n, dtype=bool)
    mask[pos] = False
    out[pos] = sample_vals
    out[mask] = rest
    return out


def sorted_column(n: int, k: int, dtype=np.int64, seed: int = 0) -> np.ndarray:
    return np.sort(column(n, k, "uniform", dtype, seed))


# Input profiles: runs of equal keys, one
# contiguous group per key, and a nearly sorted column.

def _group_sizes(n: int, k: int, seed: int) -> np.ndarray:
    """K positive sizes summing to N (uniform random proportions)."""
    w = _unit_float(splitmix64(seed, k)) + 1e-3
    sizes = np.floor(w / w.sum() * (n - k)).astype(np.int64) + 1
    sizes[0] += n - int(sizes.sum())
    return sizes


def runs_column(n: int, k: int, mean_run: float, dist: str = "uniform", dtype=np.int64,
                seed: int = 0, s: float = 1.1) -> np.ndarray:
    """Runs of equal keys: geometric run lengths with mean ``mean_run`` (>= 1),
    each run's value drawn (uniform or Zipf) from a palette of K values; a key
    recurs in many runs."""
    base = 77 + n + k
    p = 1.0 / max(mean_run, 1.0)
    m = int(n / mean_run * 1.5) + 16
    u = _unit_float(splitmix64(base ^ seed, m))
    lengths = np.ones(m, dtype=np.int64) if p >= 1.0 else \
        1 + np.floor(np.log1p(-u) / np.log1p(-p)).astype(np.int64)
    ends = np.cumsum(lengths)
    runs = int(np.searchsorted(ends, n)) + 1
    lengths = lengths[:runs]
    lengths[-1] -= int(ends[runs - 1]) - n
    pal = distinct_values(k, base ^ seed, dtype)
    ranks = (zipf_ranks(runs, k, s, base * 31 + seed) if dist == "zipf"
             else uniform_ranks(runs, k, base * 31 + seed))
    return np.repeat(pal[ranks], lengths).astype(dtype, copy=False)


def grouped_column(n: int, k: int, dtype=np.int64, seed: int = 0) -> np.ndarray:
    """Every one of K values in exactly one contiguous group, groups in random
    order (a column already grouped by key, e.g. the output of a group-by)."""
    base = 91 + n + k
    pal = shuffle(distinct_values(k, base ^ seed, dtype), base + seed)
    return np.repeat(pal, _group_sizes(n, k, base * 7 + seed)).astype(dtype, copy=False)


def almost_sorted(n: int, k: int, swaps: int, dtype=np.int64, seed: int = 0) -> np.ndarray:
    """A non-decreasing column over K values with ``swaps`` random pairs of
    positions exchanged."""
    base = 113 + n + k
    pal = np.sort(distinct_values(k, base ^ seed, dtype))
    out = np.repeat(pal, _group_sizes(n, k, base * 7 + seed)).astype(dtype, copy=False)
    if swaps and n > 1:
        ij = _uniform_index(splitmix64(base * 13 + seed, 2 * swaps), n).reshape(swaps, 2)
        for i, j in ij:
            out[i], out[j] = out[j], out[i]
    return out


def log_uniform_int(lo: float, hi: float, count: int, seed: int) -> np.ndarray:
    """Integers log-uniform in [lo, hi]."""
    u = _unit_float(splitmix64(seed, count))
    return np.floor(np.exp(np.log(lo) + u * (np.log(hi) - np.log(lo)))).astype(np.int64)


def exponential_gaps(rate: float, count: int, seed: int) -> np.ndarray:
    """Poisson-process inter-arrival times (seconds) at ``rate`` per second."""
    u = _unit_float(splitmix64(seed, count))
    return -np.log1p(-u) / rate


def batch_specs(count: int, seed: int, n_lo: float = 1e3, n_hi: float = 1e6,
                k_cap: float = 5e4) -> list[tuple[int, int]]:
    """(N, K) of a batch of columns: N log-uniform in [n_lo, n_hi], K
    log-uniform in [2, max(2, min(N/4, k_cap))]."""
    n = log_uniform_int(n_lo, n_hi, count, seed)
    u = _unit_float(splitmix64(seed + 1, count))
    khi = np.maximum(np.minimum(n / 4.0, k_cap), 2.0)
    k = np.floor(np.exp(np.log(2.0) + u * (np.log(khi) - np.log(2.0)))).astype(np.int64)
    return [(int(a), int(max(2, b))) for a, b in zip(n, k)]


def batch_column(n: int, k: int, index: int, seed: int, dtype=np.int64,
                 dist: str = "zipf") -> np.ndarray:
    """Column ``index`` of a batch (its own seed, so columns differ)."""
    return column(n, k, dist, dtype, seed=seed * 1_000_003 + index)


def mixed_specs(count: int = 64, n_lo: float = 1e3, n_hi: float = 3e7,
                spill_every: int = 16) -> list[tuple[int, int, str, str]]:
    """(N, K, dtype name, kind) of the mixed batch: dtypes alternate int32 /
    int64, N log-spaced from n_lo to n_hi, K log-spaced from 2 to N in a
    five-step cycle whose last step is K = N (all distinct), and every
    ``spill_every``-th column (the last of each group) a spill-trigger
    column."""
    out = []
    for i in range(count):
        n = int(round(n_lo * (n_hi / n_lo) ** (i / max(1, count - 1))))
        f = (i % 5) / 4.0
        k = n if f == 1.0 else max(2, int(round(2.0 * (n / 2.0) ** f)))
        kind = "spill" if (i % spill_every) == spill_every - 1 else "zipf"
        out.append((n, k, "int32" if i % 2 == 0 else "int64", kind))
    return out


def mixed_column(n: int, k: int, dtype_name: str, kind: str, index: int, seed: int = 0) -> np.ndarray:
    dtype = np.int32 if dtype_name == "int32" else np.int64
    if kind == "spill":
        return spill_trigger(n, dtype, seed=seed * 1009 + index)
    return column(n, k, "zipf", dtype, seed=seed * 1_000_003 + index)


# ---------------------------------------------------------------------------
# The same generators evaluated with torch on any device (bit-identical to the
# numpy versions above: the integer steps are exact, the Zipf table is built
# by numpy and the uniform floats take the same 53 bits).  The benchmark uses
# them to build its multi-GB inputs in device memory.
# ---------------------------------------------------------------------------
def _i64(x: int) -> int:
    x &= _MASK64
    return x - (1 << 64) if x >= (1 << 63) else x


def _srl(t, s: int):
    """Logical right shift of int64 bit patterns."""
    return (t >> s) & ((1 << (64 - s)) - 1)


def splitmix64_torch(seed: int, count: int, offset: int = 0, device="cpu"):
    import torch
    idx = torch.arange(offset + 1, offset + count + 1, dtype=torch.int64, device=device)
    z = idx * _i64(int(_GAMMA)) + _i64(seed)
    z = (z ^ _srl(z, 30)) * _i64(int(_M1))
    z = (z ^ _srl(z, 27)) * _i64(int(_M2))
    return z ^ _srl(z, 31)


def _mix32_torch(x):
    m = 0xFFFFFFFF
    x = x ^ (x >> 16)
    x = (x * 0x7FEB352D) & m
    x = x ^ (x >> 15)
    x = (x * 0x846CA68B) & m
    return x ^ (x >> 16)


def distinct_values_torch(k: int, seed: int, dtype=np.int64, start: int = 0, device="cpu"):
    import torch
    if dtype == np.int64:
        return splitmix64_torch(seed, k, offset=start, device=device)
    if k + start > (1 << 32):
        raise ValueError("at most 2^32 distinct 32-bit values")
    ctr = (torch.arange(start, start + k, dtype=torch.int64, device=device) + (seed & 0xFFFFFFFF)) & 0xFFFFFFFF
    x = _mix32_torch(ctr)
    return (x - ((x >> 31) << 32)).to(torch.int32)


def column_torch(n: int, k: int, dist: str = "uniform", dtype=np.int64, seed: int = 0,
                 s: float = 1.1, device="cpu"):
    """``column`` evaluated with torch on ``device`` (same values)."""
    import torch
    base = 42 + n + k
    if k >= n:
        return distinct_values_torch(n, base ^ seed, dtype, device=device)
    pal = torch.from_numpy(distinct_values(k, base ^ seed, dtype)).to(device)
    r = splitmix64_torch(base * 31 + seed, n, device=device)
    if dist == "uniform":
        ranks = _srl(_srl(r, 32) * k, 32)
    elif dist == "zipf":
        w = 1.0 / np.power(np.arange(1, k + 1, dtype=np.float64), s)
        cdf = np.cumsum(w)
        cdf /= cdf[-1]
        u = _srl(r, 11).to(torch.float64) * (1.0 / (1 << 53))
        ranks = torch.searchsorted(torch.from_numpy(cdf).to(device), u, right=True).clamp_(max=k - 1)
    else:
        raise ValueError(dist)
    return pal[ranks]


def spill_trigger_torch(n: int, dtype=np.int64, seed: int = 0, small_set: int = 64, device="cpu"):
    """``spill_trigger`` evaluated with torch on ``device`` (same values)."""
    import torch
    stride = max(1, n // 1024)
    npos = min(1024, n)
    pos = torch.arange(npos, dtype=torch.int64, device=device) * stride
    small = distinct_values(small_set, 1000 + seed, dtype)
    reps = -(-npos // small_set)
    sample_vals = torch.from_numpy(shuffle(np.tile(small, reps)[:npos], 2000 + seed)).to(device)
    tdt = torch.int64 if dtype == np.int64 else torch.int32
    out = torch.empty(n, dtype=tdt, device=device)
    mask = torch.ones(n, dtype=torch.bool, device=device)
    mask[pos] = False
    out[pos] = sample_vals
    out[mask] = distinct_values_torch(n - npos, 1000 + seed, dtype, start=small_set, device=device)
    return out


def batch_column_torch(n: int, k: int, index: int, seed: int, dtype=np.int64, dist: str = "zipf",
                       device="cpu"):
    return column_torch(n, k, dist, dtype, seed=seed * 1_000_003 + index, device=device)


def mixed_column_torch(n: int, k: int, dtype_name: str, kind: str, index: int, seed: int = 0,
                       device="cpu"):
    dtype = np.int32 if dtype_name == "int32" else np.int64
    if kind == "spill":
        return spill_trigger_torch(n, dtype, seed=seed * 1009 + index, device=device)
    return column_torch(n, k, "zipf", dtype, seed=seed * 1_000_003 + index, device=device)
