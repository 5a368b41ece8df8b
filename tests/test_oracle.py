"""Pins for the CPU oracle: it is checked against things other than itself.

* brute force: every sequence of length <= 6 over a 4-letter alphabet is sorted
  by an independent insertion sort and compared with ``frequency_sort``;
* invariants on larger random inputs (non-decreasing, same length, same
  histogram counted with a Python dict);
* the sampler re-run as a literal while-loop of Algorithm 2 with dict counting;
* the worked estimator and table-size values (tests/golden, Eq. 5 and Eq. 6);
* inputs that force every dispatcher branch and both sides of the guard.
"""

import itertools
import os

import numpy as np
import pytest

from oracle import cafs_oracle as O
from paper_2605_25040_gb300 import datagen as G

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _insertion_sort(seq):
    out = list(seq)
    for i in range(1, len(out)):
        v = out[i]
        j = i - 1
        while j >= 0 and out[j] > v:
            out[j + 1] = out[j]
            j -= 1
        out[j + 1] = v
    return out


def _load_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([int(t) for t in line.split()])
    return rows


@pytest.mark.parametrize("dtype", [np.int32, np.int64])
def test_frequency_sort_brute_force_tiny(dtype):
    info = np.iinfo(dtype)
    alphabet = [info.min, -1, 0, info.max]
    for length in range(0, 7):
        for seq in itertools.product(alphabet, repeat=length):
            arr = np.array(seq, dtype=dtype)
            got = O.frequency_sort(arr)
            assert got.dtype == arr.dtype
            assert got.tolist() == _insertion_sort(seq)


@pytest.mark.parametrize("n,k,dtype", [(1, 1, np.int64), (1000, 3, np.int32),
                                       (5000, 200, np.int64), (100000, 4096, np.int32),
                                       (65536, 65536, np.int64)])
def test_frequency_sort_invariants(n, k, dtype):
    x = G.column(n, k, "zipf", dtype, seed=3)
    y = O.frequency_sort(x)
    assert y.size == x.size
    assert bool(np.all(y[:-1] <= y[1:]))
    hx, hy = {}, {}
    for v in x.tolist():
        hx[v] = hx.get(v, 0) + 1
    for v in y.tolist():
        hy[v] = hy.get(v, 0) + 1
    assert hx == hy
    # the result does not depend on the input order
    assert np.array_equal(O.frequency_sort(G.shuffle(x, 5)), y)


@pytest.mark.parametrize("dtype", [np.int32, np.int64])
def test_stable_argsort_brute_force_tiny(dtype):
    # pi by the definition: positions ordered by (key, position), a stable
    # insertion sort of the positions
    info = np.iinfo(dtype)
    alphabet = [info.min, -1, 0, info.max]
    for length in range(0, 7):
        for seq in itertools.product(alphabet, repeat=length):
            arr = np.array(seq, dtype=dtype)
            pos = list(range(length))
            for i in range(1, length):
                v = pos[i]
                j = i - 1
                while j >= 0 and seq[pos[j]] > seq[v]:
                    pos[j + 1] = pos[j]
                    j -= 1
                pos[j + 1] = v
            got = O.stable_argsort(arr)
            assert got.dtype == np.uint32
            assert got.tolist() == pos


@pytest.mark.parametrize("n,k,dtype", [(5000, 3, np.int32), (20000, 200, np.int64), (30000, 30000, np.int64)])
def test_stable_argsort_invariants(n, k, dtype):
    x = G.column(n, k, "zipf", dtype, seed=4)
    pi = O.stable_argsort(x)
    # a permutation of the positions
    assert np.array_equal(np.sort(pi), np.arange(n, dtype=np.uint32))
    # keys in pi order are the sorted keys
    assert np.array_equal(x[pi], O.frequency_sort(x))
    # equal keys keep their input order
    same = x[pi][1:] == x[pi][:-1]
    assert bool(np.all(pi[1:][same] > pi[:-1][same]))
    # a stable library sort agrees
    assert np.array_equal(pi, np.argsort(x, kind="stable").astype(np.uint32))


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
def test_unsigned_brute_force_tiny(dtype):
    # natural unsigned order of Python integers
    w = np.dtype(dtype).itemsize * 8
    alphabet = [0, 1, 1 << (w - 1), (1 << w) - 1]
    for length in range(0, 6):
        for seq in itertools.product(alphabet, repeat=length):
            arr = np.array(seq, dtype=dtype)
            got = O.frequency_sort_any(arr)
            assert got.dtype == arr.dtype
            assert [int(v) for v in got] == sorted(seq)


def _total_order_key(bits: int, w: int):
    # IEEE 754 totalOrder from its definition: negatives (sign 1) before
    # positives, larger magnitude (exponent, then significand) first among
    # negatives and last among positives; NaNs sit beyond the infinities.
    mag = bits & ((1 << (w - 1)) - 1)
    return (0, -mag) if bits >> (w - 1) else (1, mag)


@pytest.mark.parametrize("fdt,idt", [(np.float32, np.uint32), (np.float64, np.uint64)])
def test_float_total_order_brute_force_tiny(fdt, idt):
    w = np.dtype(fdt).itemsize * 8
    specials = np.array([np.nan, -np.inf, -1.5, -0.0, 0.0, 2.0 ** -1030 if w == 64 else 2.0 ** -140, np.inf],
                        dtype=fdt)
    bits = [int(b) for b in specials.view(idt)]
    bits.append(bits[0] | (1 << (w - 1)))       # a negative NaN
    bits.append(bits[0] | 1)                    # a NaN with another payload
    for length in range(0, 5):
        for seq in itertools.product(bits, repeat=length):
            arr = np.array(seq, dtype=idt).view(fdt)
            got = [int(b) for b in O.frequency_sort_any(arr).view(idt)]
            assert got == sorted(seq, key=lambda b: _total_order_key(b, w))


@pytest.mark.parametrize("fdt", [np.float32, np.float64])
def test_float_finite_matches_numpy_sort(fdt):
    rng = np.random.default_rng(9)
    vals = rng.standard_normal(300).astype(fdt) * 1e3
    x = vals[rng.integers(0, vals.size, size=20_000)]
    x[x == 0] = 1
    assert np.array_equal(O.frequency_sort_any(x), np.sort(x))
    pi = O.stable_argsort_any(x)
    assert np.array_equal(pi, np.argsort(x, kind="stable").astype(np.uint32))


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64, np.float32, np.float64])
def test_ordered_signed_round_trip(dtype):
    rng = np.random.default_rng(11)
    w = np.dtype(dtype).itemsize
    raw = rng.integers(0, 256, size=4096 * w, dtype=np.uint8).view(dtype)
    back = O.from_ordered_signed(O.ordered_signed(raw), dtype)
    assert np.array_equal(back.view(np.uint8), raw.view(np.uint8))


def test_is_monotone_brute_force():
    for length in range(0, 6):
        for seq in itertools.product([0, 1, 2], repeat=length):
            want = all(seq[i] <= seq[i + 1] for i in range(len(seq) - 1))
            assert O.is_monotone(np.array(seq, dtype=np.int64)) == want


def _literal_sampler(x):
    """Algorithm 2 as a while loop with a dict as the frequency set."""
    n = len(x)
    s = 1024
    stride = max(1, n // s)
    freq = {}
    i = 0
    taken = 0
    while i < min(n, s * stride):
        v = int(x[i])
        freq[v] = freq.get(v, 0) + 1
        taken += 1
        i += stride
    u = len(freq)
    f1 = sum(1 for c in freq.values() if c == 1)
    f2 = sum(1 for c in freq.values() if c == 2)
    return stride, taken, u, f1, f2, sorted(freq)


@pytest.mark.parametrize("n", [1, 7, 1023, 1024, 1025, 2047, 2048, 3000, 10240, 99991, 300000])
@pytest.mark.parametrize("k", [2, 9, 700, 5000])
def test_chao1_spectrum_matches_literal_sampler(n, k):
    x = G.column(n, min(k, n), "zipf", np.int64, seed=n)
    est = O.chao1(x)
    stride, taken, u, f1, f2, keys = _literal_sampler(x)
    assert (est.stride, est.n_samples, est.u, est.f1, est.f2) == (stride, taken, u, f1, f2)
    assert list(est.sample_keys) == keys
    assert est.k_hat >= est.u
    assert est.f1 + 2 * est.f2 <= est.n_samples


def test_chao1_worked_values():
    for u, f1, f2, n, k_hat, sat in _load_golden("chao1_sec2_4.txt"):
        assert O.chao1_from_spectrum(u, f1, f2, n) == (k_hat, bool(sat))


def test_table_size_paper_examples():
    for k_hat, m, table_bytes in _load_golden("table_size_sec4_5.txt"):
        got_m, c, lim = O.table_size(k_hat, 10**12, 8)
        assert got_m == m
        assert 64 * got_m == table_bytes
        assert c == 4 * m and lim == 2 * m


def test_table_size_clamps():
    # lower clamp: 8 buckets
    assert O.table_size(1, 10**6, 8) == (8, 32, 16)
    assert O.table_size(1, 10**6, 4) == (8, 64, 32)
    # upper clamp bit_ceil(ceil(N/cap)): N=2048, cap 4 -> 512 buckets
    assert O.table_size(1000, 2048, 8) == (512, 2048, 1024)
    # ceil, not floor, inside the upper clamp: N = 4*1024 + 1 -> 2048 buckets
    assert O.table_size(10**6, 4097, 8)[0] == 2048
    # 32-bit keys: 8 per bucket, M = bit_ceil(K_hat)
    assert O.table_size(200, 10**7, 4) == (256, 2048, 1024)


def test_sample_example_mod8_tiny_miss():
    # N = 10240, x_i = i mod 8: stride 10 hits residues {0,2,4,6} only.
    x = (np.arange(10240) % 8).astype(np.int64)
    x = x[::-1].copy()  # not sorted; position i holds (10239 - i) mod 8
    est = O.chao1(x)
    assert est.stride == 10 and est.n_samples == 1024
    assert est.u == 4 and est.f1 == 0 and est.f2 == 0 and est.k_hat == 4
    assert est.sample_keys == (1, 3, 5, 7)
    assert O.dispatch(x) == O.TINY
    assert O.final_path(x) == O.TINY_MISS_MAIN
    assert (est.M, est.C, est.L) == (8, 32, 16)


def test_saturation_routes_high_entropy():
    x = G.shuffle(np.arange(4096, dtype=np.int64), 1)
    est = O.chao1(x)
    assert est.u == 1024 and est.saturated and est.k_hat == 4096
    assert O.dispatch(x) == O.HIGH_ENTROPY_RADIX
    assert O.dispatch(np.arange(4096, dtype=np.int64)) == O.BYPASS_SORTED


def test_dispatch_branches():
    assert O.dispatch(np.zeros(0, np.int64)) == O.EMPTY
    assert O.dispatch(np.array([5], np.int32)) == O.BYPASS_SORTED
    assert O.dispatch(np.arange(100, 0, -1).astype(np.int64)) == O.SMALL_N
    assert O.dispatch(np.array([3] * 2046 + [2], np.int64)) == O.SMALL_N
    assert O.dispatch(np.array([3] * 2047 + [2], np.int64)) == O.TINY
    x = G.column(5000, 3, "uniform", np.int64, seed=1)
    assert O.dispatch(x) == O.TINY and O.final_path(x) == O.TINY
    x = G.column(100000, 200, "uniform", np.int64, seed=1)
    assert O.dispatch(x) == O.MAIN and O.final_path(x) == O.MAIN
    x = G.column(100000, 100000, "uniform", np.int64, seed=1)
    assert O.dispatch(x) == O.HIGH_ENTROPY_RADIX
    x = G.spill_trigger(65536, np.int64, seed=2)
    est = O.chao1(x)
    assert est.u == 64 and est.k_hat == 64 and (est.M, est.C, est.L) == (128, 512, 256)
    assert O.dispatch(x) == O.MAIN and O.final_path(x) == O.MAIN_OVERFLOW_RADIX


def _guard_column(k_true, seed=0):
    """N=8192 int64: samples (stride 8) hold 16 values x 64; K_true total."""
    n = 8192
    small = G.distinct_values(16, 11 + seed, np.int64)
    x = np.empty(n, np.int64)
    pos = np.arange(1024) * 8
    x[pos] = G.shuffle(np.tile(small, 64), 12 + seed)
    extra = G.distinct_values(k_true - 16, 11 + seed, np.int64, start=16)
    rest = np.concatenate([extra, np.resize(small, n - 1024 - extra.size)])
    mask = np.ones(n, bool)
    mask[pos] = False
    x[mask] = G.shuffle(rest, 14 + seed)
    return x


def test_overflow_guard_boundary():
    at = _guard_column(64)
    est = O.chao1(at)
    assert est.k_hat == 16 and (est.M, est.C, est.L) == (32, 128, 64)
    assert O.distinct_count(at) == 64
    assert O.final_path(at) == O.MAIN
    over = _guard_column(65)
    assert O.distinct_count(over) == 65
    assert O.final_path(over) == O.MAIN_OVERFLOW_RADIX


def test_high_entropy_boundary_is_strict():
    # 1023 distinct sample values, one of them twice: K_hat = 262144; N = 2 K_hat.
    n = 524288
    stride = n // 1024
    vals = G.distinct_values(1023, 21, np.int64)
    sample = np.concatenate([vals, vals[:1]])
    sample = G.shuffle(sample, 22)
    x = np.empty(n, np.int64)
    pos = np.arange(1024) * stride
    mask = np.ones(n, bool)
    mask[pos] = False
    x[pos] = sample
    x[mask] = np.resize(vals, n - 1024)
    est = O.chao1(x)
    assert (est.u, est.f1, est.f2, est.k_hat) == (1023, 1022, 1, 262144)
    assert 2 * est.k_hat == n
    assert O.dispatch(x) == O.MAIN
    assert O.final_path(x) == O.MAIN
    y = x[: n - 1024]  # smaller N, same kind of sample: 2 K_hat > N
    est_y = O.chao1(y)
    if 2 * est_y.k_hat > y.size:
        assert O.dispatch(y) == O.HIGH_ENTROPY_RADIX


def test_datagen_is_deterministic_and_shaped():
    a = G.column(10000, 50, "zipf", np.int64, seed=9)
    b = G.column(10000, 50, "zipf", np.int64, seed=9)
    assert np.array_equal(a, b)
    assert np.unique(a).size <= 50
    c = G.column(10000, 50, "uniform", np.int32, seed=9)
    assert c.dtype == np.int32 and np.unique(c).size == 50
    p = G.paper_palette(5000, 40)
    assert np.unique(p).size <= 40


@pytest.mark.parametrize("dtype", [np.int32, np.int64, np.uint32, np.uint64, np.float32, np.float64])
def test_any_type_degenerate_inputs(dtype):
    empty = np.zeros(0, dtype=dtype)
    assert O.frequency_sort_any(empty).size == 0 and O.stable_argsort_any(empty).size == 0
    assert O.final_path_any(empty) == O.EMPTY
    one = np.ones(1, dtype=dtype)
    assert O.frequency_sort_any(one).tolist() == [1] and O.stable_argsort_any(one).tolist() == [0]
    same = np.full(3000, 7, dtype=dtype)
    assert O.final_path_any(same) == O.BYPASS_SORTED
    assert np.array_equal(O.stable_argsort_any(same), np.arange(3000, dtype=np.uint32))


@pytest.mark.parametrize("fdt,idt", [(np.float32, np.uint32), (np.float64, np.uint64)])
def test_signed_zeros_are_two_keys(fdt, idt):
    # equal keys are equal bit patterns: -0 sorts before +0, each group stable
    x = np.array([0.0, -0.0, 0.0, -0.0, 1.0, -1.0], dtype=fdt)
    got = O.frequency_sort_any(x).view(idt)
    want = np.array([-1.0, -0.0, -0.0, 0.0, 0.0, 1.0], dtype=fdt).view(idt)
    assert np.array_equal(got, want)
    assert O.stable_argsort_any(x).tolist() == [5, 1, 3, 0, 2, 4]
