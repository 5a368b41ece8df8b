"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Outputs must be bit-identical to the oracle's; the estimator fields
(u, f1, f2, K_hat, M, C, L), the dispatcher decision and the branch that
produced the output must equal the oracle's too.  Sizes span several tiles
and ragged tails; the edge cases cover empty, tiny and boundary lengths, the
type minimum (which doubles as the tables' empty marker), sorted and reverse
inputs, in-place sorting, misaligned pointers and every branch.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import cafs_oracle as O  # noqa: E402
from paper_2605_25040_gb300 import cafs  # noqa: E402
from paper_2605_25040_gb300 import datagen as G  # noqa: E402

pytestmark = pytest.mark.gpu

EST_FIELDS = ("n", "stride", "n_samples", "u", "f1", "f2", "k_hat", "M", "C", "L")


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_25040_gb300 import build
    build.build()
    cafs.load()
    yield


def check_sort(x: np.ndarray, inplace=False, offset=0):
    """Sorts x on the GPU, compares output, estimate and branch with the oracle."""
    xt = torch.from_numpy(np.concatenate([np.zeros(offset, x.dtype), x])).cuda()[offset:]
    if inplace:
        out, rep = cafs.sort_ex(xt, out=xt)
    else:
        out, rep = cafs.sort_ex(xt)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    want = O.frequency_sort(x)
    assert rep["device_status"] == 0
    assert got.dtype == want.dtype and got.size == want.size
    if not np.array_equal(got, want):
        bad = np.flatnonzero(got != want)
        raise AssertionError(f"{bad.size} mismatches, first at {bad[:5]}: got {got[bad[:5]]} want {want[bad[:5]]}")
    path = O.final_path(x)
    assert rep["path"] == path, (O.PATH_NAMES[rep["path"]], O.PATH_NAMES[path])
    if x.size:
        est = O.chao1(x)
        for f in EST_FIELDS:
            assert rep["est"][f] == getattr(est, f), f
        assert rep["est"]["dispatch"] == O.dispatch(x)
        if path in (O.TINY, O.MAIN, O.TINY_MISS_MAIN):
            assert rep["k_distinct"] == O.distinct_count(x)
    return rep


@pytest.mark.parametrize("dtype", [np.int32, np.int64])
@pytest.mark.parametrize("n", [0, 1, 2, 3, 17, 1023, 1024, 1025, 2047, 2048, 2049, 4099, 65537])
def test_lengths(n, dtype):
    check_sort(G.column(n, max(1, min(n, 5)), "uniform", dtype, seed=n))
    if n > 2:
        check_sort(G.column(n, max(1, n // 3), "zipf", dtype, seed=n + 1))


def test_config_parity_1e6_k200():
    # N = 1e6 int64 keys, K = 200 distinct values uniform over the 64-bit range
    x = G.column(1_000_000, 200, "uniform", np.int64, seed=0)
    rep = check_sort(x)
    assert rep["path"] == O.MAIN


@pytest.mark.parametrize("dtype", [np.int32, np.int64])
@pytest.mark.parametrize("k", [1, 2, 8, 9, 64, 200, 4096, 8191, 9000, 50000])
@pytest.mark.parametrize("dist", ["uniform", "zipf"])
def test_main_and_tiny_paths(k, dist, dtype):
    check_sort(G.column(300_001, k, dist, dtype, seed=k))


@pytest.mark.parametrize("dtype", [np.int32, np.int64])
def test_type_minimum_keys(dtype):
    info = np.iinfo(dtype)
    x = G.column(200_000, 50, "zipf", dtype, seed=4)
    x[::7] = info.min
    x[::11] = info.max
    check_sort(x)
    # the minimum as one of only a few keys (tiny path)
    y = np.where(np.arange(100_000) % 3 == 0, info.min, 5).astype(dtype)
    check_sort(G.shuffle(y, 3))
    # the minimum only outside the sampled positions (tiny miss)
    z = np.full(100_000, 7, dtype)
    z[1::97] = info.min
    check_sort(z)


def test_sorted_and_reverse():
    x = np.sort(G.column(500_000, 1000, "uniform", np.int64, seed=5))
    rep = check_sort(x)
    assert rep["path"] == O.BYPASS_SORTED
    check_sort(x, inplace=True)
    check_sort(x[::-1].copy())
    # samples ascend but the column does not: the full scan must find it
    y = x.copy()
    y[3], y[4] = y[4] + 1, y[3]
    check_sort(y)


def test_tiny_miss_example():
    x = (np.arange(10240) % 8).astype(np.int64)[::-1].copy()
    rep = check_sort(x)
    assert rep["path"] == O.TINY_MISS_MAIN


@pytest.mark.parametrize("dtype", [np.int32, np.int64])
def test_overflow_and_high_entropy(dtype):
    rep = check_sort(G.spill_trigger(262_144, dtype, seed=1))
    assert rep["path"] == O.MAIN_OVERFLOW_RADIX
    rep = check_sort(G.column(262_144, 262_144, "uniform", dtype, seed=2))
    assert rep["path"] == O.HIGH_ENTROPY_RADIX
    # tiny sample, many distinct keys outside it: tiny miss then overflow
    x = np.full(100_000, 3, dtype)
    x[1::3] = G.distinct_values(x[1::3].size, 9, dtype)
    stride = x.size // 1024
    x[np.arange(1024) * stride] = 3
    rep = check_sort(x)
    assert rep["path"] == O.TINY_MISS_MAIN_OVERFLOW_RADIX


@pytest.mark.parametrize("dtype", [np.int32, np.int64])
def test_inplace_all_paths(dtype):
    for x in (G.column(300_000, 300, "uniform", dtype, 1),
              G.column(300_000, 3, "uniform", dtype, 1),
              G.spill_trigger(300_000, dtype, 3),
              G.column(300_000, 300_000, "uniform", dtype, 4),
              G.column(3000, 3000, "uniform", dtype, 4)):
        check_sort(x, inplace=True)


@pytest.mark.parametrize("offset", [1, 3])
def test_misaligned_pointers(offset):
    check_sort(G.column(100_003, 77, "uniform", np.int64, 6), offset=offset)
    check_sort(G.column(100_003, 77, "uniform", np.int32, 6), offset=offset)
    check_sort(G.column(100_003, 100_003, "uniform", np.int32, 6), offset=offset)


def test_paper_palette():
    for k in (2, 40, 700, 15000):
        check_sort(G.paper_palette(400_000, k))


def test_estimate_matches_oracle():
    cases = [G.column(n, k, d, t, seed=n + k)
             for n in (1, 100, 2048, 5000, 1_000_003)
             for k in (1, 7, 300, 100_000)
             for d in ("uniform", "zipf")
             for t in (np.int32, np.int64)]
    cases.append(np.sort(G.column(50_000, 30, "uniform", np.int64, 1)))
    for x in cases:
        est = cafs.estimate_k(torch.from_numpy(x).cuda())
        ref = O.chao1(x)
        for f in EST_FIELDS:
            assert est[f] == getattr(ref, f), (f, x.size)
        assert est["dispatch"] == O.dispatch(x)
        assert bool(est["saturated"]) == ref.saturated


def test_workspace_reuse_keeps_tables_clean():
    # The global table is reset after every call; alternate branches on one stream.
    seq = [G.column(400_000, 5000, "uniform", np.int64, 1),
           G.spill_trigger(400_000, np.int64, 2),
           G.column(400_000, 5000, "zipf", np.int64, 3),
           G.column(400_000, 40_000, "uniform", np.int64, 4),
           G.column(400_000, 6, "uniform", np.int64, 5),
           G.column(400_000, 5000, "uniform", np.int64, 1)]
    for x in seq:
        check_sort(x)


def test_sort_host_end_to_end():
    x = G.column(777_777, 321, "zipf", np.int64, 8)
    out, rep = cafs.sort_host(x)
    assert np.array_equal(out, O.frequency_sort(x))
    assert rep["path"] == O.final_path(x)
    y = G.column(5000, 5000, "uniform", np.int32, 8)
    out, rep = cafs.sort_host(y)
    assert np.array_equal(out, O.frequency_sort(y))


def test_bounded_wait_reports_timeout():
    x = G.column(300_000, 100, "uniform", np.int64, 1)
    try:
        cafs.set_test_hooks(1, 20_000_000)  # CTA 0 never arrives; 20 ms wait limit
        _, rep = cafs.sort_ex(torch.from_numpy(x).cuda())
        assert rep["device_status"] == 7
    finally:
        cafs.set_test_hooks(0, 0)
    # the context is still usable
    check_sort(x)


@pytest.mark.parametrize("dtype", [np.int32, np.int64])
@pytest.mark.parametrize("offset", [0, 1])
def test_emit_tiles_with_a_few_short_runs(dtype, offset):
    # Output runs 50000, 1, 2, 3, 49994 (and variants): one emit tile holds
    # several boundaries, some inside one 16-byte vector.
    for lens in ([50_000, 1, 2, 3, 49_994], [49_999, 1, 1, 1, 1, 1, 1, 49_995],
                 [16_381, 3, 16_000, 5, 7, 30_000]):
        x = np.repeat(np.arange(len(lens), dtype=dtype) * 7 - 3, lens)
        check_sort(G.shuffle(x, sum(lens)), offset=offset)


def eq4_slots(x: np.ndarray, log2size: int) -> np.ndarray:
    """Eq. 4 for the test data: ((x * 2^64/phi) mod 2^64) >> (64 - log2 M),
    x taken as its 64-bit two's-complement pattern (int32 sign-extended)."""
    u = x.astype(np.int64).view(np.uint64)
    with np.errstate(over="ignore"):
        return (u * np.uint64(0x9E3779B97F4A7C15)) >> np.uint64(64 - log2size)


def colliding_values(groups: int, per_group: int, dtype, seed: int) -> np.ndarray:
    """groups x per_group distinct values; the values of a group share one
    slot of a 4096-slot Eq. 4 table (Alg. 2's FreqSet), so where each lands
    depends on which is inserted first."""
    rng = np.random.default_rng(seed)
    info = np.iinfo(dtype)
    cand = np.unique(rng.integers(info.min + 1, info.max, size=400_000, dtype=dtype))
    slots = eq4_slots(cand, 12)
    order = np.argsort(slots, kind="stable")
    s_sorted = slots[order]
    starts = np.flatnonzero(np.r_[True, s_sorted[1:] != s_sorted[:-1]])
    ends = np.r_[starts[1:], s_sorted.size]
    full = [(a, b) for a, b in zip(starts, ends) if b - a >= per_group][:groups]
    assert len(full) == groups
    return np.concatenate([cand[order[a:a + per_group]] for a, _ in full])


def place_samples_by_warp(x: np.ndarray, vals: np.ndarray) -> np.ndarray:
    """Alg. 2's strided sample positions i * stride (i < 1024) get vals[i //
    (1024 / len(vals))]: each value's samples are contiguous, so different
    warps of the sampler insert different values of a colliding group."""
    x = x.copy()
    stride = max(1, x.size // 1024)
    i = np.arange(1024)
    x[i * stride] = vals[i * len(vals) // 1024]
    return x


@pytest.mark.parametrize("dtype", [np.int32, np.int64])
def test_sampled_keys_colliding_in_the_sampler_table(dtype):
    # Every CTA of the grid computes the estimate and the list of sampled keys
    # itself; the list (and the tiny path's keys) must not depend on the
    # order in which colliding keys entered the FreqSet.  Repeated calls.
    vals8 = colliding_values(1, 8, dtype, seed=11)
    rng = np.random.default_rng(13)
    x = place_samples_by_warp(vals8[rng.integers(0, 8, size=300_000)], vals8)
    vals = colliding_values(32, 8, dtype, seed=12)
    y = place_samples_by_warp(vals[rng.integers(0, vals.size, size=300_000)], vals)
    for _ in range(8):
        assert check_sort(x)["path"] == O.TINY
        assert check_sort(y)["path"] == O.MAIN
    outs, reps = cafs.sort_batch([torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()] * 4,
                                 reports=True, tuning={"grid_min_n": 2048})
    for o, r, z in zip(outs, reps, [x, y] * 4):
        assert np.array_equal(o.cpu().numpy(), O.frequency_sort(z))
        assert r["path"] == O.final_path(z)
