"""Parity of the mid-K paths with the CPU oracle, through the C ABI.

Columns whose estimate exceeds one CTA's shared table are counted in the
global Eq. 4 table, pair sets larger than the rank pass are ordered by a
splitter bucket sort, and columns whose estimate was too low (the guard's
overflow branch) are still emitted from their counts when the count
completed.  None of this may change a result, the estimate, the branch or K'
(Sec. 4.2, Alg. 3, Alg. 4).  The cases span ragged lengths, both key widths,
uniform and Zipf frequencies, the type minimum, keys that all share the high
bits of one multiplicative hash, per-call hash seeds and the stable argsort
on the same columns.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import cafs_oracle as O  # noqa: E402
from paper_2605_25040_gb300 import cafs  # noqa: E402
from paper_2605_25040_gb300 import datagen as G  # noqa: E402

pytestmark = pytest.mark.gpu

EST_FIELDS = ("n", "stride", "n_samples", "u", "f1", "f2", "k_hat", "M", "C", "L")

# Multiplier of the owner hash (high 32 bits of key * m, scaled to the grid).
OWNER_MULT = 0xD6E8FEB86659FD93


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_25040_gb300 import build
    build.build()
    cafs.load()
    yield


def check(x: np.ndarray, want_path=None):
    out, rep = cafs.sort_ex(torch.from_numpy(x).cuda())
    got = out.cpu().numpy()
    assert rep["device_status"] == 0
    want = O.frequency_sort(x)
    if not np.array_equal(got, want):
        bad = np.flatnonzero(got != want)
        raise AssertionError(f"{bad.size} mismatches, first at {bad[:5]}")
    path = O.final_path(x)
    assert rep["path"] == path, (O.PATH_NAMES[rep["path"]], O.PATH_NAMES[path])
    if want_path is not None:
        assert path == want_path
    est = O.chao1(x)
    for f in EST_FIELDS:
        assert rep["est"][f] == getattr(est, f), f
    if path in (O.TINY, O.MAIN, O.TINY_MISS_MAIN):
        assert rep["k_distinct"] == O.distinct_count(x)
    return rep


@pytest.mark.parametrize("dtype", [np.int32, np.int64])
@pytest.mark.parametrize("k", [5000, 9000, 20_000, 100_000])
@pytest.mark.parametrize("dist", ["uniform", "zipf"])
def test_mid_k_columns(k, dist, dtype):
    check(G.column(2_000_003, k, dist, dtype, seed=k + 7))


@pytest.mark.parametrize("n", [70_001, 300_001, 1_048_576])
def test_mid_k_grid_sizes(n):
    # grids of 5, 19 and 64 CTAs; about n / 30 distinct keys
    check(G.column(n, max(9000, n // 30), "uniform", np.int64, seed=n))


def owner_colliding_keys(count: int, dtype, seed: int) -> np.ndarray:
    """Distinct keys whose owner-hash product has its top 32 bits below 2^24,
    so that every one of them belongs to owner 0 on any grid of <= 256 CTAs
    (int64: built through the multiplier's inverse; int32: drawn and kept)."""
    rng = np.random.default_rng(seed)
    if dtype == np.int64:
        inv = pow(OWNER_MULT, -1, 1 << 64)
        hi = rng.integers(0, 1 << 24, size=count * 2, dtype=np.uint64)
        lo = rng.integers(0, 1 << 32, size=count * 2, dtype=np.uint64)
        t = (hi << np.uint64(32)) | lo
        with np.errstate(over="ignore"):
            x = (t * np.uint64(inv)).view(np.int64)
        x = np.unique(x[x != np.iinfo(np.int64).min])
    else:
        cand = np.unique(rng.integers(-(1 << 31) + 1, 1 << 31, size=count * 600, dtype=np.int64))
        with np.errstate(over="ignore"):
            h = (cand.view(np.uint64) * np.uint64(OWNER_MULT)) >> np.uint64(32)
        x = cand[h < (1 << 24)].astype(np.int32)
    assert x.size >= count
    return rng.permutation(x)[:count].astype(dtype)


@pytest.mark.parametrize("dtype", [np.int32, np.int64])
def test_all_keys_one_owner(dtype):
    # Every key shares the high 32 bits of one multiplicative hash: the
    # counts must not depend on where such keys land.
    vals = owner_colliding_keys(20_000, dtype, seed=5)
    rng = np.random.default_rng(6)
    x = vals[rng.integers(0, vals.size, size=2_000_000)]
    check(x, want_path=O.MAIN)


@pytest.mark.parametrize("dtype", [np.int32, np.int64])
def test_mid_k_type_extremes(dtype):
    info = np.iinfo(dtype)
    x = G.column(1_500_000, 30_000, "uniform", dtype, seed=9)
    x[::13] = info.min
    x[5::17] = info.max
    check(x)


def test_mid_k_hash_seeds():
    for x in (G.column(1_200_000, 40_000, "zipf", np.int64, seed=10),
              G.column(1_200_000, 40_000, "uniform", np.int64, seed=10)):
        seeded(x)


def seeded(x):
    want = O.frequency_sort(x)
    try:
        for s in (1, 0xDEADBEEF, 12345678901):
            cafs.set_hash_seed(s)
            out, rep = cafs.sort_ex(torch.from_numpy(x).cuda())
            assert np.array_equal(out.cpu().numpy(), want)
            assert rep["path"] == O.final_path(x)
            if rep["path"] == O.MAIN:
                assert rep["k_distinct"] == O.distinct_count(x)
    finally:
        cafs.set_hash_seed(0)


@pytest.mark.parametrize("dtype", [np.int32, np.int64])
def test_mid_k_argsort(dtype):
    x = G.column(800_001, 25_000, "uniform", dtype, seed=11)
    out, perm = cafs.argsort(torch.from_numpy(x).cuda())
    assert np.array_equal(out.cpu().numpy(), O.frequency_sort(x))
    assert np.array_equal(perm.cpu().numpy().view(np.uint32), O.stable_argsort(x))


def test_mid_k_repeated_and_interleaved():
    # the global table and the pair arrays are reused call after call
    seq = [G.column(1_000_000, 50_000, "uniform", np.int64, 1),
           G.column(1_000_000, 200, "uniform", np.int64, 2),
           G.spill_trigger(1_000_000, np.int64, 3),
           G.column(1_000_000, 12_000, "zipf", np.int64, 4),
           G.column(1_000_000, 50_000, "uniform", np.int64, 1)]
    for x in seq:
        check(x)
