"""Per-call hash seeds (cafs_set_hash_seed): whatever multipliers the table
hashes use, every column's sorted keys, branch and distinct count must equal
the oracle's; keys that all collide in the Eq. 4 table under the golden-ratio
multiplier sort correctly with and without a seed."""

import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import cafs_oracle as O  # noqa: E402
from paper_2605_25040_gb300 import cafs  # noqa: E402
from paper_2605_25040_gb300 import datagen as G  # noqa: E402

pytestmark = pytest.mark.gpu

PHI = 0x9E3779B97F4A7C15
M64 = (1 << 64) - 1


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_25040_gb300 import build
    build.build()
    cafs.load()
    yield
    cafs.set_hash_seed(0)


def eq4_colliding(count: int) -> np.ndarray:
    """count distinct int64 keys whose Eq. 4 products x * phi mod 2^64 share
    their top 24 bits: one slot of any table of up to 2^24 slots."""
    inv = pow(PHI, -1, 1 << 64)
    u = [(inv * ((5 << 40) + 977 * i)) & M64 for i in range(count)]
    assert all(((x * PHI) & M64) >> 40 == 5 for x in u)
    return np.array([x - (1 << 64) if x >> 63 else x for x in u], dtype=np.int64)


def check(x, rep):
    assert rep["device_status"] == 0
    assert rep["path"] == O.final_path(x)
    if rep["path"] in (O.TINY, O.MAIN, O.TINY_MISS_MAIN):
        assert rep["k_distinct"] == O.distinct_count(x)


@pytest.mark.parametrize("seed", [0, 12345, (1 << 63) + 99])
def test_results_do_not_depend_on_the_seed(seed):
    cafs.set_hash_seed(seed)
    cols = [G.column(300_000, 5, "uniform", np.int64, seed=1),
            G.column(300_000, 200, "uniform", np.int32, seed=2),
            G.column(400_000, 4096, "zipf", np.int64, seed=3),
            G.column(400_000, 20_000, "uniform", np.int64, seed=4),
            G.spill_trigger(200_000, np.int64, seed=5),
            G.column(200_000, 200_000, "uniform", np.int32, seed=6)]
    for x in cols:
        out, rep = cafs.sort_ex(torch.from_numpy(x).cuda())
        assert np.array_equal(out.cpu().numpy(), O.frequency_sort(x))
        check(x, rep)
    outs, reps = cafs.sort_batch([torch.from_numpy(x).cuda() for x in cols], reports=True)
    for x, o, r in zip(cols, outs, reps):
        assert np.array_equal(o.cpu().numpy(), O.frequency_sort(x))
        check(x, r)
    x = cols[2]
    out, perm = cafs.argsort(torch.from_numpy(x).cuda())
    assert np.array_equal(perm.cpu().numpy().view(np.uint32), O.stable_argsort(x))


def test_keys_colliding_under_the_default_multiplier():
    vals = eq4_colliding(1000)
    x = vals[np.random.default_rng(7).integers(0, vals.size, size=200_000)]
    want = O.frequency_sort(x)
    xt = torch.from_numpy(x).cuda()
    times = {}
    for seed in (0, 777):
        cafs.set_hash_seed(seed)
        for _ in range(2):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            out, rep = cafs.sort_ex(xt)
            times[seed] = time.perf_counter() - t0
            assert np.array_equal(out.cpu().numpy(), want)
            check(x, rep)
    print(f"colliding keys: {times[0] * 1e3:.2f} ms with the golden-ratio multiplier, "
          f"{times[777] * 1e3:.2f} ms with a seeded one")
