"""Stable argsort through the C ABI (cafs_argsort): the permutation must equal
the oracle's stable_argsort element for element, the sorted keys the oracle's
frequency_sort, and the branch the oracle's final_path, on every path."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import cafs_oracle as O  # noqa: E402
from paper_2605_25040_gb300 import cafs  # noqa: E402
from paper_2605_25040_gb300 import datagen as G  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_25040_gb300 import build
    build.build()
    cafs.load()
    yield


def check_argsort(x: np.ndarray):
    xt = torch.from_numpy(x).cuda()
    out, perm, rep = cafs.argsort(xt, report=True)
    assert rep["device_status"] == 0
    got = perm.cpu().numpy().view(np.uint32)
    want = O.stable_argsort(x)
    if not np.array_equal(got, want):
        bad = np.flatnonzero(got != want)
        raise AssertionError(f"{bad.size} mismatches, first at {bad[:5]}: got {got[bad[:5]]} want {want[bad[:5]]}")
    assert np.array_equal(out.cpu().numpy(), O.frequency_sort(x))
    assert rep["path"] == O.final_path(x), (O.PATH_NAMES[rep["path"]], O.PATH_NAMES[O.final_path(x)])
    return rep


@pytest.mark.parametrize("dtype", [np.int32, np.int64])
@pytest.mark.parametrize("n", [1, 2, 17, 1023, 2047, 2048, 2049, 65537])
def test_lengths(n, dtype):
    check_argsort(G.column(n, max(1, n // 7), "zipf", dtype, seed=n))


@pytest.mark.parametrize("dtype", [np.int32, np.int64])
@pytest.mark.parametrize("k", [1, 5, 9, 200, 300, 4096, 9000, 50000])
def test_count_paths(k, dtype):
    # K' <= 256: one rank pass; <= 4096: ranks from shared memory; above:
    # the pair radix and ranks searched in global memory
    check_argsort(G.column(400_000, k, "zipf", dtype, seed=k))
    check_argsort(G.column(300_000, k, "uniform", dtype, seed=k + 1))


@pytest.mark.parametrize("dtype", [np.int32, np.int64])
def test_radix_paths(dtype):
    n = 300_000
    assert check_argsort(G.column(n, n, "uniform", dtype, seed=1))["path"] == O.HIGH_ENTROPY_RADIX
    assert check_argsort(G.spill_trigger(n, dtype, seed=2))["path"] == O.MAIN_OVERFLOW_RADIX


@pytest.mark.parametrize("dtype", [np.int32, np.int64])
def test_sorted_reverse_and_type_minimum(dtype):
    x = np.sort(G.column(200_000, 1000, "zipf", dtype, seed=3))
    assert check_argsort(x)["path"] == O.BYPASS_SORTED
    check_argsort(x[::-1].copy())
    info = np.iinfo(dtype)
    y = G.column(200_000, 50, "uniform", dtype, seed=4)
    y[::7] = info.min
    y[3::11] = info.max
    check_argsort(y)


def test_repeated_calls_and_streams():
    s = torch.cuda.Stream()
    xs = [G.column(250_000, k, "zipf", np.int64, seed=k) for k in (4, 700, 250_000)]
    for _ in range(3):
        for x in xs:
            check_argsort(x)
    with torch.cuda.stream(s):
        xt = torch.from_numpy(xs[1]).cuda()
        out, perm = cafs.argsort(xt, stream=s)
    s.synchronize()
    assert np.array_equal(perm.cpu().numpy().view(np.uint32), O.stable_argsort(xs[1]))


@pytest.mark.parametrize("spec", [("uniform", 200), ("zipf", 4096), ("uniform", 3 * 10**7)])
def test_full_size_properties(spec):
    # N = 3e7: the pure-Python oracle is too slow, so the properties that
    # determine the stable argsort are checked: perm is a permutation,
    # keys[perm] equals the oracle's sorted keys, and equal keys keep their
    # input order.
    dist, k = spec
    n = 30_000_000
    xt = G.column_torch(n, k, dist, np.int64, seed=7, device="cuda")
    out, perm, rep = cafs.argsort(xt, report=True)
    assert rep["device_status"] == 0
    p = perm.long() & 0xFFFFFFFF
    assert int(torch.bincount(p, minlength=n).max()) == 1
    sorted_keys = xt[p]
    assert torch.equal(sorted_keys, out)
    assert np.array_equal(out.cpu().numpy(), O.frequency_sort(xt.cpu().numpy()))
    same = sorted_keys[1:] == sorted_keys[:-1]
    assert bool((p[1:][same] > p[:-1][same]).all())
