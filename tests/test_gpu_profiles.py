"""Input profiles (runs of equal keys, one group per key, nearly sorted):
sorted keys, branch and argsort permutation equal the oracle's."""

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


def check(x, argsort=False):
    xt = torch.from_numpy(x).cuda()
    out, rep = cafs.sort_ex(xt)
    assert rep["device_status"] == 0
    assert np.array_equal(out.cpu().numpy(), O.frequency_sort(x))
    assert rep["path"] == O.final_path(x), (O.PATH_NAMES[rep["path"]], O.PATH_NAMES[O.final_path(x)])
    if argsort:
        _, perm = cafs.argsort(xt)
        assert np.array_equal(perm.cpu().numpy().view(np.uint32), O.stable_argsort(x))
    return rep


@pytest.mark.parametrize("dtype", [np.int32, np.int64])
@pytest.mark.parametrize("k,mean_run,dist", [(4, 1000.0, "uniform"), (200, 8.0, "uniform"),
                                             (4096, 64.0, "zipf"), (50_000, 3.0, "zipf")])
def test_runs(dtype, k, mean_run, dist):
    check(G.runs_column(300_000, k, mean_run, dist, dtype, seed=k), argsort=(k == 200))


@pytest.mark.parametrize("dtype", [np.int32, np.int64])
@pytest.mark.parametrize("k", [1, 8, 200, 4096, 100_000])
def test_grouped(dtype, k):
    check(G.grouped_column(300_000, k, dtype, seed=k), argsort=(k == 4096))


@pytest.mark.parametrize("dtype", [np.int32, np.int64])
@pytest.mark.parametrize("k,swaps", [(8, 1), (200, 30), (4096, 300), (300_000, 1000)])
def test_almost_sorted(dtype, k, swaps):
    check(G.almost_sorted(300_000, k, swaps, dtype, seed=k), argsort=(k == 200))
    check(G.almost_sorted(300_000, k, 0, dtype, seed=k))   # sorted: the bypass


@pytest.mark.parametrize("dtype", [np.int32, np.int64])
@pytest.mark.parametrize("k", [3, 50, 1500, 4000, 30_000])
@pytest.mark.parametrize("mean_run", [2.0, 9.0, 300.0])
def test_runs_in_every_table_form(k, mean_run, dtype):
    # Runs of equal keys are counted once per run with the run's length (the
    # run-length case of Sec. 4.4); K from the tiny path (3) through the
    # direct table (50), linear probing (1500), two-choice buckets (4000) to
    # the global table (30000), runs short and long, crossing vector, warp
    # and chunk boundaries.
    x = G.runs_column(700_001, k, mean_run, "uniform", dtype, seed=k + int(mean_run))
    check(x)
    check(x[::-1].copy())


@pytest.mark.parametrize("dtype", [np.int32, np.int64])
@pytest.mark.parametrize("n", [300_001, 1_048_573])
@pytest.mark.parametrize("shape", ["grouped", "runs2", "runs40"])
def test_run_folding_in_the_global_table(shape, n, dtype):
    # K_hat above one CTA's shared table: the global-table counter folds runs
    # of equal keys inside each warp's window of consecutive keys and inserts
    # every run once with its length (Sec. 4.4).  Ragged lengths give scalar
    # head and tail elements and chunks whose last warps hold fewer vectors;
    # the type minimum (the table's empty marker) is one of the run values,
    # and a window of all-distinct keys follows the plain per-key path.
    k = 60_000
    if shape == "grouped":
        x = G.grouped_column(n, k, dtype, seed=n % 97)
    else:
        x = G.runs_column(n, k, 2.0 if shape == "runs2" else 40.0, "uniform", dtype, seed=n % 89)
    x[x == x[n // 3]] = np.iinfo(dtype).min
    x[-5000:] = G.column(5000, 5000, "uniform", dtype, seed=3)   # distinct tail
    rep = check(x, argsort=(shape == "runs2" and n == 300_001))
    assert rep["path"] in (O.MAIN, O.MAIN_OVERFLOW_RADIX, O.HIGH_ENTROPY_RADIX)
