"""Unsigned and IEEE-float keys through the C ABI: sorted bits, branch and
estimate equal the oracle's (frequency_sort_any / final_path_any), and the
argsort permutation equals stable_argsort_any, for every path."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import cafs_oracle as O  # noqa: E402
from paper_2605_25040_gb300 import cafs  # noqa: E402
from paper_2605_25040_gb300 import datagen as G  # noqa: E402

pytestmark = pytest.mark.gpu

BITS = {np.dtype(np.uint32): np.int32, np.dtype(np.uint64): np.int64,
        np.dtype(np.float32): np.int32, np.dtype(np.float64): np.int64}


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_25040_gb300 import build
    build.build()
    cafs.load()
    yield


def to_device(x):
    """The keys' bits in a signed tensor of the same width."""
    return torch.from_numpy(x.view(BITS[x.dtype])).cuda()


def check(x, argsort=False):
    name = x.dtype.name
    xt = to_device(x)
    out, rep = cafs.sort_ex(xt, key_type=name)
    want = O.frequency_sort_any(x)
    got = out.cpu().numpy().view(x.dtype)
    assert np.array_equal(got.view(np.uint8), want.view(np.uint8)), name
    assert rep["device_status"] == 0
    assert rep["path"] == O.final_path_any(x), (O.PATH_NAMES[rep["path"]], O.PATH_NAMES[O.final_path_any(x)])
    assert rep["est"]["k_hat"] == O.chao1(O.ordered_signed(x)).k_hat
    if argsort:
        out2, perm = cafs.argsort(xt, key_type=name)
        assert np.array_equal(perm.cpu().numpy().view(np.uint32), O.stable_argsort_any(x))
        assert np.array_equal(out2.cpu().numpy().view(np.uint8), want.view(np.uint8))
    return rep


def float_palette(k, dtype, seed, specials=True):
    rng = np.random.default_rng(seed)
    vals = (rng.standard_normal(k) * 10.0 ** rng.integers(-30, 30, size=k)).astype(dtype)
    if specials and k >= 8:
        bits_t = np.uint32 if dtype == np.float32 else np.uint64
        sp = np.array([-0.0, 0.0, np.inf, -np.inf, np.nan, 1e-40 if dtype == np.float32 else 1e-310], dtype=dtype)
        vals[:sp.size] = sp
        vals[sp.size] = (np.array([np.nan], dtype=dtype).view(bits_t) | (bits_t(1) << bits_t(
            np.dtype(dtype).itemsize * 8 - 1))).view(dtype)[0]   # a negative NaN
    return vals


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
@pytest.mark.parametrize("k", [1, 5, 200, 4096, 300_000])
def test_unsigned(dtype, k):
    # the int columns' bits as unsigned keys: values on both sides of 2^(w-1)
    x = G.column(300_000, k, "zipf", BITS[np.dtype(dtype)], seed=k).view(dtype)
    check(x, argsort=(k in (5, 4096)))
    info = np.iinfo(dtype)
    y = x.copy()
    y[::5] = info.max
    y[1::7] = 0
    check(y)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("k", [3, 8, 200, 4096, 250_000])
def test_floats(dtype, k):
    vals = float_palette(k, dtype, seed=k)
    x = vals[np.random.default_rng(k + 1).integers(0, k, size=300_000)]
    check(x, argsort=(k in (8, 4096)))


@pytest.mark.parametrize("dtype", [np.float32, np.float64, np.uint32, np.uint64])
def test_lengths_sorted_and_host(dtype):
    for n in (1, 2047, 2048, 5000):
        x = (float_palette(max(8, n // 3), dtype, seed=n)[np.random.default_rng(n).integers(0, max(8, n // 3), n)]
             if np.dtype(dtype).kind == "f"
             else G.column(n, max(1, n // 3), "uniform", BITS[np.dtype(dtype)], seed=n).view(dtype))
        check(x, argsort=True)
        check(O.frequency_sort_any(x))   # sorted input: bypass
    x = float_palette(500, dtype, seed=3)[np.random.default_rng(4).integers(0, 500, 100_000)] \
        if np.dtype(dtype).kind == "f" else G.column(100_000, 500, "zipf", BITS[np.dtype(dtype)], seed=5).view(dtype)
    got, rep = cafs.sort_host(x)
    assert np.array_equal(got.view(np.uint8), O.frequency_sort_any(x).view(np.uint8))
    assert rep["path"] == O.final_path_any(x)
    # in place
    xt = to_device(x)
    cafs.sort(xt, out=xt, key_type=np.dtype(dtype).name)
    assert np.array_equal(xt.cpu().numpy().view(np.uint8), O.frequency_sort_any(x).view(np.uint8))


def mixed_type_columns():
    cols = []
    specs = [(np.uint32, 300_000, 5), (np.float32, 200_000, 200), (np.uint64, 250_000, 4096),
             (np.float64, 300_000, 300_000), (np.uint64, 1500, 700), (np.float64, 100_000, 8),
             (np.int64, 200_000, 50), (np.float32, 3000, 3000)]
    for i, (dt, n, k) in enumerate(specs):
        if np.dtype(dt).kind == "f":
            cols.append(float_palette(k, dt, seed=i)[np.random.default_rng(i).integers(0, k, n)])
        elif np.dtype(dt).kind == "u":
            cols.append(G.column(n, k, "zipf", BITS[np.dtype(dt)], seed=i).view(dt))
        else:
            cols.append(G.column(n, k, "uniform", dt, seed=i))
    return cols


@pytest.mark.parametrize("tuning", [None, {"grid_min_n": 2048}])
def test_batch_of_mixed_key_types(tuning):
    cols = mixed_type_columns()
    keys = [torch.from_numpy(x.view(BITS.get(x.dtype, x.dtype))).cuda() for x in cols]
    names = [x.dtype.name for x in cols]
    outs, reps = cafs.sort_batch(keys, reports=True, tuning=tuning, key_types=names)
    for x, o, r in zip(cols, outs, reps):
        assert np.array_equal(o.cpu().numpy().view(np.uint8), O.frequency_sort_any(x).view(np.uint8)), x.dtype
        assert r["path"] == O.final_path_any(x)
    # a recorded plan over the same buffers, refilled
    outs2 = [torch.empty_like(k) for k in keys]
    plan = cafs.BatchPlan(keys, outs2, key_types=names)
    try:
        for _ in range(2):
            plan.launch()
        torch.cuda.synchronize()
        for x, o in zip(cols, outs2):
            assert np.array_equal(o.cpu().numpy().view(np.uint8), O.frequency_sort_any(x).view(np.uint8))
    finally:
        plan.close()


def test_server_key_types():
    cols = mixed_type_columns()
    srv = cafs.Server(2 << 30)
    try:
        outs = [np.empty_like(x) for x in cols]
        tickets = [srv.submit(x, o) for x, o in zip(cols, outs)]
        for x, o, t in zip(cols, outs, tickets):
            rep, _ = srv.wait(t)
            assert rep["device_status"] == 0
            assert np.array_equal(o.view(np.uint8), O.frequency_sort_any(x).view(np.uint8)), x.dtype
            assert rep["path"] == O.final_path_any(x)
        # one at a time: the idle server's direct path
        for x in cols[:3]:
            o = np.empty_like(x)
            rep, _ = srv.wait(srv.submit(x, o))
            assert np.array_equal(o.view(np.uint8), O.frequency_sort_any(x).view(np.uint8))
    finally:
        srv.close()
