"""The served form: a request server with a fixed device-memory budget.

Every request's result must equal the oracle's sort with the oracle's branch,
whatever else is in flight with it; requests larger than the free arena wait
for admission instead of failing; oversized requests are refused; the
open-loop trace replay and the serial baseline give the same outputs.
"""

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


def request_columns(count, seed, n_hi=3e5):
    specs = G.batch_specs(count, seed=seed, n_lo=1e3, n_hi=n_hi, k_cap=1e5)
    cols = []
    for i, (n, k) in enumerate(specs):
        dtype = np.int64 if i % 3 else np.int32
        if i % 17 == 5:
            cols.append(G.spill_trigger(max(n, 4096), dtype, seed=i))
        elif i % 13 == 7:
            cols.append(G.column(n, n, "uniform", dtype, seed=i))
        else:
            cols.append(G.column(n, k, "zipf", dtype, seed=seed * 7919 + i))
    return cols


def check(x, got, rep):
    assert rep["device_status"] == 0
    assert np.array_equal(got, O.frequency_sort(x))
    assert rep["path"] == O.final_path(x), (x.size, rep["path"], O.final_path(x))


def test_submit_and_wait_in_any_mix():
    cols = request_columns(120, seed=1)
    cols.insert(3, np.zeros(0, np.int64))
    srv = cafs.Server(2 << 30)
    try:
        outs = [np.empty_like(x) for x in cols]
        tickets = [srv.submit(x, o) for x, o in zip(cols, outs)]
        for x, o, t in zip(cols, outs, tickets):
            rep, lat = srv.wait(t)
            assert lat >= 0
            if x.size:
                check(x, o, rep)
        st = srv.stats()
        assert st["completed"] == len(cols) - 1 and st["pending"] == 0
        assert st["launches"] >= 1 and st["arena_peak_bytes"] <= st["arena_bytes"]
    finally:
        srv.close()


def test_admission_waits_for_memory():
    # An arena of a few tens of MB: only a few 8 MB requests fit at a time.
    cfg = {"max_request_keys": 1 << 20, "max_batch_columns": 64,
           "tuning": {"cta_table_slots": 1 << 14, "defer_min_n": 1 << 15}}
    srv = cafs.Server(160 << 20, cfg)
    try:
        st = srv.stats()
        assert st["arena_bytes"] + st["workspace_bytes"] <= 160 << 20
        assert 8_000_000 < st["arena_bytes"] < 24_000_000 * 2
        cols = [G.column(1_000_000, 50 + i, "uniform", np.int64, seed=i) for i in range(24)]
        outs = [np.empty_like(x) for x in cols]
        tickets = [srv.submit(x, o) for x, o in zip(cols, outs)]
        for x, o, t in zip(cols, outs, tickets):
            rep, _ = srv.wait(t)
            check(x, o, rep)
        st = srv.stats()
        assert st["arena_peak_bytes"] <= st["arena_bytes"]
        with pytest.raises(cafs.CafsError) as e:
            srv.submit(np.zeros((1 << 20) + 1, np.int64), np.zeros((1 << 20) + 1, np.int64))
        assert e.value.code == 3
    finally:
        srv.close()


def test_trace_replay_and_serial_baseline():
    cols = request_columns(150, seed=2)
    rng_gaps = G.exponential_gaps(20_000.0, len(cols), seed=3)
    arrivals = np.cumsum(rng_gaps) - rng_gaps[0]
    pin_in = [torch.from_numpy(x).pin_memory() for x in cols]
    pin_out = [torch.empty_like(t).pin_memory() for t in pin_in]
    pairs = [(a.numpy(), b.numpy()) for a, b in zip(pin_in, pin_out)]
    srv = cafs.Server(2 << 30)
    try:
        lat, elapsed, reps = srv.run_trace(pairs, arrivals, reports=True)
        assert elapsed > 0 and np.all(lat > 0)
        for x, (_, o), r in zip(cols, pairs, reps):
            check(x, o, r)
    finally:
        srv.close()
    for _, o in pairs:
        o.fill(0)
    lat2, elapsed2 = cafs.serial_run_trace(pairs, arrivals)
    assert elapsed2 > 0 and np.all(lat2 > 0)
    for x, (_, o) in zip(cols, pairs):
        assert np.array_equal(o, O.frequency_sort(x))


def test_large_requests_set_aside_to_all_ctas():
    # requests whose Eq. 6 table exceeds the per-CTA slot go to the all-CTA stage
    cfg = {"tuning": {"cta_table_slots": 1 << 10}}
    srv = cafs.Server(2 << 30, cfg)
    try:
        cols = [G.column(400_000, k, "uniform", np.int64, seed=k) for k in (3, 500, 20_000, 90_000)]
        outs = [np.empty_like(x) for x in cols]
        tickets = [srv.submit(x, o) for x, o in zip(cols, outs)]
        for x, o, t in zip(cols, outs, tickets):
            rep, _ = srv.wait(t)
            check(x, o, rep)
    finally:
        srv.close()
