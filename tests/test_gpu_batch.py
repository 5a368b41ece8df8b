"""Parity of the batched form (cafs_sort_batch, batch plans) with the oracle.

Every column of a batch must come out bit-identical to the oracle's sort,
with the oracle's estimate and branch, and with exactly the report that the
single-column entry point gives it alone.  The cases cover every branch, both
dtypes in one batch, empty and short columns, in-place columns, each stage of
the batched kernel (all-CTA columns, the per-CTA queue, set-aside radix
columns), every scheduling knob, and the recorded-graph plan replayed over
refilled inputs.
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


def check_column(x: np.ndarray, got: np.ndarray, rep: dict, solo: dict | None = None):
    want = O.frequency_sort(x)
    assert rep["device_status"] == 0
    assert got.dtype == want.dtype and got.size == want.size
    if not np.array_equal(got, want):
        bad = np.flatnonzero(got != want)
        raise AssertionError(f"n={x.size}: {bad.size} mismatches, first at {bad[:5]}")
    path = O.final_path(x)
    assert rep["path"] == path, (x.size, O.PATH_NAMES[rep["path"]], O.PATH_NAMES[path])
    if x.size:
        est = O.chao1(x)
        for f in EST_FIELDS:
            assert rep["est"][f] == getattr(est, f), (f, x.size)
        assert rep["est"]["dispatch"] == O.dispatch(x)
        if path in (O.TINY, O.MAIN, O.TINY_MISS_MAIN):
            assert rep["k_distinct"] == O.distinct_count(x)
    if solo is not None:
        assert rep["path"] == solo["path"] and rep["k_distinct"] == solo["k_distinct"]
        assert rep["est"] == solo["est"]


def run_batch(cols, tuning=None, inplace=False, compare_solo=False):
    keys = [torch.from_numpy(x).cuda() for x in cols]
    outs = keys if inplace else [torch.empty_like(k) for k in keys]
    outs, reps = cafs.sort_batch(keys, outs=outs, tuning=tuning, reports=True)
    torch.cuda.synchronize()
    for i, x in enumerate(cols):
        solo = None
        if compare_solo:
            _, solo = cafs.sort_ex(torch.from_numpy(x).cuda())
        check_column(x, outs[i].cpu().numpy(), reps[i], solo)
    return reps


def mixed_small_columns(seed=0):
    """Every branch, both dtypes, short and ragged lengths (a few seconds of oracle)."""
    cols = []
    for i, n in enumerate([0, 1, 5, 1000, 2047, 2048, 2049, 5003, 70_001, 300_007]):
        for dtype in (np.int32, np.int64):
            k = max(1, min(n, [1, 3, 8, 9, 200, 5000][i % 6]))
            cols.append(G.column(n, k, "zipf" if i % 2 else "uniform", dtype, seed=seed + i))
    info = np.iinfo(np.int64)
    x = G.column(120_000, 40, "zipf", np.int64, seed=seed + 50)
    x[::9] = info.min                      # the type minimum (the tables' empty marker)
    cols.append(x)
    cols.append(np.sort(G.column(90_000, 500, "uniform", np.int64, seed=seed + 51)))   # bypass
    cols.append(np.sort(G.column(90_000, 500, "uniform", np.int32, seed=seed + 52))[::-1].copy())
    cols.append(G.spill_trigger(150_000, np.int64, seed=seed + 53))                      # overflow
    cols.append(G.spill_trigger(40_000, np.int32, seed=seed + 54))
    cols.append(G.column(100_000, 100_000, "uniform", np.int64, seed=seed + 55))         # 2 K_hat > N
    cols.append(G.column(20_000, 20_000, "uniform", np.int32, seed=seed + 56))
    cols.append((np.arange(10240) % 8).astype(np.int64)[::-1].copy())                   # tiny miss
    y = np.full(100_000, 3, np.int64)
    y[1::3] = G.distinct_values(y[1::3].size, 9, np.int64)
    y[np.arange(1024) * (y.size // 1024)] = 3                                            # tiny miss + overflow
    cols.append(y)
    cols.append(G.column(200_003, 6000, "uniform", np.int64, seed=seed + 57))          # > 4096 pairs
    cols.append(G.column(200_003, 30_000, "zipf", np.int32, seed=seed + 58))
    return cols


def test_batch_mixed_matches_oracle_and_solo():
    reps = run_batch(mixed_small_columns(), compare_solo=True)
    paths = {r["path"] for r in reps}
    for p in (O.EMPTY, O.BYPASS_SORTED, O.SMALL_N, O.TINY, O.MAIN, O.HIGH_ENTROPY_RADIX,
              O.MAIN_OVERFLOW_RADIX, O.TINY_MISS_MAIN, O.TINY_MISS_MAIN_OVERFLOW_RADIX):
        assert p in paths, O.PATH_NAMES[p]


def test_batch_all_columns_on_the_whole_grid():
    # grid_min_n = 2048: every column of >= 2048 keys goes through stage 1
    run_batch(mixed_small_columns(7), tuning={"grid_min_n": 2048})


def test_batch_set_aside_radix_columns():
    # defer_min_n = 2048: every radix-fallback column of the queue is set aside
    cols = mixed_small_columns(11)
    cols += [G.column(n, n, "uniform", t, seed=n) for n in (3000, 65_536, 250_001)
             for t in (np.int32, np.int64)]
    run_batch(cols, tuning={"defer_min_n": 2048})


@pytest.mark.parametrize("tuning", [
    {"cta_table_slots": 64},
    {"cta_table_slots": 4096, "defer_min_n": 1 << 30},
    {"local_slots_max": 256, "replicas_max": 1},
    {"local_slots_max": 2048, "replicas_max": 4, "emit_tile_vec": 1024},
    {"emit_tile_vec": 8192, "ctas": 7},
    {"ctas": 1, "grid_min_n": 50_000, "defer_min_n": 10_000},
])
def test_batch_knobs_never_change_results(tuning):
    run_batch(mixed_small_columns(3), tuning=tuning)


def test_batch_inplace():
    run_batch(mixed_small_columns(5), inplace=True)


def test_batch_of_config_recipe_sample():
    # 400 columns of the batched workload's recipe: N log-uniform in [1e3, 1e6],
    # K log-uniform in [2, min(N/4, 5e4)], Zipf s = 1.1
    specs = G.batch_specs(400, seed=21)
    cols = [G.batch_column(n, k, i, 21) for i, (n, k) in enumerate(specs)]
    run_batch(cols)


def test_batch_mixed_dtype_recipe_small():
    # the mixed workload's recipe scaled down to N in [1e3, 2e6] (32 columns)
    specs = G.mixed_specs(32, n_hi=2e6, spill_every=8)
    cols = [G.mixed_column(n, k, t, kind, i, 4) for i, (n, k, t, kind) in enumerate(specs)]
    run_batch(cols)
    run_batch(cols, tuning={"grid_min_n": 1 << 19})


def test_batch_empty_and_single():
    outs, reps = cafs.sort_batch([], reports=True)
    assert outs == [] and reps == []
    run_batch([G.column(0, 1, "uniform", np.int64, 0)])
    run_batch([G.column(777_777, 300, "uniform", np.int64, 1)])


def test_plan_replays_over_refilled_inputs():
    cols = mixed_small_columns(13)
    keys = [torch.from_numpy(x).cuda() for x in cols]
    outs = [torch.empty_like(k) for k in keys]
    plan = cafs.BatchPlan(keys, outs, tuning={"defer_min_n": 4096})
    try:
        for rnd in range(3):
            if rnd:
                cols = [G.column(x.size, max(1, min(x.size, 37 * rnd)), "zipf", x.dtype, seed=100 * rnd + i)
                        for i, x in enumerate(cols)]
                for k, x in zip(keys, cols):
                    k.copy_(torch.from_numpy(x))
            plan.launch()
            reps = plan.reports()
            for i, x in enumerate(cols):
                check_column(x, outs[i].cpu().numpy(), reps[i])
    finally:
        plan.close()


def test_batch_launch_count_is_one():
    cols = [G.column(50_000 + i, 100, "uniform", np.int64, seed=i) for i in range(64)]
    keys = [torch.from_numpy(x).cuda() for x in cols]
    cafs.sort_batch(keys)  # workspace grows here
    torch.cuda.synchronize()
    before = cafs.kernel_launch_count()
    cafs.sort_batch(keys)
    torch.cuda.synchronize()
    assert cafs.kernel_launch_count() - before == 1


def test_autotuner_times_candidates_and_caches(tmp_path):
    from paper_2605_25040_gb300 import autotune
    cols = mixed_small_columns(17)
    keys = [torch.from_numpy(x).cuda() for x in cols]
    outs = [torch.empty_like(k) for k in keys]
    ms = cafs.time_tunings(keys, outs, [{}, {"emit_tile_vec": 1024}, {"local_slots_max": 2048}], reps=2)
    assert len(ms) == 3 and all(m > 0 for m in ms)
    for x, o in zip(cols, outs):        # the tuner's launches sorted the columns too
        assert np.array_equal(o.cpu().numpy(), O.frequency_sort(x))
    cache = str(tmp_path / "tune.json")
    small = {"emit_tile_vec": [2048, 4096], "replicas_max": [8, 32]}
    r1 = autotune.tuned(keys, outs, cache_path=cache, reps=1, rounds=1, space=small)
    assert not r1["cached"] and r1["ms"] > 0 and r1["trials"] == 5
    r2 = autotune.tuned(keys, outs, cache_path=cache, space=small)
    assert r2["cached"] and r2["tuning"] == r1["tuning"]
    run_batch(cols, tuning=r1["tuning"])
