"""The torch twins of the seeded generators give the numpy generators' values
bit for bit (the benchmark builds its inputs with the former, the tests with
the latter)."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2605_25040_gb300 import datagen as G  # noqa: E402


@pytest.mark.parametrize("n,k,dist,dtype", [
    (1000, 7, "uniform", np.int64), (100_000, 300, "zipf", np.int64),
    (50_000, 50_000, "uniform", np.int32), (70_001, 1234, "zipf", np.int32),
    (5, 3, "uniform", np.int32), (300_000, 299_999, "uniform", np.int64),
])
def test_column_twin(n, k, dist, dtype):
    a = G.column(n, k, dist, dtype, seed=9)
    b = G.column_torch(n, k, dist, dtype, seed=9).numpy()
    assert a.dtype == b.dtype and np.array_equal(a, b)


@pytest.mark.parametrize("dtype", [np.int32, np.int64])
def test_spill_trigger_twin(dtype):
    assert np.array_equal(G.spill_trigger(100_000, dtype, seed=3),
                          G.spill_trigger_torch(100_000, dtype, seed=3).numpy())


def test_batch_and_mixed_twins():
    for i, (n, k) in enumerate(G.batch_specs(12, seed=5, n_hi=2e5)):
        assert np.array_equal(G.batch_column(n, k, i, 5), G.batch_column_torch(n, k, i, 5).numpy())
    for i, (n, k, t, kind) in enumerate(G.mixed_specs(20, n_hi=3e5, spill_every=5)):
        assert np.array_equal(G.mixed_column(n, k, t, kind, i, 2),
                              G.mixed_column_torch(n, k, t, kind, i, 2).numpy())


def test_specs_follow_the_recipes():
    specs = G.batch_specs(4096, seed=3)
    n = np.array([a for a, _ in specs])
    k = np.array([b for _, b in specs])
    assert n.min() >= 1000 and n.max() <= 1_000_000
    assert k.min() >= 2 and np.all(k <= np.maximum(2, np.minimum(n // 4 + 1, 50_000)))
    mixed = G.mixed_specs()
    assert len(mixed) == 64 and mixed[0][0] == 1000 and mixed[-1][0] == 30_000_000
    assert sum(1 for m in mixed if m[3] == "spill") == 4
    assert sum(1 for m in mixed if m[0] == m[1]) >= 10           # K = N columns
    assert {m[2] for m in mixed} == {"int32", "int64"}


def test_input_profiles_have_their_shape():
    x = G.runs_column(100_000, 300, 16.0, "zipf", np.int64, seed=3)
    assert x.size == 100_000 and np.array_equal(x, G.runs_column(100_000, 300, 16.0, "zipf", np.int64, seed=3))
    runs = 1 + int(np.count_nonzero(x[1:] != x[:-1]))
    assert 100_000 / 16.0 * 0.8 < runs < 100_000 / 16.0 * 1.2   # geometric runs, mean ~16
    g = G.grouped_column(50_000, 700, np.int32, seed=4)
    assert g.size == 50_000 and g.dtype == np.int32
    starts = np.flatnonzero(np.r_[True, g[1:] != g[:-1]])
    assert starts.size == 700 and np.unique(g).size == 700        # one contiguous group per key
    a = G.almost_sorted(50_000, 500, 40, np.int64, seed=5)
    assert np.count_nonzero(a[1:] < a[:-1]) <= 2 * 40
    assert np.count_nonzero(G.almost_sorted(50_000, 500, 0, np.int64, seed=5)[1:] <
                            G.almost_sorted(50_000, 500, 0, np.int64, seed=5)[:-1]) == 0
