"""Parity at the benchmark's full sizes, in the launch configurations that
bench.py times.

The single-array sweep (N = 3e7 int64, one cooperative launch of one CTA per
SM per column): representative columns of every branch are compared element
by element with the oracle.  The batched workload (4096 columns, N up to
1e6, one batched launch): a seeded sample of columns is compared with the
oracle element by element, and every column is checked for the properties
that hold at any size (non-decreasing, same length, same key sum and the
same count of the type minimum as its input).
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import cafs_oracle as O  # noqa: E402
from paper_2605_25040_gb300 import cafs  # noqa: E402
from paper_2605_25040_gb300 import datagen as G  # noqa: E402

pytestmark = pytest.mark.gpu

N = 30_000_000


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_25040_gb300 import build
    build.build()
    cafs.load()
    yield


@pytest.mark.parametrize("kind,k", [("uniform", 200), ("zipf", 4096), ("uniform", 4),
                                    ("uniform", 130_000), ("uniform", N), ("spill", 0),
                                    ("mid_uniform", 10_000), ("mid_uniform", 100_000),
                                    ("mid_zipf", 30_000)])
def test_sweep_column_full_size(kind, k):
    # the same columns (and seeds) as the benchmark's sweep and mid-K leg
    seed = {("uniform", 200): 3, ("zipf", 4096): 13, ("uniform", 4): 0, ("uniform", 130_000): 5,
            ("uniform", N): 8, ("spill", 0): 18, ("mid_uniform", 10_000): 1000 + 10_000,
            ("mid_uniform", 100_000): 1000 + 100_000, ("mid_zipf", 30_000): 2000 + 30_000}[(kind, k)]
    if kind.startswith("mid_"):
        kind = kind[4:]
    if kind == "spill":
        xt = G.spill_trigger_torch(N, np.int64, seed=seed, device="cuda")
    else:
        xt = G.column_torch(N, min(k, N), kind, np.int64, seed=seed, device="cuda")
    out, rep = cafs.sort_ex(xt)
    torch.cuda.synchronize()
    x = xt.cpu().numpy()
    got = out.cpu().numpy()
    assert rep["device_status"] == 0
    assert np.array_equal(got, O.frequency_sort(x))
    assert rep["path"] == O.final_path(x)
    est = O.chao1(x)
    for f in ("u", "f1", "f2", "k_hat", "M", "C", "L"):
        assert rep["est"][f] == getattr(est, f), f


def test_batched_workload_full_size():
    specs = G.batch_specs(4096, seed=3)
    keys = [G.batch_column_torch(n, k, i, 3, device="cuda") for i, (n, k) in enumerate(specs)]
    outs = [torch.empty_like(t) for t in keys]
    plan = cafs.BatchPlan(keys, outs)
    try:
        plan.launch()
        reps = plan.reports()
    finally:
        plan.close()
    torch.cuda.synchronize()
    lo = torch.iinfo(torch.int64).min
    for t, o, r in zip(keys, outs, reps):
        assert r["device_status"] == 0
        assert o.numel() == t.numel()
        if o.numel() > 1:
            assert bool((o[1:] >= o[:-1]).all())
        assert int(o.sum()) == int(t.sum())                      # wrapping int64 sums
        assert int((o == lo).sum()) == int((t == lo).sum())
    rng = np.random.default_rng(7)
    for i in sorted(rng.choice(len(keys), size=48, replace=False)):
        x = keys[i].cpu().numpy()
        assert np.array_equal(outs[i].cpu().numpy(), O.frequency_sort(x)), i
        assert reps[i]["path"] == O.final_path(x), i
