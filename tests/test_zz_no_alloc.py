"""The allocation-free entry point, cafs_sort_noalloc.

Callers that cannot allocate device memory (engines that hand out only
pre-reserved pools, processes held to a fixed device-memory budget, loops
that cannot afford the device synchronisation of cudaMalloc) use
cafs_sort_noalloc, whose scratch lives in one static device array.  This test
calls it through the C ABI twice in a row on each column and checks every
result against the CPU oracle and against cafs_sort's output on the same keys
(the integer sort is exact: tolerance zero), that the calls leave the free
device memory unchanged, and the size limit.  The file is named so that
pytest collects it last.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import cafs_oracle as O  # noqa: E402
from paper_2605_25040_gb300 import cafs  # noqa: E402
from paper_2605_25040_gb300 import datagen as G  # noqa: E402

pytestmark = pytest.mark.gpu

MAX_KEYS = 1 << 19


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_25040_gb300 import build
    build.build()
    return cafs.load()


def _noalloc(lib, x: torch.Tensor, out: torch.Tensor) -> None:
    code = lib.cafs_sort_noalloc(x.data_ptr(), x.numel(), cafs._dtype_code(x.dtype), out.data_ptr(),
                                 torch.cuda.current_stream().cuda_stream)
    assert code == 0, cafs.STATUS.get(code, code)


@pytest.mark.parametrize("dtype", [np.int64, np.int32])
def test_noalloc_matches_oracle_and_cafs_sort_twice(lib, dtype):
    cols = [G.column(MAX_KEYS, 300, "zipf", dtype, seed=1),          # main path
            G.column(MAX_KEYS, 20_000, "uniform", dtype, seed=5),     # large pair set
            G.spill_trigger(300_000, dtype, seed=2),                  # guard -> radix
            G.column(5000, 3, "uniform", dtype, seed=3),              # tiny
            G.column(1500, 1500, "uniform", dtype, seed=4)]           # N < 2048
    keys = [torch.from_numpy(x).cuda() for x in cols]
    refs = [cafs.sort(k) for k in keys]                  # the existing entry point
    outs = [(torch.empty_like(k), torch.empty_like(k)) for k in keys]
    _noalloc(lib, keys[0], outs[0][0])                   # first call: device set-up
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    for k, (a, b) in zip(keys, outs):
        _noalloc(lib, k, a)
        _noalloc(lib, k, b)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free_before
    for x, ref, (a, b) in zip(cols, refs, outs):
        want = O.frequency_sort(x)
        assert np.array_equal(a.cpu().numpy(), want)
        assert np.array_equal(b.cpu().numpy(), want)
        assert torch.equal(a, ref) and torch.equal(b, ref)


def test_noalloc_rejects_too_large(lib):
    x = torch.zeros(MAX_KEYS + 1, dtype=torch.int64, device="cuda")
    out = torch.empty_like(x)
    code = lib.cafs_sort_noalloc(x.data_ptr(), x.numel(), cafs.INT64, out.data_ptr(),
                                 torch.cuda.current_stream().cuda_stream)
    assert code == 3  # CAFS_ERR_TOO_LARGE
    assert lib.cafs_sort_noalloc(None, 0, cafs.INT64, None, None) == 0
