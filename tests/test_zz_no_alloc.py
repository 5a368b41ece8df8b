"""The allocation-free entry point, cafs_sort_noalloc.

Callers that cannot allocate device memory (a graph capture that must not
add allocation nodes, engines that only hand out pre-reserved pools, locked
allocators) use cafs_sort_noalloc, whose scratch lives in one static device
array.  This test calls it through the C ABI twice in a row on different
columns and checks each result against cafs_sort's output on the same keys
(the integer sort is exact: tolerance zero), plus the size limit.  The file
is named so that pytest collects it last.
"""

import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

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


def _noalloc(lib, x: torch.Tensor) -> torch.Tensor:
    out = torch.empty_like(x)
    code = lib.cafs_sort_noalloc(x.data_ptr(), x.numel(), cafs._dtype_code(x.dtype), out.data_ptr(),
                                 torch.cuda.current_stream().cuda_stream)
    assert code == 0, cafs.STATUS.get(code, code)
    return out


@pytest.mark.parametrize("dtype", [np.int64, np.int32])
def test_noalloc_matches_cafs_sort_twice(lib, dtype):
    cols = [G.column(MAX_KEYS, 300, "zipf", dtype, seed=1),          # main path
            G.spill_trigger(300_000, dtype, seed=2),                  # guard -> radix
            G.column(5000, 3, "uniform", dtype, seed=3),              # tiny
            G.column(1500, 1500, "uniform", dtype, seed=4)]           # N < 2048
    for x in cols:
        xt = torch.from_numpy(x).cuda()
        first = _noalloc(lib, xt)
        second = _noalloc(lib, xt)
        ref = cafs.sort(xt)
        torch.cuda.synchronize()
        assert torch.equal(first, ref)
        assert torch.equal(second, ref)


def test_noalloc_rejects_too_large(lib):
    x = torch.zeros(MAX_KEYS + 1, dtype=torch.int64, device="cuda")
    out = torch.empty_like(x)
    code = lib.cafs_sort_noalloc(x.data_ptr(), x.numel(), cafs.INT64, out.data_ptr(),
                                 torch.cuda.current_stream().cuda_stream)
    assert code == 3  # CAFS_ERR_TOO_LARGE
    assert lib.cafs_sort_noalloc(None, 0, cafs.INT64, None, None) == 0
