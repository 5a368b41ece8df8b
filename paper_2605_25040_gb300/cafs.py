"""Thin ctypes binding of libcafs.so (include/cafs.h); argument marshalling only.

Every step of the sort runs in the CUDA library.  There is no CPU fallback:
when the library has not been built, or no CUDA device is present, the calls
raise.  PyTorch supplies device memory and the current CUDA stream.
"""

from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libcafs.so")

INT32, INT64 = 0, 1

STATUS = {
    0: "ok", 1: "invalid argument", 2: "unsupported dtype", 3: "too large", 4: "alias",
    5: "out of memory", 6: "cuda error", 7: "timeout", 8: "internal", 9: "busy",
}
PATHS = {
    0: "empty", 1: "bypass_sorted", 2: "small_n", 3: "tiny", 4: "main",
    5: "high_entropy_radix", 6: "main_overflow_radix", 7: "tiny_miss_main",
    8: "tiny_miss_main_overflow_radix",
}


class Estimate(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_uint64), ("stride", ctypes.c_uint64), ("n_samples", ctypes.c_uint32),
        ("u", ctypes.c_uint32), ("f1", ctypes.c_uint32), ("f2", ctypes.c_uint32),
        ("k_hat", ctypes.c_uint64), ("saturated", ctypes.c_int32),
        ("sample_nondecreasing", ctypes.c_int32), ("M", ctypes.c_uint64), ("C", ctypes.c_uint64),
        ("L", ctypes.c_uint64), ("dispatch", ctypes.c_int),
    ]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class Report(ctypes.Structure):
    _fields_ = [("est", Estimate), ("path", ctypes.c_int), ("k_distinct", ctypes.c_uint64),
                ("device_status", ctypes.c_int), ("timeline_ns", ctypes.c_uint64 * 6)]

    def as_dict(self) -> dict:
        return {"est": self.est.as_dict(), "path": self.path, "k_distinct": self.k_distinct,
                "device_status": self.device_status, "timeline_ns": list(self.timeline_ns)}


class CafsError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {STATUS.get(code, code)} ({code})")
        self.code = code


_lib = None
_lock = threading.Lock()

# name -> (restype, argtypes) for every symbol the header declares
SIGNATURES = {
    "cafs_sort": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_void_p,
                                 ctypes.c_void_p]),
    "cafs_sort_ex": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_void_p,
                                    ctypes.POINTER(Report), ctypes.c_void_p]),
    "cafs_estimate_k": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int,
                                       ctypes.POINTER(Estimate), ctypes.c_void_p]),
    "cafs_sort_host": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int,
                                      ctypes.c_void_p, ctypes.POINTER(Report), ctypes.c_void_p]),
    "cafs_sort_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_void_p,
                                         ctypes.c_void_p]),
    "cafs_set_test_hooks": (None, [ctypes.c_uint32, ctypes.c_uint64]),
    "cafs_kernel_launch_count": (ctypes.c_uint64, []),
    "cafs_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "cafs_path_string": (ctypes.c_char_p, [ctypes.c_int]),
}


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Loads libcafs.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with paper_2605_25040_gb300.build.build()")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _dtype_code(dtype) -> int:
    import torch
    if dtype in (torch.int64, np.int64, np.dtype(np.int64)):
        return INT64
    if dtype in (torch.int32, np.int32, np.dtype(np.int32)):
        return INT32
    raise TypeError(f"unsupported key dtype {dtype}: int32 or int64 only")


def _check(code: int, what: str) -> None:
    if code != 0:
        raise CafsError(code, what)


def _stream_handle(stream) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def _device_tensor(t):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("keys must be a CUDA tensor")
    if t.dim() != 1 or not t.is_contiguous():
        raise ValueError("keys must be a contiguous 1-D tensor")
    return t


def sort(keys, out=None, stream=None):
    """Sorts a 1-D int32/int64 CUDA tensor ascending; returns ``out``."""
    import torch
    lib = load()
    keys = _device_tensor(keys)
    if out is None:
        out = torch.empty_like(keys)
    if out.dtype != keys.dtype or out.numel() != keys.numel() or not out.is_contiguous():
        raise ValueError("out must match keys in dtype and size")
    with torch.cuda.device(keys.device):
        _check(lib.cafs_sort(keys.data_ptr(), keys.numel(), _dtype_code(keys.dtype), out.data_ptr(),
                             _stream_handle(stream)), "cafs_sort")
    return out


def sort_ex(keys, out=None, stream=None):
    """Like ``sort`` but waits and returns (out, report dict)."""
    import torch
    lib = load()
    keys = _device_tensor(keys)
    if out is None:
        out = torch.empty_like(keys)
    rep = Report()
    with torch.cuda.device(keys.device):
        _check(lib.cafs_sort_ex(keys.data_ptr(), keys.numel(), _dtype_code(keys.dtype),
                                out.data_ptr(), ctypes.byref(rep), _stream_handle(stream)),
               "cafs_sort_ex")
    return out, rep.as_dict()


def estimate_k(keys, stream=None) -> dict:
    """Sampler + Chao1 + dispatcher result for a CUDA tensor of keys."""
    import torch
    lib = load()
    keys = _device_tensor(keys)
    est = Estimate()
    with torch.cuda.device(keys.device):
        _check(lib.cafs_estimate_k(keys.data_ptr(), keys.numel(), _dtype_code(keys.dtype),
                                   ctypes.byref(est), _stream_handle(stream)), "cafs_estimate_k")
    return est.as_dict()


def sort_host(keys: np.ndarray, out: np.ndarray | None = None, stream=None):
    """End-to-end sort of a host numpy array (copies in, sorts on the GPU, copies out)."""
    lib = load()
    keys = np.ascontiguousarray(keys)
    if out is None:
        out = np.empty_like(keys)
    rep = Report()
    _check(lib.cafs_sort_host(keys.ctypes.data, keys.size, _dtype_code(keys.dtype), out.ctypes.data,
                              ctypes.byref(rep), _stream_handle(stream)), "cafs_sort_host")
    return out, rep.as_dict()


def sort_host_ptr(src_ptr: int, n: int, dtype, dst_ptr: int, stream=None) -> dict:
    """End-to-end sort between raw host pointers (e.g. pinned torch tensors)."""
    lib = load()
    rep = Report()
    _check(lib.cafs_sort_host(src_ptr, n, _dtype_code(dtype), dst_ptr, ctypes.byref(rep),
                              _stream_handle(stream)), "cafs_sort_host")
    return rep.as_dict()


def set_test_hooks(flags: int, wait_timeout_ns: int = 0) -> None:
    load().cafs_set_test_hooks(flags, wait_timeout_ns)


def kernel_launch_count() -> int:
    return int(load().cafs_kernel_launch_count())


def path_name(code: int) -> str:
    return PATHS.get(code, str(code))
