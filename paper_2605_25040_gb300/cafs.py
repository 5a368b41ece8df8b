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

INT32, INT64, UINT32, UINT64, FLOAT32, FLOAT64 = 0, 1, 2, 3, 4, 5
KEY_TYPES = {"int32": (INT32, 4), "int64": (INT64, 8), "uint32": (UINT32, 4), "uint64": (UINT64, 8),
             "float32": (FLOAT32, 4), "float64": (FLOAT64, 8)}

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


class Column(ctypes.Structure):
    _fields_ = [("keys", ctypes.c_void_p), ("out", ctypes.c_void_p), ("n", ctypes.c_size_t),
                ("dtype", ctypes.c_int), ("reserved", ctypes.c_int32)]


class BatchTuning(ctypes.Structure):
    _fields_ = [("grid_min_n", ctypes.c_uint64), ("defer_min_n", ctypes.c_uint64),
                ("cta_table_slots", ctypes.c_uint64), ("local_slots_max", ctypes.c_uint32), ("replicas_max", ctypes.c_uint32),
                ("emit_tile_vec", ctypes.c_uint32), ("ctas", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32), ("reserved2", ctypes.c_uint32)]

    KNOBS = ("grid_min_n", "defer_min_n", "cta_table_slots", "local_slots_max", "replicas_max",
             "emit_tile_vec", "ctas")

    def as_dict(self) -> dict:
        return {f: int(getattr(self, f)) for f in self.KNOBS}

    @classmethod
    def from_dict(cls, d: dict | None) -> "BatchTuning":
        t = cls()
        for k, v in (d or {}).items():
            if k not in cls.KNOBS:
                raise KeyError(f"unknown batch tuning knob {k!r}")
            setattr(t, k, int(v))
        return t


class ServerConfig(ctypes.Structure):
    _fields_ = [("max_batch_columns", ctypes.c_uint32), ("max_inflight", ctypes.c_uint32),
                ("max_request_keys", ctypes.c_uint64), ("tuning", BatchTuning),
                ("reserved", ctypes.c_uint32), ("reserved2", ctypes.c_uint32)]


class ServerStats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_uint64) for f in ("launches", "completed", "keys_done", "pending", "arena_bytes",
                                                "arena_peak_bytes", "workspace_bytes")]

    def as_dict(self) -> dict:
        return {f: int(getattr(self, f)) for f, _ in self._fields_}


class Request(ctypes.Structure):
    _fields_ = [("host_keys", ctypes.c_void_p), ("host_out", ctypes.c_void_p), ("n", ctypes.c_size_t),
                ("dtype", ctypes.c_int), ("reserved", ctypes.c_int32)]


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
    "cafs_argsort": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.POINTER(Report), ctypes.c_void_p]),
    "cafs_set_hash_seed": (None, [ctypes.c_uint64]),
    "cafs_sort_host": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int,
                                      ctypes.c_void_p, ctypes.POINTER(Report), ctypes.c_void_p]),
    "cafs_sort_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_void_p,
                                         ctypes.c_void_p]),
    "cafs_batch_tuning_default": (ctypes.c_int, [ctypes.POINTER(BatchTuning)]),
    "cafs_sort_batch": (ctypes.c_int, [ctypes.POINTER(Column), ctypes.c_size_t, ctypes.POINTER(Report),
                                       ctypes.c_void_p]),
    "cafs_sort_batch_tuned": (ctypes.c_int, [ctypes.POINTER(Column), ctypes.c_size_t,
                                             ctypes.POINTER(BatchTuning), ctypes.POINTER(Report),
                                             ctypes.c_void_p]),
    "cafs_batch_plan_create": (ctypes.c_int, [ctypes.POINTER(Column), ctypes.c_size_t,
                                              ctypes.POINTER(BatchTuning), ctypes.POINTER(ctypes.c_void_p)]),
    "cafs_batch_plan_launch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "cafs_batch_plan_reports": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Report), ctypes.c_void_p]),
    "cafs_batch_plan_columns": (ctypes.c_size_t, [ctypes.c_void_p]),
    "cafs_batch_plan_destroy": (None, [ctypes.c_void_p]),
    "cafs_batch_autotune": (ctypes.c_int, [ctypes.POINTER(Column), ctypes.c_size_t, ctypes.POINTER(BatchTuning),
                                           ctypes.c_size_t, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                           ctypes.POINTER(ctypes.c_size_t), ctypes.c_void_p]),
    "cafs_server_config_default": (ctypes.c_int, [ctypes.POINTER(ServerConfig)]),
    "cafs_server_create": (ctypes.c_int, [ctypes.c_size_t, ctypes.POINTER(ServerConfig),
                                          ctypes.POINTER(ctypes.c_void_p)]),
    "cafs_server_submit": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int,
                                          ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint64)]),
    "cafs_server_wait": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(Report),
                                        ctypes.POINTER(ctypes.c_double)]),
    "cafs_server_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ServerStats)]),
    "cafs_server_destroy": (None, [ctypes.c_void_p]),
    "cafs_server_run_trace": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Request), ctypes.c_size_t,
                                             ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                             ctypes.POINTER(Report), ctypes.POINTER(ctypes.c_double)]),
    "cafs_serial_run_trace": (ctypes.c_int, [ctypes.POINTER(Request), ctypes.c_size_t,
                                             ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                             ctypes.POINTER(Report), ctypes.POINTER(ctypes.c_double),
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
    names = {torch.int64: "int64", torch.int32: "int32", torch.float32: "float32", torch.float64: "float64"}
    for attr in ("uint32", "uint64"):
        if hasattr(torch, attr):
            names[getattr(torch, attr)] = attr
    if isinstance(dtype, torch.dtype):
        if dtype in names:
            return KEY_TYPES[names[dtype]][0]
    else:
        name = np.dtype(dtype).name
        if name in KEY_TYPES:
            return KEY_TYPES[name][0]
    raise TypeError(f"unsupported key dtype {dtype}")


def _key_code(t, key_type) -> int:
    """The key type of tensor t, or ``key_type`` (a name of KEY_TYPES) read
    from t's bits when given (e.g. uint64 keys held in an int64 tensor)."""
    if key_type is None:
        return _dtype_code(t.dtype)
    code, width = KEY_TYPES[str(key_type)]
    if t.element_size() != width:
        raise ValueError(f"key_type {key_type} needs {width}-byte elements")
    return code


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


def sort(keys, out=None, stream=None, key_type=None):
    """Sorts a 1-D CUDA tensor of keys ascending (int32/int64/uint32/uint64/
    float32/float64; ``key_type`` names the type when the tensor's dtype only
    holds the bits); returns ``out``."""
    import torch
    lib = load()
    keys = _device_tensor(keys)
    if out is None:
        out = torch.empty_like(keys)
    if out.dtype != keys.dtype or out.numel() != keys.numel() or not out.is_contiguous():
        raise ValueError("out must match keys in dtype and size")
    with torch.cuda.device(keys.device):
        _check(lib.cafs_sort(keys.data_ptr(), keys.numel(), _key_code(keys, key_type), out.data_ptr(),
                             _stream_handle(stream)), "cafs_sort")
    return out


def sort_ex(keys, out=None, stream=None, key_type=None):
    """Like ``sort`` but waits and returns (out, report dict)."""
    import torch
    lib = load()
    keys = _device_tensor(keys)
    if out is None:
        out = torch.empty_like(keys)
    rep = Report()
    with torch.cuda.device(keys.device):
        _check(lib.cafs_sort_ex(keys.data_ptr(), keys.numel(), _key_code(keys, key_type),
                                out.data_ptr(), ctypes.byref(rep), _stream_handle(stream)),
               "cafs_sort_ex")
    return out, rep.as_dict()


def argsort(keys, out=None, perm=None, stream=None, report: bool = False, key_type=None):
    """Stable argsort of a 1-D int32/int64 CUDA tensor: returns (sorted keys,
    perm) with keys[perm] == sorted keys and equal keys in input order
    (perm is int32 holding the uint32 positions); with ``report`` also the
    report dict (then the call waits for the stream)."""
    import torch
    lib = load()
    keys = _device_tensor(keys)
    if out is None:
        out = torch.empty_like(keys)
    if perm is None:
        perm = torch.empty(keys.numel(), dtype=torch.int32, device=keys.device)
    if out.dtype != keys.dtype or out.numel() != keys.numel() or not out.is_contiguous():
        raise ValueError("out must match keys in dtype and size")
    if perm.dtype != torch.int32 or perm.numel() != keys.numel() or not perm.is_contiguous():
        raise ValueError("perm must be a contiguous int32 tensor of keys' size")
    rep = Report() if report else None
    with torch.cuda.device(keys.device):
        _check(lib.cafs_argsort(keys.data_ptr(), keys.numel(), _key_code(keys, key_type), out.data_ptr(),
                                perm.data_ptr(), ctypes.byref(rep) if report else None,
                                _stream_handle(stream)), "cafs_argsort")
    if report:
        return out, perm, rep.as_dict()
    return out, perm


def set_hash_seed(seed: int) -> None:
    """0: golden-ratio table hashes (default); else each later call draws its
    own odd multipliers from the seed (never changes a result or a path)."""
    load().cafs_set_hash_seed(int(seed) & 0xFFFFFFFFFFFFFFFF)


def estimate_k(keys, stream=None, key_type=None) -> dict:
    """Sampler + Chao1 + dispatcher result for a CUDA tensor of keys."""
    import torch
    lib = load()
    keys = _device_tensor(keys)
    est = Estimate()
    with torch.cuda.device(keys.device):
        _check(lib.cafs_estimate_k(keys.data_ptr(), keys.numel(), _key_code(keys, key_type),
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


# ---------------------------------------------------------------------------
# Batched form.
# ---------------------------------------------------------------------------
def _columns(keys_list, outs, key_types=None):
    """Column descriptors; ``key_types`` (optional, one name of KEY_TYPES or
    None per column) reads a column's bits as that type."""
    n = len(keys_list)
    if key_types is not None and len(key_types) != n:
        raise ValueError("one key type per column")
    if outs is not None and len(outs) != n:
        raise ValueError("one output per column")
    arr = (Column * max(n, 1))()
    for i, k in enumerate(keys_list):
        k = _device_tensor(k)
        o = outs[i] if outs is not None else None
        if o is None:
            raise ValueError("missing output tensor")
        if o.dtype != k.dtype or o.numel() != k.numel() or not o.is_contiguous():
            raise ValueError("out must match keys in dtype and size")
        arr[i].keys = k.data_ptr() if k.numel() else None
        arr[i].out = o.data_ptr() if o.numel() else None
        arr[i].n = k.numel()
        arr[i].dtype = _key_code(k, key_types[i] if key_types is not None else None)
        arr[i].reserved = 0
    return arr


def default_tuning() -> dict:
    t = BatchTuning()
    _check(load().cafs_batch_tuning_default(ctypes.byref(t)), "cafs_batch_tuning_default")
    return t.as_dict()


def sort_batch(keys_list, outs=None, tuning: dict | None = None, reports: bool = False, stream=None,
               key_types=None):
    """Sorts many 1-D CUDA tensors with one batched launch (``key_types``: an
    optional key type name per column, as for ``sort``).

    Returns the outputs, and the per-column report dicts when ``reports``."""
    import torch
    lib = load()
    if outs is None:
        outs = [torch.empty_like(k) for k in keys_list]
    arr = _columns(keys_list, outs, key_types)
    n = len(keys_list)
    reps = (Report * max(n, 1))() if reports else None
    t = BatchTuning.from_dict(tuning) if tuning else None
    dev = keys_list[0].device if n else torch.device("cuda", torch.cuda.current_device())
    with torch.cuda.device(dev):
        _check(lib.cafs_sort_batch_tuned(arr, n, ctypes.byref(t) if t is not None else None,
                                         reps, _stream_handle(stream)), "cafs_sort_batch")
    if reports:
        return outs, [reps[i].as_dict() for i in range(n)]
    return outs


def time_tunings(keys_list, outs, tunings: list, reps: int = 3, stream=None) -> list:
    """Median batched-launch time (ms) of each knob setting on these columns."""
    import torch
    lib = load()
    arr = _columns(keys_list, outs)
    cand = (BatchTuning * len(tunings))()
    for i, t in enumerate(tunings):
        cand[i] = BatchTuning.from_dict(t)
    ms = (ctypes.c_double * len(tunings))()
    best = ctypes.c_size_t()
    dev = keys_list[0].device if keys_list else torch.device("cuda", torch.cuda.current_device())
    with torch.cuda.device(dev):
        _check(lib.cafs_batch_autotune(arr, len(keys_list), cand, len(tunings), reps, ms, ctypes.byref(best),
                                       _stream_handle(stream)), "cafs_batch_autotune")
    return [float(ms[i]) for i in range(len(tunings))]


class BatchPlan:
    """A recorded batched launch (CUDA graph) over fixed column buffers."""

    def __init__(self, keys_list, outs, tuning: dict | None = None, key_types=None):
        import torch
        self._lib = load()
        self.keys = list(keys_list)
        self.outs = list(outs)
        self.n = len(self.keys)
        arr = _columns(self.keys, self.outs, key_types)
        t = BatchTuning.from_dict(tuning) if tuning else None
        h = ctypes.c_void_p()
        self.device = self.keys[0].device if self.n else torch.device("cuda", torch.cuda.current_device())
        with torch.cuda.device(self.device):
            _check(self._lib.cafs_batch_plan_create(arr, self.n, ctypes.byref(t) if t is not None else None,
                                                    ctypes.byref(h)), "cafs_batch_plan_create")
        self._h = h

    def launch(self, stream=None) -> None:
        import torch
        with torch.cuda.device(self.device):
            _check(self._lib.cafs_batch_plan_launch(self._h, _stream_handle(stream)), "cafs_batch_plan_launch")

    def reports(self, stream=None) -> list:
        import torch
        reps = (Report * max(self.n, 1))()
        with torch.cuda.device(self.device):
            _check(self._lib.cafs_batch_plan_reports(self._h, reps, _stream_handle(stream)),
                   "cafs_batch_plan_reports")
        return [reps[i].as_dict() for i in range(self.n)]

    def close(self) -> None:
        if getattr(self, "_h", None):
            self._lib.cafs_batch_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# Served form.
# ---------------------------------------------------------------------------
def default_server_config() -> dict:
    c = ServerConfig()
    _check(load().cafs_server_config_default(ctypes.byref(c)), "cafs_server_config_default")
    return {"max_batch_columns": c.max_batch_columns, "max_inflight": c.max_inflight,
            "max_request_keys": c.max_request_keys, "tuning": c.tuning.as_dict()}


def _server_config(cfg: dict | None) -> ServerConfig:
    c = ServerConfig()
    _check(load().cafs_server_config_default(ctypes.byref(c)), "cafs_server_config_default")
    for k, v in (cfg or {}).items():
        if k == "tuning":
            for tk, tv in v.items():
                if tk not in BatchTuning.KNOBS:
                    raise KeyError(tk)
                setattr(c.tuning, tk, int(tv))
        elif k in ("max_batch_columns", "max_inflight", "max_request_keys"):
            setattr(c, k, int(v))
        else:
            raise KeyError(f"unknown server option {k!r}")
    return c


def _requests(pairs):
    """(host_in, host_out) numpy arrays -> ctypes request array."""
    arr = (Request * max(len(pairs), 1))()
    for i, (a, b) in enumerate(pairs):
        arr[i].host_keys = a.ctypes.data if a.size else None
        arr[i].host_out = b.ctypes.data if b.size else None
        arr[i].n = a.size
        arr[i].dtype = _dtype_code(a.dtype)
        arr[i].reserved = 0
    return arr


class Server:
    """Request server of the served form (native threads, fixed memory budget)."""

    def __init__(self, mem_budget_bytes: int, config: dict | None = None, device=None):
        import torch
        self._lib = load()
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        c = _server_config(config)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _check(self._lib.cafs_server_create(mem_budget_bytes, ctypes.byref(c), ctypes.byref(h)),
                   "cafs_server_create")
        self._h = h

    def submit(self, keys: np.ndarray, out: np.ndarray) -> int:
        if keys.dtype != out.dtype or keys.size != out.size:
            raise ValueError("out must match keys")
        t = ctypes.c_uint64()
        _check(self._lib.cafs_server_submit(self._h, keys.ctypes.data if keys.size else None, keys.size,
                                            _dtype_code(keys.dtype), out.ctypes.data if out.size else None,
                                            ctypes.byref(t)), "cafs_server_submit")
        return int(t.value)

    def wait(self, ticket: int):
        rep = Report()
        lat = ctypes.c_double()
        _check(self._lib.cafs_server_wait(self._h, ticket, ctypes.byref(rep), ctypes.byref(lat)),
               "cafs_server_wait")
        return rep.as_dict(), float(lat.value)

    def stats(self) -> dict:
        st = ServerStats()
        _check(self._lib.cafs_server_stats(self._h, ctypes.byref(st)), "cafs_server_stats")
        return st.as_dict()

    def run_trace(self, pairs, arrival_s: np.ndarray, reports: bool = False):
        """Open-loop replay; returns (latencies_us, elapsed_s[, reports])."""
        n = len(pairs)
        req = _requests(pairs)
        arr = np.ascontiguousarray(arrival_s, dtype=np.float64)
        lat = np.zeros(max(n, 1), dtype=np.float64)
        reps = (Report * max(n, 1))() if reports else None
        el = ctypes.c_double()
        _check(self._lib.cafs_server_run_trace(
            self._h, req, n, arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
            lat.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), reps, ctypes.byref(el)), "cafs_server_run_trace")
        if reports:
            return lat[:n], float(el.value), [reps[i].as_dict() for i in range(n)]
        return lat[:n], float(el.value)

    def close(self) -> None:
        if getattr(self, "_h", None):
            self._lib.cafs_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def serial_run_trace(pairs, arrival_s: np.ndarray, stream=None):
    """The trace served one request at a time (cafs_sort_host); (latencies_us, elapsed_s)."""
    lib = load()
    n = len(pairs)
    req = _requests(pairs)
    arr = np.ascontiguousarray(arrival_s, dtype=np.float64)
    lat = np.zeros(max(n, 1), dtype=np.float64)
    el = ctypes.c_double()
    _check(lib.cafs_serial_run_trace(req, n, arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                     lat.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), None,
                                     ctypes.byref(el), _stream_handle(stream)), "cafs_serial_run_trace")
    return lat[:n], float(el.value)
