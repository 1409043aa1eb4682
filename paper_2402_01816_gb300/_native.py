"""ctypes binding of libgns.so -- argument marshalling only.

Every function has the name of the C entry point it calls (include/gns.h) and
does nothing but check tensor types, take raw pointers and the current CUDA
stream, call the library and turn a non-zero return code into an exception.
There is no fallback: if the compiled library is missing the call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libgns.so")

GNS_OK, GNS_ERR_INVALID, GNS_ERR_UNSUPPORTED, GNS_ERR_OOM, GNS_ERR_CUDA, GNS_ERR_TIMEOUT = 0, -1, -2, -3, -4, -5
GNS_ERR_INTERNAL = -6
ASCENDING, DESCENDING = 0, 1
KEY_F64, KEY_I64 = 0, 1
FROGSORT1, GECKOSORT1, SQUIDSORT1 = 0, 1, 2
WS_SORT, WS_LEARNED = 0, 1

_lock = threading.Lock()
_lib = None


class GnsError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {strerror(code)} ({code})")


def lib() -> ctypes.CDLL:
    """Load libgns.so (built by paper_2402_01816_gb300.build)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing "
                                   "(run paper_2402_01816_gb300.build.build())")
            L = ctypes.CDLL(LIB_PATH)
            P, i64, i32, u64, f64 = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_int,
                                     ctypes.c_uint64, ctypes.c_double)
            sig = {
                "gns_sort": ([P, P, i64, i32, f64, P], i32),
                "gns_sort_i64": ([P, P, i64, i32, f64, P], i32),
                "gns_sort_symmetric": ([P, i32, P, i64, i32, f64, i32, P], i32),
                "gns_sort_host": ([P, P, i64, i32, i32, f64, P], i32),
                "gns_sort_noalloc": ([P, P, i64, i32, P], i32),
                "gns_learned_sort": ([P, P, i64, i32, f64, P, P, P], i32),
                "gns_mlp_forward": ([P, P, i64, P, P], i32),
                "gns_mlp_loss_grad": ([P, P, P, i64, P, P, P], i32),
                "gns_mlp_train": ([P, P, i64, P, P, P, i32, i32, ctypes.c_float, P], i32),
                "gns_mlp_init_params": ([P], None),
                "gns_segmented_sort": ([P, P, P, i64, P], i32),
                "gns_segmented_sort_ex": ([P, i32, P, P, i64, i64, i32, P], i32),
                "gns_workspace_bytes": ([i64, f64, i32], ctypes.c_size_t),
                "gns_segmented_schedule": ([i64, i64, P], i32),
                "gns_segmented_release": ([P], None),
                "gns_set_allocator": ([P, P, P], None),
                "gns_stream_status": ([P], i32),
                "gns_release_workspace_cache": ([], i32),
                "gns_strerror": ([i32], ctypes.c_char_p),
                "gns_version": ([], ctypes.c_char_p),
                "gns_launch_count": ([], u64),
                "gns_profile_enable": ([i32], None),
                "gns_profile_read": ([P, P, i32], i32),
                "gns_kernel_name": ([i32], ctypes.c_char_p),
                "gns_set_wait_limit_ns": ([u64], None),
                "gns_debug_skip_publish": ([i64], None),
                "gns_learned_half_plan_ok": ([i64], i32),
                "gns_debug_learned_fault": ([i32], None),
                "gns_debug_jitter": ([ctypes.c_uint32], None),
                "gns_debug_merge_partition": ([P, i64, i64, P, P], i32),
                "gns_debug_ordered_segments": ([P, i32, P, i64, P, i64, i32, P], i32),
            }
            for name, (args, res) in sig.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = res
            _lib = L
    return _lib


def strerror(code: int) -> str:
    try:
        return lib().gns_strerror(code).decode()
    except RuntimeError:
        return f"error {code}"


def _check(rc: int, where: str) -> None:
    if rc != GNS_OK:
        raise GnsError(rc, where)


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _dev_ptr(t, dtype, name):
    import torch
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def gns_sort(keys, payload=None, order: int = ASCENDING, buffer_fraction: float = 1.0, stream=None) -> None:
    """In-place stable sort of a CUDA float64 or int64 tensor (+ uint32 payload
    passed as an int32 tensor, reinterpreted bit for bit)."""
    import torch
    n = keys.numel()
    if payload is not None and payload.numel() != n:
        raise ValueError("payload must have as many elements as keys")
    if keys.dtype == torch.float64:
        fn, kd = lib().gns_sort, torch.float64
    elif keys.dtype == torch.int64:
        fn, kd = lib().gns_sort_i64, torch.int64
    else:
        raise TypeError("keys must be float64 or int64")
    _check(fn(_dev_ptr(keys, kd, "keys"), _dev_ptr(payload, torch.int32, "payload"), n, order,
              float(buffer_fraction), _stream(stream)), "gns_sort")


def gns_sort_symmetric(keys, payload=None, order: int = ASCENDING, variant: int = SQUIDSORT1,
                       buffer_fraction: float = 0.5, stream=None) -> None:
    """In-place stable sort on an in-place tier's layout (Frogsort1's tree for
    buffer_fraction in [0.5, 1), Frogsort2's below) in one of the symmetric
    variants: FROGSORT1, GECKOSORT1 or SQUIDSORT1."""
    import torch
    n = keys.numel()
    if payload is not None and payload.numel() != n:
        raise ValueError("payload must have as many elements as keys")
    if keys.dtype == torch.float64:
        kt = KEY_F64
    elif keys.dtype == torch.int64:
        kt = KEY_I64
    else:
        raise TypeError("keys must be float64 or int64")
    _check(lib().gns_sort_symmetric(_dev_ptr(keys, keys.dtype, "keys"), kt,
                                    _dev_ptr(payload, torch.int32, "payload"), n, order,
                                    float(buffer_fraction), int(variant), _stream(stream)), "gns_sort_symmetric")


def gns_sort_host(keys: np.ndarray, payload: np.ndarray | None = None, order: int = ASCENDING,
                  buffer_fraction: float = 1.0, stream=None) -> None:
    """Same sort on host arrays (copied to the device and back inside the call)."""
    if keys.dtype == np.float64:
        kt = KEY_F64
    elif keys.dtype == np.int64:
        kt = KEY_I64
    else:
        raise TypeError("keys must be float64 or int64")
    if not keys.flags.c_contiguous or (payload is not None and not payload.flags.c_contiguous):
        raise ValueError("arrays must be C-contiguous")
    if payload is not None and (payload.dtype != np.uint32 or payload.size != keys.size):
        raise TypeError("payload must be uint32 with as many elements as keys")
    pp = None if payload is None else ctypes.c_void_p(payload.ctypes.data)
    _check(lib().gns_sort_host(ctypes.c_void_p(keys.ctypes.data), pp, keys.size, kt, order,
                               float(buffer_fraction), _stream(stream)), "gns_sort_host")


NOALLOC_MAX_N = 1 << 20


def gns_sort_noalloc(keys, payload=None, order: int = ASCENDING, stream=None) -> None:
    """gns_sort_noalloc: the 100%-buffer sort of float64 keys using the library's
    fixed scratch array instead of any allocation (n <= NOALLOC_MAX_N)."""
    import torch
    n = keys.numel()
    if payload is not None and payload.numel() != n:
        raise ValueError("payload must have as many elements as keys")
    _check(lib().gns_sort_noalloc(_dev_ptr(keys, torch.float64, "keys"), _dev_ptr(payload, torch.int32, "payload"),
                                  n, order, _stream(stream)), "gns_sort_noalloc")


class LearnedParams(ctypes.Structure):
    _fields_ = [("train_steps", ctypes.c_int), ("batch", ctypes.c_int), ("learning_rate", ctypes.c_float),
                ("overfull_factor", ctypes.c_float)]


class LearnedReport(ctypes.Structure):
    _fields_ = [("fallback", ctypes.c_int), ("nonempty_buckets", ctypes.c_int), ("max_bucket", ctypes.c_int64),
                ("overfull_buckets", ctypes.c_int), ("tied_buckets", ctypes.c_int), ("final_loss", ctypes.c_float),
                ("fit_ms", ctypes.c_float),
                ("partition_ms", ctypes.c_float), ("bucket_sort_ms", ctypes.c_float),
                ("verify_failed", ctypes.c_int)]


def gns_learned_sort(keys, payload=None, order: int = ASCENDING, buffer_fraction: float = 1.0,
                     train_steps: int = 32, batch: int = 1024, learning_rate: float = 1e-2,
                     overfull_factor: float = 4.0, report: bool = False, stream=None):
    """Learned-splitter stable sort of a CUDA float64 tensor; with report=True the
    call synchronises and returns the report as a dict."""
    import torch
    n = keys.numel()
    if payload is not None and payload.numel() != n:
        raise ValueError("payload must have as many elements as keys")
    prm = LearnedParams(train_steps, batch, learning_rate, overfull_factor)
    rep = LearnedReport() if report else None
    _check(lib().gns_learned_sort(_dev_ptr(keys, torch.float64, "keys"), _dev_ptr(payload, torch.int32, "payload"),
                                  n, order, float(buffer_fraction), ctypes.byref(prm),
                                  ctypes.byref(rep) if rep is not None else None, _stream(stream)),
           "gns_learned_sort")
    if rep is None:
        return None
    return {name: getattr(rep, name) for name, _ in LearnedReport._fields_}


def gns_learned_half_plan_ok(n: int) -> bool:
    """True if gns_learned_sort at a buffer fraction in [0.5, 1) runs its
    half-buffer form for n keys (host-side plan only; needs no GPU)."""
    return bool(lib().gns_learned_half_plan_ok(int(n)))


def gns_mlp_init_params():
    out = np.zeros(1153, dtype=np.float32)
    lib().gns_mlp_init_params(ctypes.c_void_p(out.ctypes.data))
    return out


def gns_mlp_forward(params, x, stream=None):
    import torch
    y = torch.empty_like(x)
    _check(lib().gns_mlp_forward(_dev_ptr(params, torch.float32, "params"), _dev_ptr(x, torch.float32, "x"),
                                 x.numel(), _dev_ptr(y, torch.float32, "y"), _stream(stream)), "gns_mlp_forward")
    return y


def gns_mlp_loss_grad(params, x, t, stream=None):
    import torch
    grad = torch.empty(1153, dtype=torch.float32, device=x.device)
    loss = torch.empty(1, dtype=torch.float32, device=x.device)
    _check(lib().gns_mlp_loss_grad(_dev_ptr(params, torch.float32, "params"), _dev_ptr(x, torch.float32, "x"),
                                   _dev_ptr(t, torch.float32, "t"), x.numel(), _dev_ptr(grad, torch.float32, "grad"),
                                   _dev_ptr(loss, torch.float32, "loss"), _stream(stream)), "gns_mlp_loss_grad")
    return loss, grad


def gns_mlp_train(x, t, params, steps: int, batch: int = 1024, learning_rate: float = 1e-2, stream=None):
    import torch
    out = torch.empty(1153, dtype=torch.float32, device=x.device)
    loss = torch.zeros(1, dtype=torch.float32, device=x.device)
    _check(lib().gns_mlp_train(_dev_ptr(x, torch.float32, "x"), _dev_ptr(t, torch.float32, "t"), x.numel(),
                               _dev_ptr(params, torch.float32, "params"), _dev_ptr(out, torch.float32, "out"),
                               _dev_ptr(loss, torch.float32, "loss"), steps, batch, float(learning_rate),
                               _stream(stream)), "gns_mlp_train")
    return out, loss


def gns_segmented_sort(keys, payload, offsets, order: int = ASCENDING, stream=None) -> None:
    """Stable sort of every segment [offsets[s], offsets[s+1]) independently."""
    import torch
    if keys.dtype == torch.int64:
        kt = KEY_I64
    elif keys.dtype == torch.float64:
        kt = KEY_F64
    else:
        raise TypeError("keys must be int64 or float64")
    nseg = offsets.numel() - 1
    if nseg < 0:
        raise ValueError("offsets needs nseg + 1 entries")
    _check(lib().gns_segmented_sort_ex(_dev_ptr(keys, keys.dtype, "keys"), kt,
                                       _dev_ptr(payload, torch.int32, "payload"),
                                       _dev_ptr(offsets, torch.int64, "offsets"), nseg, keys.numel(),
                                       order, _stream(stream)), "gns_segmented_sort")


def gns_segmented_schedule(total_n: int, offsets) -> int:
    return int(lib().gns_segmented_schedule(total_n, offsets.numel() - 1, ctypes.c_void_p(offsets.data_ptr())))


def gns_segmented_release(stream=None) -> None:
    lib().gns_segmented_release(_stream(stream))


def gns_workspace_bytes(n: int, buffer_fraction: float = 1.0, kind: int = WS_SORT) -> int:
    return int(lib().gns_workspace_bytes(n, float(buffer_fraction), kind))


def gns_stream_status(stream=None) -> int:
    return int(lib().gns_stream_status(_stream(stream)))


def gns_release_workspace_cache() -> None:
    _check(lib().gns_release_workspace_cache(), "gns_release_workspace_cache")


def gns_version() -> str:
    return lib().gns_version().decode()


def gns_launch_count() -> int:
    return int(lib().gns_launch_count())


def gns_profile_enable(on: bool) -> None:
    lib().gns_profile_enable(1 if on else 0)


def gns_profile_read(cap: int = 1 << 16):
    """[(kernel name, milliseconds)] of the launches since the last read."""
    ids = np.zeros(cap, dtype=np.int32)
    ms = np.zeros(cap, dtype=np.float32)
    n = lib().gns_profile_read(ctypes.c_void_p(ids.ctypes.data), ctypes.c_void_p(ms.ctypes.data), cap)
    n = min(n, cap)
    return [(lib().gns_kernel_name(int(i)).decode(), float(t)) for i, t in zip(ids[:n], ms[:n])]


def gns_set_wait_limit_ns(ns: int) -> None:
    lib().gns_set_wait_limit_ns(int(ns))


def gns_debug_skip_publish(ticket: int) -> None:
    lib().gns_debug_skip_publish(int(ticket))


FAULT_NONE, FAULT_BUCKETS_SWAPPED, FAULT_GARBAGE_WEIGHTS, FAULT_SPLITTERS_REVERSED = 0, 1, 2, 3


def gns_debug_learned_fault(kind: int) -> None:
    """Plant one fault into the next gns_learned_sort call (test hook)."""
    lib().gns_debug_learned_fault(int(kind))


def gns_debug_jitter(max_ns: int) -> None:
    """Test hook: perturb the load order of the in-place levels' tickets."""
    lib().gns_debug_jitter(int(max_ns))


def gns_debug_ordered_segments(keys, payload, offsets, order: int = ASCENDING, stream=None) -> None:
    """Test hook: the learned sort's bucket sort on caller-given ordered
    segments (offsets: CUDA int64 tensor of nseg + 1 entries)."""
    import torch
    if keys.dtype == torch.int64:
        kt = KEY_I64
    elif keys.dtype == torch.float64:
        kt = KEY_F64
    else:
        raise TypeError("keys must be int64 or float64")
    _check(lib().gns_debug_ordered_segments(_dev_ptr(keys, keys.dtype, "keys"), kt,
                                            _dev_ptr(payload, torch.int32, "payload"), keys.numel(),
                                            _dev_ptr(offsets, torch.int64, "offsets"), offsets.numel() - 1,
                                            order, _stream(stream)), "gns_debug_ordered_segments")


def gns_debug_merge_partition(keys, w: int, stream=None):
    """Test hook: co-ranks of one merge level (keys: CUDA int64 tensor holding
    order-mapped keys as raw bits); returns a CUDA int64 tensor of splits."""
    import torch
    n = keys.numel()
    splits = torch.empty((n + 2047) // 2048, dtype=torch.int64, device=keys.device)
    _check(lib().gns_debug_merge_partition(_dev_ptr(keys, torch.int64, "keys"), n, int(w),
                                           _dev_ptr(splits, torch.int64, "splits"), _stream(stream)),
           "gns_debug_merge_partition")
    return splits
