"""Python binding of the GB300 Adaptive Hybrid Sort library (libahs.so).

Argument marshalling only: every step of the sort runs in the library's CUDA
kernels.  The raw C entry points are available as ``lib.ahs_*`` with the
signatures of ``include/ahs.h``; ``Context`` wraps them for torch tensors
(device memory and streams come from PyTorch).

The library must be built first (``python -c "import __graft_entry__ as g;
g.build()"`` or ``python paper_2506_20677_gb300/build.py``); importing this
package without it raises ImportError — there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libahs.so")

# ---------------------------------------------------------------- constants
AHS_OK, AHS_ERR_INVALID_ARG, AHS_ERR_DTYPE, AHS_ERR_OOM, AHS_ERR_BUDGET, AHS_ERR_CUDA, \
    AHS_ERR_DEVICE_TIMEOUT, AHS_ERR_AGAIN, AHS_ERR_NOT_FOUND, AHS_ERR_UNIMPLEMENTED, \
    AHS_ERR_RANGE = range(11)
AHS_U32, AHS_U64, AHS_I32, AHS_I64 = range(4)
AHS_AUTO, AHS_IDENTITY, AHS_SMALL, AHS_COUNTING, AHS_RADIX, AHS_GENERAL, AHS_REVERSE = range(7)
AHS_SEL_PAPER, AHS_SEL_LISTING6, AHS_SEL_GB300, AHS_SEL_MODEL, AHS_SEL_CUSTOM, AHS_SEL_LEMMA32 = range(6)
AHS_DEBUG_STALL_ONE_TILE = 1
AHS_DEBUG_K2_SPLIT = 2
STRATEGY_NAMES = ("AUTO", "IDENTITY", "SMALL", "COUNTING", "RADIX", "GENERAL", "REVERSE")


class ahs_features_t(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint64), ("min_bits", ctypes.c_uint64),
                ("max_bits", ctypes.c_uint64), ("span", ctypes.c_uint64),
                ("hist_shift", ctypes.c_uint32), ("nbins", ctypes.c_uint32),
                ("entropy_bits", ctypes.c_double), ("entropy_norm", ctypes.c_double),
                ("descents", ctypes.c_uint64), ("distinct", ctypes.c_uint64),
                ("ascents", ctypes.c_uint64)]


class ahs_thresholds_t(ctypes.Structure):
    _fields_ = [("n_t", ctypes.c_uint64), ("k_t", ctypes.c_uint64), ("k_max", ctypes.c_uint64),
                ("h_max", ctypes.c_double), ("use_entropy", ctypes.c_int32),
                ("sorted_identity", ctypes.c_int32)]


class ahs_config_t(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("select_mode", ctypes.c_int),
                ("thresholds", ahs_thresholds_t), ("model_path", ctypes.c_char_p),
                ("workspace_limit", ctypes.c_uint64), ("timing", ctypes.c_int32),
                ("debug_flags", ctypes.c_uint32), ("tuning_path", ctypes.c_char_p)]


class ahs_sort_info_t(ctypes.Structure):
    _fields_ = [("strategy", ctypes.c_int), ("features_valid", ctypes.c_int32),
                ("features", ahs_features_t), ("passes", ctypes.c_uint32),
                ("buckets", ctypes.c_uint32), ("ms_features", ctypes.c_float),
                ("ms_sort", ctypes.c_float), ("workspace_bytes", ctypes.c_uint64)]


class ahs_batch_info_t(ctypes.Structure):
    _fields_ = [("n_keys", ctypes.c_uint64), ("n_seg", ctypes.c_uint32),
                ("seg_per_strategy", ctypes.c_uint32 * 6),
                ("keys_per_strategy", ctypes.c_uint64 * 6),
                ("ms_features", ctypes.c_float), ("ms_select", ctypes.c_float),
                ("ms_sort", ctypes.c_float)]


class ahs_serve_config_t(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_uint64), ("max_inflight", ctypes.c_uint32),
                ("tick_us", ctypes.c_uint32)]


class ahs_request_t(ctypes.Structure):
    _fields_ = [("d_keys_in", ctypes.c_void_p), ("d_keys_out", ctypes.c_void_p),
                ("n", ctypes.c_uint64), ("type", ctypes.c_int), ("flags", ctypes.c_uint32),
                ("d_vals_in", ctypes.c_void_p), ("d_vals_out", ctypes.c_void_p),
                ("gen_seed", ctypes.c_uint64), ("gen_id", ctypes.c_uint64),
                ("gen_kind", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


AHS_REQ_GENERATE = 1


class ahs_result_t(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("strategy", ctypes.c_int),
                ("latency_ms", ctypes.c_double), ("queue_ms", ctypes.c_double)]


class ahs_serve_stats_t(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_uint64), ("keys", ctypes.c_uint64),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("peak_reserved_bytes", ctypes.c_uint64), ("batches", ctypes.c_uint64)]


class ahs_host_array_t(ctypes.Structure):
    _fields_ = [("h_keys_in", ctypes.c_void_p), ("h_keys_out", ctypes.c_void_p),
                ("h_vals_in", ctypes.c_void_p), ("h_vals_out", ctypes.c_void_p),
                ("n", ctypes.c_uint64)]


class ahs_trace_entry_t(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_char_p), ("items", ctypes.c_uint64), ("ms", ctypes.c_float),
                ("start_ms", ctypes.c_float)]


# Every symbol include/ahs.h declares, with (restype, argtypes).
_P = ctypes.POINTER
_vp, _u64, _u32, _i32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int32
_ctx = ctypes.c_void_p
SIGNATURES = {
    "ahs_default_config": (None, [_P(ahs_config_t)]),
    "ahs_profile_thresholds": (ctypes.c_int, [ctypes.c_int, _P(ahs_thresholds_t)]),
    "ahs_create": (ctypes.c_int, [_P(_ctx), _P(ahs_config_t)]),
    "ahs_destroy": (None, [_ctx]),
    "ahs_status_str": (ctypes.c_char_p, [ctypes.c_int]),
    "ahs_last_cuda_error": (ctypes.c_char_p, [_ctx]),
    "ahs_load_model": (ctypes.c_int, [_ctx, ctypes.c_char_p]),
    "ahs_load_tuning": (ctypes.c_int, [_ctx, ctypes.c_char_p]),
    "ahs_tuned_radix_bits": (ctypes.c_int, [_ctx, _u32, _i32, _u64, _P(_u32), _P(_u32)]),
    "ahs_trace_enable": (ctypes.c_int, [_ctx, _i32]),
    "ahs_trace_collect": (ctypes.c_int, [_ctx, _P(ahs_trace_entry_t), _u32, _P(_u32)]),
    "ahs_features": (ctypes.c_int, [_ctx, _vp, _u64, ctypes.c_int, _vp, _P(ahs_features_t)]),
    "ahs_features_noalloc": (ctypes.c_int, [_vp, _u64, ctypes.c_int, _vp, _P(ahs_features_t)]),
    "ahs_entropy_exact": (ctypes.c_int, [_ctx, _vp, _u64, ctypes.c_int, _vp, _P(ctypes.c_double),
                                         _P(_u64)]),
    "ahs_select_fsm": (ctypes.c_int, [_P(ahs_features_t), _P(ahs_thresholds_t), _P(ctypes.c_int)]),
    "ahs_select": (ctypes.c_int, [_ctx, _P(ahs_features_t), ctypes.c_int, _u32, _i32,
                                  _P(ctypes.c_int)]),
    "ahs_sort": (ctypes.c_int, [_ctx, _vp, _vp, _vp, _vp, _u64, ctypes.c_int, ctypes.c_int, _vp,
                                _P(ahs_sort_info_t)]),
    "ahs_small_capacity": (_u64, [ctypes.c_int, _i32]),
    "ahs_sort_host": (ctypes.c_int, [_ctx, _P(ahs_host_array_t), _u32, ctypes.c_int, ctypes.c_int,
                                     _vp, _i32, _P(ctypes.c_int)]),
    "ahs_wait_host": (ctypes.c_int, [_ctx, _vp]),
    "ahs_sort_batch": (ctypes.c_int, [_ctx, _vp, _vp, _vp, _vp, _P(_u64), _u32, ctypes.c_int,
                                      _vp, _P(ahs_batch_info_t)]),
    "ahs_sort_batch_dev": (ctypes.c_int, [_ctx, _vp, _vp, _vp, _vp, _vp, _u32, ctypes.c_int,
                                          _vp, _P(ahs_batch_info_t)]),
    "ahs_serve_start": (ctypes.c_int, [_ctx, _P(ahs_serve_config_t)]),
    "ahs_serve_submit": (ctypes.c_int, [_ctx, _P(ahs_request_t), _P(_u64)]),
    "ahs_serve_poll": (ctypes.c_int, [_ctx, _u64, _i32, _P(ahs_result_t)]),
    "ahs_serve_stats": (ctypes.c_int, [_ctx, _P(ahs_serve_stats_t)]),
    "ahs_serve_stop": (ctypes.c_int, [_ctx]),
}


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: build the CUDA library first "
            "(python paper_2506_20677_gb300/build.py); there is no CPU fallback")
    L = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    return L


lib = _load()


class AhsError(RuntimeError):
    def __init__(self, status: int, what: str, detail: str = ""):
        self.status = status
        msg = f"{what}: {lib.ahs_status_str(status).decode()} (status {status})"
        if detail:
            msg += f": {detail}"
        super().__init__(msg)


def check(status: int, what: str, ctx=None):
    if status != AHS_OK:
        detail = lib.ahs_last_cuda_error(ctx).decode() if ctx else ""
        raise AhsError(status, what, detail)


def key_type_of(tensor) -> int:
    """C key type for a torch tensor's dtype; floating dtypes are refused (Section III-K)."""
    import torch
    m = {torch.int32: AHS_I32, torch.int64: AHS_I64}
    for name, t in (("uint32", AHS_U32), ("uint64", AHS_U64)):
        if hasattr(torch, name):
            m[getattr(torch, name)] = t
    if tensor.dtype not in m:
        raise AhsError(AHS_ERR_DTYPE, "key dtype " + str(tensor.dtype))
    return m[tensor.dtype]


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


@dataclass
class SortResult:
    keys: object
    vals: object
    strategy: int
    info: ahs_sort_info_t

    @property
    def strategy_name(self) -> str:
        return STRATEGY_NAMES[self.strategy]


# Tree table trained on GB300 timing labels (selector/labels_gb300.json);
# the default for AHS_SEL_MODEL contexts.
SHIPPED_TREES = os.path.join(os.path.dirname(os.path.abspath(__file__)), "selector", "ahs_trees.txt")
# Kernel shapes tuned on GB300 (autotune.py); every context loads it when present.
SHIPPED_TUNING = os.path.join(os.path.dirname(os.path.abspath(__file__)), "selector",
                              "tuning_gb300.txt")


class Context:
    """An ahs_ctx on one device (owns the device workspace)."""

    def __init__(self, device: int = 0, select_mode: int = AHS_SEL_GB300, model_path=None,
                 timing: bool = False, workspace_limit: int = 0, thresholds=None,
                 debug_flags: int = 0, tuning_path="shipped"):
        cfg = ahs_config_t()
        lib.ahs_default_config(ctypes.byref(cfg))
        cfg.device = device
        cfg.select_mode = select_mode
        cfg.timing = int(timing)
        cfg.workspace_limit = workspace_limit
        cfg.debug_flags = debug_flags
        if model_path is None and select_mode == AHS_SEL_MODEL:
            model_path = SHIPPED_TREES
        self._model_path = None if model_path is None else os.fsencode(model_path)
        cfg.model_path = self._model_path
        if tuning_path == "shipped":
            tuning_path = SHIPPED_TUNING if os.path.exists(SHIPPED_TUNING) else None
        self._tuning_path = None if tuning_path is None else os.fsencode(tuning_path)
        cfg.tuning_path = self._tuning_path
        if thresholds is not None:
            cfg.thresholds = thresholds
        self.handle = ctypes.c_void_p()
        check(lib.ahs_create(ctypes.byref(self.handle), ctypes.byref(cfg)), "ahs_create")
        self.device = device

    def close(self):
        if self.handle:
            lib.ahs_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False

    # ------------------------------------------------------------- tracing
    def trace(self, on: bool = True):
        check(lib.ahs_trace_enable(self.handle, int(on)), "ahs_trace_enable")

    def trace_collect(self):
        """[(kernel, items, ms, start_ms)] of the launches traced since the last
        collect; start_ms is measured from the start of the first of them."""
        cnt = ctypes.c_uint32()
        cap = 1 << 16
        buf = (ahs_trace_entry_t * cap)()
        check(lib.ahs_trace_collect(self.handle, buf, cap, ctypes.byref(cnt)), "ahs_trace_collect",
              self.handle)
        return [(buf[i].kernel.decode(), buf[i].items, buf[i].ms, buf[i].start_ms)
                for i in range(min(cnt.value, cap))]

    # ------------------------------------------------------------ features
    def features(self, keys, key_type=None, stream=None) -> ahs_features_t:
        f = ahs_features_t()
        kt = key_type_of(keys) if key_type is None else key_type
        check(lib.ahs_features(self.handle, ctypes.c_void_p(keys.data_ptr()), keys.numel(), kt,
                               _stream_handle(stream), ctypes.byref(f)), "ahs_features", self.handle)
        return f

    def load_tuning(self, path):
        """Replace the tuned-shape table (None: compiled defaults)."""
        check(lib.ahs_load_tuning(self.handle, None if path is None else os.fsencode(path)),
              "ahs_load_tuning", self.handle)

    def radix_plan(self, span: int, key_bytes: int = 4, has_payload: bool = False):
        """(passes, digit bits of the first pass) of the stable LSD radix for a key range."""
        p, b = ctypes.c_uint32(), ctypes.c_uint32()
        check(lib.ahs_tuned_radix_bits(self.handle, key_bytes, int(has_payload), span,
                                       ctypes.byref(p), ctypes.byref(b)), "ahs_tuned_radix_bits")
        return p.value, b.value

    def entropy_exact(self, keys, key_type=None, stream=None):
        """(H over every distinct value, number of distinct values), on the device."""
        h, k = ctypes.c_double(), ctypes.c_uint64()
        kt = key_type_of(keys) if key_type is None else key_type
        check(lib.ahs_entropy_exact(self.handle, ctypes.c_void_p(keys.data_ptr()), keys.numel(), kt,
                                    _stream_handle(stream), ctypes.byref(h), ctypes.byref(k)),
              "ahs_entropy_exact", self.handle)
        return h.value, k.value

    def select(self, f: ahs_features_t, mode: int, key_bytes: int = 4, has_payload: bool = False):
        out = ctypes.c_int()
        check(lib.ahs_select(self.handle, ctypes.byref(f), mode, key_bytes, int(has_payload),
                             ctypes.byref(out)), "ahs_select", self.handle)
        return out.value

    # --------------------------------------------------------------- sorts
    def sort(self, keys, vals=None, out=None, vals_out=None, force: int = AHS_AUTO,
             key_type=None, stream=None) -> SortResult:
        import torch
        kt = key_type_of(keys) if key_type is None else key_type
        if not keys.is_contiguous():
            raise AhsError(AHS_ERR_INVALID_ARG, "keys must be contiguous")
        if out is None:
            out = torch.empty_like(keys)
        if vals is not None and vals_out is None:
            vals_out = torch.empty_like(vals)
        info = ahs_sort_info_t()
        vp = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None
        check(lib.ahs_sort(self.handle, vp(keys), vp(out), vp(vals), vp(vals_out), keys.numel(),
                           kt, force, _stream_handle(stream), ctypes.byref(info)),
              "ahs_sort", self.handle)
        return SortResult(out, vals_out, info.strategy, info)

    def sort_host(self, host_keys, host_out, key_type=None, force: int = AHS_AUTO,
                  stream=None, wait: bool = True, host_vals=None, host_vals_out=None):
        """Sort a sequence of host arrays (torch CPU tensors, pinned for
        asynchronous copies) into the matching host outputs through
        ahs_sort_host: the library copies array i + 1 in and array i - 1 out
        while it sorts array i.  wait=False: returns once queued; call
        wait_host(stream) and synchronise before reading host_out.  Returns
        the strategy of each array."""
        n = len(host_keys)
        if len(host_out) != n or any(
                h.dtype != host_keys[0].dtype or o.dtype != h.dtype or o.numel() != h.numel()
                for h, o in zip(host_keys, host_out)):
            raise AhsError(AHS_ERR_INVALID_ARG, "sort_host: one dtype, matching output sizes")
        if n == 0:
            return []
        kt = key_type_of(host_keys[0]) if key_type is None else key_type
        arr = (ahs_host_array_t * n)()
        for i in range(n):
            arr[i].h_keys_in = host_keys[i].data_ptr()
            arr[i].h_keys_out = host_out[i].data_ptr()
            arr[i].n = host_keys[i].numel()
            if host_vals is not None:
                arr[i].h_vals_in = host_vals[i].data_ptr()
                arr[i].h_vals_out = host_vals_out[i].data_ptr()
        picks = (ctypes.c_int * n)()
        check(lib.ahs_sort_host(self.handle, arr, n, kt, force, _stream_handle(stream), int(wait),
                                picks), "ahs_sort_host", self.handle)
        self._host_refs = (host_keys, host_out, host_vals, host_vals_out)   # alive until waited on
        return list(picks)

    def wait_host(self, stream=None):
        """Make `stream` (default: the current stream) wait for every
        sort_host call issued so far."""
        check(lib.ahs_wait_host(self.handle, _stream_handle(stream)), "ahs_wait_host", self.handle)

    def sort_batch(self, keys, seg_offsets, out=None, vals=None, vals_out=None, key_type=None,
                   stream=None):
        import torch
        kt = key_type_of(keys) if key_type is None else key_type
        if out is None:
            out = torch.empty_like(keys)
        if vals is not None and vals_out is None:
            vals_out = torch.empty_like(vals)
        info = ahs_batch_info_t()
        vp = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None
        if isinstance(seg_offsets, torch.Tensor) and seg_offsets.is_cuda:
            # offsets resident on the device (int64 tensor of n_seg + 1)
            check(lib.ahs_sort_batch_dev(self.handle, vp(keys), vp(out), vp(vals), vp(vals_out),
                                         vp(seg_offsets), seg_offsets.numel() - 1, kt,
                                         _stream_handle(stream), ctypes.byref(info)),
                  "ahs_sort_batch_dev", self.handle)
            return out, vals_out, info
        offs = (ctypes.c_uint64 * len(seg_offsets))(*[int(x) for x in seg_offsets])
        check(lib.ahs_sort_batch(self.handle, vp(keys), vp(out), vp(vals), vp(vals_out), offs,
                                 len(seg_offsets) - 1, kt, _stream_handle(stream),
                                 ctypes.byref(info)), "ahs_sort_batch", self.handle)
        return out, vals_out, info


AHS_NOALLOC_MAX_KEYS = (1 << 32) - 1


def features_noalloc(keys, key_type=None, stream=None) -> ahs_features_t:
    """ahs_features_noalloc: the state vector with no allocation and no context,
    for callers that cannot allocate device memory (see include/ahs.h)."""
    f = ahs_features_t()
    kt = key_type_of(keys) if key_type is None else key_type
    check(lib.ahs_features_noalloc(ctypes.c_void_p(keys.data_ptr()), keys.numel(), kt,
                                   _stream_handle(stream), ctypes.byref(f)), "ahs_features_noalloc")
    return f


def profile_thresholds(mode: int) -> ahs_thresholds_t:
    t = ahs_thresholds_t()
    check(lib.ahs_profile_thresholds(mode, ctypes.byref(t)), "ahs_profile_thresholds")
    return t


def select_fsm(f: ahs_features_t, t: ahs_thresholds_t) -> int:
    out = ctypes.c_int()
    check(lib.ahs_select_fsm(ctypes.byref(f), ctypes.byref(t), ctypes.byref(out)), "ahs_select_fsm")
    return out.value
