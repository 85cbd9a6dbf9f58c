"""CPU oracle for Adaptive Hybrid Sort — TEST INFRASTRUCTURE ONLY.

Thin ctypes wrapper over ``oracle/ahs_oracle.c``.  Only tests/,
``__graft_entry__.smoke()`` and bench.py's CPU-baseline / reference legs may
import this package; the product library never does.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ahs_oracle.c")
_LIB = os.path.join(_HERE, "libahs_oracle.so")

U32, U64, I32, I64 = 0, 1, 2, 3
AUTO, IDENTITY, SMALL, COUNTING, RADIX, GENERAL, REVERSE = range(7)
STRATEGY_NAMES = ("AUTO", "IDENTITY", "SMALL", "COUNTING", "RADIX", "GENERAL", "REVERSE")

_DTYPE_TO_TYPE = {np.dtype(np.uint32): U32, np.dtype(np.uint64): U64,
                  np.dtype(np.int32): I32, np.dtype(np.int64): I64}


class Features(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint64), ("min_bits", ctypes.c_uint64),
                ("max_bits", ctypes.c_uint64), ("span", ctypes.c_uint64),
                ("shift", ctypes.c_uint32), ("nbins", ctypes.c_uint32),
                ("entropy", ctypes.c_double), ("entropy_norm", ctypes.c_double),
                ("descents", ctypes.c_uint64), ("ascents", ctypes.c_uint64)]


class Fsm(ctypes.Structure):
    _fields_ = [("n_t", ctypes.c_uint64), ("k_t", ctypes.c_uint64),
                ("k_max", ctypes.c_uint64), ("h_max", ctypes.c_double),
                ("use_entropy", ctypes.c_int32), ("sorted_identity", ctypes.c_int32)]


@dataclass(frozen=True)
class Profile:
    n_t: int
    k_t: int
    k_max: int
    h_max: float = 0.7
    use_entropy: bool = True
    sorted_identity: bool = False

    def c(self) -> Fsm:
        return Fsm(self.n_t, self.k_t, self.k_max, self.h_max,
                   int(self.use_entropy), int(self.sorted_identity))


# Section III-A text and Listing 6: n_t = 20, k_t = 1000, k_max = 10^6, H < 0.7 log2 k.
PAPER = Profile(20, 1000, 10**6)
# Listing 6 itself: the same thresholds without the entropy test.
LISTING6 = Profile(20, 1000, 10**6, use_entropy=False)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, -O2, no vector intrinsics)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "ahs_oracle.h"))):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=gnu99", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_STD_SRC = os.path.join(_HERE, "stdsort.cpp")
_STD_LIB = os.path.join(_HERE, "libahs_stdsort.so")


def build_std(force: bool = False) -> str:
    """Compile the std::sort context routine (g++, -O2)."""
    if force or not os.path.exists(_STD_LIB) or os.path.getmtime(_STD_LIB) < os.path.getmtime(_STD_SRC):
        tmp = _STD_LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-o", tmp, _STD_SRC])
        os.replace(tmp, _STD_LIB)
    return _STD_LIB


_std = None


def std_sort(keys: np.ndarray, stable: bool = False) -> np.ndarray:
    """libstdc++ std::sort (or std::stable_sort) of uint32 keys: context for the
    CPU baseline, not part of the oracle."""
    global _std
    if _std is None:
        _std = ctypes.CDLL(build_std())
        _std.orc_std_sort_u32.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64,
                                          ctypes.c_int]
    keys = np.ascontiguousarray(keys, dtype=np.uint32)
    out = np.empty_like(keys)
    _check(_std.orc_std_sort_u32(_ptr(keys), _ptr(out), len(keys), int(stable)), "std_sort")
    return out


_lib = None


def open_library(path: str):
    """Load an oracle build at `path` and declare its signatures."""
    L = ctypes.CDLL(path)
    vp, u64, i32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int
    L.orc_features.argtypes = [vp, u64, i32, ctypes.POINTER(Features)]
    L.orc_entropy_exact.argtypes = [vp, u64, i32, ctypes.POINTER(ctypes.c_double)]
    L.orc_select.argtypes = [ctypes.POINTER(Features), ctypes.POINTER(Fsm)]
    L.orc_distinct.argtypes = [vp, u64, i32, ctypes.POINTER(ctypes.c_uint64)]
    L.orc_select_lemma32.argtypes = [ctypes.POINTER(Features), ctypes.POINTER(Fsm), u64]
    L.orc_radix_passes.argtypes = [u64]
    L.orc_radix_passes.restype = ctypes.c_uint32
    for name in ("orc_insertion_sort", "orc_counting_sort", "orc_radix_sort", "orc_merge_sort"):
        getattr(L, name).argtypes = [vp, vp, vp, vp, u64, i32]
    L.orc_radix_sort_signed_listing7.argtypes = [vp, vp, u64, i32]
    L.orc_quicksort.argtypes = [vp, vp, u64, i32]
    L.orc_sort.argtypes = [vp, vp, vp, vp, u64, i32, i32, ctypes.POINTER(Fsm),
                           ctypes.POINTER(ctypes.c_int), ctypes.POINTER(Features)]
    L.orc_model_load.argtypes = [ctypes.c_char_p]
    L.orc_model_load.restype = vp
    L.orc_model_free.argtypes = [vp]
    L.orc_model_predict.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
    L.orc_select_model.argtypes = [ctypes.POINTER(Features), vp, ctypes.c_uint32, i32,
                                   ctypes.POINTER(Fsm), u64]
    return L


class using_library:
    """Context manager: route this module's calls to another oracle build
    (the mutation tests load deliberately broken copies this way)."""

    def __init__(self, path: str):
        self.path = path

    def __enter__(self):
        global _lib
        self.saved = _lib
        _lib = open_library(self.path)
        return self

    def __exit__(self, *exc):
        global _lib
        _lib = self.saved
        return False


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = open_library(_LIB)
    return _lib


def _key_type(a: np.ndarray) -> int:
    try:
        return _DTYPE_TO_TYPE[a.dtype]
    except KeyError:
        raise TypeError(f"keys must be integers (uint32/uint64/int32/int64), got {a.dtype}")


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with status {rc}")


def features(keys: np.ndarray) -> Features:
    keys = np.ascontiguousarray(keys)
    f = Features()
    _check(lib().orc_features(_ptr(keys), len(keys), _key_type(keys), ctypes.byref(f)), "features")
    return f


def entropy_exact(keys: np.ndarray) -> float:
    keys = np.ascontiguousarray(keys)
    out = ctypes.c_double()
    _check(lib().orc_entropy_exact(_ptr(keys), len(keys), _key_type(keys), ctypes.byref(out)),
           "entropy_exact")
    return out.value


def distinct(keys: np.ndarray) -> int:
    keys = np.ascontiguousarray(keys)
    out = ctypes.c_uint64()
    _check(lib().orc_distinct(_ptr(keys), len(keys), _key_type(keys), ctypes.byref(out)), "distinct")
    return out.value


def select_lemma32(f: Features, profile: Profile = None, distinct: int = 0) -> int:
    p = (profile or PAPER).c()
    return lib().orc_select_lemma32(ctypes.byref(f), ctypes.byref(p), distinct)


def select(f: Features, profile: Profile) -> int:
    p = profile.c()
    return lib().orc_select(ctypes.byref(f), ctypes.byref(p))


def radix_passes(span: int) -> int:
    return lib().orc_radix_passes(span)


def _run2(name: str, keys, vals):
    keys = np.ascontiguousarray(keys)
    out = np.empty_like(keys)
    vo = None
    if vals is not None:
        vals = np.ascontiguousarray(vals, dtype=np.uint32)
        assert len(vals) == len(keys)
        vo = np.empty_like(vals)
    _check(getattr(lib(), name)(_ptr(keys), _ptr(out), _ptr(vals), _ptr(vo), len(keys),
                                _key_type(keys)), name)
    return out if vals is None else (out, vo)


def insertion_sort(keys, vals=None):
    return _run2("orc_insertion_sort", keys, vals)


def counting_sort(keys, vals=None):
    return _run2("orc_counting_sort", keys, vals)


def radix_sort(keys, vals=None):
    return _run2("orc_radix_sort", keys, vals)


def merge_sort(keys, vals=None):
    return _run2("orc_merge_sort", keys, vals)


def radix_sort_signed_listing7(keys):
    keys = np.ascontiguousarray(keys)
    out = np.empty_like(keys)
    _check(lib().orc_radix_sort_signed_listing7(_ptr(keys), _ptr(out), len(keys), _key_type(keys)),
           "radix_listing7")
    return out


def quicksort(keys):
    keys = np.ascontiguousarray(keys)
    out = np.empty_like(keys)
    _check(lib().orc_quicksort(_ptr(keys), _ptr(out), len(keys), _key_type(keys)), "quicksort")
    return out


def sort(keys, vals=None, force: int = AUTO, profile: Profile = PAPER):
    """Features -> FSM -> strategy.  Returns (keys_out, vals_out|None, chosen, features)."""
    keys = np.ascontiguousarray(keys)
    out = np.empty_like(keys)
    vo = None
    if vals is not None:
        vals = np.ascontiguousarray(vals, dtype=np.uint32)
        vo = np.empty_like(vals)
    chosen = ctypes.c_int()
    f = Features()
    p = profile.c()
    _check(lib().orc_sort(_ptr(keys), _ptr(out), _ptr(vals), _ptr(vo), len(keys), _key_type(keys),
                          force, ctypes.byref(p), ctypes.byref(chosen), ctypes.byref(f)), "sort")
    return out, vo, chosen.value, f


class Model:
    """A tree table loaded by the oracle's own evaluator."""

    def __init__(self, path: str):
        self.h = lib().orc_model_load(os.fsencode(path))
        if not self.h:
            raise RuntimeError(f"oracle could not load tree table {path}")

    def predict(self, x) -> int:
        arr = (ctypes.c_double * len(x))(*[float(v) for v in x])
        return lib().orc_model_predict(self.h, arr)

    def select(self, f: Features, key_bytes: int, payload: bool, rules: Profile,
               small_capacity: int) -> int:
        p = rules.c()
        return lib().orc_select_model(ctypes.byref(f), self.h, key_bytes, int(payload),
                                      ctypes.byref(p), small_capacity)

    def __del__(self):
        try:
            if self.h:
                lib().orc_model_free(self.h)
        except Exception:
            pass
