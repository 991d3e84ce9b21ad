"""Oracle for the LOFAR Online Flagger hot path -- TEST INFRASTRUCTURE ONLY.

A plain single-threaded C restatement of the paper's method (lof_ref.c),
compiled with gcc at -O2 -ffp-contract=off, wrapped here with ctypes and numpy.
Only the tests, the smoke check and the benchmark's CPU-baseline leg may import
this package; the CUDA library never does, and the two share no code.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lof_ref.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liblof_ref.so")
_lock = threading.Lock()
_lib = None

CI8, CI16, F32, CF32 = 1, 2, 3, 4
SIGMA_MAD, SIGMA_STD, SIGMA_WINSOR = 0, 1, 2


class Params(ctypes.Structure):
    _fields_ = [
        ("p", ctypes.c_double),
        ("sensitivity", ctypes.c_double),
        ("start_threshold", ctypes.c_double),
        ("max_window", ctypes.c_int),
        ("history_len", ctypes.c_int),
        ("history_min", ctypes.c_int),
        ("history_k", ctypes.c_double),
        ("sigma_estimator", ctypes.c_int),
        ("enable_freq", ctypes.c_int),
        ("enable_time", ctypes.c_int),
        ("enable_history", ctypes.c_int),
        ("sir_percent", ctypes.c_int),
        ("time_mode", ctypes.c_int),
        ("stats_scope", ctypes.c_int),
        ("integ_chan", ctypes.c_int),
        ("integ_time", ctypes.c_int),
    ]


class Stats(ctypes.Structure):
    _fields_ = [
        ("median_f", ctypes.c_double),
        ("sigma_f", ctypes.c_double),
        ("median_t", ctypes.c_double),
        ("sigma_t", ctypes.c_double),
        ("n_chan_freq", ctypes.c_int64),
        ("n_flag_time", ctypes.c_int64),
        ("n_chan_hist", ctypes.c_int64),
        ("n_flag_total", ctypes.c_int64),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def default_params(**kw) -> Params:
    """Paper defaults (Section 2.1: p=1.5, sensitivity=1, 6 sigma at I=1)."""
    d = dict(p=1.5, sensitivity=1.0, start_threshold=6.0, max_window=64, history_len=60,
             history_min=8, history_k=6.0, sigma_estimator=SIGMA_MAD, enable_freq=1,
             enable_time=1, enable_history=1, sir_percent=0, time_mode=0, stats_scope=0,
             integ_chan=1, integ_time=1)
    d.update(kw)
    return Params(**d)


def build(force: bool = False) -> str:
    """Compile lof_ref.c into a shared library (idempotent)."""
    with _lock:
        if not force and os.path.exists(_LIB_PATH) and \
                os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(_SRC),
                                                   os.path.getmtime(os.path.join(_HERE, "lof_ref.h"))):
            return _LIB_PATH
        os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-std=gnu11", "-O2", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = ctypes.CDLL(path)
        P = ctypes.POINTER
        L.lof_ref_factor.argtypes = [P(Params), ctypes.c_int]
        L.lof_ref_factor.restype = ctypes.c_double
        L.lof_ref_threshold.argtypes = [P(Params), ctypes.c_double, ctypes.c_double, ctypes.c_int]
        L.lof_ref_threshold.restype = ctypes.c_double
        L.lof_ref_median.argtypes = [ctypes.c_void_p, ctypes.c_int64]
        L.lof_ref_median.restype = ctypes.c_double
        L.lof_ref_sigma.argtypes = [P(Params), ctypes.c_void_p, ctypes.c_int64, ctypes.c_int,
                                    P(ctypes.c_double)]
        L.lof_ref_sigma.restype = ctypes.c_double
        L.lof_ref_sum_threshold.argtypes = [P(Params), ctypes.c_void_p, ctypes.c_int64,
                                            ctypes.c_double, ctypes.c_double, ctypes.c_void_p]
        L.lof_ref_sum_threshold.restype = None
        L.lof_ref_flag_unit.argtypes = [P(Params), ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                        ctypes.c_int, ctypes.c_int64, ctypes.c_void_p,
                                        ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p, P(Stats)]
        L.lof_ref_flag_unit.restype = ctypes.c_int
        L.lof_ref_history_commit.argtypes = [P(Params), ctypes.c_int, ctypes.c_void_p,
                                             ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        L.lof_ref_history_commit.restype = None
        L.lof_ref_sir.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                                  ctypes.c_void_p, ctypes.c_int64]
        L.lof_ref_sir.restype = None
        _lib = L
    return _lib


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def factor(params: Params, k: int) -> float:
    return lib().lof_ref_factor(ctypes.byref(params), k)


def threshold(params: Params, median: float, sigma: float, k: int) -> float:
    return lib().lof_ref_threshold(ctypes.byref(params), median, sigma, k)


def median(x) -> float:
    x = np.ascontiguousarray(x, dtype=np.float64)
    return lib().lof_ref_median(_ptr(x), x.size)


def sigma(params: Params, x, is_int: bool):
    """Return (median, sigma) as the flagger computes them."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    m = ctypes.c_double(0.0)
    s = lib().lof_ref_sigma(ctypes.byref(params), _ptr(x), x.size, int(is_int), ctypes.byref(m))
    return m.value, s


def sum_threshold(params: Params, v, median: float, sigma: float, entry=None) -> np.ndarray:
    v = np.ascontiguousarray(v, dtype=np.float64)
    f = np.zeros(v.size, np.uint8) if entry is None else np.array(entry, dtype=np.uint8).copy()
    lib().lof_ref_sum_threshold(ctypes.byref(params), _ptr(v), v.size, median, sigma, _ptr(f))
    return f


def sir(mask, percent: int) -> np.ndarray:
    """Section 2.2 scale-invariant rank operator on one line of a 0/1 mask."""
    f = np.ascontiguousarray(mask, dtype=np.uint8).ravel()
    g = np.zeros(f.size, np.uint8)
    lib().lof_ref_sir(_ptr(f), f.size, 1, int(percent), _ptr(g), 1)
    return g


def dtype_code(arr: np.ndarray) -> int:
    if arr.dtype == np.int8:
        return CI8
    if arr.dtype == np.int16:
        return CI16
    if arr.dtype == np.float32:
        return F32
    if arr.dtype == np.complex64:
        return CF32
    raise TypeError(arr.dtype)


class History:
    """Per-channel rings, oldest -> newest, as the oracle keeps them."""

    def __init__(self, n_chan: int, params: Params):
        self.params = params
        self.ring = np.zeros((n_chan, params.history_len), np.float64)
        self.count = np.zeros(n_chan, np.int32)

    def commit(self, c0: int, pending: np.ndarray, has_pending: np.ndarray):
        C = pending.size
        ring = np.ascontiguousarray(self.ring[c0:c0 + C])
        cnt = np.ascontiguousarray(self.count[c0:c0 + C])
        lib().lof_ref_history_commit(ctypes.byref(self.params), C, _ptr(ring), _ptr(cnt),
                                     _ptr(np.ascontiguousarray(pending, np.float64)),
                                     _ptr(np.ascontiguousarray(has_pending, np.uint8)))
        self.ring[c0:c0 + C] = ring
        self.count[c0:c0 + C] = cnt


def flag_unit(params: Params, data: np.ndarray, history: History | None = None, c0: int = 0,
              want_out: bool = True):
    """Flag one unit.  data: int8/int16 array [C, T, 2] (complex voltages),
    float32 [C, T] (Stokes I) or complex64 [C, T] (visibilities).  Returns dict(mask, out, pending, has_pending, stats)."""
    dt = dtype_code(data)
    data = np.ascontiguousarray(data)
    C, T = data.shape[0], data.shape[1]
    mask = np.zeros((C, T), np.uint8)
    out = np.zeros_like(data) if want_out else None
    pending = np.zeros(C, np.float64)
    has_pending = np.zeros(C, np.uint8)
    st = Stats()
    ring = cnt = None
    if history is not None:
        ring = np.ascontiguousarray(history.ring[c0:c0 + C])
        cnt = np.ascontiguousarray(history.count[c0:c0 + C])
    rc = lib().lof_ref_flag_unit(ctypes.byref(params), dt, _ptr(data), C, T, T, _ptr(out), T,
                                 _ptr(mask), T, _ptr(ring), _ptr(cnt), _ptr(pending),
                                 _ptr(has_pending), ctypes.byref(st))
    if rc != 0:
        raise ValueError("lof_ref_flag_unit rejected its arguments")
    return dict(mask=mask, out=out, pending=pending, has_pending=has_pending, stats=st.as_dict())
