"""ctypes binding of the CUDA flagger library (include/lof.h).

Argument marshalling only: every step of the flagger runs in liblof.so.  The
functions keep the C names; `Flagger` is a thin owner of one lof_ctx that
turns PyTorch tensors into lof_unit descriptors.  If the library cannot be
built or loaded, every call raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

LOF_OK = 0
LOF_ERR_INVALID = -1
LOF_ERR_NOMEM = -2
LOF_ERR_CUDA = -3
LOF_ERR_TIMEOUT = -4
LOF_ERR_STATE = -5
LOF_ERR_UNSUPPORTED = -6
LOF_CI8, LOF_CI16, LOF_F32, LOF_CF32 = 1, 2, 3, 4
LOF_SIGMA_MAD, LOF_SIGMA_STD, LOF_SIGMA_WINSOR = 0, 1, 2
LOF_TIME_PER_CHANNEL, LOF_TIME_INTEGRATED, LOF_TIME_2D = 0, 1, 2
LOF_SCOPE_POOLED, LOF_SCOPE_CHANNEL = 0, 1
(LOF_SCHED_PACKED, LOF_SCHED_BOUND64, LOF_SCHED_COALESCED, LOF_SCHED_VALUE_WINDOW, LOF_SCHED_F32_CLUSTER,
 LOF_SCHED_SET) = 1, 2, 4, 8, 16, 0x80

EXPORTED = [
    "lof_default_params", "lof_create", "lof_flag_block", "lof_flag_block_host",
    "lof_history_update", "lof_history_export", "lof_history_import", "lof_status",
    "lof_max_time", "lof_set_tuning", "lof_get_tuning", "lof_last_error", "lof_destroy",
    "lof_flag_block_noalloc", "lof_autotune", "lof_graph_create", "lof_graph_launch",
    "lof_graph_status", "lof_graph_destroy", "lof_block_counters",
]


class lof_params(ctypes.Structure):
    _fields_ = [
        ("p", ctypes.c_double),
        ("sensitivity", ctypes.c_double),
        ("start_threshold", ctypes.c_double),
        ("max_window", ctypes.c_int32),
        ("history_len", ctypes.c_int32),
        ("history_min", ctypes.c_int32),
        ("history_k", ctypes.c_double),
        ("sigma_estimator", ctypes.c_int32),
        ("enable_freq", ctypes.c_int32),
        ("enable_time", ctypes.c_int32),
        ("enable_history", ctypes.c_int32),
        ("sir_percent", ctypes.c_int32),
        ("time_mode", ctypes.c_int32),
        ("stats_scope", ctypes.c_int32),
        ("integ_chan", ctypes.c_int32),
        ("integ_time", ctypes.c_int32),
    ]


class lof_unit_stats(ctypes.Structure):
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


STATS_FIELDS = [k for k, _ in lof_unit_stats._fields_]
STATS_DOUBLES = 4  # first four fields are binary64, the rest int64


class lof_unit(ctypes.Structure):
    _fields_ = [
        ("in_", ctypes.c_void_p),
        ("out", ctypes.c_void_p),
        ("mask", ctypes.c_void_p),
        ("n_chan", ctypes.c_int32),
        ("n_time", ctypes.c_int32),
        ("in_row_stride", ctypes.c_int64),
        ("out_row_stride", ctypes.c_int64),
        ("mask_row_stride", ctypes.c_int64),
        ("history_slot", ctypes.c_int64),
        ("stats", ctypes.c_void_p),
    ]


class lof_tuning(ctypes.Structure):
    _fields_ = [
        ("threads", ctypes.c_int32),
        ("ctas_per_sm", ctypes.c_int32),
        ("tile_bytes", ctypes.c_int32),
        ("fine_bins", ctypes.c_int32),
        ("flag_rows", ctypes.c_int32),
        ("stat_samples", ctypes.c_int32),
        ("schedule", ctypes.c_int32),
    ]


_lib = None


class LofError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{msg} (status {code})")
        self.code = code


def library(build: bool = True):
    """Load liblof.so (building it first if needed)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build else _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA flagger library missing: {path}")
    L = ctypes.CDLL(path)
    P, V = ctypes.POINTER, ctypes.c_void_p
    L.lof_default_params.argtypes = [P(lof_params)]
    L.lof_default_params.restype = None
    L.lof_create.argtypes = [P(lof_params), ctypes.c_int, ctypes.c_int64, P(V)]
    L.lof_flag_block.argtypes = [V, ctypes.c_int, P(lof_unit), ctypes.c_int, ctypes.c_uint64, V]
    L.lof_flag_block_host.argtypes = [V, ctypes.c_int, P(lof_unit), ctypes.c_int, ctypes.c_uint64, V]
    L.lof_history_update.argtypes = [V, P(lof_unit), ctypes.c_int, V]
    L.lof_history_export.argtypes = [V, ctypes.c_int64, ctypes.c_int64, V, V]
    L.lof_history_import.argtypes = [V, ctypes.c_int64, ctypes.c_int64, V, V]
    L.lof_status.argtypes = [V, V]
    L.lof_max_time.argtypes = [V, ctypes.c_int]
    L.lof_set_tuning.argtypes = [V, P(lof_tuning)]
    L.lof_get_tuning.argtypes = [V, P(lof_tuning)]
    L.lof_last_error.argtypes = [V]
    L.lof_last_error.restype = ctypes.c_char_p
    L.lof_destroy.argtypes = [V]
    L.lof_flag_block_noalloc.argtypes = [P(lof_params), ctypes.c_int, P(lof_unit), ctypes.c_int, V, V]
    L.lof_autotune.argtypes = [V, ctypes.c_int, P(lof_unit), ctypes.c_int, ctypes.c_int, V,
                               P(lof_tuning), P(ctypes.c_float)]
    L.lof_graph_create.argtypes = [V, ctypes.c_int, P(lof_unit), ctypes.c_int, P(V)]
    L.lof_graph_launch.argtypes = [V, ctypes.c_uint64, V]
    L.lof_graph_status.argtypes = [V, V]
    L.lof_graph_destroy.argtypes = [V]
    L.lof_block_counters.argtypes = [V, V, P(ctypes.c_int64)]
    for name in ("lof_create", "lof_flag_block", "lof_flag_block_host", "lof_history_update",
                 "lof_history_export", "lof_history_import", "lof_status", "lof_max_time",
                 "lof_set_tuning", "lof_get_tuning", "lof_destroy", "lof_flag_block_noalloc",
                 "lof_autotune", "lof_graph_create", "lof_graph_launch", "lof_graph_status",
                 "lof_graph_destroy", "lof_block_counters"):
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def lof_default_params(**overrides) -> lof_params:
    p = lof_params()
    library().lof_default_params(ctypes.byref(p))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def lof_last_error(ctx=None) -> str:
    s = library().lof_last_error(ctx)
    return s.decode() if s else ""


def _check(rc, ctx=None):
    if rc != LOF_OK:
        raise LofError(rc, lof_last_error(ctx))
    return rc


def lof_create(params: lof_params | None, device: int, n_history_slots: int):
    ctx = ctypes.c_void_p()
    rc = library().lof_create(ctypes.byref(params) if params is not None else None, device,
                              n_history_slots, ctypes.byref(ctx))
    _check(rc, None)
    return ctx


def _units_array(units):
    arr = (lof_unit * max(1, len(units)))(*units)
    return arr, len(units)


def lof_flag_block(ctx, dtype: int, units, block_seq: int, stream: int) -> int:
    arr, n = _units_array(units)
    return library().lof_flag_block(ctx, dtype, arr, n, block_seq, ctypes.c_void_p(stream))


def lof_flag_block_host(ctx, dtype: int, units, block_seq: int, stream: int) -> int:
    arr, n = _units_array(units)
    return library().lof_flag_block_host(ctx, dtype, arr, n, block_seq, ctypes.c_void_p(stream))


def lof_flag_block_noalloc(params, dtype: int, units, status_ptr: int, stream: int) -> int:
    """Context-free, allocation-free flagging of one block (no history)."""
    arr, n = _units_array(units)
    return library().lof_flag_block_noalloc(ctypes.byref(params) if params is not None else None,
                                            dtype, arr, n, ctypes.c_void_p(status_ptr or None),
                                            ctypes.c_void_p(stream))


def lof_history_update(ctx, units, stream: int) -> int:
    arr, n = _units_array(units)
    return library().lof_history_update(ctx, arr, n, ctypes.c_void_p(stream))


def lof_history_export(ctx, slot0: int, n: int, values_ptr: int, counts_ptr: int) -> int:
    return library().lof_history_export(ctx, slot0, n, ctypes.c_void_p(values_ptr),
                                        ctypes.c_void_p(counts_ptr))


def lof_history_import(ctx, slot0: int, n: int, values_ptr: int, counts_ptr: int) -> int:
    return library().lof_history_import(ctx, slot0, n, ctypes.c_void_p(values_ptr),
                                        ctypes.c_void_p(counts_ptr))


def lof_status(ctx, stream: int) -> int:
    return library().lof_status(ctx, ctypes.c_void_p(stream))


def lof_max_time(ctx, dtype: int) -> int:
    return library().lof_max_time(ctx, dtype)


def lof_set_tuning(ctx, threads=0, ctas_per_sm=0, tile_bytes=0, fine_bins=0, flag_rows=0,
                   stat_samples=0, schedule=0) -> int:
    t = lof_tuning(threads, ctas_per_sm, tile_bytes, fine_bins, flag_rows, stat_samples, schedule)
    return library().lof_set_tuning(ctx, ctypes.byref(t))


def lof_get_tuning(ctx) -> dict:
    t = lof_tuning()
    _check(library().lof_get_tuning(ctx, ctypes.byref(t)), ctx)
    return {k: getattr(t, k) for k, _ in lof_tuning._fields_}


def lof_destroy(ctx) -> int:
    return library().lof_destroy(ctx)


# ---------------------------------------------------------------- torch glue

def dtype_of(t) -> int:
    import torch
    if t.dtype == torch.int8:
        return LOF_CI8
    if t.dtype == torch.int16:
        return LOF_CI16
    if t.dtype == torch.float32:
        return LOF_F32
    raise TypeError(f"unsupported sample type {t.dtype}")


def _row_stride(t) -> int:
    """Row stride in elements (complex samples for [C, T, 2] voltages)."""
    if t.dim() == 3:  # [C, T, 2] complex voltages
        if t.stride(2) != 1 or t.stride(1) != 2 or t.stride(0) % 2:
            raise ValueError("voltages must be [C, T, 2] with interleaved, contiguous rows")
        return t.stride(0) // 2
    if t.dim() == 2:
        if t.stride(1) != 1:
            raise ValueError("rows must be contiguous")
        return t.stride(0)
    raise ValueError("expected [C, T, 2] voltages or [C, T] Stokes I")


def make_unit(inp, out=None, mask=None, history_slot: int = -1, stats=None) -> lof_unit:
    """Descriptor for one unit from tensors (device or host, same layout rules)."""
    C, T = inp.shape[0], inp.shape[1]
    u = lof_unit()
    u.in_ = inp.data_ptr()
    u.n_chan, u.n_time = C, T
    u.in_row_stride = _row_stride(inp)
    if out is not None:
        u.out = out.data_ptr()
        u.out_row_stride = _row_stride(out)
    if mask is not None:
        if mask.dim() != 2 or mask.stride(1) != 1:
            raise ValueError("mask must be [C, T] uint8 with contiguous rows")
        u.mask = mask.data_ptr()
        u.mask_row_stride = mask.stride(0)
    u.history_slot = history_slot
    if stats is not None:
        u.stats = stats.data_ptr()
    return u


def stats_tensor(n_units: int, device):
    """Zeroed storage for n_units lof_unit_stats records (int64 view)."""
    import torch
    return torch.zeros((n_units, len(STATS_FIELDS)), dtype=torch.int64, device=device)


def decode_stats(row) -> dict:
    """One lof_unit_stats record (int64 tensor row or array) -> dict."""
    import numpy as np
    a = np.asarray(row.cpu() if hasattr(row, "cpu") else row, dtype=np.int64)
    d = a[:STATS_DOUBLES].view(np.float64)
    out = {k: float(d[i]) for i, k in enumerate(STATS_FIELDS[:STATS_DOUBLES])}
    for i, k in enumerate(STATS_FIELDS[STATS_DOUBLES:]):
        out[k] = int(a[STATS_DOUBLES + i])
    return out


class Flagger:
    """Owns one lof_ctx on a CUDA device.

    params are fields of lof_params (include/lof.h), defaults otherwise: p,
    sensitivity, start_threshold, max_window, history_len, history_min,
    history_k, sigma_estimator (LOF_SIGMA_MAD / _STD / _WINSOR), enable_freq,
    enable_time, enable_history, sir_percent, time_mode
    (LOF_TIME_PER_CHANNEL / _INTEGRATED / _2D), stats_scope
    (LOF_SCOPE_POOLED / _CHANNEL), integ_chan, integ_time.  Invalid
    combinations raise LofError here, at creation.
    """

    def __init__(self, device: int = 0, n_history_slots: int = 0, **params):
        self.params = lof_default_params(**params)
        self.device = device
        self.n_history_slots = n_history_slots
        self.ctx = lof_create(self.params, device, n_history_slots)

    def close(self):
        if self.ctx:
            lof_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _stream(stream):
        if stream is None:
            import torch
            return torch.cuda.current_stream().cuda_stream
        return stream if isinstance(stream, int) else stream.cuda_stream

    def flag_block(self, dtype: int, units, block_seq: int = 0, stream=None):
        _check(lof_flag_block(self.ctx, dtype, units, block_seq, self._stream(stream)), self.ctx)

    def flag_block_host(self, dtype: int, units, block_seq: int = 0, stream=None):
        _check(lof_flag_block_host(self.ctx, dtype, units, block_seq, self._stream(stream)), self.ctx)

    def history_update(self, units, stream=None):
        _check(lof_history_update(self.ctx, units, self._stream(stream)), self.ctx)

    def status(self, stream=None):
        _check(lof_status(self.ctx, self._stream(stream)), self.ctx)

    def counters(self, stream=None) -> dict:
        """Work counters of the last flag_block (lof_block_counters)."""
        c = (ctypes.c_int64 * 2)()
        _check(library().lof_block_counters(self.ctx, ctypes.c_void_p(self._stream(stream)), c), self.ctx)
        return {"units_refined": int(c[0]), "refine_passes": int(c[1])}

    def set_tuning(self, **kw):
        _check(lof_set_tuning(self.ctx, **kw), self.ctx)

    def tuning(self) -> dict:
        return lof_get_tuning(self.ctx)

    def autotune(self, dtype: int, units, reps: int = 3, stream=None):
        """Pick the fastest launch shape for these units; returns (tuning dict, ms)."""
        arr = (lof_unit * len(units))(*units)
        best = lof_tuning()
        ms = ctypes.c_float()
        _check(library().lof_autotune(self.ctx, dtype, arr, len(units), reps, self._stream(stream),
                                      ctypes.byref(best), ctypes.byref(ms)), self.ctx)
        return {k: getattr(best, k) for k, _ in lof_tuning._fields_}, ms.value

    def graph(self, dtype: int, units):
        """Capture the block of these units (fixed buffers) as a replayable graph."""
        return Graph(self, dtype, units)

    def max_time(self, dtype: int) -> int:
        return lof_max_time(self.ctx, dtype)

    def history_export(self, slot0: int, n: int):
        import numpy as np
        vals = np.zeros((n, self.params.history_len), np.float64)
        cnt = np.zeros(n, np.int32)
        _check(lof_history_export(self.ctx, slot0, n, vals.ctypes.data, cnt.ctypes.data), self.ctx)
        return vals, cnt

    def history_import(self, slot0: int, values, counts):
        import numpy as np
        vals = np.ascontiguousarray(values, np.float64)
        cnt = np.ascontiguousarray(counts, np.int32)
        _check(lof_history_import(self.ctx, slot0, cnt.size, vals.ctypes.data, cnt.ctypes.data),
               self.ctx)


class Graph:
    """A captured block (lof_graph_*): replay with launch(block_seq)."""

    def __init__(self, flagger: "Flagger", dtype: int, units):
        self.fl = flagger
        self.units = list(units)
        arr = (lof_unit * len(self.units))(*self.units)
        h = ctypes.c_void_p()
        _check(library().lof_graph_create(flagger.ctx, dtype, arr, len(self.units), ctypes.byref(h)),
               flagger.ctx)
        self.h = h

    def launch(self, block_seq: int = 0, stream=None):
        _check(library().lof_graph_launch(self.h, block_seq, Flagger._stream(stream)), self.fl.ctx)

    def status(self, stream=None):
        _check(library().lof_graph_status(self.h, Flagger._stream(stream)), self.fl.ctx)

    def close(self):
        if self.h:
            library().lof_graph_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
