"""CPU checks of the C ABI: the library builds, loads and exports every entry
point include/lof.h declares; host-side validation works without a GPU."""
import ctypes
import os
import re

from paper_1701_08197_gb300 import lof

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "lof.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lof_[a-z_]+)\s*\(", src)))


def test_header_declares_the_binding_names():
    assert declared_functions() == sorted(lof.EXPORTED)


def test_library_exports_every_declared_symbol():
    L = lof.library()
    for name in declared_functions():
        assert hasattr(L, name), name


def test_struct_sizes_match_header_layout():
    # lof_params: 3 doubles, 3 ints (+pad), double, 4 ints
    # ... + sir_percent, time_mode, stats_scope, integ_chan, integ_time (int32, padded to 8)
    assert ctypes.sizeof(lof.lof_params) == 3 * 8 + 4 * 4 + 8 + 4 * 4 + 5 * 4 + 4
    assert lof.lof_params.sir_percent.offset == 64
    assert lof.lof_params.time_mode.offset == 68
    assert lof.lof_params.stats_scope.offset == 72
    assert lof.lof_params.integ_chan.offset == 76
    assert lof.lof_params.integ_time.offset == 80
    assert ctypes.sizeof(lof.lof_unit) == 3 * 8 + 2 * 4 + 4 * 8 + 8
    assert ctypes.sizeof(lof.lof_unit_stats) == 8 * 8


def test_default_params_follow_the_paper():
    p = lof.lof_default_params()
    assert (p.p, p.sensitivity, p.start_threshold, p.max_window) == (1.5, 1.0, 6.0, 64)
    assert (p.history_len, p.history_min, p.history_k) == (60, 8, 6.0)
    assert (p.enable_freq, p.enable_time, p.enable_history) == (1, 1, 1)


def test_null_context_is_rejected_without_a_gpu():
    L = lof.library()
    assert L.lof_flag_block(None, lof.LOF_CI16, None, 0, 0, None) == lof.LOF_ERR_INVALID
    assert L.lof_history_update(None, None, 0, None) == lof.LOF_ERR_INVALID
    assert L.lof_status(None, None) == lof.LOF_ERR_INVALID
    assert L.lof_destroy(None) == lof.LOF_OK


def test_bad_parameters_are_rejected_before_touching_a_device():
    L = lof.library()
    ctx = ctypes.c_void_p()
    p = lof.lof_default_params(max_window=48)
    assert L.lof_create(ctypes.byref(p), 0, 0, ctypes.byref(ctx)) == lof.LOF_ERR_INVALID
    assert "max_window" in lof.lof_last_error()
    p = lof.lof_default_params(sensitivity=0.0)
    assert L.lof_create(ctypes.byref(p), 0, 0, ctypes.byref(ctx)) == lof.LOF_ERR_INVALID


def test_noalloc_rejects_bad_parameters_before_launch():
    """The allocation-free entry point checks its parameters as lof_create
    does, before it reads a unit or touches a device."""
    x = (ctypes.c_int16 * 128)()
    u = lof.lof_unit()
    u.in_ = ctypes.addressof(x)
    u.n_chan, u.n_time, u.in_row_stride, u.history_slot = 1, 64, 64, -1
    for bad, word in ((dict(max_window=128), "max_window"),
                      (dict(time_mode=lof.LOF_TIME_2D, integ_chan=0), "integ_chan"),
                      (dict(sensitivity=0.0), "sensitivity"),
                      (dict(sigma_estimator=7), "sigma_estimator"),
                      (dict(time_mode=9), "time_mode")):
        p = lof.lof_default_params(**bad)
        rc = lof.lof_flag_block_noalloc(p, lof.LOF_CI16, [u], 0, 0)
        assert rc == lof.LOF_ERR_INVALID, bad
        assert word in lof.lof_last_error(), (bad, lof.lof_last_error())
