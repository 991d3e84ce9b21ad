"""Value-window statistics: a unit whose history slot holds the previous
block's median and MAD counts its pooled powers value by value in a window
around them (LOF_SCHED_VALUE_WINDOW).  Whatever path a block takes -- no
hint, a window hit, a window miss (full recount), a hint too wide for a
window -- its statistics, mask and data must equal the oracle's bit for bit,
and the schedule bit must not change any result."""
import numpy as np
import pytest
import torch

import oracle
from paper_1701_08197_gb300 import lof, synth

from helpers import compare_unit, gpu_units

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
SHAPES = [(256, 768), (64, 3072), (17, 1000), (5, 33)]


def _blocks(seed, block, sigma, dtype=torch.int16):
    datas = []
    for i, (C, T) in enumerate(SHAPES):
        spec = synth.VoltageSpec(C=C, T=T, sigma=sigma, dtype=dtype, n_tones=min(3, C // 4),
                                 n_impulses=1 if T > 64 else 0)
        datas.append(synth.voltage_block(spec, seed=seed + i, block=block)[0, 0, 0].numpy())
    return datas


def _slots():
    out, off = [], 0
    for C, _ in SHAPES:
        out.append(off)
        off += C
    return out, off


def _run(fl, datas, seq, P, dtype=lof.LOF_CI16):
    slots, _ = _slots()
    ins, outs, masks, stats, units = gpu_units(datas, DEV, slots=slots)
    fl.flag_block(dtype, units, seq)
    fl.status()
    for i, d in enumerate(datas):
        r = oracle.flag_unit(P, d)
        compare_unit(d, r, outs[i], masks[i], stats[i], tag=f"block {seq} unit {i} {d.shape[:2]}")
    return fl.counters(), [m.cpu().numpy() for m in masks], stats.cpu()


def test_window_hit_miss_and_wide_hint_match_oracle():
    """sigma 32 (no hint), 32 (window), 128 (the data leave the window: every
    unit is counted again), 32 (hint too wide for a window: general path),
    32 (window again)."""
    P = oracle.default_params(enable_history=0)
    _, ns = _slots()
    with lof.Flagger(0, n_history_slots=ns, enable_history=0) as fl:
        cn = []
        for seq, sigma in enumerate((32.0, 32.0, 128.0, 32.0, 32.0)):
            c, _, _ = _run(fl, _blocks(11, seq, sigma), seq, P)
            cn.append(c)
        # the miss recounts the units that were in window mode (all but the
        # 5-sample-wide unit of 5 x 33 values, whose hint may or may not hit)
        assert cn[2]["units_refined"] >= 3 and cn[2]["refine_passes"] >= 3, cn
        assert cn[1]["units_refined"] == 0 and cn[4]["units_refined"] == 0, cn


def test_window_schedule_bit_changes_no_result():
    P = oracle.default_params(enable_history=0)
    _, ns = _slots()
    res = {}
    for win in (0, lof.LOF_SCHED_VALUE_WINDOW):
        with lof.Flagger(0, n_history_slots=ns, enable_history=0) as fl:
            t = fl.tuning()
            fl.set_tuning(schedule=(t["schedule"] & ~lof.LOF_SCHED_VALUE_WINDOW) | win)
            out = []
            for seq in range(3):
                _, m, s = _run(fl, _blocks(23, seq, 32.0), seq, P)
                out.append((m, s))
            res[win] = out
    for (ma, sa), (mb, sb) in zip(res[0], res[lof.LOF_SCHED_VALUE_WINDOW]):
        assert all(np.array_equal(a, b) for a, b in zip(ma, mb))
        assert torch.equal(sa, sb)


def test_window_ci8_and_zero_mad():
    """ci8 units in window mode, and units whose MAD is zero (most powers
    equal): the window resolves the median, then the exact moments."""
    P = oracle.default_params(enable_history=0)
    _, ns = _slots()
    rng = np.random.default_rng(3)
    with lof.Flagger(0, n_history_slots=ns, enable_history=0) as fl:
        for seq in range(3):
            _run(fl, _blocks(31, seq, 6.0, dtype=torch.int8), seq, P, dtype=lof.LOF_CI8)
        for seq in range(3, 6):
            datas = []
            for C, T in SHAPES:
                x = np.zeros((C, T, 2), np.int16)
                x[..., 0] = 3
                k = rng.random((C, T)) < 0.2
                x[k, 1] = rng.integers(-40, 40, int(k.sum()))
                datas.append(x)
            _run(fl, datas, seq, P)
