"""GPU parity of the two-dimensional mode (time_mode = 2: SumThreshold on
cells of summed powers, along time then along frequency for each window
size), bit for bit against the oracle on integer units: masks, data,
statistics and history rings."""
import numpy as np
import pytest
import torch

import oracle
from paper_1701_08197_gb300 import lof, synth

from helpers import compare_unit, gpu_units, oracle_params

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
G2 = lof.LOF_TIME_2D


def _run(fl, dtype, datas, P, slots=None, hist=None, seq=0, inplace=False):
    ins, outs, masks, stats, units = gpu_units(datas, DEV, slots=slots, inplace=inplace)
    fl.flag_block(dtype, units, seq)
    fl.status()
    res = []
    for i, d in enumerate(datas):
        r = oracle.flag_unit(P, d, history=hist, c0=(slots[i] if slots else 0))
        compare_unit(d, r, outs[i], masks[i], stats[i], tag=f"unit {i} C={d.shape[0]} T={d.shape[1]}")
        res.append(r)
    return res, units


def _noise(rng, C, T, sigma=32, np_dtype=np.int16):
    lim = 127 if np_dtype == np.int8 else 32767
    d = np.clip(np.round(rng.normal(0, sigma, (C, T, 2))), -lim, lim).astype(np_dtype)
    if C > 2 and T > 40:
        d[rng.integers(0, C), :, 0] = np.clip(d[rng.integers(0, C), :, 0] + 3 * sigma, -lim, lim)
        t0 = int(rng.integers(0, T - 30))
        d[:, t0:t0 + 2, 1] = np.clip(d[:, t0:t0 + 2, 1] + 4 * sigma, -lim, lim)
        c0 = int(rng.integers(0, C - 2))
        d[c0:c0 + 2, t0 // 2:t0 // 2 + 20, 0] = min(lim, 6 * sigma)
    return d


@pytest.mark.parametrize("cells", [(1, 1), (4, 16), (2, 8), (8, 1), (1, 32)])
def test_2d_units_match_oracle(cells):
    Fi, Ti = cells
    rng = np.random.default_rng(Fi * 100 + Ti)
    a = synth.voltage_block(synth.VoltageSpec(C=64, T=768, sigma=32.0, n_tones=2, n_impulses=3),
                            seed=4, block=0)[0, 0, 0].numpy()
    b = _noise(rng, 16 * Fi, 64 * Ti)
    c = np.round(rng.normal(0, 32, (Fi, Ti, 2))).astype(np.int16)     # one cell
    z = np.zeros((8 * Fi, 4 * Ti, 2), np.int16)                           # sigma 0: nothing flagged
    e = _noise(rng, 32 * Fi, 96 * Ti if Ti > 1 else 512, 8, np.int8)
    P = oracle_params(time_mode=G2, integ_chan=Fi, integ_time=Ti)
    with lof.Flagger(0, n_history_slots=0, time_mode=G2, integ_chan=Fi, integ_time=Ti) as fl:
        _run(fl, lof.LOF_CI16, [x for x in (a, b, c, z) if x.shape[0] % Fi == 0 and x.shape[1] % Ti == 0
                                and (x.shape[0] // Fi) * (x.shape[1] // Ti) <= 16384], P)
        _run(fl, lof.LOF_CI8, [e], P)


@pytest.mark.parametrize("kw", [dict(enable_time=0), dict(enable_freq=0), dict(sigma_estimator=1),
                                dict(sigma_estimator=2), dict(sir_percent=20), dict(max_window=8, p=1.2)])
def test_2d_variants(kw):
    rng = np.random.default_rng(6)
    datas = [_noise(rng, 64, 1024), _noise(rng, 32, 2048)]
    P = oracle_params(time_mode=G2, integ_chan=2, integ_time=4, **kw)
    with lof.Flagger(0, n_history_slots=0, time_mode=G2, integ_chan=2, integ_time=4, **kw) as fl:
        _run(fl, lof.LOF_CI16, datas, P)


def test_2d_largest_grid_in_place():
    # 16320 one-sample cells (the limit is 16384) and a station-size unit in 4 x 16 cells
    rng = np.random.default_rng(9)
    a = _noise(rng, 24, 680)
    b = _noise(rng, 256, 3072)
    with lof.Flagger(0, n_history_slots=0, time_mode=G2) as fl:
        _run(fl, lof.LOF_CI16, [a], oracle_params(time_mode=G2), inplace=True)
    with lof.Flagger(0, n_history_slots=0, time_mode=G2, integ_chan=4, integ_time=16) as fl:
        _run(fl, lof.LOF_CI16, [b], oracle_params(time_mode=G2, integ_chan=4, integ_time=16), inplace=True)


def test_2d_block_sequence_with_history():
    P = oracle_params(time_mode=G2, integ_time=8)
    spec = synth.VoltageSpec(C=64, T=768, sigma=32.0, n_tones=2, n_impulses=2)
    H = oracle.History(64, P)
    with lof.Flagger(0, n_history_slots=64, time_mode=G2, integ_time=8) as fl:
        for blk in range(12):
            spec.contaminated = (blk == 10)
            d = synth.voltage_block(spec, seed=6, block=blk)[0, 0, 0].numpy()
            res, units = _run(fl, lof.LOF_CI16, [d], P, slots=[0], hist=H, seq=blk)
            fl.history_update(units)
            H.commit(0, res[0]["pending"], res[0]["has_pending"])
            vals, cnt = fl.history_export(0, 64)
            assert np.array_equal(cnt, H.count) and np.array_equal(vals, H.ring), f"block {blk}"


def test_2d_limits():
    with pytest.raises(lof.LofError):
        lof.Flagger(0, time_mode=G2, integ_chan=0)
    with pytest.raises(lof.LofError):
        lof.Flagger(0, time_mode=G2, integ_chan=512, integ_time=256)     # 131072 samples per cell
    with pytest.raises(lof.LofError):
        lof.Flagger(0, time_mode=G2, stats_scope=lof.LOF_SCOPE_CHANNEL)
    with lof.Flagger(0, time_mode=G2, integ_chan=2, integ_time=4) as fl:
        x = torch.zeros((4, 100), dtype=torch.float32, device=DEV)
        with pytest.raises(lof.LofError):
            fl.flag_block(lof.LOF_F32, [lof.make_unit(x, torch.empty_like(x))])
        y = torch.zeros((6, 102, 2), dtype=torch.int16, device=DEV)       # 102 % 4 != 0
        with pytest.raises(lof.LofError):
            fl.flag_block(lof.LOF_CI16, [lof.make_unit(y, torch.empty_like(y))])
        w = torch.zeros((8, 16384, 2), dtype=torch.int16, device=DEV)     # 4 x 4096 cells fit
        fl.flag_block(lof.LOF_CI16, [lof.make_unit(w, torch.empty_like(w))])
        fl.status()
        v = torch.zeros((16, 16384, 2), dtype=torch.int16, device=DEV)    # 8 x 4096 cells do not
        with pytest.raises(lof.LofError):
            fl.flag_block(lof.LOF_CI16, [lof.make_unit(v, torch.empty_like(v))])
