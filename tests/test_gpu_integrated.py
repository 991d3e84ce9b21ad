"""GPU parity of the integrated time mode (Section 3: the frequency direction
integrated fully for time-domain flagging), bit for bit against the oracle on
integer units: masks, data, statistics and history rings."""
import numpy as np
import pytest
import torch

import oracle
from paper_1701_08197_gb300 import lof, synth

from helpers import compare_unit, gpu_units, oracle_params

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
INTEG = lof.LOF_TIME_INTEGRATED


def _run(fl, dtype, datas, P, slots=None, hist=None, seq=0):
    ins, outs, masks, stats, units = gpu_units(datas, DEV, slots=slots)
    fl.flag_block(dtype, units, seq)
    fl.status()
    res = []
    for i, d in enumerate(datas):
        r = oracle.flag_unit(P, d, history=hist, c0=(slots[i] if slots else 0))
        compare_unit(d, r, outs[i], masks[i], stats[i], tag=f"unit {i} C={d.shape[0]} T={d.shape[1]}")
        res.append(r)
    return res, units


@pytest.mark.parametrize("kw", [dict(), dict(sigma_estimator=1), dict(enable_time=0), dict(enable_freq=0),
                                dict(sir_percent=20), dict(max_window=8)])
def test_integrated_units_match_oracle(kw):
    rng = np.random.default_rng(7)
    a = synth.voltage_block(synth.VoltageSpec(C=256, T=768, sigma=32.0, n_tones=3, n_impulses=4),
                            seed=3, block=0)[0, 0, 0].numpy()
    b = np.round(rng.normal(0, 32, (37, 3001, 2))).astype(np.int16)
    b[:, 1200:1206, 0] += 60                     # weak broadband impulse
    b[:, 2000] = 3000                            # strong single-sample one
    b[9] += np.int16(70)                         # hot channel
    c = np.round(rng.normal(0, 32, (1, 500, 2))).astype(np.int16)
    z = np.zeros((8, 64, 2), np.int16)           # sigma 0: nothing flagged
    e = np.clip(np.round(rng.normal(0, 8, (64, 2048, 2))), -127, 127).astype(np.int8)
    e[:, 100:103] = 90
    P = oracle_params(time_mode=INTEG, **kw)
    with lof.Flagger(0, n_history_slots=0, time_mode=INTEG, **kw) as fl:
        _run(fl, lof.LOF_CI16, [a, b, c, z], P)
        _run(fl, lof.LOF_CI8, [e], P)


def test_integrated_longest_rows():
    rng = np.random.default_rng(2)
    d = np.round(rng.normal(0, 32, (24, 16384, 2))).astype(np.int16)
    d[:, 9000:9040, 1] += 80                     # flagged in every channel
    P = oracle_params(time_mode=INTEG)
    with lof.Flagger(0, n_history_slots=0, time_mode=INTEG) as fl:
        _run(fl, lof.LOF_CI16, [d], P)


def test_integrated_block_sequence_with_history():
    P = oracle_params(time_mode=INTEG)
    spec = synth.VoltageSpec(C=64, T=768, sigma=32.0, n_tones=2, n_impulses=2)
    H = oracle.History(64, P)
    with lof.Flagger(0, n_history_slots=64, time_mode=INTEG) as fl:
        for blk in range(12):
            spec.contaminated = (blk == 10)
            d = synth.voltage_block(spec, seed=6, block=blk)[0, 0, 0].numpy()
            res, units = _run(fl, lof.LOF_CI16, [d], P, slots=[0], hist=H, seq=blk)
            fl.history_update(units)
            H.commit(0, res[0]["pending"], res[0]["has_pending"])
            vals, cnt = fl.history_export(0, 64)
            assert np.array_equal(cnt, H.count) and np.array_equal(vals, H.ring), f"block {blk}"


def test_integrated_mode_limits():
    with lof.Flagger(0, time_mode=INTEG) as fl:
        x = torch.zeros((4, 100), dtype=torch.float32, device=DEV)
        with pytest.raises(lof.LofError):
            fl.flag_block(lof.LOF_F32, [lof.make_unit(x, torch.empty_like(x))])
        y = torch.zeros((2, 16385, 2), dtype=torch.int16, device=DEV)
        with pytest.raises(lof.LofError):
            fl.flag_block(lof.LOF_CI16, [lof.make_unit(y, torch.empty_like(y))])
