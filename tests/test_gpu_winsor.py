"""GPU parity of the winsorized sigma estimator (sigma_estimator = 2; Section
4.2 lists winsorized means among the statistics) in the pooled per-channel
time pass, the integrated time mode and the per-channel statistics scope, bit
for bit against the oracle on integer units: masks, data, statistics and
history rings."""
import numpy as np
import pytest
import torch

import oracle
from paper_1701_08197_gb300 import lof, synth

from helpers import compare_unit, gpu_units, oracle_params

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
W = lof.LOF_SIGMA_WINSOR
MODES = {"pooled": dict(), "integrated": dict(time_mode=lof.LOF_TIME_INTEGRATED),
         "scope": dict(stats_scope=lof.LOF_SCOPE_CHANNEL)}


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


def _units(rng):
    a = synth.voltage_block(synth.VoltageSpec(C=256, T=768, sigma=32.0, n_tones=3, n_impulses=4),
                            seed=12, block=0)[0, 0, 0].numpy()
    b = np.round(rng.normal(0, 32, (37, 3001, 2))).astype(np.int16)
    b[:, 1200:1206, 0] += 90
    b[:, 2000] = 3000
    b[9] += np.int16(70)
    b[20, 100:400] += np.int16(120)
    c = np.round(rng.normal(0, 32, (1, 1, 2))).astype(np.int16)
    t = np.round(rng.normal(0, 32, (11, 9, 2))).astype(np.int16)     # n < 10: nothing clamped
    z = np.zeros((8, 64, 2), np.int16)                                # sigma 0: nothing flagged
    k = np.full((12, 200, 2), 7, np.int16)                            # clamped stddev 0: the
    k[3, 50:52] = 400                                                 # plain stddev instead
    return [a, b, c, t, z, k]


@pytest.mark.parametrize("mode", list(MODES))
def test_winsor_units_match_oracle(mode):
    rng = np.random.default_rng(13)
    e = np.clip(np.round(rng.normal(0, 8, (64, 2048, 2))), -127, 127).astype(np.int8)
    e[:, 100:103] = 90
    e[7, 1000:1010] = 40
    P = oracle_params(sigma_estimator=W, **MODES[mode])
    with lof.Flagger(0, n_history_slots=0, sigma_estimator=W, **MODES[mode]) as fl:
        _run(fl, lof.LOF_CI16, _units(rng), P)
        _run(fl, lof.LOF_CI8, [e], P)


@pytest.mark.parametrize("kw", [dict(sir_percent=20), dict(enable_freq=0), dict(enable_time=0),
                                dict(max_window=8, p=1.2)])
def test_winsor_pooled_variants(kw):
    rng = np.random.default_rng(5)
    P = oracle_params(sigma_estimator=W, **kw)
    with lof.Flagger(0, n_history_slots=0, sigma_estimator=W, **kw) as fl:
        _run(fl, lof.LOF_CI16, _units(rng)[:2], P)


def test_winsor_pooled_large_unit_and_in_place():
    rng = np.random.default_rng(8)
    d = np.round(rng.normal(0, 32, (1024, 1024, 2))).astype(np.int16)
    d[rng.integers(0, 1024, 40)] += np.int16(150)
    d[:, 300:302, 1] += 500
    r = np.round(rng.normal(0, 32, (33, 2049, 2))).astype(np.int16)
    r[4, 60:64] = 900
    P = oracle_params(sigma_estimator=W)
    with lof.Flagger(0, n_history_slots=0, sigma_estimator=W) as fl:
        _run(fl, lof.LOF_CI16, [d, r], P, inplace=True)


def test_winsor_block_sequence_with_history():
    P = oracle_params(sigma_estimator=W)
    spec = synth.VoltageSpec(C=64, T=768, sigma=32.0, n_tones=2, n_impulses=2)
    H = oracle.History(64, P)
    with lof.Flagger(0, n_history_slots=64, sigma_estimator=W) as fl:
        for blk in range(12):
            spec.contaminated = (blk == 10)
            d = synth.voltage_block(spec, seed=6, block=blk)[0, 0, 0].numpy()
            res, units = _run(fl, lof.LOF_CI16, [d], P, slots=[0], hist=H, seq=blk)
            fl.history_update(units)
            H.commit(0, res[0]["pending"], res[0]["has_pending"])
            vals, cnt = fl.history_export(0, 64)
            assert np.array_equal(cnt, H.count) and np.array_equal(vals, H.ring), f"block {blk}"


def test_winsor_limits():
    with pytest.raises(lof.LofError):
        lof.Flagger(0, sigma_estimator=3)
    with lof.Flagger(0, sigma_estimator=W) as fl:
        x = torch.zeros((4, 100), dtype=torch.float32, device=DEV)
        with pytest.raises(lof.LofError):
            fl.flag_block(lof.LOF_F32, [lof.make_unit(x, torch.empty_like(x))])
        y = torch.zeros((2, 16385, 2), dtype=torch.int16, device=DEV)
        with pytest.raises(lof.LofError):
            fl.flag_block(lof.LOF_CI16, [lof.make_unit(y, torch.empty_like(y))])
