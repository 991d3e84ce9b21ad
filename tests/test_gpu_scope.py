"""GPU parity of the per-channel statistics scope (stats_scope = 1: each kept
channel's time pass thresholds with the median and sigma of its own samples),
bit for bit against the oracle on integer units: masks, data, statistics and
history rings."""
import numpy as np
import pytest
import torch

import oracle
from paper_1701_08197_gb300 import lof, synth

from helpers import compare_unit, gpu_units, oracle_params

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
CHAN = lof.LOF_SCOPE_CHANNEL


def _run(fl, dtype, datas, P, slots=None, hist=None, seq=0, inplace=False):
    ins, outs, masks, stats, units = gpu_units(datas, DEV, slots=slots, inplace=inplace)
    fl.flag_block(dtype, units, seq)
    fl.status()
    res = []
    for i, d in enumerate(datas):
        r = oracle.flag_unit(P, d, history=hist, c0=(slots[i] if slots else 0))
        compare_unit(d, r, outs[i], masks[i], stats[i], tag=f"unit {i} C={d.shape[0]} T={d.shape[1]}")
        res.append(r)
    return res, units, masks


def _loud_and_quiet(rng, C=24, T=2048):
    # rows of very different levels: pooled statistics flag the loud rows'
    # ordinary samples, each row's own statistics do not
    lv = np.where(np.arange(C) % 3 == 0, 200.0, 20.0)
    d = np.round(rng.normal(0, 1, (C, T, 2)) * lv[:, None, None]).astype(np.int16)
    d[4, 700:706] = 150                          # an impulse visible only against row 4's level
    d[9, 1500:1540, 0] += 90
    return d


@pytest.mark.parametrize("kw", [dict(), dict(sigma_estimator=1), dict(enable_time=0), dict(enable_freq=0),
                                dict(sir_percent=20), dict(max_window=8)])
def test_scope_units_match_oracle(kw):
    rng = np.random.default_rng(11)
    a = synth.voltage_block(synth.VoltageSpec(C=256, T=768, sigma=32.0, n_tones=3, n_impulses=4),
                            seed=8, block=0)[0, 0, 0].numpy()
    b = _loud_and_quiet(rng)
    c = np.round(rng.normal(0, 32, (1, 1, 2))).astype(np.int16)
    z = np.zeros((8, 64, 2), np.int16)           # sigma 0: nothing flagged
    e = np.clip(np.round(rng.normal(0, 8, (64, 2048, 2))), -127, 127).astype(np.int8)
    e[:, 100:103] = 90
    e[7, 1000:1010] = 40
    P = oracle_params(stats_scope=CHAN, **kw)
    with lof.Flagger(0, n_history_slots=0, stats_scope=CHAN, **kw) as fl:
        _run(fl, lof.LOF_CI16, [a, b, c, z], P)
        _run(fl, lof.LOF_CI8, [e], P)


def test_scope_ragged_shapes_in_place():
    rng = np.random.default_rng(23)
    datas = []
    for C, T in [(1, 5), (3, 31), (5, 33), (17, 100), (40, 257), (9, 4097), (256, 96), (33, 2049)]:
        x = np.round(rng.normal(0, 32, (C, T, 2)))
        if C > 4 and T > 40:
            x[rng.integers(0, C), :, :] += 640
            t0 = rng.integers(0, T - 20)
            x[:, t0:t0 + rng.integers(1, 20), 0] += 800
        datas.append(np.clip(x, -32768, 32767).astype(np.int16))
    P = oracle_params(stats_scope=CHAN)
    with lof.Flagger(0, n_history_slots=0, stats_scope=CHAN) as fl:
        _run(fl, lof.LOF_CI16, datas, P, inplace=True)


def test_scope_longest_rows_and_differs_from_pooled():
    rng = np.random.default_rng(4)
    d = _loud_and_quiet(rng, C=12, T=16384)
    P = oracle_params(stats_scope=CHAN)
    with lof.Flagger(0, n_history_slots=0, stats_scope=CHAN) as fl:
        _, _, m_scope = _run(fl, lof.LOF_CI16, [d], P)
    with lof.Flagger(0, n_history_slots=0) as fl:
        _, _, m_pool = _run(fl, lof.LOF_CI16, [d], oracle_params())
    assert not torch.equal(m_scope[0], m_pool[0])


def test_scope_block_sequence_with_history():
    P = oracle_params(stats_scope=CHAN)
    spec = synth.VoltageSpec(C=64, T=768, sigma=32.0, n_tones=2, n_impulses=2)
    H = oracle.History(64, P)
    with lof.Flagger(0, n_history_slots=64, stats_scope=CHAN) as fl:
        for blk in range(12):
            spec.contaminated = (blk == 10)
            d = synth.voltage_block(spec, seed=6, block=blk)[0, 0, 0].numpy()
            res, units, _ = _run(fl, lof.LOF_CI16, [d], P, slots=[0], hist=H, seq=blk)
            fl.history_update(units)
            H.commit(0, res[0]["pending"], res[0]["has_pending"])
            vals, cnt = fl.history_export(0, 64)
            assert np.array_equal(cnt, H.count) and np.array_equal(vals, H.ring), f"block {blk}"
        assert res[0]["stats"]["median_t"] == 0.0


def test_scope_limits():
    with pytest.raises(lof.LofError):
        lof.Flagger(0, stats_scope=CHAN, time_mode=lof.LOF_TIME_INTEGRATED)
    with pytest.raises(lof.LofError):
        lof.Flagger(0, stats_scope=2)
    with lof.Flagger(0, stats_scope=CHAN) as fl:
        x = torch.zeros((4, 100), dtype=torch.float32, device=DEV)
        with pytest.raises(lof.LofError):
            fl.flag_block(lof.LOF_F32, [lof.make_unit(x, torch.empty_like(x))])
        y = torch.zeros((2, 16385, 2), dtype=torch.int16, device=DEV)
        with pytest.raises(lof.LofError):
            fl.flag_block(lof.LOF_CI16, [lof.make_unit(y, torch.empty_like(y))])
