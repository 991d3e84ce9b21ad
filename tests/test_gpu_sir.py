"""GPU parity of the scale-invariant rank operator (Section 2.2) on the final
mask, along time and then frequency: bit for bit against the oracle on
integer units, and at the full station-block size against the oracle's
operator applied to the same kernel's mask without SIR."""
import numpy as np
import pytest
import torch

import bench
import oracle
from paper_1701_08197_gb300 import lof, synth

from helpers import compare_unit, gpu_units, oracle_params

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _sir_2d(mask, percent):
    """Oracle operator along time on every row, then along frequency."""
    m = np.stack([oracle.sir(r, percent) for r in mask])
    return np.stack([oracle.sir(c, percent) for c in m.T]).T


@pytest.mark.parametrize("percent", [20, 45])
def test_sir_units_match_oracle(percent):
    rng = np.random.default_rng(percent)
    a = synth.voltage_block(synth.VoltageSpec(C=256, T=768, sigma=32.0, n_tones=3, n_impulses=4),
                            seed=5, block=0)[0, 0, 0].numpy()
    b = np.round(rng.normal(0, 32, (300, 2500, 2))).astype(np.int16)   # 3 tiles along time,
    b[40:44, 1000:1100] += 300                                          # 2 along frequency
    b[:, 2000:2003] += 500
    b[120] += 90
    c = np.clip(np.round(rng.normal(0, 8, (70, 4100, 2))), -127, 127).astype(np.int8)
    c[10:12, 4000:4090] = 100
    P = oracle_params(sir_percent=percent)
    with lof.Flagger(0, n_history_slots=0, sir_percent=percent) as fl:
        for dtype, datas in ((lof.LOF_CI16, [a, b]), (lof.LOF_CI8, [c])):
            ins, outs, masks, stats, units = gpu_units(datas, DEV)
            fl.flag_block(dtype, units, 0)
            fl.status()
            for i, d in enumerate(datas):
                compare_unit(d, oracle.flag_unit(P, d), outs[i], masks[i], stats[i], tag=f"unit {i}")


@pytest.mark.parametrize("shape", [(1, 100), (33, 129), (255, 7), (32, 1000), (64, 130), (257, 64)])
def test_sir_edge_shapes_match_oracle(shape):
    """Channel counts around the 32-channel blocks of the frequency pass (one
    thread per time step up to 256 channels, the line form above), time
    steps around its 128-thread CTAs."""
    C, T = shape
    rng = np.random.default_rng(C * 1000 + T)
    d = np.round(rng.normal(0, 32, (C, T, 2))).astype(np.int16)
    d[:, T // 3:T // 3 + 3] += 400
    d[C // 2] += 100
    d[:, :: 7] += 60
    P = oracle_params(sir_percent=30)
    with lof.Flagger(0, n_history_slots=0, sir_percent=30) as fl:
        ins, outs, masks, stats, units = gpu_units([d], DEV)
        fl.flag_block(lof.LOF_CI16, units, 0)
        fl.status()
        compare_unit(d, oracle.flag_unit(P, d), outs[0], masks[0], stats[0], tag=str(shape))


def test_sir_full_station_block_against_mask_without_sir():
    dev = torch.device(DEV)
    x = bench.make_block(dev, seed=2, n_station=4)
    n_units = x.shape[0] * 2 * 8
    C, T = 256, 3072
    res = {}
    for percent in (0, 20):
        out = torch.empty_like(x)
        mask = torch.empty(x.shape[:-1], dtype=torch.uint8, device=dev)
        stats = lof.stats_tensor(n_units, dev)
        with lof.Flagger(0, n_history_slots=n_units * C, sir_percent=percent) as fl:
            fl.flag_block(lof.LOF_CI16, bench.build_units(x, out, mask, stats), 0)
            fl.status()
        res[percent] = (mask.reshape(n_units, C, T).cpu().numpy(), out.reshape(n_units, C, T, 2), stats.cpu())
    m0, m1 = res[0][0], res[20][0]
    xs = x.reshape(n_units, C, T, 2)
    for ui in (0, 17, 63):
        assert np.array_equal(m1[ui], _sir_2d(m0[ui], 20)), f"unit {ui}"
    assert (m1 >= m0).all() and m1.sum() > m0.sum()
    keep = torch.as_tensor(1 - m1).to(dev).to(torch.int16).unsqueeze(-1)
    assert torch.equal(res[20][1], xs * keep)
    for ui in range(0, n_units, 9):
        assert lof.decode_stats(res[20][2][ui])["n_flag_total"] == int(m1[ui].sum())


def test_sir_needs_the_mask():
    d = np.zeros((4, 64, 2), np.int16)
    with lof.Flagger(0, sir_percent=20) as fl:
        x = torch.as_tensor(d).to(DEV)
        with pytest.raises(lof.LofError):
            fl.flag_block(lof.LOF_CI16, [lof.make_unit(x, torch.empty_like(x), None)])
