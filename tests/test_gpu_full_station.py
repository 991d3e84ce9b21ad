"""Parity at full size, in the launch configuration bench.py times: the whole
LOFAR pre-beamformer block (48 stations x 2 pols x 8 subbands = 768 units of
256 x 3072 complex int16, history rings filled to 60 means) in one launch;
sampled units against the oracle, bit for bit, plus properties that hold for
every unit.  Also the largest shapes the C ABI accepts and an empty block."""
import numpy as np
import pytest
import torch

import bench
import oracle
from paper_1701_08197_gb300 import lof

from helpers import compare_unit, gpu_units, oracle_params

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def test_full_station_block_sampled_units_match_oracle():
    dev = torch.device(DEV)
    x = bench.make_block(dev, seed=2)                          # [48, 2, 8, 256, 3072, 2]
    out = torch.full_like(x, 77)
    mask = torch.full(x.shape[:-1], 9, dtype=torch.uint8, device=dev)
    n_units = x.shape[0] * 2 * 8
    stats = lof.stats_tensor(n_units, dev)
    C, T, H = 256, 3072, 60
    with lof.Flagger(0, n_history_slots=n_units * C) as fl:
        pw = (x.to(torch.float32) ** 2).sum(-1).mean(-1).reshape(-1).double().cpu().numpy()
        rng = np.random.default_rng(7)
        ring = pw[:, None] * (1.0 + 0.01 * rng.standard_normal((pw.size, H)))
        counts = np.full(pw.size, H, np.int32)
        fl.history_import(0, ring, counts)
        units = bench.build_units(x, out, mask, stats)
        fl.flag_block(lof.LOF_CI16, units, 5)
        fl.status()
        torch.cuda.synchronize()
        # every unit: the data output is the input with the mask applied, and
        # the mask is 0/1
        m_all = mask.reshape(n_units, C, T)
        assert int(m_all.max()) <= 1
        keep = (1 - m_all).to(torch.int16).unsqueeze(-1)
        assert torch.equal(out.reshape(n_units, C, T, 2), x.reshape(n_units, C, T, 2) * keep)
        st = stats.cpu()
        assert all(lof.decode_stats(st[i])["n_flag_total"] == int(m_all[i].sum()) for i in range(0, n_units, 37))
        # sampled units against the oracle with the same rings
        P = oracle_params()
        xs = x.reshape(n_units, C, T, 2)
        # fixed corners plus a seeded draw of 16 more units across the stations
        draw = np.random.default_rng(20261204).choice(n_units, 16, replace=False).tolist()
        for ui in sorted({0, 1, 131, 402, 767, *draw}):
            hist = oracle.History(C, P)
            hist.ring[:] = ring[ui * C:(ui + 1) * C]
            hist.count[:] = H
            d = xs[ui].cpu().numpy()
            r = oracle.flag_unit(P, d, history=hist)
            compare_unit(d, r, out.reshape(n_units, C, T, 2)[ui], m_all[ui], st[ui], tag=f"unit {ui}")


def test_largest_shapes_and_empty_block():
    rng = np.random.default_rng(11)
    # the channel limit, and a long row (several time-pass segments)
    a = np.round(rng.normal(0, 32, (2048, 48, 2))).astype(np.int16)
    a[100, :, 0] += 900
    b = np.round(rng.normal(0, 32, (3, 40000, 2))).astype(np.int16)
    b[:, 12345:12400, 1] += 1500
    P = oracle_params()
    with lof.Flagger(0) as fl:
        ins, outs, masks, stats, units = gpu_units([a, b], DEV)
        fl.flag_block(lof.LOF_CI16, units, 0)
        fl.status()
        for i, d in enumerate([a, b]):
            compare_unit(d, oracle.flag_unit(P, d), outs[i], masks[i], stats[i], tag=f"unit {i}")
        # an empty block is a no-op
        fl.flag_block(lof.LOF_CI16, [], 0)
        fl.status()
