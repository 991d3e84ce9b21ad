"""GPU parity: the CUDA path against the oracle, element by element, through
the C ABI.  Integer voltages must match bit for bit (mask, zeroed output,
statistics, history rings)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1701_08197_gb300 import lof, synth

from helpers import compare_unit, gpu_units, oracle_params

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _flag(fl, dtype, datas, P, slots=None, hist=None, seq=0, inplace=False, check=True):
    ins, outs, masks, stats, units = gpu_units(datas, DEV, slots=slots, inplace=inplace)
    fl.flag_block(dtype, units, seq)
    fl.status()
    res = []
    off = 0
    for i, d in enumerate(datas):
        r = oracle.flag_unit(P, d, history=hist, c0=(slots[i] if slots else 0))
        res.append(r)
        if check:
            compare_unit(d, r, outs[i], masks[i], stats[i], tag=f"unit {i} C={d.shape[0]} T={d.shape[1]}")
    return res, units


def test_tiny_block_sequence_with_history():
    """16 blocks of one 256 x 768 ci16 unit with tones, impulses and one fully
    contaminated block: masks, data, statistics and rings match every block."""
    P = oracle_params()
    spec = synth.VoltageSpec(C=256, T=768, sigma=32.0, n_tones=3, n_impulses=2)
    H = oracle.History(256, P)
    with lof.Flagger(0, n_history_slots=256) as fl:
        for b in range(16):
            spec.contaminated = (b == 11)
            d = synth.voltage_block(spec, seed=1, block=b)[0, 0, 0].numpy()
            res, units = _flag(fl, lof.LOF_CI16, [d], P, slots=[0], hist=H, seq=b)
            fl.history_update(units)
            H.commit(0, res[0]["pending"], res[0]["has_pending"])
            vals, cnt = fl.history_export(0, 256)
            assert np.array_equal(cnt, H.count)
            assert np.array_equal(vals, H.ring), f"block {b}: history rings differ"
        assert res[0]["stats"]["n_chan_hist"] == 0


def test_contaminated_block_history_flags():
    P = oracle_params()
    spec = synth.VoltageSpec(C=64, T=768, sigma=32.0)
    H = oracle.History(64, P)
    with lof.Flagger(0, n_history_slots=64) as fl:
        for b in range(12):
            spec.contaminated = (b == 10)
            d = synth.voltage_block(spec, seed=4, block=b)[0, 0, 0].numpy()
            res, units = _flag(fl, lof.LOF_CI16, [d], P, slots=[0], hist=H, seq=b)
            fl.history_update(units)
            H.commit(0, res[0]["pending"], res[0]["has_pending"])
            if b == 10:
                assert res[0]["stats"]["n_chan_hist"] == 64


@pytest.mark.parametrize("dtype", [lof.LOF_CI8, lof.LOF_CI16])
def test_ragged_shapes_in_one_launch(dtype):
    """Many uneven units (ragged C and T, tiny to several tiles) in one launch."""
    rng = np.random.default_rng(17)
    npdt = np.int8 if dtype == lof.LOF_CI8 else np.int16
    sigma = 8.0 if dtype == lof.LOF_CI8 else 32.0
    shapes = [(1, 1), (1, 5), (3, 31), (2, 32), (5, 33), (17, 100), (64, 768), (7, 1000),
              (40, 257), (256, 96), (9, 4097), (33, 2049), (128, 640)]
    datas = []
    for C, T in shapes:
        x = np.round(rng.normal(0, sigma, (C, T, 2)))
        if C > 4 and T > 40:
            x[rng.integers(0, C), :, :] += 20 * sigma            # a narrowband channel
            t0 = rng.integers(0, T - 20)
            x[:, t0:t0 + rng.integers(1, 20), 0] += 25 * sigma   # a broadband burst
        info = np.iinfo(npdt)
        datas.append(np.clip(x, info.min, info.max).astype(npdt))
    P = oracle_params()
    with lof.Flagger(0, n_history_slots=0) as fl:
        _flag(fl, dtype, datas, P)


def test_saturated_and_degenerate_values():
    """Saturated int16 (powers >= 2^26: 64-bit window sums), constant rows (MAD = 0
    falls back to the stddev), all-zero units (nothing flagged)."""
    rng = np.random.default_rng(3)
    a = np.round(rng.normal(0, 8000, (16, 512, 2))).clip(-32768, 32767).astype(np.int16)
    a[3, 100:110] = 32767
    b = np.full((8, 300, 2), 5, np.int16)
    b[2, 7] = (40, 40)
    c = np.zeros((4, 64, 2), np.int16)
    d = np.full((6, 200, 2), -32768, np.int16)
    P = oracle_params()
    with lof.Flagger(0, n_history_slots=0) as fl:
        _flag(fl, lof.LOF_CI16, [a, b, c, d], P)


@pytest.mark.parametrize("kw", [dict(sigma_estimator=1), dict(max_window=1), dict(max_window=8),
                                dict(enable_freq=0), dict(enable_time=0), dict(sensitivity=1.7),
                                dict(p=1.2, start_threshold=5.0)])
def test_parameter_variants(kw):
    spec = synth.VoltageSpec(C=96, T=1536, sigma=8.0, dtype=torch.int8, n_tones=2, n_impulses=3)
    d = synth.voltage_block(spec, seed=9, block=0)[0, 0, 0].numpy()
    P = oracle_params(**kw)
    with lof.Flagger(0, n_history_slots=0, **kw) as fl:
        _flag(fl, lof.LOF_CI8, [d, d[:50, :700]], P)


def test_in_place_and_strided_rows():
    rng = np.random.default_rng(5)
    d = np.round(rng.normal(0, 32, (20, 300, 2))).astype(np.int16)
    d[4, 50:60] = 2000
    P = oracle_params()
    want = oracle.flag_unit(P, d)
    with lof.Flagger(0) as fl:
        # in place
        x = torch.as_tensor(d).to(DEV)
        m = torch.zeros((20, 300), dtype=torch.uint8, device=DEV)
        fl.flag_block(lof.LOF_CI16, [lof.make_unit(x, x, m)])
        fl.status()
        assert np.array_equal(m.cpu().numpy(), want["mask"])
        assert np.array_equal(x.cpu().numpy(), want["out"])
        # rows inside a wider buffer (unaligned strides: element-wise staging)
        big = torch.zeros((20, 301, 2), dtype=torch.int16, device=DEV)
        big[:, 1:] = torch.as_tensor(d).to(DEV)
        view = big[:, 1:]
        ob = torch.zeros((20, 303, 2), dtype=torch.int16, device=DEV)[:, :300]
        mb = torch.zeros((20, 305), dtype=torch.uint8, device=DEV)[:, :300]
        fl.flag_block(lof.LOF_CI16, [lof.make_unit(view, ob, mb)])
        fl.status()
        assert np.array_equal(mb.cpu().numpy(), want["mask"])
        assert np.array_equal(ob.cpu().numpy(), want["out"])


@pytest.mark.parametrize("p,sigma", [(2.5, 300.0), (5.0, 34.0)])
def test_growing_window_factors(p, sigma):
    # p >= 2 makes threshold_I grow with I: for p = 2.5 at sigma 300 the
    # 32-sample table leaves the register (low-bit) form and the units take the
    # general path; for p = 5 at sigma 34 the windows up to 32 stay packed while
    # the 64-sample prefilter bound degrades to c = 0 (every block a candidate)
    rng = np.random.default_rng(31)
    d = np.clip(np.round(rng.normal(0, sigma, (40, 3072, 2))), -32000, 32000).astype(np.int16)
    d[5, 1000:1200] = np.int16(min(32000, 12 * sigma))
    d[:, 2500:2503] = np.int16(min(32000, 20 * sigma))
    P = oracle_params(p=p)
    with lof.Flagger(0, n_history_slots=0, p=p) as fl:
        _flag(fl, lof.LOF_CI16, [d], P)


@pytest.mark.parametrize("np_dtype,dtype,sigma", [(np.int16, lof.LOF_CI16, 32), (np.int8, lof.LOF_CI8, 8)])
def test_in_place_multi_segment_rows(np_dtype, dtype, sigma):
    # rows of several time-pass segments (1024 samples each, overlapping by
    # 120-sample halos): flagged samples inside the halos must not be seen
    # zeroed by the next segment, so in place equals out of place
    rng = np.random.default_rng(21)
    T = 3072
    d = np.clip(np.round(rng.normal(0, sigma, (24, T, 2))), -120 if np_dtype == np.int8 else -30000,
                120 if np_dtype == np.int8 else 30000).astype(np_dtype)
    hi = 100 if np_dtype == np.int8 else 2000
    for r in range(24):
        for a in (760 + 7 * r, 800 + 5 * r, 880 + 3 * r, 1660 + 4 * r, 1750 + 2 * r, 2580 + 6 * r):
            d[r, a:a + 3 + (r % 5)] = hi
    P = oracle_params()
    want = oracle.flag_unit(P, d)
    with lof.Flagger(0) as fl:
        x = torch.as_tensor(d).to(DEV)
        m = torch.zeros((24, T), dtype=torch.uint8, device=DEV)
        fl.flag_block(dtype, [lof.make_unit(x, x, m)])
        fl.status()
        assert np.array_equal(m.cpu().numpy(), want["mask"])
        assert np.array_equal(x.cpu().numpy(), want["out"])


def test_host_buffer_entry_point():
    rng = np.random.default_rng(8)
    d = np.round(rng.normal(0, 8, (33, 777, 2))).astype(np.int8)
    d[:, 300:305, 1] = 100
    P = oracle_params()
    want = oracle.flag_unit(P, d)
    x = torch.as_tensor(d).pin_memory()
    o = torch.zeros_like(x).pin_memory()
    m = torch.zeros((33, 777), dtype=torch.uint8).pin_memory()
    st = torch.zeros((1, 8), dtype=torch.int64).pin_memory()
    with lof.Flagger(0) as fl:
        s = torch.cuda.current_stream()
        fl.flag_block_host(lof.LOF_CI8, [lof.make_unit(x, o, m, -1, st[0])], 0, s)
        s.synchronize()
        fl.status()
    assert np.array_equal(m.numpy(), want["mask"])
    assert np.array_equal(o.numpy(), want["out"])
    g = lof.decode_stats(st[0])
    assert g["median_t"] == want["stats"]["median_t"] and g["sigma_t"] == want["stats"]["sigma_t"]


def test_host_buffer_pipeline_matches_device_path():
    """Enough units for several upload / flag / download chunks, compact
    (merged copies) and strided (2-D copies) host rows, two calls in a row:
    equal to lof_flag_block on device copies, bit for bit."""
    rng = np.random.default_rng(81)
    C, T, n = 64, 3072, 120                     # 120 x 0.75 MiB of ci16 input, > 64 MiB
    with lof.Flagger(0) as fl:
        s = torch.cuda.current_stream()
        for call in range(2):
            blk = np.round(rng.normal(0, 32, (n, C, T, 2))).astype(np.int16)
            blk[:, :, 1000 + 7 * call:1010 + 7 * call, 0] += 900
            hx = torch.as_tensor(blk).pin_memory()
            wide = torch.zeros((C, T + 8, 2), dtype=torch.int16).pin_memory()   # strided rows
            wide[:, :T] = hx[0]
            ho = torch.zeros_like(hx).pin_memory()
            hm = torch.zeros((n, C, T), dtype=torch.uint8).pin_memory()
            hs = torch.zeros((n, 8), dtype=torch.int64).pin_memory()
            units = [lof.make_unit(wide[:, :T], ho[0], hm[0], -1, hs[0])]
            units += [lof.make_unit(hx[i], ho[i], hm[i], -1, hs[i]) for i in range(1, n)]
            fl.flag_block_host(lof.LOF_CI16, units, call, s)
            s.synchronize()
            fl.status()
            dx = hx.to(DEV)
            do = torch.zeros_like(dx)
            dm = torch.zeros((n, C, T), dtype=torch.uint8, device=DEV)
            ds = lof.stats_tensor(n, DEV)
            fl.flag_block(lof.LOF_CI16, [lof.make_unit(dx[i], do[i], dm[i], -1, ds[i]) for i in range(n)],
                          call, s)
            fl.status()
            assert torch.equal(hm, dm.cpu()), f"call {call}: masks differ"
            assert torch.equal(ho, do.cpu()), f"call {call}: data differs"
            assert torch.equal(hs, ds.cpu()), f"call {call}: statistics differ"
            assert int(hm.sum()) > 0


def test_history_export_import_roundtrip():
    P = oracle_params()
    with lof.Flagger(0, n_history_slots=40) as fl:
        rng = np.random.default_rng(2)
        vals = rng.normal(100, 3, (40, P.history_len))
        cnt = rng.integers(0, P.history_len + 1, 40).astype(np.int32)
        vals[np.arange(P.history_len)[None, :] >= cnt[:, None]] = 0.0
        fl.history_import(0, vals, cnt)
        v2, c2 = fl.history_export(0, 40)
        assert np.array_equal(c2, cnt) and np.array_equal(v2, vals)


def test_invalid_descriptors_are_rejected():
    with lof.Flagger(0, n_history_slots=4) as fl:
        x = torch.zeros((8, 16, 2), dtype=torch.int16, device=DEV)
        u = lof.make_unit(x, None, None, history_slot=0)  # 8 channels > 4 slots
        with pytest.raises(lof.LofError) as e:
            fl.flag_block(lof.LOF_CI16, [u])
        assert e.value.code == lof.LOF_ERR_INVALID
        u = lof.make_unit(x)
        u.n_chan = 0
        with pytest.raises(lof.LofError):
            fl.flag_block(lof.LOF_CI16, [u])
        with pytest.raises(lof.LofError):
            fl.flag_block(7, [lof.make_unit(x)])
