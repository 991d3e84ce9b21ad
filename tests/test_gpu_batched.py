"""Batched uneven units (complex int8, mixed channel counts and block
lengths) in one persistent launch, captured once as a CUDA graph and
replayed, with the launch shape picked by the autotuner: bit-exact against
the oracle, and identical to the direct call whatever the tuning."""
import numpy as np
import pytest
import torch

import oracle
from paper_1701_08197_gb300 import lof, synth

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _units(seed, n_units=18, block=0):
    shapes = synth.random_units(n_units, (16, 64, 256), (768, 3072, 12288), seed=seed)
    xs = []
    for i, (C, T) in enumerate(shapes):
        spec = synth.VoltageSpec(C=C, T=T, dtype=torch.int8, sigma=8.0, tone_frac=0.02,
                                 impulse_frac=0.01)
        xs.append(synth.voltage_block(spec, seed=synth._mix(seed, i), block=block, device=DEV)[0, 0, 0])
    return xs


def _bufs(xs):
    outs = [torch.full_like(x, 5) for x in xs]
    masks = [torch.full(x.shape[:2], 3, dtype=torch.uint8, device=DEV) for x in xs]
    stats = lof.stats_tensor(len(xs), DEV)
    units = [lof.make_unit(x, o, m, -1, stats[i]) for i, (x, o, m) in enumerate(zip(xs, outs, masks))]
    return outs, masks, stats, units


def _snap(outs, masks, stats):
    torch.cuda.synchronize()
    return ([o.cpu().numpy().copy() for o in outs], [m.cpu().numpy().copy() for m in masks],
            [lof.decode_stats(s) for s in stats.cpu()])


def test_graph_replay_matches_direct_call_and_oracle():
    xs = _units(31)
    outs, masks, stats, units = _bufs(xs)
    with lof.Flagger(0) as fl:
        fl.flag_block(lof.LOF_CI8, units, 1)
        fl.status()
        direct = _snap(outs, masks, stats)
        for o, m in zip(outs, masks):
            o.fill_(5)
            m.fill_(3)
        with fl.graph(lof.LOF_CI8, units) as g:
            g.launch(1)
            g.status()
            replay = _snap(outs, masks, stats)
            for i in range(len(xs)):
                assert np.array_equal(replay[1][i], direct[1][i]), f"unit {i}: mask"
                assert np.array_equal(replay[0][i], direct[0][i]), f"unit {i}: data"
                assert replay[2][i] == direct[2][i]
            # new data in the same buffers, replayed again
            ys = _units(31, block=1)
            for x, y in zip(xs, ys):
                x.copy_(y)
            g.launch(2)
            g.status()
            second = _snap(outs, masks, stats)
    p = oracle.default_params()
    rng = np.random.default_rng(0)
    for i in sorted(rng.choice(len(xs), 4, replace=False)):
        ref = oracle.flag_unit(p, xs[i].cpu().numpy())
        assert np.array_equal(second[1][i], ref["mask"]), f"unit {i} {tuple(xs[i].shape)}: mask"
        assert np.array_equal(second[0][i], ref["out"]), f"unit {i}: data"
        assert second[2][i]["median_t"] == ref["stats"]["median_t"]
        assert second[2][i]["sigma_t"] == ref["stats"]["sigma_t"]


def test_autotuned_shape_gives_identical_results():
    xs = _units(33, n_units=12)
    outs, masks, stats, units = _bufs(xs)
    with lof.Flagger(0) as fl:
        fl.flag_block(lof.LOF_CI8, units, 0)
        fl.status()
        before = _snap(outs, masks, stats)
        tuning, ms = fl.autotune(lof.LOF_CI8, units, reps=1)
        assert ms > 0 and tuning["threads"] in (128, 256)
        assert fl.tuning() == tuning
        for o, m in zip(outs, masks):
            o.fill_(5)
            m.fill_(3)
        fl.flag_block(lof.LOF_CI8, units, 0)
        fl.status()
        after = _snap(outs, masks, stats)
    for i in range(len(xs)):
        assert np.array_equal(after[1][i], before[1][i])
        assert np.array_equal(after[0][i], before[0][i])
        assert after[2][i] == before[2][i]


@pytest.mark.parametrize("kw", [dict(flag_rows=5), dict(stat_samples=4096), dict(threads=256, ctas_per_sm=1)])
def test_launch_shapes_do_not_change_results(kw):
    xs = _units(34, n_units=6)
    outs, masks, stats, units = _bufs(xs)
    with lof.Flagger(0) as fl:
        fl.flag_block(lof.LOF_CI8, units, 0)
        fl.status()
        base = _snap(outs, masks, stats)
        fl.set_tuning(**kw)
        fl.flag_block(lof.LOF_CI8, units, 0)
        fl.status()
        other = _snap(outs, masks, stats)
    for i in range(len(xs)):
        assert np.array_equal(other[1][i], base[1][i])
        assert np.array_equal(other[0][i], base[0][i])


def _ragged_ci16(seed):
    """Ragged complex int16 units: row lengths off every segment and chunk
    boundary, one unit with rows past the packed form's range."""
    rng = np.random.default_rng(seed)
    out = []
    for C, T in [(7, 1001), (33, 3071), (5, 4097), (64, 769), (3, 37)]:
        x = np.round(rng.normal(0, 32, (C, T, 2)))
        x[rng.integers(0, C), :, 0] += 25 * 32
        t0 = int(rng.integers(0, max(1, T - 70)))
        x[:, t0:t0 + 60, 1] += 40 * 32
        out.append(np.clip(x, -32768, 32767).astype(np.int16))
    big = np.round(rng.normal(0, 3000, (4, 2000, 2)))           # threshold_1 above 2^20: general path
    out.append(np.clip(big, -32768, 32767).astype(np.int16))
    return out


@pytest.mark.parametrize("dtype", [lof.LOF_CI8, lof.LOF_CI16])
def test_every_window_schedule_gives_identical_results(dtype):
    """The autotuner's window schedules (packed or general time pass, the
    bound on the 64-sample windows on or off, coalesced or bulk data stores)
    change the work, never the result: bit-identical masks, data and
    statistics on ragged units, equal to the oracle."""
    if dtype == lof.LOF_CI8:
        xs = [x.cpu().numpy() for x in _units(36, n_units=8)]
    else:
        xs = _ragged_ci16(37)
    ins = [torch.as_tensor(x).to(DEV) for x in xs]
    outs, masks, stats, units = _bufs(ins)
    results = {}
    with lof.Flagger(0) as fl:
        for sc in range(8):
            fl.set_tuning(schedule=lof.LOF_SCHED_SET | sc)
            assert fl.tuning()["schedule"] == lof.LOF_SCHED_SET | sc
            for o, m in zip(outs, masks):
                o.fill_(5)
                m.fill_(3)
            fl.flag_block(dtype, units, 0)
            fl.status()
            results[sc] = _snap(outs, masks, stats)
    base = results[7]
    for sc, r in results.items():
        for i in range(len(xs)):
            assert np.array_equal(r[1][i], base[1][i]), f"schedule {sc} unit {i}: mask"
            assert np.array_equal(r[0][i], base[0][i]), f"schedule {sc} unit {i}: data"
            assert r[2][i] == base[2][i], f"schedule {sc} unit {i}: statistics"
    P = oracle.default_params()
    for i, x in enumerate(xs):
        want = oracle.flag_unit(P, x)
        assert np.array_equal(base[1][i], want["mask"]), f"unit {i}: oracle mask"
        assert np.array_equal(base[0][i], want["out"]), f"unit {i}: oracle data"
