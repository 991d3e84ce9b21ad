"""The graph form (lof_graph_*) replays exactly what lof_flag_block computes,
for every kernel family: the float path (Stokes I and visibilities), the
exact-statistics kernel (integrated time mode, two-dimensional mode, pooled
winsorized statistics; it takes a second argument) and the SIR pass."""
import numpy as np
import pytest
import torch

from paper_1701_08197_gb300 import lof, synth

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _both(dtype, xs, **params):
    """Masks, data and stats from lof_flag_block and from a graph replay."""
    res = []
    for use_graph in (False, True):
        outs = [torch.zeros_like(x) for x in xs]
        masks = [torch.full(x.shape[:2], 9, dtype=torch.uint8, device=DEV) for x in xs]
        stats = lof.stats_tensor(len(xs), DEV)
        units = [lof.make_unit(x, o, m, -1, stats[k]) for k, (x, o, m) in enumerate(zip(xs, outs, masks))]
        with lof.Flagger(0, **params) as fl:
            if use_graph:
                with fl.graph(dtype, units) as g:
                    g.launch(0)
                    g.status()
            else:
                fl.flag_block(dtype, units, 0)
                fl.status()
        res.append(([m.cpu() for m in masks], [o.cpu() for o in outs], stats.cpu()))
    return res


@pytest.mark.parametrize("case", ["f32", "cf32", "integrated", "2d", "winsor", "sir"])
def test_graph_replay_equals_flag_block(case):
    rng = np.random.default_rng(3)
    if case == "f32":
        spec = synth.PulsarSpec(n_subband=3, C=16, T=3000)
        xs = [t.contiguous() for t in synth.stokes_block(spec, seed=2, block=0, device=DEV)]
        dtype, params = lof.LOF_F32, {}
    elif case == "cf32":
        v = (rng.normal(0, 1, (3, 32, 2000)) + 1j * rng.normal(0, 1, (3, 32, 2000))).astype(np.complex64)
        v[:, :, 700] *= 8
        xs = [torch.as_tensor(a).to(DEV) for a in v]
        dtype, params = lof.LOF_CF32, {}
    else:
        spec = synth.VoltageSpec(C=128, T=1536, sigma=32.0, n_tones=2, n_impulses=3)
        xs = [synth.voltage_block(spec, seed=s, block=0, device=DEV)[0, 0, 0].contiguous() for s in (1, 2)]
        dtype = lof.LOF_CI16
        params = {"integrated": {"time_mode": lof.LOF_TIME_INTEGRATED},
                  "2d": {"time_mode": lof.LOF_TIME_2D, "integ_chan": 4, "integ_time": 8},
                  "winsor": {"sigma_estimator": lof.LOF_SIGMA_WINSOR},
                  "sir": {"sir_percent": 20}}[case]
    (m0, o0, s0), (m1, o1, s1) = _both(dtype, xs, **params)
    for a, b in zip(m0, m1):
        assert torch.equal(a, b)
    for a, b in zip(o0, o1):
        assert torch.equal(a.view(torch.uint8), b.view(torch.uint8))
    assert torch.equal(s0, s1)
    assert int(sum(m.sum() for m in m1)) > 0
