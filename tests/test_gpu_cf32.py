"""Complex float32 visibilities (post-correlation placement): GPU path against
the oracle under the float contract of the Stokes I path (statistics within
1e-6 relative, masks equal outside the uncertain set of the binary64 replay:
near-threshold windows and what they cascade into), and the
complex output equal to the input with the GPU's own mask applied."""
import numpy as np
import pytest
import torch

import oracle
from paper_1701_08197_gb300 import lof

from test_gpu_f32 import _check_unit

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _vis(seed, C, T):
    rng = np.random.default_rng(seed)
    v = (rng.normal(0, 1, (C, T)) + 1j * rng.normal(0, 1, (C, T))).astype(np.complex64)
    v[rng.integers(0, C), :] *= 4                  # a narrowband interferer
    v[:, rng.integers(0, T, 3)] *= 6               # broadband impulses
    v[rng.integers(0, C), rng.integers(0, T)] = complex(np.nan, 0.0)
    return v


@pytest.mark.parametrize("shape", [(16, 12288), (64, 3000), (3, 37)])
def test_cf32_matches_oracle_within_tolerance(shape):
    C, T = shape
    xs = [_vis(200 + i, C, T) for i in range(2)]
    p = oracle.default_params()
    ins = [torch.as_tensor(x).to(DEV) for x in xs]
    outs = [torch.full_like(t, 7.0 + 7.0j) for t in ins]
    masks = [torch.full(t.shape, 9, dtype=torch.uint8, device=DEV) for t in ins]
    stats = lof.stats_tensor(len(xs), DEV)
    units = [lof.make_unit(i, o, m, -1, stats[k]) for k, (i, o, m) in enumerate(zip(ins, outs, masks))]
    with lof.Flagger(0) as fl:
        fl.flag_block(lof.LOF_CF32, units, 0)
        fl.status()
    for k, x in enumerate(xs):
        m = masks[k].cpu().numpy()
        o = outs[k].cpu().numpy()
        assert np.array_equal(o, np.where(m.astype(bool), np.complex64(0), x))
        pw = (x.real.astype(np.float64) ** 2 + x.imag.astype(np.float64) ** 2)
        pw = np.where(np.isfinite(x.real) & np.isfinite(x.imag), pw, np.nan).astype(np.float32)
        ref = oracle.flag_unit(p, x)
        nd, nn, nc = _check_unit(p, pw, m, np.where(m.astype(bool), np.float32(0), pw),
                                 lof.decode_stats(stats.cpu()[k]), ref, tag=f"cf32 unit {k}")
        assert nd <= nn + nc
