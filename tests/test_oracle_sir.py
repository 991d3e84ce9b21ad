"""Pins of the oracle's scale-invariant rank operator (Section 2.2) against
its definition and closed forms: a sample is flagged when some interval
holding it is at least (100 - percent)% flagged."""
import numpy as np
import pytest

import oracle


def _brute(f, percent):
    """The definition, interval by interval (exact integer arithmetic)."""
    L = len(f)
    c = np.concatenate([[0], np.cumsum(f)])
    g = np.zeros(L, np.uint8)
    for a in range(L):
        for b in range(a + 1, L + 1):
            if 100 * (c[b] - c[a]) >= (100 - percent) * (b - a):
                g[a:b] = 1
    return g


@pytest.mark.parametrize("percent", [0, 5, 20, 33, 50, 80, 99])
def test_matches_the_definition_on_random_masks(percent):
    rng = np.random.default_rng(percent + 1)
    for L in (1, 2, 3, 7, 19, 40):
        for density in (0.05, 0.3, 0.6):
            f = (rng.random(L) < density).astype(np.uint8)
            assert np.array_equal(oracle.sir(f, percent), _brute(f, percent)), (L, density, f)


@pytest.mark.parametrize("percent,run", [(20, 1), (20, 4), (20, 7), (20, 40), (20, 101), (50, 9), (10, 30)])
def test_isolated_run_grows_by_the_closed_form(percent, run):
    # a run of L flags far from any other grows by floor(percent * L / (100 - percent))
    # samples on each side: 100 * L >= (100 - percent) * (L + d)
    d = (percent * run) // (100 - percent)
    f = np.zeros(run + 4 * d + 20, np.uint8)
    s = 2 * d + 10
    f[s:s + run] = 1
    want = np.zeros_like(f)
    want[s - d:s + run + d] = 1
    assert np.array_equal(oracle.sir(f, percent), want)


def test_special_cases():
    rng = np.random.default_rng(3)
    f = (rng.random(500) < 0.2).astype(np.uint8)
    assert np.array_equal(oracle.sir(f, 0), f)                     # eta = 0: unchanged
    assert not oracle.sir(np.zeros(64, np.uint8), 20).any()         # nothing to extend
    assert oracle.sir(np.ones(64, np.uint8), 20).all()
    g = oracle.sir(f, 20)
    assert np.all(g >= f)                                           # flags are only added
    assert np.array_equal(oracle.sir(f[::-1], 20), g[::-1])         # no direction
    # two runs whose joint density reaches 80 % merge across their gap
    h = np.zeros(60, np.uint8)
    h[10:26] = 1
    h[30:46] = 1                                                    # 32 flags in 36 samples
    assert oracle.sir(h, 20)[26:30].all()


def test_unit_applies_time_then_frequency_on_the_final_mask():
    rng = np.random.default_rng(9)
    d = np.round(rng.normal(0, 32, (24, 300, 2))).astype(np.int16)
    d[5, 100:104] = 900
    d[:, 200:202] = 700
    d[17] += np.int16(60)
    P0 = oracle.default_params()
    P1 = oracle.default_params(sir_percent=20)
    m0 = oracle.flag_unit(P0, d)["mask"]
    r1 = oracle.flag_unit(P1, d)
    want = np.stack([_brute(row, 20) for row in m0])
    want = np.stack([_brute(col, 20) for col in want.T]).T
    assert np.array_equal(r1["mask"], want)
    assert r1["stats"]["n_flag_total"] == int(want.sum())
    assert np.array_equal(r1["out"], d * (1 - want)[:, :, None].astype(np.int16))
