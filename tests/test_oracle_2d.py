"""Pins of the oracle's two-dimensional mode (time_mode = 2: SumThreshold on
cells of integ_chan x integ_time summed powers, along time on every row of
cells and then along frequency on every column, for each window size; the
paper mentions a 2-D flagger with partial integration in Sections 2.1 and 3).
Each pin reduces it to an independently written branch or to a brute force."""
import numpy as np
import pytest

import oracle

rng0 = np.random.default_rng


def _unit(seed, C, T, sigma=32):
    rng = rng0(seed)
    d = np.round(rng.normal(0, sigma, (C, T, 2))).astype(np.int16)
    d[rng.integers(0, C), :, 0] += np.int16(4 * sigma)            # a narrowband channel
    t0 = int(rng.integers(0, max(1, T - 4)))
    d[:, t0:t0 + 3, 1] += np.int16(5 * sigma)                     # a broadband burst
    d[rng.integers(0, C), rng.integers(0, T)] = np.int16(20 * sigma)
    return d


def _power(d):
    return (d.astype(np.int64) ** 2).sum(-1)


def _p(**kw):
    kw.setdefault("enable_history", 0)
    return oracle.default_params(**kw)


def test_time_direction_alone_is_the_pooled_per_channel_pass():
    # one-sample cells, frequency direction off: the per-channel mode with its
    # frequency pass off (pooled statistics over every sample, SumThreshold
    # along every row)
    d = _unit(1, 24, 700)
    a = oracle.flag_unit(_p(time_mode=2, enable_freq=0), d)
    b = oracle.flag_unit(_p(time_mode=0, enable_freq=0), d)
    assert np.array_equal(a["mask"], b["mask"]) and np.array_equal(a["out"], b["out"])
    for k in ("median_t", "sigma_t", "n_flag_time", "n_flag_total"):
        assert a["stats"][k] == b["stats"][k], k
    assert a["mask"].sum() > 0


def test_frequency_direction_alone_is_the_column_pass():
    d = _unit(2, 40, 90)
    P = _power(d).astype(np.float64)
    a = oracle.flag_unit(_p(time_mode=2, enable_time=0), d)
    med, sig = oracle.sigma(_p(), P.reshape(-1), True)
    want = np.stack([oracle.sum_threshold(_p(), P[:, t], med, sig) for t in range(P.shape[1])], 1)
    assert np.array_equal(a["mask"], want)
    assert (a["stats"]["median_t"], a["stats"]["sigma_t"]) == (med, sig)
    assert a["mask"].sum() > 0


def test_one_row_of_cells_is_the_integrated_series():
    # cells spanning every channel: the integrated time mode with its
    # frequency pass off
    d = _unit(3, 16, 1000)
    a = oracle.flag_unit(_p(time_mode=2, integ_chan=16, enable_freq=0), d)
    b = oracle.flag_unit(_p(time_mode=1, enable_freq=0), d)
    assert np.array_equal(a["mask"], b["mask"])
    for k in ("median_t", "sigma_t", "n_flag_time"):
        assert a["stats"][k] == b["stats"][k], k


def _brute(P, Fi, Ti, max_window=64, time_first=True):
    """Cells by reshape, library statistics, substituted-sum windows."""
    stats = pytest.importorskip("scipy.stats")
    C, T = P.shape
    V = P.reshape(C // Fi, Fi, T // Ti, Ti).sum((1, 3)).astype(np.float64)
    med = float(np.median(V))
    sig = float(stats.median_abs_deviation(V.reshape(-1), scale="normal"))
    if sig == 0:
        sig = float(np.std(V))
    Cg, Tg = V.shape
    F = np.zeros(V.shape, bool)
    dirs = [(V, F), (V.T, F.T)]               # along time (rows), along frequency (columns)
    if not time_first:
        dirs.reverse()
    k = 0
    while True:
        I = 1 << k
        if I > max_window or (I > Tg and I > Cg):
            break
        thr = med + sig * (6.0 * 1.5 ** k / I)
        for Vv, Fv in dirs:
            if I > Vv.shape[1]:
                continue
            new = Fv.copy()
            for r in range(Vv.shape[0]):
                for t in range(Vv.shape[1] - I + 1):
                    w = np.where(Fv[r, t:t + I], thr, Vv[r, t:t + I])
                    if w.sum() > I * thr:
                        new[r, t:t + I] = True
            Fv[...] = new
        k += 1
    return np.repeat(np.repeat(F, Fi, 0), Ti, 1), med, sig


@pytest.mark.parametrize("C,T,Fi,Ti", [(8, 24, 1, 1), (12, 40, 2, 4), (16, 64, 4, 2), (6, 96, 3, 8),
                                       (32, 8, 2, 1)])
def test_brute_force_cells_and_interleaved_directions(C, T, Fi, Ti):
    for seed in range(4):
        d = _unit(10 * seed + C, C, T)
        P = _power(d)
        want, med, sig = _brute(P, Fi, Ti)
        a = oracle.flag_unit(_p(time_mode=2, integ_chan=Fi, integ_time=Ti), d)
        assert a["stats"]["median_t"] == pytest.approx(med, rel=1e-15)
        assert a["stats"]["sigma_t"] == pytest.approx(sig, rel=1e-12)
        assert np.array_equal(a["mask"], want), (C, T, Fi, Ti, seed)


def test_order_matters_and_is_time_first():
    # a grid on which the two direction orders give different masks (cells
    # flagged along time at I >= 2 enter the frequency windows substituted):
    # the oracle takes the time-first order
    rng = rng0(126)
    d = np.round(rng.normal(0, 4, (10, 10, 2))).astype(np.int16)
    for _ in range(6):
        r, c = rng.integers(0, 10, 2)
        d[r, c, 0] += np.int16(rng.integers(8, 20))
    P = _power(d)
    a = oracle.flag_unit(_p(time_mode=2), d)
    tf, _, _ = _brute(P, 1, 1)
    ft, _, _ = _brute(P, 1, 1, time_first=False)
    assert not np.array_equal(tf, ft)
    assert np.array_equal(a["mask"], tf)


def test_cells_must_divide_the_unit():
    d = _unit(4, 12, 100)
    with pytest.raises(ValueError):
        oracle.flag_unit(_p(time_mode=2, integ_chan=5), d)
    with pytest.raises(ValueError):
        oracle.flag_unit(_p(time_mode=2, integ_time=3), d)
