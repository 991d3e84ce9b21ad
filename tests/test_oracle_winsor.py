"""Pins of the oracle's winsorized sigma estimator (sigma_estimator = 2; the
statistics of Section 4.2 include winsorized means): 10% winsorizing on each
side, population stddev of the clamped values, scaled to estimate sigma of
normal data."""
import numpy as np
import pytest

import oracle

W = oracle.SIGMA_WINSOR


def _p():
    return oracle.default_params(sigma_estimator=W)


def _sig(params, x, is_int):
    return oracle.sigma(params, x, is_int)[1]


def test_consistency_factor_from_the_normal_distribution():
    # the scale 1/sqrt(c) with c the variance of a standard normal clamped at
    # its 10% and 90% quantiles, by numerical integration: a normal sample of
    # known sigma is estimated within its sampling error (large n)
    stats = pytest.importorskip("scipy.stats")
    integrate = pytest.importorskip("scipy.integrate")
    z = stats.norm.ppf(0.9)
    c = integrate.quad(lambda x: x * x * stats.norm.pdf(x), -z, z)[0] + 2 * 0.1 * z * z
    rng = np.random.default_rng(0)
    x = rng.normal(1000.0, 37.0, 2_000_000)
    s = _sig(_p(), x, False)
    assert s == pytest.approx(37.0, rel=3e-3)
    # the same sample's clamped stddev times 1/sqrt(c) (library winsorizing)
    mst = pytest.importorskip("scipy.stats.mstats")
    w = np.asarray(mst.winsorize(x, limits=(0.1, 0.1)))
    assert s == pytest.approx(np.std(w) / np.sqrt(c), rel=1e-9)   # quad is good to ~1e-11


@pytest.mark.parametrize("n", [1, 2, 9, 10, 11, 19, 20, 101, 1000])
def test_matches_library_winsorizing_on_integers(n):
    mst = pytest.importorskip("scipy.stats.mstats")
    rng = np.random.default_rng(n)
    x = rng.integers(0, 5000, n).astype(np.float64)
    x[: max(1, n // 20)] = 4_000_000_000.0            # outliers beyond the clamp
    w = np.asarray(mst.winsorize(x, limits=(0.1, 0.1)), dtype=np.float64)
    want_raw = np.std(w)
    s = _sig(_p(), x, True)
    if want_raw > 0:
        assert s == pytest.approx(1.2138796046717422 * want_raw, rel=1e-12)
    else:
        assert s == pytest.approx(np.std(x), rel=1e-12)   # degenerate: plain stddev


def test_robust_to_outliers_and_median_unchanged():
    rng = np.random.default_rng(3)
    x = rng.integers(900, 1100, 1000).astype(np.float64)
    s0 = _sig(_p(), x, True)
    m0 = oracle.median(x)
    y = x.copy()
    y[rng.choice(1000, 50, replace=False)] = 1e12          # 5% of the values, far out
    s1 = _sig(_p(), y, True)
    assert s1 < 1.2 * s0                                   # plain stddev would grow ~1e10x
    assert _sig(oracle.default_params(sigma_estimator=oracle.SIGMA_STD), y, True) > 1e9
    assert m0 == oracle.median(x)


def test_flag_unit_uses_it_for_both_passes():
    # a unit whose spectrum and pooled time series differ between estimators:
    # the reported sigmas are the winsorized ones of the same values
    rng = np.random.default_rng(9)
    d = np.round(rng.normal(0, 32, (64, 1024, 2))).astype(np.int16)
    d[5] += 200
    d[:, 500:504, 0] += 400
    r = oracle.flag_unit(_p(), d)
    P = (d.astype(np.int64) ** 2).sum(-1)
    S = P.sum(1).astype(np.float64)
    assert r["stats"]["sigma_f"] == _sig(_p(), S, True)
    assert r["stats"]["median_f"] == oracle.median(S)
    kept = r["mask"].sum(1) < 1024                          # channels the frequency pass left
    U = P[kept].reshape(-1).astype(np.float64)
    assert (r["stats"]["median_t"], r["stats"]["sigma_t"]) == oracle.sigma(_p(), U, True)
    mad = oracle.flag_unit(oracle.default_params(), d)
    assert r["stats"]["sigma_f"] != mad["stats"]["sigma_f"]
