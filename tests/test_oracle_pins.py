"""Pins of the oracle against what the paper and the mathematics fix.

Every test here runs on the CPU (no GPU marker).  The oracle is checked against
values printed in the paper (Section 2.1: 6 sigma at I=1, 4.5 sigma at I=2),
hand-worked examples of the definition (tests/golden/), a brute-force window
enumerator written in the "substituted sum" form, numpy/scipy statistics and
special cases that reduce to textbook operations.
"""
import itertools
import math
import os

import numpy as np
import pytest

import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    out = []
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                out.append(line)
    return out


# ---------------------------------------------------------------- thresholds

def test_factor_table_matches_section_2_1():
    P = oracle.default_params()
    for line in _rows("factor_table.txt"):
        k, I, f = line.split()
        assert oracle.factor(P, int(k)) == float(f), line


def test_printed_sigmas():
    # Section 2.1 prints 6 sigma for the first iteration and 4.5 sigma for the second.
    P = oracle.default_params()
    assert oracle.threshold(P, 0.0, 1.0, 0) == 6.0
    assert oracle.threshold(P, 0.0, 1.0, 1) == 4.5
    assert oracle.threshold(P, 100.0, 2.0, 0) == 112.0


def test_threshold_scales_with_sensitivity_and_p():
    P = oracle.default_params(sensitivity=2.0, p=2.0, start_threshold=5.0)
    # factor_I = 5 * 2^k / 2^k = 5 for every I when p = 2
    for k in range(7):
        assert oracle.factor(P, k) == 5.0
        assert oracle.threshold(P, 1.0, 3.0, k) == 1.0 + 3.0 * 5.0 * 2.0


# ---------------------------------------------------------------- SumThreshold

def _bits(mask):
    return "".join(str(int(b)) for b in mask)


def test_hand_worked_examples():
    P = oracle.default_params()
    for line in _rows("sumthreshold_examples.txt"):
        name, vals, m, s, want = [x.strip() for x in line.split("|")]
        v = np.array([float(x) for x in vals.split()])
        got = oracle.sum_threshold(P, v, float(m), float(s))
        assert _bits(got) == want, name


def test_hand_worked_example_with_statistics():
    P = oracle.default_params()
    for line in _rows("sumthreshold_stats_examples.txt"):
        name, vals, m, mad, s, t1, t2, want = [x.strip() for x in line.split("|")]
        v = np.array([float(x) for x in vals.split()])
        med, sig = oracle.sigma(P, v, is_int=True)
        assert med == float(m)
        assert sig == float(s)
        assert oracle.threshold(P, med, sig, 0) == float(t1)
        assert oracle.threshold(P, med, sig, 1) == float(t2)
        assert _bits(oracle.sum_threshold(P, v, med, sig)) == want, name


def brute_force(v, m, s, max_window=64, p=1.5, sens=1.0, start=6.0, entry=None):
    """Independent enumerator in the 'substituted sum' form of Section 2.1: the
    window sum with every flagged sample replaced by threshold_I exceeds
    I * threshold_I.  Threshold schedule from the printed 6 / 4.5 sigma."""
    L = len(v)
    flags = [False] * L if entry is None else [bool(e) for e in entry]
    if not s > 0:
        return flags
    I, k = 1, 0
    while I <= max_window and I <= L:
        thr = m + s * (start * p ** k / I) * sens
        new = list(flags)
        for t in range(L - I + 1):
            tot = sum(thr if flags[j] else v[j] for j in range(t, t + I))
            if tot > I * thr:
                for j in range(t, t + I):
                    new[j] = True
        flags = new
        I, k = 2 * I, k + 1
    return flags


def test_brute_force_random_rows():
    """Random small integer rows with dyadic thresholds (m integer, sigma a power
    of two), where both forms are exact, must agree bit for bit."""
    rng = np.random.default_rng(7)
    P = oracle.default_params()
    n = 0
    for L in list(range(1, 20)) + [31, 32, 33, 63, 64, 65, 100]:
        for _ in range(12):
            m = int(rng.integers(0, 4))
            s = float(2.0 ** int(rng.integers(-1, 3)))
            v = rng.exponential(3.0, L).round() + m
            if rng.random() < 0.5:
                v[rng.integers(0, L, size=max(1, L // 8))] += rng.integers(5, 40)
            got = oracle.sum_threshold(P, v, float(m), s)
            want = brute_force(list(v), m, s)
            assert _bits(got) == _bits(want), (L, m, s, list(v))
            n += 1
    assert n > 300


def test_brute_force_with_entry_flags_and_windows():
    rng = np.random.default_rng(11)
    for maxw in (1, 2, 8, 64):
        P = oracle.default_params(max_window=maxw)
        for L in (5, 17, 70):
            for _ in range(10):
                v = rng.integers(0, 12, L).astype(float)
                entry = rng.random(L) < 0.1
                got = oracle.sum_threshold(P, v, 2.0, 1.0, entry=entry.astype(np.uint8))
                want = brute_force(list(v), 2.0, 1.0, max_window=maxw, entry=entry)
                assert _bits(got) == _bits(want)
                assert np.all(got[entry] == 1)  # entry flags are kept


def test_max_window_one_is_a_simple_thresholder():
    rng = np.random.default_rng(3)
    P = oracle.default_params(max_window=1)
    v = rng.exponential(10.0, 1000)
    got = oracle.sum_threshold(P, v, 5.0, 2.0)
    assert np.array_equal(got.astype(bool), v > 5.0 + 6.0 * 2.0)


def test_zero_sigma_flags_nothing():
    P = oracle.default_params()
    v = np.array([0.0, 100.0, 0.0])
    assert not oracle.sum_threshold(P, v, 0.0, 0.0).any()


def test_window_longer_than_row_is_skipped():
    # a 3-sample row only runs I = 1 and I = 2
    P = oracle.default_params()
    v = np.array([3.0, 3.0, 3.0])   # I=4 would see 9 > 4*2.53 = 10.1? no; I=2: 6 > 9? no
    assert not oracle.sum_threshold(P, v, 0.0, 1.0).any()
    v = np.array([5.0, 5.0])        # I=2: 10 > 9 -> both
    assert _bits(oracle.sum_threshold(P, v, 0.0, 1.0)) == "11"


# ---------------------------------------------------------------- statistics

def test_median_matches_numpy():
    rng = np.random.default_rng(5)
    for n in (1, 2, 3, 10, 11, 1000, 1001):
        x = rng.integers(0, 50, n).astype(float)
        assert oracle.median(x) == np.median(x)
        y = rng.normal(3, 2, n)
        assert oracle.median(y) == np.median(y)


def test_mad_sigma_matches_scipy():
    stats = pytest.importorskip("scipy.stats")
    P = oracle.default_params()
    rng = np.random.default_rng(6)
    for n in (2, 5, 64, 1000, 1001):
        x = rng.integers(0, 10000, n).astype(float)
        m, s = oracle.sigma(P, x, is_int=True)
        assert m == np.median(x)
        ref = stats.median_abs_deviation(x, scale="normal")
        assert s == pytest.approx(ref, rel=1e-15, abs=0)
        y = rng.exponential(2.0, n)
        m, s = oracle.sigma(P, y, is_int=False)
        assert s == pytest.approx(stats.median_abs_deviation(y, scale="normal"), rel=1e-15)


def test_sigma_hand_example():
    # v = [1,20,1,5,5,0,2,4]: median 3, |v-3| = 2,17,2,2,2,3,1,1 -> MAD 2
    P = oracle.default_params()
    m, s = oracle.sigma(P, np.array([1, 20, 1, 5, 5, 0, 2, 4.0]), is_int=True)
    assert m == 3.0 and s == 2 * 1.482602218505602
    Pstd = oracle.default_params(sigma_estimator=oracle.SIGMA_STD)
    m, s = oracle.sigma(Pstd, np.array([1, 20, 1, 5, 5, 0, 2, 4.0]), is_int=True)
    assert s == pytest.approx(np.std([1, 20, 1, 5, 5, 0, 2, 4.0]), rel=1e-15)


def test_std_fallback_when_mad_is_zero():
    P = oracle.default_params()
    x = np.array([5, 5, 5, 5, 9, 9, 100.0])  # MAD = 0
    m, s = oracle.sigma(P, x, is_int=True)
    assert m == 5.0
    assert s == pytest.approx(np.std(x), rel=1e-15)
    # exact integer moments: sigma = sqrt((n*sum x^2 - (sum x)^2)) / n
    n, s1, s2 = len(x), int(x.sum()), int((x.astype(np.int64) ** 2).sum())
    assert s == math.sqrt((n * s2 - s1 * s1) / (n * n))


def test_integer_std_is_exact_for_large_values():
    P = oracle.default_params(sigma_estimator=oracle.SIGMA_STD)
    x = np.array([2.0 ** 31, 0.0, 2.0 ** 31, 1.0])
    _, s = oracle.sigma(P, x, is_int=True)
    n, s1 = 4, int(sum(int(v) for v in x))
    s2 = sum(int(v) ** 2 for v in x)
    assert s == math.sqrt(float(n * s2 - s1 * s1) / float(n * n))


# ---------------------------------------------------------------- whole unit

def test_unit_power_and_apply():
    """Power is re^2 + im^2 (Section 4); flagged samples are zeroed in the output
    and reported in the mask."""
    P = oracle.default_params(enable_freq=0, enable_history=0, max_window=1)
    rng = np.random.default_rng(1)
    d = rng.integers(-3, 4, (4, 50, 2)).astype(np.int16)
    d[2, 17] = (300, -400)  # power 250000
    r = oracle.flag_unit(P, d)
    assert r["mask"][2, 17] == 1
    assert (r["out"][2, 17] == 0).all()
    keep = r["mask"] == 0
    assert np.array_equal(r["out"][keep], d[keep])
    pw = (d.astype(np.int64) ** 2).sum(-1).astype(float)
    m, s = oracle.sigma(P, pw.ravel(), True)
    assert r["stats"]["median_t"] == m and r["stats"]["sigma_t"] == s
    assert np.array_equal(r["mask"].astype(bool), pw > m + 6 * s)


def test_unit_frequency_pass_flags_whole_channels():
    P = oracle.default_params(enable_history=0)
    rng = np.random.default_rng(2)
    d = np.round(rng.normal(0, 32, (64, 256, 2))).astype(np.int16)
    t = np.arange(256)
    d[10, :, 0] = (d[10, :, 0] + 600 * np.cos(0.3 * t)).astype(np.int16)
    d[10, :, 1] = (d[10, :, 1] + 600 * np.sin(0.3 * t)).astype(np.int16)
    r = oracle.flag_unit(P, d)
    assert r["mask"][10].all()
    assert r["stats"]["n_chan_freq"] >= 1
    # the spectrum statistics are those of the per-channel power sums
    pw = (d.astype(np.int64) ** 2).sum(-1)
    S = pw.sum(1).astype(float)
    m, s = oracle.sigma(P, S, True)
    assert r["stats"]["median_f"] == m and r["stats"]["sigma_f"] == s


def test_time_statistics_exclude_frequency_flagged_channels():
    # with the time pass off, the fully flagged rows are exactly the frequency flags
    P = oracle.default_params(enable_history=0, enable_time=0)
    rng = np.random.default_rng(4)
    d = np.round(rng.normal(0, 8, (32, 128, 2))).astype(np.int8)
    d[5] = 120
    r = oracle.flag_unit(P, d)
    assert r["mask"][5].all()
    fc = r["mask"].all(1)
    assert r["stats"]["n_chan_freq"] == fc.sum() and r["mask"][~fc].sum() == 0
    pw = (d.astype(np.int64) ** 2).sum(-1).astype(float)
    m, s = oracle.sigma(P, pw[~fc].ravel(), True)
    assert r["stats"]["median_t"] == m and r["stats"]["sigma_t"] == s
    m_all, _ = oracle.sigma(P, pw.ravel(), True)
    assert m_all != m or fc.sum() == 0


def test_history_hand_worked_sequence():
    P = oracle.default_params(history_min=4, history_len=4, history_k=6.0)
    H = oracle.History(1, P)
    for line in _rows("history_examples.txt"):
        step, cur, flag, staged, ring = [x.strip() for x in line.split("|")]
        d = np.full((1, 8), float(cur), np.float32)
        r = oracle.flag_unit(P, d, history=H)
        assert r["stats"]["n_chan_hist"] == int(flag), step
        assert bool(r["mask"].all()) == bool(int(flag)), step
        assert r["has_pending"][0] == 1 and r["pending"][0] == float(staged), step
        H.commit(0, r["pending"], r["has_pending"])
        want = [float(x) for x in ring.split()]
        assert H.count[0] == len(want)
        assert list(H.ring[0, :len(want)]) == want, step


def test_history_no_test_before_warmup_and_no_stage_when_all_flagged():
    P = oracle.default_params(history_min=3)
    H = oracle.History(1, P)
    for v in (5.0, 5.0, 500.0):   # only two entries stored when the 500 arrives
        r = oracle.flag_unit(P, np.full((1, 4), v, np.float32), history=H)
        assert r["stats"]["n_chan_hist"] == 0
        H.commit(0, r["pending"], r["has_pending"])
    d = np.full((1, 4), np.nan, np.float32)   # nothing unflagged: nothing staged
    r = oracle.flag_unit(P, d, history=H)
    assert r["has_pending"][0] == 0 and r["mask"].all()


def test_f32_non_finite_are_flagged_on_entry():
    P = oracle.default_params(enable_history=0)
    rng = np.random.default_rng(9)
    d = rng.chisquare(4, (8, 64)).astype(np.float32)
    d[3, 7] = np.nan
    d[4, 9] = np.inf
    r = oracle.flag_unit(P, d)
    assert r["mask"][3, 7] == 1 and r["mask"][4, 9] == 1
    assert r["out"][3, 7] == 0 and r["out"][4, 9] == 0
    fin = np.isfinite(d)
    m, _ = oracle.sigma(P, d[fin].astype(float), False)
    assert r["stats"]["median_t"] == m


def test_empty_and_degenerate_units():
    P = oracle.default_params()
    r = oracle.flag_unit(P, np.zeros((0, 10, 2), np.int16))
    assert r["mask"].size == 0
    r = oracle.flag_unit(P, np.zeros((3, 0, 2), np.int16))
    assert r["mask"].size == 0
    r = oracle.flag_unit(P, np.zeros((3, 5, 2), np.int16))   # all zero: nothing flagged
    assert r["mask"].sum() == 0
    r = oracle.flag_unit(P, np.ones((1, 1, 2), np.int8))
    assert r["mask"].sum() == 0
