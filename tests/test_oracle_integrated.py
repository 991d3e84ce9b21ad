"""Pins of the oracle's integrated time mode (Section 3: the frequency
direction integrated fully for time-domain flagging)."""
import numpy as np
import pytest

import oracle


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_one_channel_reduces_to_the_per_channel_pass(seed):
    # with a single channel the integrated series is the channel itself, its
    # statistics are the pooled ones and SumThreshold runs on the same values
    rng = np.random.default_rng(seed)
    d = np.round(rng.normal(0, 32, (1, 2000, 2))).astype(np.int16)
    d[0, 500:520] += 150
    d[0, 1500] = (3000, 0)
    r0 = oracle.flag_unit(oracle.default_params(time_mode=0), d)
    r1 = oracle.flag_unit(oracle.default_params(time_mode=1), d)
    assert np.array_equal(r0["mask"], r1["mask"])
    for k in ("median_t", "sigma_t", "n_flag_time", "n_flag_total"):
        assert r0["stats"][k] == r1["stats"][k], k


def test_weak_broadband_impulse_found_only_when_integrated():
    # +4 sigma of amplitude in every channel for 6 samples: each channel's
    # samples stay below the per-channel thresholds, the integrated series
    # (sum over 128 channels) does not
    rng = np.random.default_rng(5)
    d = np.round(rng.normal(0, 32, (128, 1024, 2))).astype(np.int16)
    d[:, 400:406, 0] += 60
    r0 = oracle.flag_unit(oracle.default_params(time_mode=0), d)
    r1 = oracle.flag_unit(oracle.default_params(time_mode=1), d)
    assert r1["mask"][:, 400:406].all()
    assert r0["mask"][:, 400:406].mean() < 0.5
    # the integrated mode flags whole time steps of the kept channels
    cols = r1["mask"].any(axis=0)
    assert np.array_equal(r1["mask"], np.broadcast_to(cols, r1["mask"].shape).astype(np.uint8))


def test_integrated_statistics_are_those_of_the_series():
    rng = np.random.default_rng(8)
    d = np.round(rng.normal(0, 32, (16, 300, 2))).astype(np.int16)
    d[3] += 40                                   # a hot channel the frequency pass removes
    P = oracle.default_params(time_mode=1, enable_time=0)
    r = oracle.flag_unit(P, d)
    p = (d.astype(np.float64) ** 2).sum(-1)
    keep = ~r["mask"].all(axis=1)                # rows the frequency pass kept
    g = p[keep].sum(axis=0)
    med = np.median(g)
    mad = np.median(np.abs(g - med))
    assert r["stats"]["median_t"] == med
    assert abs(r["stats"]["sigma_t"] - 1.482602218505602 * mad) <= 1e-9 * mad
