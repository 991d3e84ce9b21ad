"""Pins of the oracle's per-channel statistics scope: each kept channel's
time pass runs with its own median and sigma."""
import numpy as np

import oracle


def test_channel_scope_runs_each_row_with_its_own_statistics():
    # a unit whose rows differ in level: row by row, the scoped pass equals
    # the pooled pass on that row alone (a one-channel unit, where pooled =
    # the row's own statistics)
    rng = np.random.default_rng(12)
    rows = []
    for c in range(6):
        r = np.round(rng.normal(0, 20 + 10 * c, (1, 800, 2))).astype(np.int16)
        r[0, 100 + 50 * c:104 + 50 * c] += np.int16(8 * (20 + 10 * c))
        rows.append(r)
    d = np.concatenate(rows)
    P = oracle.default_params(stats_scope=1, enable_freq=0)
    r = oracle.flag_unit(P, d)
    n_time = 0
    for c in range(6):
        one = oracle.flag_unit(oracle.default_params(enable_freq=0), rows[c])
        assert np.array_equal(r["mask"][c], one["mask"][0]), c
        n_time += one["stats"]["n_flag_time"]
    assert r["stats"]["n_flag_time"] == n_time
    assert r["stats"]["median_t"] == 0.0 and r["stats"]["sigma_t"] == 0.0


def test_channel_scope_differs_from_pooled_on_uneven_rows():
    # a quiet row next to loud rows: pooled thresholds never fire on its
    # modest burst, its own statistics do
    rng = np.random.default_rng(13)
    d = np.round(rng.normal(0, 200, (16, 1024, 2))).astype(np.int16)
    d[3] = np.round(rng.normal(0, 10, (1024, 2))).astype(np.int16)
    d[3, 500:508] += 120
    pooled = oracle.flag_unit(oracle.default_params(enable_freq=0), d)
    scoped = oracle.flag_unit(oracle.default_params(enable_freq=0, stats_scope=1), d)
    assert scoped["mask"][3, 500:508].all()
    assert not pooled["mask"][3, 500:508].any()
