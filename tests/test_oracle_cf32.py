"""Pins of the oracle's complex float32 (visibility) input: the flagger on
|V|^2 equals the Stokes I path on the same powers."""
import numpy as np

import oracle


def test_complex_input_equals_the_power_path_on_exact_powers():
    # small integer parts: re^2 + im^2 is exact in float32 and binary64
    rng = np.random.default_rng(4)
    re = np.round(rng.normal(0, 20, (24, 1500)))
    im = np.round(rng.normal(0, 20, (24, 1500)))
    re[5, 300:310] = 400
    re[:, 900] = 300
    v = (re + 1j * im).astype(np.complex64)
    pw = (re ** 2 + im ** 2).astype(np.float32)
    P = oracle.default_params()
    rv, rp = oracle.flag_unit(P, v), oracle.flag_unit(P, pw)
    assert np.array_equal(rv["mask"], rp["mask"])
    assert rv["stats"] == rp["stats"]
    assert np.array_equal(rv["out"], np.where(rv["mask"].astype(bool), np.complex64(0), v))


def test_non_finite_parts_flag_the_sample():
    v = np.ones((4, 64), np.complex64)
    v[1, 10] = complex(np.nan, 1.0)
    v[2, 20] = complex(1.0, np.inf)
    r = oracle.flag_unit(oracle.default_params(), v)
    assert r["mask"][1, 10] == 1 and r["mask"][2, 20] == 1
    assert r["out"][1, 10] == 0 and r["out"][2, 20] == 0
