"""Flagging quality on beamformed Stokes I data (the paper's pulsar
evaluation, Section 5.1): the folded-profile S/N of a seeded dispersed pulsar
after the flagger is above the S/N after no flagging and above the S/N after a
simple per-unit 5-sigma thresholder, as the paper reports for its observation
(it also reports the flagger removing more samples than the thresholder)."""
import pytest

from paper_1701_08197_gb300 import quality

pytestmark = pytest.mark.gpu


def test_flagger_beats_no_flagging_and_the_simple_thresholder():
    res = quality.evaluate(n_subband=64, n_block=4, seed=4)
    print({k: (round(v["snr"], 2), round(v["flagged_fraction"], 4)) for k, v in res.items()})
    lof_snr, raw_snr, thr_snr = res["lof"]["snr"], res["none"]["snr"], res["threshold_5sigma"]["snr"]
    assert lof_snr > raw_snr, res
    assert lof_snr > thr_snr, res
    assert res["lof"]["flagged_fraction"] > res["threshold_5sigma"]["flagged_fraction"], res
    assert res["lof"]["flagged_fraction"] < 0.2, res
    assert res["none"]["flagged_fraction"] == 0.0
