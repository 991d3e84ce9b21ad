"""Flagging quality on beamformed Stokes I data (the paper's pulsar
evaluation): the folded-profile S/N of a seeded dispersed pulsar improves
when the flagger removes the injected RFI."""
import pytest

from paper_1701_08197_gb300 import quality

pytestmark = pytest.mark.gpu


def test_flagger_raises_folded_snr_over_no_flagging():
    res = quality.evaluate(n_subband=32, n_block=3, seed=4)
    lof_snr, raw_snr = res["lof"]["snr"], res["none"]["snr"]
    assert lof_snr > raw_snr, res
    assert res["lof"]["flagged_fraction"] < 0.2, res
    assert res["none"]["flagged_fraction"] == 0.0
