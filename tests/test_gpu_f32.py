"""Float32 Stokes I units (power given): GPU path against the oracle.

Parity rule for float inputs (the float contract of the Stokes I path): the
spectrum and pooled statistics agree within 1e-6 relative; a mask may differ
only on samples the binary64 replay of tests/float_parity.py marks uncertain:
samples of windows whose substituted sum lies within 1e-5 relative of its
threshold I * T_I (near), and samples of later windows whose sums those
uncertain samples can move across that band (cascade).  Any other difference
fails.  Both counts are reported for every unit (pytest warnings summary).
The data output must equal the input with the GPU's own mask applied."""
import warnings

import numpy as np
import pytest
import torch

import oracle
from paper_1701_08197_gb300 import lof, synth

from float_parity import allowed_differences

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
REL_STATS = 1e-6


class FloatParityCounts(UserWarning):
    """near-threshold / cascade / differing sample counts of a float unit"""


def _check_unit(p, x, res_gpu_mask, res_gpu_out, gpu_stats, ref, tag=""):
    """x: float32 powers [C, T] (non-finite = flagged on entry).  Returns
    (differing samples, near-threshold samples, cascade samples)."""
    C, T = x.shape
    rs = ref["stats"]
    entry = ~np.isfinite(x)
    P = np.where(entry, 0.0, x.astype(np.float64))
    allowed, fc_unc, n_near, n_casc = allowed_differences(p, P, entry, rs)
    # the statistics are compared unless a channel's frequency decision is
    # itself uncertain and the two sides took it differently (the pooled set
    # then differs by that channel)
    if not (fc_unc.any() and gpu_stats["n_chan_freq"] != rs["n_chan_freq"]):
        for key in ("median_f", "sigma_f", "median_t", "sigma_t"):
            a, b = gpu_stats[key], rs[key]
            assert abs(a - b) <= REL_STATS * max(abs(b), 1e-30), (tag, key, a, b)
    diff = res_gpu_mask != ref["mask"]
    bad = diff & ~allowed
    assert not bad.any(), f"{tag}: {int(bad.sum())} differing samples outside the uncertain set " \
                          f"(first at {np.argwhere(bad)[:3].tolist()})"
    # the output is the input with the GPU mask applied
    exp = np.where(res_gpu_mask.astype(bool), np.float32(0), x)
    assert np.array_equal(res_gpu_out.view(np.uint32), exp.view(np.uint32))
    nd = int(diff.sum())
    warnings.warn(FloatParityCounts(f"{tag} {C}x{T}: near_threshold_count={n_near} "
                                    f"cascade_count={n_casc} differing={nd}"))
    return nd, n_near, n_casc


def _stokes(seed, C, T, nonfinite=0):
    spec = synth.PulsarSpec(n_subband=1, C=C, T=T)
    x = synth.stokes_block(spec, seed=seed, block=0, device="cpu")[0].numpy().copy()
    rng = np.random.default_rng(seed)
    for _ in range(nonfinite):
        x[rng.integers(0, C), rng.integers(0, T)] = rng.choice([np.nan, np.inf, -np.inf])
    return x.astype(np.float32)


def _run_gpu(fl, xs, p=None):
    ins = [torch.as_tensor(x).to(DEV) for x in xs]
    outs = [torch.full_like(t, 7.0) for t in ins]
    masks = [torch.full(t.shape, 9, dtype=torch.uint8, device=DEV) for t in ins]
    stats = lof.stats_tensor(len(xs), DEV)
    units = [lof.make_unit(i, o, m, -1, stats[k]) for k, (i, o, m) in enumerate(zip(ins, outs, masks))]
    fl.flag_block(lof.LOF_F32, units, 0)
    fl.status()
    return ([m.cpu().numpy() for m in masks], [o.cpu().numpy() for o in outs],
            [lof.decode_stats(s) for s in stats.cpu()])


@pytest.mark.parametrize("shape", [(16, 12288), (13, 1000), (64, 3072), (1, 37), (5, 1)])
def test_f32_matches_oracle_within_tolerance(shape):
    C, T = shape
    xs = [_stokes(100 + i, C, T, nonfinite=3 if T > 1 else 0) for i in range(2)]
    p = oracle.default_params()
    with lof.Flagger(0) as fl:
        masks, outs, stats = _run_gpu(fl, xs)
    for k, x in enumerate(xs):
        ref = oracle.flag_unit(p, x)
        nd, nn, nc = _check_unit(p, x, masks[k], outs[k], stats[k], ref, tag=f"f32 unit {k}")
        assert nd <= nn + nc
        if T > 1:
            assert ref["mask"].sum() > 0


def test_f32_nonfinite_samples_are_flagged_and_zeroed():
    x = _stokes(7, 8, 2048)
    x[3, 100] = np.nan
    x[5, 7] = np.inf
    with lof.Flagger(0) as fl:
        masks, outs, _ = _run_gpu(fl, [x])
    assert masks[0][3, 100] == 1 and masks[0][5, 7] == 1
    assert outs[0][3, 100] == 0.0 and outs[0][5, 7] == 0.0


def test_f32_pure_noise_thresholds_flag_little():
    # chi-square(4) noise without RFI: the flag fraction stays near the method's
    # own false-alarm rate (well below 5 %)
    spec = synth.PulsarSpec(n_subband=1, C=16, T=12288)
    x = synth.stokes_block(spec, seed=3, block=0, device="cpu", with_pulsar=False,
                           with_rfi=False)[0].numpy().astype(np.float32)
    with lof.Flagger(0) as fl:
        masks, _, st = _run_gpu(fl, [x])
    frac = masks[0].mean()
    assert frac < 0.05, frac
    assert st[0]["n_chan_freq"] == 0


@pytest.mark.parametrize("shape", [(16, 12288), (13, 1000), (256, 768), (1, 37), (17, 4096)])
def test_cluster_and_single_cta_kernels_agree(shape):
    """LOF_SCHED_F32_CLUSTER on (one thread-block cluster per unit, the unit in
    shared memory) and off (one CTA per unit): the same row sums, order
    statistics and window sums, so bit-identical masks, data and statistics."""
    C, T = shape
    xs = [_stokes(300 + i, C, T, nonfinite=2 if T > 1 else 0) for i in range(3)]
    res = {}
    for on in (0, lof.LOF_SCHED_F32_CLUSTER):
        with lof.Flagger(0) as fl:
            t = fl.tuning()
            fl.set_tuning(schedule=(t["schedule"] & ~lof.LOF_SCHED_F32_CLUSTER) | on)
            res[on] = _run_gpu(fl, xs)
    (ma, oa, sa), (mb, ob, sb) = res[0], res[lof.LOF_SCHED_F32_CLUSTER]
    for k in range(len(xs)):
        assert np.array_equal(ma[k], mb[k]), f"unit {k}: masks differ"
        assert np.array_equal(oa[k].view(np.uint32), ob[k].view(np.uint32)), f"unit {k}: data differ"
        assert sa[k] == sb[k], (k, sa[k], sb[k])


def test_cluster_kernel_std_estimator_within_tolerance():
    """The std estimator's binary64 sums follow the cluster's CTAs: within the
    float rule against the oracle."""
    xs = [_stokes(400, 16, 12288)]
    p = oracle.default_params(sigma_estimator=1)
    with lof.Flagger(0, sigma_estimator=lof.LOF_SIGMA_STD) as fl:
        masks, outs, stats = _run_gpu(fl, xs)
    ref = oracle.flag_unit(p, xs[0])
    _check_unit(p, xs[0], masks[0], outs[0], stats[0], ref, tag="f32 cluster std")


def test_hinted_window_selection_equals_radix_selection():
    """Units with history slots take the previous block's median and MAD as
    hints (two window passes each); without slots, the three radix passes.
    Both give the same order statistics, so identical results, on a hit
    (block 1 after block 0), a miss (block 2 scaled by 10) and again a hit."""
    C, T = 16, 12288
    xs = {}
    for b in range(4):
        spec = synth.PulsarSpec(n_subband=3, C=C, T=T)
        x = synth.stokes_block(spec, seed=77, block=b, device="cpu").numpy().astype(np.float32)
        xs[b] = x * (10.0 if b == 2 else 1.0)
    with lof.Flagger(0, n_history_slots=3 * C, enable_history=0) as fa, \
            lof.Flagger(0, enable_history=0) as fb:
        for b in range(4):
            ins = [torch.as_tensor(xs[b][s]).to(DEV) for s in range(3)]
            res = []
            for fl, slots in ((fa, True), (fb, False)):
                masks = [torch.empty(t.shape, dtype=torch.uint8, device=DEV) for t in ins]
                stats = lof.stats_tensor(3, DEV)
                units = [lof.make_unit(ins[s], None, masks[s], s * C if slots else -1, stats[s]) for s in range(3)]
                fl.flag_block(lof.LOF_F32, units, b)
                fl.status()
                res.append(([m.cpu().numpy() for m in masks], [lof.decode_stats(s) for s in stats.cpu()]))
            (ma, sa), (mb, sb) = res
            for s in range(3):
                assert np.array_equal(ma[s], mb[s]), f"block {b} unit {s}: masks differ"
                assert sa[s] == sb[s], (b, s, sa[s], sb[s])
