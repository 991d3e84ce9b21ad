"""CPU checks of the float parity rule (tests/float_parity.py): the binary64
replay follows the oracle's SumThreshold, marks exactly the near-threshold
windows when nothing else is uncertain, and propagates uncertainty only
through windows whose decision the uncertain samples can flip."""
import numpy as np

import oracle
from float_parity import allowed_differences, replay

P = oracle.default_params()


def test_replay_flags_follow_the_oracle_on_random_rows():
    rng = np.random.default_rng(5)
    for trial in range(20):
        T = int(rng.integers(1, 700))
        x = (rng.chisquare(4, (3, T))).astype(np.float32)
        x[rng.integers(0, 3), rng.integers(0, T)] = 60.0
        ref = oracle.flag_unit(P, x)
        entry = ~np.isfinite(x)
        allowed, _, _, _ = allowed_differences(P, x.astype(np.float64), entry, ref["stats"])
        # replaying with the oracle's statistics gives the oracle's mask, up to
        # the uncertain samples (summation order of binary64 sums)
        Pz = x.astype(np.float64)
        spec = Pz.sum(axis=1)
        fc, _, _ = replay(P, spec, np.zeros(3, bool), ref["stats"]["median_f"], ref["stats"]["sigma_f"])
        for c in range(3):
            if fc[c]:
                assert ref["mask"][c].all()
                continue
            fl, unc, _ = replay(P, Pz[c], entry[c], ref["stats"]["median_t"], ref["stats"]["sigma_t"])
            d = fl != ref["mask"][c].astype(bool)
            assert not (d & ~unc).any(), (trial, c)


def test_near_threshold_sample_and_its_cascade():
    # m = 0, sigma = 1: T_1 = 6, T_2 = 4.5.  Sample 0 lies within 1e-5 of T_1
    # (near); if it is flagged, window [0, 1] sums 4.5 + 4 = 8.5 < 9 = 2 T_2
    # (no fire, far from the band), if not, 6.00003 + 4 > 9 (fire): sample 1
    # is a cascade, not a near sample.  The samples far away are certain.
    v = np.array([6.00003, 4.0, 0.0, 0.0, 0.0, 0.0, 7.0, 0.0, 0.0, 0.0, 0.0, 0.0])
    fl, unc, near = replay(P, v, np.zeros(v.size, bool), 0.0, 1.0)
    assert near[0] and not near[1]
    assert unc[0] and unc[1]
    assert not unc[2:].any()
    assert fl[6] and not unc[6]          # 7 > 6 by far: flagged on both sides


def test_uncertain_sample_that_cannot_flip_a_window_is_no_cascade():
    # sample 0 is near T_1 again, but its window of two with a zero neighbour
    # stays far below 2 T_2 either way: no cascade
    v = np.array([6.00003, 0.0, 0.0, 0.0])
    _, unc, near = replay(P, v, np.zeros(v.size, bool), 0.0, 1.0)
    assert unc[0] and near[0]
    assert not unc[1:].any()


def test_counts_split_near_and_cascade():
    x = np.zeros((2, 12), np.float64)
    x[0] = [6.00003, 4.0, 0, 0, 0, 0, 7.0, 0, 0, 0, 0, 0]
    stats = {"median_f": 0.0, "sigma_f": 0.0, "median_t": 0.0, "sigma_t": 1.0}
    allowed, fc_unc, n_near, n_casc = allowed_differences(P, x, np.zeros(x.shape, bool), stats)
    assert not fc_unc.any()
    assert n_near == 1 and n_casc == 1
    assert allowed[0, :2].all() and not allowed[1].any()
