"""Parity rule of the float paths (Stokes I, visibilities): which flag
differences between the GPU (float32 window sums and statistics) and the
oracle (binary64) the arithmetic allows, and how many samples that covers.

SumThreshold (Section 2.1) is replayed here in binary64, level by level, on
the oracle's own statistics.  Every sample carries the oracle's flag and an
"uncertain" mark.  For each window the substituted sum is bounded over the
states the uncertain samples may take on the GPU (flagged: threshold_I,
unflagged: the power): S_lo and S_hi.  A window's decision is
  * certain to fire when S_lo > I * T_I (1 + rel),
  * certain not to fire when S_hi <= I * T_I (1 - rel),
  * uncertain otherwise; its samples become uncertain, unless a certain
    firing window of the same level covers them.
With no uncertain sample in the window, S_lo = S_hi = the oracle's sum and
this is the near-threshold rule: the sum lies within rel of I * T_I.  A
window with uncertain samples is uncertain only when those samples can move
its sum across that band (the cascade), not merely because it overlaps them.

near  = samples covered by a window whose oracle sum is within rel of its
        threshold;
cascade = the other uncertain samples (reached through cascaded windows).
The frequency pass is replayed the same way over the spectrum; an uncertain
channel may differ as a whole row.  This module holds none of the CUDA
path's code; it is test infrastructure beside the oracle.
"""
from __future__ import annotations

import numpy as np

REL_NEAR = 1e-5


def factor(p, k):
    """Section 2.1: start_threshold * p^k / 2^k, p^k by k products."""
    pk = 1.0
    for _ in range(k):
        pk = pk * p.p
    return p.start_threshold * pk / float(1 << k)


def threshold(p, m, s, k):
    return m + (s * factor(p, k)) * p.sensitivity


def _cover(starts: np.ndarray, I: int, L: int) -> np.ndarray:
    """Samples covered by windows of I starting where starts is True."""
    d = np.zeros(L + 1, np.int64)
    idx = np.nonzero(starts)[0]
    np.add.at(d, idx, 1)
    np.add.at(d, idx + I, -1)
    return np.cumsum(d[:L]) > 0


def replay(p, v: np.ndarray, entry: np.ndarray, m: float, s: float, rel: float = REL_NEAR):
    """SumThreshold over one sequence with uncertainty propagation.

    v: binary64 values (powers; anything at entry-flagged positions),
    entry: flagged on entry (certain on both sides).
    Returns (oracle flags, uncertain, near)."""
    L = len(v)
    flags = entry.copy()        # the oracle's flags
    sure = entry.copy()         # flagged on both sides (flags never clear)
    unc = np.zeros(L, bool)     # may differ between the two sides
    near = np.zeros(L, bool)
    if not (s > 0) or L == 0:
        return flags, unc, near
    k = 0
    while (1 << k) <= min(p.max_window, L):
        I = 1 << k
        t = threshold(p, m, s, k)
        lim = I * t
        band = rel * abs(lim)
        sub = np.where(flags, t, v)                     # the oracle's substituted values
        lo_v = np.where(unc, np.minimum(v, t), sub)     # either state of an uncertain sample
        hi_v = np.where(unc, np.maximum(v, t), sub)

        def wsum(a):
            c = np.concatenate([[0.0], np.cumsum(a)])
            return c[I:] - c[:-I]

        S, S_lo, S_hi = wsum(sub), wsum(lo_v), wsum(hi_v)
        fire = S > lim
        fires_sure = S_lo > lim + band
        maybe = ~fires_sure & (S_hi > lim - band)
        near |= _cover(np.abs(S - lim) <= band, I, L)
        sure |= _cover(fires_sure, I, L)
        unc = (unc | _cover(maybe, I, L)) & ~sure
        flags = flags | _cover(fire, I, L)
        k += 1
    return flags, unc, near


def allowed_differences(p, P: np.ndarray, entry: np.ndarray, stats: dict, rel: float = REL_NEAR):
    """Uncertain samples of a [C, T] float unit under the oracle's statistics
    (median_f, sigma_f, median_t, sigma_t), and the near / cascade counts.
    P: binary64 powers, entry: flagged on entry.  Returns (allowed [C, T],
    uncertain channels [C], near count, cascade count)."""
    C, T = P.shape
    Pz = np.where(entry, 0.0, P)
    spec = Pz.sum(axis=1)
    fc, fc_unc, fc_near = replay(p, spec, np.zeros(C, bool), stats["median_f"], stats["sigma_f"], rel)
    if not p.enable_freq:
        fc = np.zeros(C, bool)
        fc_unc = np.zeros(C, bool)
        fc_near = np.zeros(C, bool)
    allowed = np.zeros((C, T), bool)
    near = np.zeros((C, T), bool)
    for c in range(C):
        if fc_unc[c]:
            allowed[c] = True
            near[c] = fc_near[c]
            continue
        if fc[c] or not p.enable_time:
            continue
        _, unc, nr = replay(p, P[c], entry[c], stats["median_t"], stats["sigma_t"], rel)
        allowed[c] = unc
        near[c] = nr
    n_near = int(near.sum())
    n_cascade = int((allowed & ~near).sum())
    return allowed, fc_unc, n_near, n_cascade
