"""Flagging quality on beamformed Stokes I data: folded-profile S/N of a
dispersed pulsar after no flagging, after a simple per-unit 5-sigma
thresholder and after the flagger (the paper's pulsar evaluation, with a
seeded synthetic pulsar standing in for the observed one).

Each block of n_subband x C x T float32 power samples (chi-square(4) noise,
a dispersed pulsar, narrowband and impulsive RFI; see synth.stokes_block) is
flagged, dedispersed and folded into n_bin phase bins: every unflagged
sample adds to the bin of its pulse phase (the arrival time minus the cold
plasma delay of its channel, modulo the period).  The profile is the mean
per bin; S/N = sum over the on-pulse bins of (p - mean_off) /
(std_off * sqrt(N_on)), on-pulse = the bins whose phase lies in the duty
cycle.

  python -m paper_1701_08197_gb300.quality [--subbands N] [--blocks B]
"""
from __future__ import annotations

import argparse
import json
import math

import torch

from . import lof, synth


def pulse_phase(spec: synth.PulsarSpec, block: int, device) -> torch.Tensor:
    """Pulse phase in [0, 1) of every sample, [n_subband, C, T] (float64)."""
    f = synth.stokes_channel_freqs_mhz(spec.n_subband, spec.C).to(device)
    f_hi = float(f.max())
    delay = 4.148808e3 * spec.dm * (f ** -2 - f_hi ** -2)
    t = (torch.arange(spec.T, device=device, dtype=torch.float64) + block * spec.T) * spec.tsamp
    ph = torch.remainder((t[None, :] - delay[:, None]) / spec.period, 1.0)
    return ph.reshape(spec.n_subband, spec.C, spec.T)


def threshold_5sigma(x: torch.Tensor) -> torch.Tensor:
    """Simple thresholder: flag samples above median + 5 * 1.4826 * MAD of
    their unit (one unit = one subband)."""
    flat = x.reshape(x.shape[0], -1)
    med = flat.median(dim=1).values
    mad = (flat - med[:, None]).abs().median(dim=1).values
    thr = med + 5.0 * 1.482602218505602 * mad
    return (x > thr[:, None, None])


class Folder:
    def __init__(self, n_bin: int, device):
        self.n_bin = n_bin
        self.s = torch.zeros(n_bin, dtype=torch.float64, device=device)
        self.n = torch.zeros(n_bin, dtype=torch.float64, device=device)

    def add(self, x: torch.Tensor, flagged: torch.Tensor, phase: torch.Tensor):
        keep = ~flagged
        b = torch.clamp((phase * self.n_bin).long(), 0, self.n_bin - 1)[keep]
        self.s.index_add_(0, b, x[keep].double())
        self.n.index_add_(0, b, torch.ones_like(b, dtype=torch.float64))

    def snr(self, duty: float) -> float:
        p = self.s / torch.clamp(self.n, min=1.0)
        centers = (torch.arange(self.n_bin, device=p.device, dtype=torch.float64) + 0.5) / self.n_bin
        on = centers < duty
        off = ~on
        mu, sd = p[off].mean(), p[off].std()
        return float(((p[on] - mu).sum() / (sd * math.sqrt(int(on.sum())))).item())


def evaluate(n_subband=64, n_block=4, seed=4, n_bin=256, device="cuda:0", flagger=None):
    """Folded S/N for none / 5-sigma thresholder / flagger, and the flagged fractions."""
    dev = torch.device(device)
    spec = synth.PulsarSpec(n_subband=n_subband)
    folders = {k: Folder(n_bin, dev) for k in ("none", "threshold_5sigma", "lof")}
    frac = {k: 0.0 for k in folders}
    own = flagger is None
    fl = flagger or lof.Flagger(dev.index or 0, n_history_slots=n_subband * spec.C)
    try:
        for b in range(n_block):
            x = synth.stokes_block(spec, seed=seed, block=b, device=dev).contiguous()
            ph = pulse_phase(spec, b, dev)
            mask = torch.empty(x.shape, dtype=torch.uint8, device=dev)
            units = [lof.make_unit(x[s], None, mask[s], s * spec.C) for s in range(n_subband)]
            fl.flag_block(lof.LOF_F32, units, b)
            fl.history_update(units)
            fl.status()
            marks = {"none": torch.zeros_like(x, dtype=torch.bool),
                     "threshold_5sigma": threshold_5sigma(x),
                     "lof": mask.bool()}
            for k, m in marks.items():
                folders[k].add(x, m, ph)
                frac[k] += float(m.float().mean().item()) / n_block
    finally:
        if own:
            fl.close()
    return {k: {"snr": folders[k].snr(spec.duty), "flagged_fraction": frac[k]} for k in folders}


def time_block(n_subband=488, seed=4, reps=5, device="cuda:0"):
    """Flag-kernel time of one full Stokes I block (CUDA events, median), as
    in streaming: every unit has its history slots (so the previous block's
    statistics serve as hints) and two distinct blocks alternate."""
    dev = torch.device(device)
    spec = synth.PulsarSpec(n_subband=n_subband)
    xs = [synth.stokes_block(spec, seed=seed, block=b, device=dev).contiguous() for b in (0, 1)]
    out = torch.empty_like(xs[0])
    mask = torch.empty(xs[0].shape, dtype=torch.uint8, device=dev)
    with lof.Flagger(dev.index or 0, n_history_slots=n_subband * spec.C) as fl:
        units = [[lof.make_unit(x[s], out[s], mask[s], s * spec.C) for s in range(n_subband)] for x in xs]
        st = torch.cuda.current_stream()
        for b in (0, 1):
            fl.flag_block(lof.LOF_F32, units[b], b)
        fl.status()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ts = []
        for r in range(reps):
            e0.record(st)
            fl.flag_block(lof.LOF_F32, units[r % 2], 2 + r)
            e1.record(st)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        fl.status()
    x = xs[0]
    ms = sorted(ts)[reps // 2]
    n = x.numel()
    return {"ms": ms, "Msamples_s": n / ms / 1e3, "GBs_9B_per_sample": 9 * n / ms / 1e6}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--subbands", type=int, default=488)
    ap.add_argument("--blocks", type=int, default=8)
    ap.add_argument("--seed", type=int, default=4)
    args = ap.parse_args()
    res = evaluate(args.subbands, args.blocks, args.seed)
    print(json.dumps({"workload": f"Stokes I {args.subbands} sb x 16 ch x 12288 t, {args.blocks} "
                                  f"blocks, chi2(4) noise, pulsar P=0.714 s DM=26.8, seed {args.seed}",
                      "folded_snr": res, "flag_block": time_block(args.subbands, args.seed)}))


if __name__ == "__main__":
    main()
