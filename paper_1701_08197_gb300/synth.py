"""Seeded synthetic inputs shaped like LOFAR / SKA flagger blocks.

This module only draws noise and injects RFI; it contains none of the
flagger's arithmetic.  Both the CUDA path and the oracle consume what it
produces (the oracle gets a host copy of the very same tensors).

Workloads (shapes from the paper: 256-channel pre-correlation blocks of
~1.3 ms samples, Section 3; 16-channel subbands at 12 kHz / 82 us for the
beam-formed pulsar data, Section 5.1):

* complex voltages: re, im ~ round(N(0, sigma^2)) clipped to the integer range;
  narrowband tones (constant amplitude a*sigma, a ~ U[10, 40], random start
  phase and per-channel phase rate) in a fraction of the channels;
  broadband impulses (all channels of a station, 1..64 samples, amplitude
  U[5, 50]*sigma, random phase per sample); optionally one fully contaminated
  block (extra complex noise of 2*sigma per component, i.e. 5x the power).
* Stokes I: chi-square(4) noise (mean 4, std sqrt 8), a dispersed pulsar and
  narrowband / impulsive RFI added in power.

Everything is drawn with torch.Generator on the requested device, so large
workloads are generated on the GPU in milliseconds.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import torch


def _gen(seed: int, device) -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(int(seed) & 0x7FFFFFFFFFFFFFFF)
    return g


def _mix(*xs: int) -> int:
    """Derive a sub-seed from integers (splitmix64 finaliser)."""
    h = 0x9E3779B97F4A7C15
    for x in xs:
        h = (h ^ (int(x) & 0xFFFFFFFFFFFFFFFF)) & 0xFFFFFFFFFFFFFFFF
        h = (h * 0xBF58476D1CE4E5B9) & 0xFFFFFFFFFFFFFFFF
        h ^= h >> 31
        h = (h * 0x94D049BB133111EB) & 0xFFFFFFFFFFFFFFFF
        h ^= h >> 29
    return h & 0x7FFFFFFFFFFFFFFF


@dataclass
class VoltageSpec:
    n_station: int = 1
    n_pol: int = 1
    n_subband: int = 1
    C: int = 256
    T: int = 768
    dtype: torch.dtype = torch.int16
    sigma: float = 32.0
    tone_frac: float = 0.0          # per-channel probability of a tone (per station, subband)
    n_tones: int | None = None      # or an exact tone count per (station, subband)
    impulse_frac: float = 0.0       # expected fraction of samples covered by impulses
    n_impulses: int | None = None   # or an exact impulse count per station
    impulse_amp: tuple = (5.0, 50.0)
    tone_amp: tuple = (10.0, 40.0)
    contaminated: bool = False      # add 2*sigma complex noise to the whole block
    extra: dict = field(default_factory=dict)


def voltage_block(spec: VoltageSpec, seed: int, block: int, device="cpu", return_truth=False):
    """One block of complex voltages, shape [station, pol, subband, C, T, 2]."""
    dev = torch.device(device)
    S, Pn, B, C, T = spec.n_station, spec.n_pol, spec.n_subband, spec.C, spec.T
    g = _gen(_mix(seed, block, 1), dev)
    re = torch.randn((S, Pn, B, C, T), generator=g, device=dev, dtype=torch.float32) * spec.sigma
    im = torch.randn((S, Pn, B, C, T), generator=g, device=dev, dtype=torch.float32) * spec.sigma
    truth = torch.zeros((S, Pn, B, C, T), dtype=torch.float32, device=dev) if return_truth else None
    if spec.contaminated:
        re += torch.randn(re.shape, generator=g, device=dev) * (2.0 * spec.sigma)
        im += torch.randn(im.shape, generator=g, device=dev) * (2.0 * spec.sigma)
    # narrowband tones: the same channels in both polarisations of a station-subband;
    # constant over the observation (seeded without the block index)
    gt = _gen(_mix(seed, 2), dev)
    if spec.n_tones is not None:
        sel = torch.zeros((S, B, C), dtype=torch.bool, device=dev)
        for s in range(S):
            for b in range(B):
                idx = torch.randperm(C, generator=gt, device=dev)[: spec.n_tones]
                sel[s, b, idx] = True
    else:
        sel = torch.rand((S, B, C), generator=gt, device=dev) < spec.tone_frac
    amp = (spec.tone_amp[0] + (spec.tone_amp[1] - spec.tone_amp[0]) *
           torch.rand((S, B, C), generator=gt, device=dev)) * spec.sigma
    ph0 = torch.rand((S, B, C), generator=gt, device=dev) * (2 * math.pi)
    rate = (torch.rand((S, B, C), generator=gt, device=dev) - 0.5) * 0.2
    if bool(sel.any()):
        t = torch.arange(T, device=dev, dtype=torch.float32) + float(block * T)
        phase = ph0[..., None] + 2 * math.pi * rate[..., None] * t  # [S,B,C,T]
        a = (amp * sel)[..., None]
        re += (a * torch.cos(phase))[:, None]
        im += (a * torch.sin(phase))[:, None]
        if truth is not None:
            truth = torch.maximum(truth, (amp / spec.sigma * sel)[:, None, :, :, None].expand_as(truth))
    # broadband impulses per station: all subbands, pols and channels
    gi = _gen(_mix(seed, block, 3), dev)
    for s in range(S):
        if spec.n_impulses is not None:
            n_imp = spec.n_impulses
        else:
            lam = spec.impulse_frac * T / 32.5
            n_imp = int(torch.poisson(torch.tensor([lam], dtype=torch.float32), generator=_gen(_mix(seed, block, s, 4), "cpu")).item()) if lam > 0 else 0
        for _ in range(n_imp):
            dur = int(torch.randint(1, 65, (1,), generator=gi, device=dev).item())
            start = int(torch.randint(0, max(1, T - dur + 1), (1,), generator=gi, device=dev).item())
            A = (spec.impulse_amp[0] + (spec.impulse_amp[1] - spec.impulse_amp[0]) *
                 torch.rand((1,), generator=gi, device=dev).item()) * spec.sigma
            ph = torch.rand((Pn, B, C, dur), generator=gi, device=dev) * (2 * math.pi)
            re[s, :, :, :, start:start + dur] += A * torch.cos(ph)
            im[s, :, :, :, start:start + dur] += A * torch.sin(ph)
            if truth is not None:
                truth[s, :, :, :, start:start + dur] = torch.maximum(
                    truth[s, :, :, :, start:start + dur], torch.tensor(A / spec.sigma, device=dev))
    info = torch.iinfo(spec.dtype)
    out = torch.stack([re, im], dim=-1).round_().clamp_(info.min, info.max).to(spec.dtype)
    if return_truth:
        return out, truth
    return out


def stokes_channel_freqs_mhz(n_subband: int, n_chan: int, f0_mhz=100.0, df_khz=12.207):
    """Channel centre frequencies: f = f0 + (n_chan*s + c + 1/2) * df."""
    k = torch.arange(n_subband * n_chan, dtype=torch.float64)
    return f0_mhz + (k + 0.5) * df_khz * 1e-3


@dataclass
class PulsarSpec:
    n_subband: int = 488
    C: int = 16
    T: int = 12288
    tsamp: float = 81.92e-6
    period: float = 0.714
    dm: float = 26.8
    duty: float = 0.05
    snr_per_sample: float = 0.05    # in units of the noise std (sqrt 8)
    rfi_chan_frac: float = 0.02
    rfi_chan_amp: tuple = (0.5, 3.0)   # in units of the noise mean, added in power
    rfi_impulse_frac: float = 0.01
    rfi_impulse_amp: tuple = (5.0, 50.0)  # in units of the noise std


def pulsar_on(spec: PulsarSpec, block: int, device="cpu"):
    """Boolean [n_subband, C, T]: is the (dispersed) pulse on at each sample."""
    dev = torch.device(device)
    f = stokes_channel_freqs_mhz(spec.n_subband, spec.C).to(dev)
    f_hi = float(f.max())
    delay = 4.148808e3 * spec.dm * (f ** -2 - f_hi ** -2)  # seconds
    t = (torch.arange(spec.T, device=dev, dtype=torch.float64) + block * spec.T) * spec.tsamp
    phase = torch.remainder((t[None, :] - delay[:, None]) / spec.period, 1.0)
    return (phase < spec.duty).reshape(spec.n_subband, spec.C, spec.T)


def stokes_block(spec: PulsarSpec, seed: int, block: int, device="cpu", with_pulsar=True,
                 with_rfi=True, return_truth=False):
    """Stokes I power [n_subband, C, T] float32: chi2(4) noise + pulsar + RFI."""
    dev = torch.device(device)
    g = _gen(_mix(seed, block, 11), dev)
    shape = (spec.n_subband, spec.C, spec.T)
    x = torch.zeros(shape, device=dev, dtype=torch.float32)
    for _ in range(4):
        z = torch.randn(shape, generator=g, device=dev, dtype=torch.float32)
        x += z * z
    sd = math.sqrt(8.0)
    if with_pulsar:
        x += pulsar_on(spec, block, dev).to(torch.float32) * (spec.snr_per_sample * sd)
    truth = torch.zeros(shape, dtype=torch.bool, device=dev) if return_truth else None
    if with_rfi:
        gr = _gen(_mix(seed, 12), dev)
        sel = torch.rand((spec.n_subband, spec.C), generator=gr, device=dev) < spec.rfi_chan_frac
        amp = spec.rfi_chan_amp[0] + (spec.rfi_chan_amp[1] - spec.rfi_chan_amp[0]) * \
            torch.rand((spec.n_subband, spec.C), generator=gr, device=dev)
        x += (sel * amp * 4.0)[..., None]
        gi = _gen(_mix(seed, block, 13), dev)
        n_imp = max(0, int(round(spec.rfi_impulse_frac * spec.T / 32.5)))
        for _ in range(n_imp):
            dur = int(torch.randint(1, 65, (1,), generator=gi, device=dev).item())
            start = int(torch.randint(0, max(1, spec.T - dur + 1), (1,), generator=gi, device=dev).item())
            A = (spec.rfi_impulse_amp[0] + (spec.rfi_impulse_amp[1] - spec.rfi_impulse_amp[0]) *
                 torch.rand((1,), generator=gi, device=dev).item()) * sd
            x[:, :, start:start + dur] += A
            if truth is not None:
                truth[:, :, start:start + dur] = True
        if truth is not None:
            truth |= sel[..., None]
    if return_truth:
        return x, truth
    return x


def random_units(n_units: int, C_choices, T_choices, seed: int, device="cpu"):
    """Shapes for a batch of uneven units: list of (C, T), drawn from a seed."""
    g = torch.Generator().manual_seed(_mix(seed, 21))
    Ci = torch.randint(0, len(C_choices), (n_units,), generator=g)
    Ti = torch.randint(0, len(T_choices), (n_units,), generator=g)
    return [(int(C_choices[a]), int(T_choices[b])) for a, b in zip(Ci.tolist(), Ti.tolist())]
