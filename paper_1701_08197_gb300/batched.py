"""Batched uneven units: every station x polarisation x subband of a block,
with mixed channel counts {16, 64, 256} and block lengths {768, 3072, 12288}
drawn per subband from a seed (shared by the stations and polarisations of
the subband), complex int8 (sigma 8, saturated), flagged by ONE persistent
launch captured in a CUDA graph, with the launch shape picked by the
autotuner -- against the same units flagged by one launch per unit.

  python -m paper_1701_08197_gb300.batched [--subbands N] [--stations S]
"""
from __future__ import annotations

import argparse
import json

import torch

from . import lof, synth


def build(n_subband=61, n_station=48, seed=3, device="cuda:0", block=0):
    """Device tensors of one block: per subband one [S, 2, C, T, 2] int8 tensor
    (the shapes depend on the seed only, the samples on the block index too)."""
    shapes = synth.random_units(n_subband, (16, 64, 256), (768, 3072, 12288), seed=seed)
    xs = []
    for b, (C, T) in enumerate(shapes):
        spec = synth.VoltageSpec(n_station=n_station, n_pol=2, n_subband=1, C=C, T=T,
                                 dtype=torch.int8, sigma=8.0, tone_frac=0.02, impulse_frac=0.01)
        xs.append(synth.voltage_block(spec, seed=synth._mix(seed, b), block=block, device=device)[:, :, 0])
    return xs


def units_of(xs, outs, masks, history=False):
    """Descriptors of every station x pol of every subband; with history,
    each unit owns its channels' history slots (consecutive), so the
    statistics of one block serve as hints for the next."""
    out = []
    slot = 0
    for x, o, m in zip(xs, outs, masks):
        for s in range(x.shape[0]):
            for p in range(2):
                out.append(lof.make_unit(x[s, p], o[s, p], m[s, p], slot if history else -1))
                slot += x.shape[2]
    return out


def time_ms(fn, reps, stream):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ts = []
    for _ in range(reps):
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    ts.sort()
    return ts[len(ts) // 2]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--subbands", type=int, default=61)
    ap.add_argument("--stations", type=int, default=48)
    ap.add_argument("--reps", type=int, default=5)
    args = ap.parse_args()
    dev = torch.device("cuda", 0)
    xs = build(args.subbands, args.stations, device=dev)
    outs = [torch.empty_like(x) for x in xs]
    masks = [torch.empty(x.shape[:-1], dtype=torch.uint8, device=dev) for x in xs]
    units = units_of(xs, outs, masks)
    samples = sum(int(x.numel() // 2) for x in xs)
    st = torch.cuda.current_stream()
    res = {"workload": f"{args.subbands} subbands x {args.stations} stations x 2 pols = {len(units)} "
                       f"uneven units (C in 16/64/256, T in 768/3072/12288), complex int8",
           "samples": samples}
    with lof.Flagger(0) as fl:
        default_ms = time_ms(lambda: fl.flag_block(lof.LOF_CI8, units, 0), args.reps, st)
        tuning, tuned_ms = fl.autotune(lof.LOF_CI8, units, reps=2)
        with fl.graph(lof.LOF_CI8, units) as g:
            g.launch(0)
            g.status()
            graph_ms = time_ms(lambda: g.launch(1), args.reps, st)
            g.status()
        # one launch per unit (the plain, per-block form)
        fl.set_tuning(threads=128, ctas_per_sm=4, flag_rows=16, stat_samples=65536)
        plain_ms = time_ms(lambda: [fl.flag_block(lof.LOF_CI8, [u], 0) for u in units], 2, st)
        fl.status()
    alg_bytes = samples * 5
    res.update({
        "batched_default_ms": default_ms, "autotuned": tuning, "autotuned_ms": tuned_ms,
        "graph_ms": graph_ms, "plain_per_unit_ms": plain_ms,
        "graph_Msamples_s": samples / graph_ms / 1e3,
        "graph_GBs": alg_bytes / graph_ms / 1e6,
        "plain_vs_graph": plain_ms / graph_ms,
    })
    print(json.dumps(res))


if __name__ == "__main__":
    main()
