"""Benchmark: LOFAR Online Flagger hot path on GB300.

Workload (one "step" = one block of the full LOFAR pre-beamformer
configuration through the whole hot path): 48 stations x 2 polarisations x 8
subbands = 768 units of 256 channels x 3072 samples of complex int16 voltages
(sigma 32, seeded tones and broadband impulses), flagged by ONE persistent
launch (lof_flag_block), followed by the history commit (lof_history_update)
with rings pre-filled to 60 means.  Inputs (2.4 GB) stay resident in HBM and
are larger than L2, so no flush is needed between steps.

Reported: input Msamples/s (value), the same through the host-buffer entry
point with PCIe/C2C copies inside the timed region (e2e), the HBM roofline
fraction of the flag kernel, the oracle timed on the host cores
(cpu_baseline), per-step p50/p99 latency of the batched launch against the
plain form (one launch per station-subband), clocks during the timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Options of the method, each timed on the same block (the oracle legs take
them too): --sir P (Section 2.2 SIR operator), --integrated (Section 3
integrated time flagging), --channel-scope (per-channel time-pass
statistics), --sigma {mad,std,winsor} (Section 4.2 estimators), --grid FxT
(two-dimensional SumThreshold on F x T cells).  The launch shape is the
library default unless --autotune.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_STATION, N_POL, N_SUBBAND, C, T = 48, 2, 8, 256, 3072
BYTES_PER_SAMPLE = 4 + 4 + 1          # ci16 in + ci16 out + uint8 mask
METRIC = "input Msamples/s (full LOFAR pre-beamformer block, 768 units x 256 ch x 3072 t, ci16)"


PROFILE = os.path.join(ROOT, "profiles", "lof_block_kernel_ci16_full_station.md")


def measured_traffic(n_units, tuning):
    """DRAM bytes per launch of the block kernel from the committed ncu summary
    (read + write bytes per unit x units), or None when the kernel sources or
    the launch shape differ from the ones the counters were taken with."""
    import hashlib
    try:
        text = open(PROFILE).read()
    except OSError:
        return None
    kv = {}
    inside = False
    for line in text.splitlines():
        if line.startswith("```counters"):
            inside = True
        elif line.startswith("```"):
            inside = False
        elif inside and ":" in line:
            k, v = line.split(":", 1)
            kv[k.strip()] = v.strip()
    csrc = os.path.join(ROOT, "paper_1701_08197_gb300", "csrc")
    for f, key in (("lof_kernels.cu", "kernel_sha256_lof_kernels_cu"),
                   ("lof_internal.h", "kernel_sha256_lof_internal_h")):
        h = hashlib.sha256(open(os.path.join(csrc, f), "rb").read()).hexdigest()
        if kv.get(key) != h:
            return None
    def shape(t):
        # resident CTAs per SM are capped by the kernel's launch bounds
        cap = 4 if int(t["threads"]) == 128 else 2
        return (int(t["threads"]), min(int(t["ctas_per_sm"]), cap), int(t["tile_bytes"]),
                int(t["fine_bins"]), int(t["flag_rows"]), int(t["stat_samples"]),
                int(t.get("schedule", -1)))
    try:
        taken = dict(f.split("=") for f in kv["tuning"].split())
        if shape(taken) != shape(tuning):
            return None
        return int(kv["traffic_bytes_per_unit"]) * n_units
    except (KeyError, ValueError):
        return None


SIGMA = {"mad": 0, "std": 1, "winsor": 2}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--autotune", action="store_true",
                    help="time with the autotuner's launch shape instead of the library default "
                         "(the shape the recorded DRAM counters were taken with)")
    ap.add_argument("--no-autotune", action="store_true", help="the default; kept for old command lines")
    ap.add_argument("--integrated", action="store_true",
                    help="integrated time mode (Section 3): one SumThreshold on the frequency-"
                         "integrated series of the kept channels instead of one per channel")
    ap.add_argument("--channel-scope", action="store_true",
                    help="per-channel statistics scope: each kept channel's time pass with the "
                         "median and sigma of its own samples instead of the pooled ones")
    ap.add_argument("--grid", default=None, metavar="FxT",
                    help="two-dimensional mode on cells of F channels x T samples (e.g. 4x16)")
    ap.add_argument("--sigma", default="mad", choices=list(SIGMA),
                    help="sigma estimator of the statistics (Section 4.2): 1.4826 * MAD, "
                         "population stddev or winsorized stddev")
    ap.add_argument("--sir", type=int, default=0,
                    help="SIR operator percentage (Section 2.2) on the final mask; 0 = off")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--stations", type=int, default=48,
                    help="stations per block (48 = the full configuration; fewer for profiling)")
    ap.add_argument("--no-configs", dest="configs", action="store_false",
                    help="skip the legs of the other configurations (batched uneven, Stokes I, serving)")
    ap.add_argument("--same-block", action="store_true",
                    help="flag one block every step (the statistics hints then always hit); the "
                         "default alternates two distinct seeded blocks, as a stream does")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def measured_peak_hbm():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


NOMINAL_HBM_GBS = 7900.0   # GB300 HBM3e, nominal


def timed_kernel_name(args) -> str:
    """The flag kernel a bench configuration times (plus the SIR pass)."""
    name = ("lof_integ_kernel<CI16, two-dimensional>" if args.grid
            else "lof_integ_kernel<CI16, integrated>" if args.integrated
            else "lof_integ_kernel<CI16, channel scope>" if args.channel_scope
            else "lof_integ_kernel<CI16, pooled exact>" if args.sigma == "winsor"
            else "lof_block_kernel<CI16>")
    return name + (" + SIR" if args.sir else "")


def roofline_entry(alg_bytes: float, kernel_ms: float, peak: float, peak_kind: str, traffic, kernel: str):
    """The roofline object: algorithmic bytes per launch over the kernel's
    average CUDA-event time, against the measured copy peak (frac) and the
    nominal HBM bandwidth (frac_nominal)."""
    achieved = alg_bytes / (kernel_ms * 1e-3) / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": traffic, "kernel": kernel,
            "bytes_per_launch": alg_bytes, "kernel_ms": kernel_ms, "peak_kind": peak_kind,
            "nominal_peak": NOMINAL_HBM_GBS, "frac_nominal": achieved / NOMINAL_HBM_GBS}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for n, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def make_block(dev, seed=2, block=0, n_station=None):
    """Config-2 block [station, pol, subband, C, T, 2] int16 on the device: tones in
    ~2% of the channels of each station-subband, impulses covering ~1% of the
    samples of each station (all its subbands and pols), independent stations."""
    import torch
    from paper_1701_08197_gb300 import synth
    parts = []
    for s in range(n_station or N_STATION):
        spec = synth.VoltageSpec(n_station=1, n_pol=N_POL, n_subband=N_SUBBAND, C=C, T=T,
                                 sigma=32.0, tone_frac=0.02, impulse_frac=0.01)
        parts.append(synth.voltage_block(spec, seed=synth._mix(seed, s), block=block, device=dev))
    return torch.cat(parts, dim=0).contiguous()


def build_units(x, out, mask, stats, slot_base=0):
    from paper_1701_08197_gb300 import lof
    units = []
    u = 0
    for s in range(x.shape[0]):
        for p in range(N_POL):
            for b in range(N_SUBBAND):
                units.append(lof.make_unit(x[s, p, b], out[s, p, b], mask[s, p, b],
                                           slot_base + u * C, stats[u]))
                u += 1
    return units


def grid_cells(grid):
    """(channels, samples) per cell of the two-dimensional mode, or None."""
    if not grid:
        return None
    f, t = grid.lower().split("x")
    return int(f), int(t)


def workload_config(stations: int, sir: int = 0, integrated: bool = False, scope: bool = False,
                    sigma: str = "mad", grid=None) -> dict:
    c = {"workload": f"full LOFAR pre-beamformer block: {stations} st x 2 pol x 8 sb "
                     f"= {stations * 16} units x 256 ch x 3072 t, complex int16, history 60",
         "launch": "batched persistent (1 launch per block) + history commit",
         "l2": "inputs > L2 (2.4 GB at 48 stations), no flush",
         "per_rank_units": stations * 16}
    if sir:
        c["sir_percent"] = sir
    if integrated:
        c["time_mode"] = "integrated (Section 3)"
    if scope:
        c["stats_scope"] = "per channel"
    if sigma != "mad":
        c["sigma_estimator"] = sigma
    if grid_cells(grid):
        c["time_mode"] = "two-dimensional on %d x %d cells" % grid_cells(grid)
    return c


def max_over_ranks(ms: float, world: int, device) -> float:
    """Slowest rank's time: the whole job ends when its last rank does."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_msamples_per_s(samples_per_rank: int, world: int, steps: int, t_max_ms: float) -> float:
    """Whole-job throughput: every rank flags its own block of samples_per_rank
    samples per step (weak scaling, no data exchange between ranks)."""
    return samples_per_rank * world * steps / (t_max_ms * 1e-3) / 1e6


def run_gpu(args):
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_1701_08197_gb300 import lof

    rank, world, local = dist_env()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    n_units = args.stations * N_POL * N_SUBBAND
    samples = n_units * C * T
    # two distinct seeded blocks (the same generator, block index 0 and 1),
    # alternated step by step: every launch meets data it has not seen, and
    # the statistics hints come from the other block
    x = make_block(dev, seed=2 + 1000 * rank, n_station=args.stations)
    x1 = x if args.same_block else make_block(dev, seed=2 + 1000 * rank, block=1,
                                               n_station=args.stations)
    out = torch.empty_like(x)
    mask = torch.empty(x.shape[:-1], dtype=torch.uint8, device=dev)
    stats = lof.stats_tensor(n_units, dev)
    fl = lof.Flagger(local, n_history_slots=n_units * C, sir_percent=args.sir,
                     time_mode=(lof.LOF_TIME_2D if args.grid else
                                lof.LOF_TIME_INTEGRATED if args.integrated else lof.LOF_TIME_PER_CHANNEL),
                     stats_scope=lof.LOF_SCOPE_CHANNEL if args.channel_scope else lof.LOF_SCOPE_POOLED,
                     sigma_estimator=SIGMA[args.sigma],
                     integ_chan=(grid_cells(args.grid) or (1, 1))[0],
                     integ_time=(grid_cells(args.grid) or (1, 1))[1])
    # rings pre-filled with 60 means per channel (steady state of the history flagger)
    pw = (x.to(torch.float32) ** 2).sum(-1).mean(-1).reshape(-1).double().cpu().numpy()
    rng = np.random.default_rng(7)
    H = fl.params.history_len
    ring = pw[:, None] * (1.0 + 0.01 * rng.standard_normal((pw.size, H)))
    fl.history_import(0, ring, np.full(pw.size, H, np.int32))
    units = build_units(x, out, mask, stats)
    units1 = units if args.same_block else build_units(x1, out, mask, stats)
    blocks = [units, units1]
    stream = torch.cuda.Stream(dev)

    def step(seq):
        fl.flag_block(lof.LOF_CI16, blocks[seq % 2], seq, stream)
        fl.history_update(units, stream)

    # launch shape: the library default, or the autotuner's pick (untimed;
    # results do not depend on it)
    tuning = None
    if args.autotune and not args.no_autotune:
        tuning, _ = fl.autotune(lof.LOF_CI16, units, reps=2, stream=stream)
        torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        for i in range(args.warmup):
            step(i)
        fl.status(stream)
    torch.cuda.synchronize()
    # timed region: K steps, events per step, and the flag kernel alone
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        time.sleep(0.3)
        ev[0].record(stream)
        for i in range(args.steps):
            kev[i][0].record(stream)
            fl.flag_block(lof.LOF_CI16, blocks[i % 2], 1000 + i, stream)
            kev[i][1].record(stream)
            fl.history_update(units, stream)
            ev[i + 1].record(stream)
        stream.synchronize()
        time.sleep(0.2)
    fl.status(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    # the exact selection's refinement work on fresh data: one more launch of
    # each block, untimed, after the other block's (the steady state above)
    refine = []
    for b in (0, 1):
        fl.flag_block(lof.LOF_CI16, blocks[b], 0, stream)
        refine.append(fl.counters(stream))
    step_ms = [ev[i].elapsed_time(ev[i + 1]) for i in range(args.steps)]
    total_ms = ev[0].elapsed_time(ev[-1])
    kern_ms = [a.elapsed_time(b) for a, b in kev]
    t_max = max_over_ranks(total_ms, world, dev)
    value = job_msamples_per_s(samples, world, args.steps, t_max)
    res = {"rank": rank, "value": value, "ms_per_step": t_max / args.steps, "step_ms": step_ms,
           "kern_ms": kern_ms, "clocks": clk.summary(), "samples": samples,
           "tuning": tuning or fl.tuning(), "refine": refine}

    # plain form: one launch per station-subband (its two polarisations)
    if not args.no_plain and rank == 0:
        groups = [[units[(s * N_POL + p) * N_SUBBAND + b] for p in range(N_POL)]
                  for s in range(args.stations) for b in range(N_SUBBAND)]
        with torch.cuda.stream(stream):
            for g in groups[:8]:
                fl.flag_block(lof.LOF_CI16, g, 0, stream)
        torch.cuda.synchronize()
        pev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        reps = []
        for r in range(3):
            a, b = pev[0], pev[1]
            a.record(stream)
            for g in groups:
                fl.flag_block(lof.LOF_CI16, g, 0, stream)
            b.record(stream)
            stream.synchronize()
            reps.append(a.elapsed_time(b))
        fl.status(stream)
        res["plain_ms"] = reps

    # end to end through the host-buffer entry point
    if not args.no_e2e and rank == 0:
        # the host buffers on the GPU's own NUMA node: allocated (first touch)
        # from the CPUs local to the GPU, the process's affinity restored after
        saved_cpus = None
        local = gpu_local_cpus(dev)
        if local:
            try:
                saved_cpus = os.sched_getaffinity(0)
                os.sched_setaffinity(0, local)
            except OSError:
                saved_cpus = None
        res["e2e_host_cpus"] = (f"{len(local)} CPUs local to the GPU" if saved_cpus is not None
                                else "unchanged (the GPU's local CPUs not found)")
        hx = x.cpu().pin_memory()
        hout = torch.empty_like(hx).pin_memory()
        hmask = torch.empty(hx.shape[:-1], dtype=torch.uint8).pin_memory()
        hst = torch.zeros_like(stats, device="cpu").pin_memory()
        hunits = build_units(hx, hout, hmask, hst)
        e2e_steps = max(2, min(5, args.steps))
        fl.flag_block_host(lof.LOF_CI16, hunits, 0, stream)  # warm staging
        stream.synchronize()
        fl.status(stream)
        t0 = time.perf_counter()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(e2e_steps):
            fl.flag_block_host(lof.LOF_CI16, hunits, 2000 + i, stream)
            fl.history_update(units, stream)
        e1.record(stream)
        stream.synchronize()
        wall = time.perf_counter() - t0
        fl.status(stream)
        e2e_ms = e0.elapsed_time(e1) / e2e_steps
        if saved_cpus is not None:
            os.sched_setaffinity(0, saved_cpus)
        res["e2e"] = {"value": samples / (e2e_ms * 1e-3) / 1e6, "unit": "Msamples/s",
                      "h2d_bytes_per_step": int(hx.numel() * hx.element_size()),
                      "d2h_bytes_per_step": int(hout.numel() * hout.element_size() + hmask.numel()
                                                + hst.numel() * 8),
                      "ms_per_step": e2e_ms, "wall_ms_per_step": wall * 1e3 / e2e_steps,
                      "host_buffers": res.pop("e2e_host_cpus")}
    fl.close()
    # the other configurations (rank 0, one GPU): the headline's buffers go first
    if args.configs and rank == 0 and world == 1:
        del x, x1, out, mask, units, units1, blocks
        torch.cuda.empty_cache()
        legs = {}
        for name, fn in (("config3_batched", lambda: leg_batched(dev)),
                         ("config4_stokes", lambda: leg_stokes(dev)),
                         ("config5_serving", lambda: leg_serving(dev))):
            try:
                legs[name] = fn()
            except Exception as e:  # a leg's failure is recorded, not hidden
                legs[name] = {"error": f"{type(e).__name__}: {e}"}
        if isinstance(legs.get("config4_stokes"), tuple):
            legs["config4_stokes"], res["stokes_kept"] = legs["config4_stokes"]
        res["legs"] = legs
    if world > 1:
        dist.destroy_process_group()
    return res


def parse_cpulist(text):
    """CPU ids of a Linux cpulist string ("0-3,8,10-11")."""
    cpus = set()
    for part in text.strip().split(","):
        part = part.strip()
        if "-" in part:
            lo, hi = part.split("-")
            cpus.update(range(int(lo), int(hi) + 1))
        elif part:
            cpus.add(int(part))
    return cpus


def gpu_local_cpus(dev):
    """The CPUs (of those this process may use) that Linux lists as local to
    the GPU `dev` (sysfs local_cpulist of its PCI device), or an empty set."""
    import torch
    try:
        pr = torch.cuda.get_device_properties(dev)
        dom, bus, devn = (getattr(pr, "pci_domain_id", None), getattr(pr, "pci_bus_id", None),
                          getattr(pr, "pci_device_id", None))
        if bus is None:
            return set()
        path = f"/sys/bus/pci/devices/{dom or 0:04x}:{bus:02x}:{devn or 0:02x}.0/local_cpulist"
        with open(path) as fh:
            return parse_cpulist(fh.read()) & os.sched_getaffinity(0)
    except Exception:  # no GPU, no such sysfs entry, no affinity interface: leave things as they are
        return set()


# ---------------------------------------------------------------- other configurations
# Short legs after the headline measurement (rank 0, N = 1): the batched
# uneven block (config 3), the Stokes I pulsar block (config 4) and the
# serving loop (config 5), each with the sizes stated in its record.

def _events_ms(fn, reps, stream):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ts = []
    for _ in range(reps):
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    return sorted(ts)[len(ts) // 2]


def leg_batched(dev, n_subband=244, n_station=48, plain_seconds=3.0, peak=6789.0):
    """Config 3: every station x pol x subband of a block of uneven complex
    int8 units (C in 16/64/256, T in 768/3072/12288 drawn per subband from
    seed 3) in ONE persistent launch captured in a CUDA graph, against one
    launch per unit (timed on the first units for plain_seconds, scaled to all
    units).  Units own history slots; blocks 0 and 1 alternate, so each
    replay meets new data with the other block's statistics as hints."""
    import torch
    from paper_1701_08197_gb300 import batched, lof
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    xa = batched.build(n_subband, n_station, device=dev, block=0)
    xb = batched.build(n_subband, n_station, device=dev, block=1)
    gen_s = time.perf_counter() - t0
    outs = [torch.empty_like(x) for x in xa]
    masks = [torch.empty(x.shape[:-1], dtype=torch.uint8, device=dev) for x in xa]
    ua = batched.units_of(xa, outs, masks, history=True)
    ub = batched.units_of(xb, outs, masks, history=True)
    samples = sum(int(x.numel() // 2) for x in xa)
    slots = sum(int(x.shape[0] * 2 * x.shape[2]) for x in xa)
    res = {"workload": f"{n_subband} subbands x {n_station} stations x 2 pols = {len(ua)} uneven units, "
                       f"C in 16/64/256, T in 768/3072/12288 (seed 3), complex int8 sigma 8, "
                       f"{samples} samples, blocks 0/1 alternated", "samples": samples,
           "generate_s": gen_s}
    with lof.Flagger(dev.index or 0, n_history_slots=slots) as fl:
        ga, gb = fl.graph(lof.LOF_CI8, ua), fl.graph(lof.LOF_CI8, ub)
        for i in range(3):
            (ga if i % 2 == 0 else gb).launch(i, stream)
        ga.status(stream)
        k = [0]

        def replay():
            (gb if k[0] % 2 == 0 else ga).launch(10 + k[0], stream)
            k[0] += 1
        graph_ms = _events_ms(replay, 4, stream)
        ga.status(stream)
        direct_ms = _events_ms(lambda: fl.flag_block(lof.LOF_CI8, ua, 0, stream), 2, stream)
        fl.status(stream)
        refine = fl.counters(stream)
        ga.close()
        gb.close()
        # plain form: one launch per unit, as long as plain_seconds allows
        n_plain, tp0 = 0, time.perf_counter()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        while n_plain < len(ua) and time.perf_counter() - tp0 < plain_seconds:
            for u in ua[n_plain:n_plain + 64]:
                fl.flag_block(lof.LOF_CI8, [u], 0, stream)
            n_plain = min(len(ua), n_plain + 64)
            stream.synchronize()
        e1.record(stream)
        e1.synchronize()
        fl.status(stream)
        plain_part_ms = e0.elapsed_time(e1)
        plain_samples = sum(ua[i].n_chan * ua[i].n_time for i in range(n_plain))
    plain_ms = plain_part_ms * samples / max(1, plain_samples)
    res.update({"graph_ms": graph_ms, "direct_launch_ms": direct_ms,
                "graph_Msamples_s": samples / graph_ms / 1e3,
                "graph_GBs": 5 * samples / graph_ms / 1e6,
                "graph_frac_of_measured_hbm": 5 * samples / graph_ms / 1e6 / peak,
                "plain_per_unit_ms_scaled": plain_ms,
                "plain_note": f"one launch per unit on the first {n_plain} units ({plain_part_ms:.0f} ms), "
                              f"scaled by samples to all {len(ua)}",
                "plain_vs_graph": plain_ms / graph_ms,
                "units_refined_last_direct_launch": refine["units_refined"]})
    del xa, xb, outs, masks
    torch.cuda.empty_cache()
    return res


def leg_stokes(dev, n_subband=488, n_block=60, peak=6789.0, keep_units=8):
    """Config 4: Stokes I float32, 488 subbands x 16 channels x 12288 samples
    per block (chi-square(4) noise, a dispersed pulsar P = 0.714 s, DM 26.8,
    narrowband and impulsive RFI): flag-kernel time of one block, and the
    folded-profile S/N over n_block blocks for no flagging, a simple per-unit
    5 sigma thresholder and the flagger.  Keeps block 0's first keep_units
    subbands and their GPU masks for the float parity counts."""
    import torch
    from paper_1701_08197_gb300 import lof, quality, synth
    t0 = time.perf_counter()
    q = quality.evaluate(n_subband=n_subband, n_block=n_block, seed=4, device=str(dev))
    tb = quality.time_block(n_subband, seed=4, reps=5, device=str(dev))
    spec = synth.PulsarSpec(n_subband=keep_units)
    x = synth.stokes_block(synth.PulsarSpec(n_subband=n_subband), seed=4, block=0, device=dev)[:keep_units]
    x = x.contiguous()
    mask = torch.empty(x.shape, dtype=torch.uint8, device=dev)
    st = lof.stats_tensor(keep_units, dev)
    with lof.Flagger(dev.index or 0) as fl:
        fl.flag_block(lof.LOF_F32, [lof.make_unit(x[i], None, mask[i], -1, st[i]) for i in range(keep_units)], 0)
        fl.status()
    kept = {"x": x.cpu().numpy(), "mask": mask.cpu().numpy(), "stats": st.cpu().numpy()}
    n = n_subband * spec.C * spec.T
    res = {"workload": f"Stokes I f32 {n_subband} sb x 16 ch x 12288 t, {n_block} blocks, pulsar "
                       f"P=0.714 s DM=26.8, seed 4",
           "flag_kernel_ms": tb["ms"], "Msamples_s": tb["Msamples_s"], "GBs_9B_per_sample": tb["GBs_9B_per_sample"],
           "frac_of_measured_hbm": tb["GBs_9B_per_sample"] / peak,
           "folded_snr": {k: v["snr"] for k, v in q.items()},
           "flagged_fraction": {k: v["flagged_fraction"] for k, v in q.items()},
           "samples_per_block": n, "wall_s": time.perf_counter() - t0}
    return res, kept


def leg_serving(dev, n_streams=32, n_blocks=3, budget_gb=2.0):
    """Config 5: 32 concurrent complex int8 streams (1-16 stations x 2 pols x
    64-384 channels x 1024-8192 samples, seed 5) arriving every 1 s with
    +-100 ms jitter, admitted by a device-memory budget, continuously batched;
    p50/p99 block latency against the 1 s deadline."""
    from paper_1701_08197_gb300 import serve
    streams = serve.make_streams(n_streams)
    srv, wall = serve.run(streams, n_blocks, int(budget_gb * 2 ** 30), accelerated=False,
                          gen_device=str(dev))
    rep = serve.report(srv, wall)
    srv.close()
    rep.update({"workload": f"{n_streams} streams x {n_blocks} blocks, real-time 1 s cadence +-100 ms, "
                            f"device budget {budget_gb} GB", "wall_s": wall})
    return rep


def float_parity_counts(kept):
    """Config 4 sample on the host cores: the oracle on the kept Stokes I
    subbands against the GPU masks, with the binary64 replay's near-threshold
    and cascade counts (the float contract)."""
    import numpy as np

    import oracle
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from float_parity import allowed_differences
    from paper_1701_08197_gb300 import lof
    P = oracle.default_params()
    tot = {"units": 0, "samples": 0, "differing": 0, "near_threshold_count": 0, "cascade_count": 0,
           "outside_allowed": 0}
    for i in range(kept["x"].shape[0]):
        x = kept["x"][i]
        ref = oracle.flag_unit(P, x)
        entry = ~np.isfinite(x)
        allowed, _, nn, nc = allowed_differences(P, np.where(entry, 0.0, x.astype(np.float64)), entry,
                                                 ref["stats"])
        diff = kept["mask"][i] != ref["mask"]
        tot["units"] += 1
        tot["samples"] += int(x.size)
        tot["differing"] += int(diff.sum())
        tot["near_threshold_count"] += nn
        tot["cascade_count"] += nc
        tot["outside_allowed"] += int((diff & ~allowed).sum())
    return tot


def oracle_sample(seconds: float, seed=2, sir=0, integrated=False, scope=False, sigma="mad", grid=None,
                  threads=None):
    """The oracle (as it stands) on host cores: units of the same workload, one
    per thread (the paper's thread-per-subband CPU layout), bounded in time.
    threads = None: every host core; 1: a single thread."""
    from concurrent.futures import ThreadPoolExecutor

    import torch

    import oracle
    from paper_1701_08197_gb300 import synth
    cells = grid_cells(grid) or (1, 1)
    P = oracle.default_params(sir_percent=sir, time_mode=2 if grid else 1 if integrated else 0,
                              stats_scope=1 if scope else 0, sigma_estimator=SIGMA[sigma],
                              integ_chan=cells[0], integ_time=cells[1])
    cores = threads or os.cpu_count() or 1
    spec = synth.VoltageSpec(n_station=1, n_pol=N_POL, n_subband=N_SUBBAND, C=C, T=T,
                             sigma=32.0, tone_frac=0.02, impulse_frac=0.01)
    blk = synth.voltage_block(spec, seed=synth._mix(seed, 0), block=0, device="cpu")
    units = [blk[0, p, b].numpy() for p in range(N_POL) for b in range(N_SUBBAND)]
    oracle.lib()
    done = [0]
    lock = threading.Lock()

    def work(i):
        k = i
        while time.perf_counter() < deadline or k == i:
            oracle.flag_unit(P, units[k % len(units)], want_out=True)
            with lock:
                done[0] += 1
            k += cores
        return 0

    t0 = time.perf_counter()
    deadline = t0 + seconds
    with ThreadPoolExecutor(cores) as ex:
        list(ex.map(work, range(cores)))
    wall = time.perf_counter() - t0
    n = done[0]
    value = n * C * T / wall / 1e6 if n else 0.0
    return {"value": value, "unit": "Msamples/s", "cores": cores, "kind": "oracle",
            "sample": f"{n} units of 256 x 3072 ci16 (one station's 16 units, cycled), "
                      f"{cores} threads, one unit per thread at a time, {wall:.1f} s wall"}


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        if rank != 0:
            return
        steps = []
        cb = None
        for i in range(args.warmup + args.steps):
            r = oracle_sample(max(2.0, args.cpu_seconds / max(1, args.steps)), sir=args.sir,
                              integrated=args.integrated, scope=args.channel_scope, sigma=args.sigma,
                              grid=args.grid)
            if i >= args.warmup:
                steps.append(r)
            cb = r
        vals = [r["value"] for r in steps]
        v = statistics.mean(vals) if vals else 0.0
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "Msamples/s",
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": (N_STATION * N_POL * N_SUBBAND * C * T / (v * 1e6) * 1e3) if v else None,
                "ms_per_step_note": "extrapolated: one full block's samples at the sampled oracle rate "
                                    "(each step times a bounded sample of the block's units)",
                "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "int64+f64",
                "data": "synthetic (seeded)",
                "config": workload_config(args.stations, args.sir, args.integrated, args.channel_scope, args.sigma,
                                    args.grid),
                "cpu_baseline": {"value": v, "unit": "Msamples/s", "cores": cb["cores"],
                                 "kind": "oracle", "sample": cb["sample"]},
                "e2e": {"value": v, "unit": "Msamples/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    res = run_gpu(args)
    if rank != 0:
        return
    peak, peak_kind = measured_peak_hbm()
    samples = res["samples"]
    kern_avg = statistics.mean(res["kern_ms"])
    alg_bytes = samples * BYTES_PER_SAMPLE
    step_sorted = sorted(res["step_ms"])

    def pct(a, q):
        return a[min(len(a) - 1, int(math.ceil(q * len(a))) - 1)]

    line = {
        "metric": METRIC, "value": res["value"], "unit": "Msamples/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32/u64",
        "data": "synthetic (seeded noise + tones + impulses)",
        "config": dict(workload_config(args.stations, args.sir, args.integrated, args.channel_scope, args.sigma,
                                    args.grid), tuning=res["tuning"],
                       data_blocks="one block, every step" if args.same_block else
                       "two distinct seeded blocks (block index 0, 1), alternated step by step"),
        "roofline": roofline_entry(
            alg_bytes, kern_avg, peak, peak_kind,
            # the recorded counters are those of the block kernel alone
            None if (args.integrated or args.channel_scope or args.sir or args.sigma == "winsor"
                     or args.grid) else measured_traffic(args.stations * 16, res["tuning"]),
            timed_kernel_name(args)),
        "latency_ms": {"batched_p50": pct(step_sorted, 0.5), "batched_p99": pct(step_sorted, 0.99),
                       "deadline_ms": T * 1.31072},
        "clocks": res["clocks"],
        # per step: the flag kernel, the history commit and, with --sir, its two kernels
        "gpu_launches": (2 + (2 if args.sir else 0)) * args.steps,
    }
    if "plain_ms" in res:
        pm = sorted(res["plain_ms"])
        line["latency_ms"]["plain_block_ms"] = pm[len(pm) // 2]
        line["plain_vs_batched"] = pm[len(pm) // 2] / kern_avg
    if "e2e" in res:
        line["e2e"] = res["e2e"]
    line["stats_refinement"] = {
        "units_refined_per_launch": [r["units_refined"] for r in res["refine"]],
        "refine_passes_per_launch": [r["refine_passes"] for r in res["refine"]],
        "note": "block 0 after block 1 and block 1 after block 0: units whose pooled median/MAD "
                "needed a refinement pass beyond the first counting pass (the previous block's "
                "statistics as hints)" if not args.same_block else "same block every step"}
    if "legs" in res:
        line["configs"] = res["legs"]
    if not args.no_cpu:
        if "stokes_kept" in res:
            try:
                line["configs"]["config4_stokes"]["float_parity"] = float_parity_counts(res["stokes_kept"])
            except Exception as e:
                line["configs"]["config4_stokes"]["float_parity"] = {"error": f"{type(e).__name__}: {e}"}
        opts = dict(sir=args.sir, integrated=args.integrated, scope=args.channel_scope, sigma=args.sigma,
                    grid=args.grid)
        cb = oracle_sample(args.cpu_seconds * 0.7, **opts)
        one = oracle_sample(max(3.0, args.cpu_seconds * 0.3), threads=1, **opts)
        cb["single_thread"] = {"value": one["value"], "unit": one["unit"], "cores": 1,
                               "sample": one["sample"]}
        line["cpu_baseline"] = cb
    print(json.dumps(line))


if __name__ == "__main__":
    main()
