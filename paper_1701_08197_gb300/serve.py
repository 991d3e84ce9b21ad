"""Serving loop: flags data blocks arriving from many concurrent streams
(stations x polarisations x subbands of different shapes, each stream one
real-time source), with continuous batching.

* Admission by device memory: every request (one block of one stream) needs
  its input, output, mask and statistics on the device.  Those live in one
  preallocated arena; a request is admitted when a first-fit allocation of
  its bytes succeeds and freed as soon as its results are back on the host.
* Per-stream state stays on the device: every stream owns history slots of
  the one flagger context (one ring per channel, Section 4.1).  A stream's
  blocks must pass the history flagger in order, so one launch holds at most
  one block of a stream; later blocks of that stream go to later launches,
  which the compute stream orders after the earlier history commit.
* Continuous batching: whenever the compute stream can take work, every
  admitted request whose upload has finished (and whose stream is not yet in
  the batch) joins ONE persistent launch (lof_flag_block + lof_history_update);
  uploads and downloads run on copy streams and overlap with the kernels of
  other requests.
* Latency of a block = results on the host - arrival time; p50/p99 against
  the real-time deadline are reported beside the throughput.
"""
from __future__ import annotations

import bisect
import collections
import dataclasses
import time

import numpy as np
import torch

from . import lof

ALIGN = 256


class Arena:
    """First-fit allocator over one device byte buffer."""

    def __init__(self, nbytes: int, device):
        self.buf = torch.empty(nbytes, dtype=torch.uint8, device=device)
        self.size = nbytes
        self.free = [(0, nbytes)]  # sorted (offset, length)

    def alloc(self, n: int):
        n = (n + ALIGN - 1) // ALIGN * ALIGN
        for i, (off, ln) in enumerate(self.free):
            if ln >= n:
                if ln == n:
                    self.free.pop(i)
                else:
                    self.free[i] = (off + n, ln - n)
                return off, n
        return None

    def release(self, off: int, n: int):
        i = bisect.bisect_left(self.free, (off, 0))
        self.free.insert(i, (off, n))
        merged = []
        for o, l in self.free:
            if merged and merged[-1][0] + merged[-1][1] == o:
                merged[-1] = (merged[-1][0], merged[-1][1] + l)
            else:
                merged.append((o, l))
        self.free = merged

    def view(self, off: int, shape, dtype):
        nbytes = int(np.prod(shape)) * torch.empty((), dtype=dtype).element_size()
        return self.buf[off:off + nbytes].view(dtype).view(shape)


@dataclasses.dataclass
class StreamSpec:
    """One real-time source: n_station x 2 pols x C channels x T samples per block."""
    sid: int
    n_station: int
    C: int
    T: int
    period_s: float = 1.0     # block cadence
    dtype: torch.dtype = torch.int8

    @property
    def n_units(self):
        return self.n_station * 2

    @property
    def shape(self):
        return (self.n_station, 2, self.C, self.T, 2)

    @property
    def samples(self):
        return self.n_station * 2 * self.C * self.T


@dataclasses.dataclass
class Request:
    spec: StreamSpec
    block: int
    arrival: float                 # host clock (s)
    data: torch.Tensor             # pinned host [S, 2, C, T, 2]
    # filled by the server
    mem: tuple | None = None
    d_in: torch.Tensor | None = None
    d_out: torch.Tensor | None = None
    d_mask: torch.Tensor | None = None
    d_stats: torch.Tensor | None = None
    up_done: torch.cuda.Event | None = None
    down_done: torch.cuda.Event | None = None
    h_out: torch.Tensor | None = None
    h_mask: torch.Tensor | None = None
    h_stats: torch.Tensor | None = None
    done: float | None = None

    def device_bytes(self):
        es = self.data.element_size()
        n = self.spec.samples
        return 2 * n * 2 * es + n + self.spec.n_units * 64 + 4 * ALIGN


class Server:
    """Continuous-batching flagger for a fixed set of streams."""

    def __init__(self, streams, mem_budget: int, device: int = 0, keep_results: bool = True):
        self.dev = torch.device("cuda", device)
        self.streams = {s.sid: s for s in streams}
        slots, self.slot0 = 0, {}
        for s in streams:
            self.slot0[s.sid] = slots
            slots += s.n_units * s.C
        self.fl = lof.Flagger(device, n_history_slots=slots)
        self.arena = Arena(mem_budget, self.dev)
        self.s_up = torch.cuda.Stream(self.dev)
        self.s_comp = torch.cuda.Stream(self.dev)
        self.s_down = torch.cuda.Stream(self.dev)
        self.waiting = collections.deque()   # arrived, not admitted (FIFO)
        self.admitted = []                   # uploading or waiting for a batch
        self.running = []                    # launched, results on the way back
        self.finished = []
        self.keep = keep_results
        self.launches = 0
        self.inflight = []  # completion events of the queued launches
        self.next_block = {s.sid: 0 for s in streams}  # blocks must be flagged in order

    def close(self):
        torch.cuda.synchronize(self.dev)
        self.fl.close()

    # -- steps of the loop
    def submit(self, req: Request):
        if req.device_bytes() > self.arena.size:
            raise ValueError(f"block of stream {req.spec.sid} needs {req.device_bytes()} bytes, "
                             f"more than the device budget {self.arena.size}")
        self.waiting.append(req)

    def _admit(self):
        while self.waiting:
            req = self.waiting[0]
            a = self.arena.alloc(req.device_bytes())
            if a is None:
                break  # FIFO: wait for memory
            self.waiting.popleft()
            req.mem = a
            off = a[0]
            shp, S = req.spec.shape, req.spec
            n = S.samples
            es = req.data.element_size()
            req.d_in = self.arena.view(off, shp, req.data.dtype)
            off2 = off + (2 * n * es + ALIGN - 1) // ALIGN * ALIGN
            req.d_out = self.arena.view(off2, shp, req.data.dtype)
            off3 = off2 + (2 * n * es + ALIGN - 1) // ALIGN * ALIGN
            req.d_mask = self.arena.view(off3, shp[:4], torch.uint8)
            off4 = off3 + (n + ALIGN - 1) // ALIGN * ALIGN
            req.d_stats = self.arena.view(off4, (S.n_units, len(lof.STATS_FIELDS)), torch.int64)
            with torch.cuda.stream(self.s_up):
                req.d_in.copy_(req.data, non_blocking=True)
                req.up_done = torch.cuda.Event()
                req.up_done.record(self.s_up)
            self.admitted.append(req)

    def _units(self, req: Request):
        S = req.spec
        base = self.slot0[S.sid]
        out = []
        for st in range(S.n_station):
            for p in range(2):
                u = st * 2 + p
                out.append(lof.make_unit(req.d_in[st, p], req.d_out[st, p], req.d_mask[st, p],
                                         base + u * S.C, req.d_stats[u]))
        return out

    def _launch(self):
        batch, in_batch = [], set()
        for req in list(self.admitted):
            sid = req.spec.sid
            if sid in in_batch or req.block != self.next_block[sid] or not req.up_done.query():
                continue
            batch.append(req)
            in_batch.add(sid)
        if not batch:
            return False
        for req in batch:
            self.admitted.remove(req)
            self.next_block[req.spec.sid] += 1
        units = [u for req in batch for u in self._units(req)]
        dt = lof.dtype_of(batch[0].d_in)
        for req in batch:
            self.s_comp.wait_event(req.up_done)
        self.fl.flag_block(dt, units, self.launches, self.s_comp)
        self.fl.history_update(units, self.s_comp)
        self.launches += 1
        ev = torch.cuda.Event()
        ev.record(self.s_comp)
        self.inflight.append(ev)
        self.s_down.wait_event(ev)
        with torch.cuda.stream(self.s_down):
            for req in batch:
                if self.keep:
                    req.h_mask = torch.empty(req.d_mask.shape, dtype=torch.uint8, pin_memory=True)
                    req.h_out = torch.empty(req.d_out.shape, dtype=req.d_out.dtype, pin_memory=True)
                    req.h_mask.copy_(req.d_mask, non_blocking=True)
                    req.h_out.copy_(req.d_out, non_blocking=True)
                else:  # the mask alone leaves the device (the data stays for the beamformer)
                    req.h_mask = torch.empty(req.d_mask.shape, dtype=torch.uint8, pin_memory=True)
                    req.h_mask.copy_(req.d_mask, non_blocking=True)
                req.h_stats = torch.empty(req.d_stats.shape, dtype=torch.int64, pin_memory=True)
                req.h_stats.copy_(req.d_stats, non_blocking=True)
                req.down_done = torch.cuda.Event()
                req.down_done.record(self.s_down)
        self.running.extend(batch)
        return True

    def _retire(self):
        still = []
        for req in self.running:
            if req.down_done.query():
                req.done = time.perf_counter()
                self.arena.release(*req.mem)
                req.d_in = req.d_out = req.d_mask = req.d_stats = None
                self.finished.append(req)
            else:
                still.append(req)
        self.running = still

    def step(self):
        """One pass of the loop; returns whether anything is still pending."""
        self._retire()
        self._admit()
        # at most two launches queued on the compute stream: work that arrives
        # meanwhile joins the next batch instead of a queue of small launches
        self.inflight = [e for e in self.inflight if not e.query()]
        if len(self.inflight) < 2:
            self._launch()
        return bool(self.waiting or self.admitted or self.running)

    def check(self):
        self.fl.status(self.s_comp)


def make_streams(n_streams=32, seed=5, period_s=1.0):
    """Seeded SKA-Low-like stream shapes: 1-16 stations x 2 pols x C in [64, 384]
    (multiple of 16) x T in {1024, ..., 8192}."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_streams):
        S = int(rng.integers(1, 17))
        C = int(rng.integers(4, 25)) * 16
        T = int(2 ** rng.integers(10, 14))
        out.append(StreamSpec(i, S, C, T, period_s))
    return out


def make_block(spec: StreamSpec, block: int, seed=5, device="cpu"):
    """Seeded complex int8 block (sigma 8, tones and impulses) in pinned host
    memory, drawn on `device` (a CUDA device draws large blocks in
    milliseconds; the values depend on the device's generator)."""
    from . import synth
    vs = synth.VoltageSpec(n_station=spec.n_station, n_pol=2, n_subband=1, C=spec.C, T=spec.T,
                           dtype=spec.dtype, sigma=8.0, tone_frac=0.02, impulse_frac=0.01)
    x = synth.voltage_block(vs, seed=synth._mix(seed, spec.sid), block=block, device=device)
    return x[:, :, 0].contiguous().cpu().pin_memory()


def run(streams, n_blocks: int, mem_budget: int, accelerated=False, jitter_s=0.1, seed=5,
        keep_results=False, blocks=None, gen_device="cpu"):
    """Drive the server with every stream's blocks 0..n_blocks-1 arriving on
    its cadence (jittered), or all at once when accelerated; returns the server
    (finished requests hold latencies and results) and the wall time."""
    rng = np.random.default_rng(seed + 1)
    events = []
    for s in streams:
        for b in range(n_blocks):
            t = 0.0 if accelerated else b * s.period_s + float(rng.uniform(-jitter_s, jitter_s)) + jitter_s
            events.append((t, s.sid, b))
    events.sort()
    data = {} if blocks is None else blocks
    for _, sid, b in events:
        if (sid, b) not in data:
            data[(sid, b)] = make_block(next(s for s in streams if s.sid == sid), b, seed, gen_device)
    srv = Server(streams, mem_budget, keep_results=keep_results)
    by_id = {s.sid: s for s in streams}
    t0 = time.perf_counter()
    i = 0
    pending = True
    while i < len(events) or pending:
        now = time.perf_counter() - t0
        while i < len(events) and events[i][0] <= now:
            _, sid, b = events[i]
            srv.submit(Request(by_id[sid], b, t0 + events[i][0], data[(sid, b)]))
            i += 1
        pending = srv.step()
        if not pending and i < len(events):
            time.sleep(max(0.0, min(0.002, events[i][0] - (time.perf_counter() - t0))))
    torch.cuda.synchronize()
    srv.check()
    return srv, time.perf_counter() - t0


def report(srv: Server, wall: float, deadline_s: float = 1.0):
    lat = np.array([r.done - r.arrival for r in srv.finished])
    samples = sum(r.spec.samples for r in srv.finished)
    return {"blocks": len(srv.finished), "launches": srv.launches,
            "throughput_Msamples_s": samples / wall / 1e6,
            "latency_ms": {"p50": float(np.percentile(lat, 50) * 1e3),
                           "p99": float(np.percentile(lat, 99) * 1e3),
                           "max": float(lat.max() * 1e3)},
            "deadline_ms": deadline_s * 1e3,
            "deadline_misses": int((lat > deadline_s).sum())}


def main():
    import argparse
    import json
    ap = argparse.ArgumentParser()
    ap.add_argument("--streams", type=int, default=32)
    ap.add_argument("--blocks", type=int, default=4)
    ap.add_argument("--budget-gb", type=float, default=2.0)
    ap.add_argument("--accelerated", action="store_true")
    args = ap.parse_args()
    streams = make_streams(args.streams)
    srv, wall = run(streams, args.blocks, int(args.budget_gb * 2 ** 30), args.accelerated)
    rep = report(srv, wall)
    rep["mode"] = "accelerated" if args.accelerated else "real-time (1 s cadence, +-100 ms jitter)"
    rep["streams"] = args.streams
    rep["device_budget_GB"] = args.budget_gb
    print(json.dumps(rep))
    srv.close()


if __name__ == "__main__":
    main()
