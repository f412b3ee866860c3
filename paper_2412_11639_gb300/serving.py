"""Streaming request loop with continuous batching over live spike streams.

Each request is a camera stream of H x W pixels and T steps that starts at its arrival
time and then produces `rate` steps per second.  The server

* admits requests first-come first-served while the device memory they need (per-pixel
  scan state, the frames, a piece buffer) fits the budget and a slot is free;
* every tick gathers the steps each active stream has produced since the last tick and
  reconstructs all of these pieces in ONE spk_run launch (continuous batching: streams
  that arrived while others were running join the next launch, and their work shares the
  device with everyone else's);
* keeps every stream's per-pixel stability state on the device between pieces
  (spk_stream_*), so the frames are exactly those of one reconstruction of the whole
  stream;
* records, for every frame, the latency from the moment its sampling step was produced to
  the moment the frame became final for every pixel (a frame is final once the stable
  span covering it closes -- for a static pixel that can be the end of the stream);
* lets any thread cancel a request (cancel(rid)): a waiting request is dropped, an active
  one gives back its slot, its device state and its memory at the next tick.

The scheduling is host logic; every step of the reconstruction runs in libspk.
"""
from __future__ import annotations

import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import Reconstructor, Stream, spk_run


@dataclass
class Request:
    rid: int
    stream: np.ndarray   # host uint8 [T][pitch]: what the camera will produce
    H: int
    W: int
    arrival: float       # seconds after the loop starts
    rate: float          # steps produced per second once arrived
    threshold: float = 1.0

    @property
    def T(self) -> int:
        return self.stream.shape[0]


@dataclass
class _Live:
    req: Request
    s: Stream
    staging: object          # pinned host copy of the whole stream (the camera's buffer)
    dev_buf: object          # device buffer for one piece
    mem: int
    ready: int = 0
    latencies: list = field(default_factory=list)


@dataclass
class ServeStats:
    frames: int
    pixel_frames: int
    wall_s: float
    busy_s: float
    launches: int
    p50_ms: float
    p99_ms: float
    max_ms: float
    peak_active: int
    admitted_late_s: float   # total time requests waited for admission
    cancelled: int = 0       # requests cancelled before they finished


def stream_state_bytes(order: int, stability_order: int = 3) -> int:
    """Device bytes per pixel of a live stream's state: the scan's 20 int32, or for the
    n-order tree (order 5) its carried rows (11 scalars and 8 fields of each of its 7
    register-level nodes and max(1, 2^n - 8) deeper ones) and its pending-cut rings (64 cuts
    of two int32 at first), each with the copy taken before a launch."""
    if order != 5:
        return 20 * 4
    n = stability_order
    return 2 * 4 * (11 + 8 * (7 + max(1, 2 ** n - 8))) + 2 * 2 * 64 * 4


class Server:
    """Continuous-batching server over one libspk context."""

    def __init__(self, order: int = 2, stride: int = 1, dtype=None, device: int = 0,
                 mem_budget: int = 8 << 30, max_streams: int = 64, max_piece: int = 4096,
                 stability_order: int = 3):
        import torch
        self.torch = torch
        self.rec = Reconstructor(order=order, stride=stride, dtype=dtype, device=device,
                                 stability_order=stability_order)
        self.stride = stride
        self.esz = {torch.float16: 2, torch.uint8: 1}.get(self.rec.dtype, 4)
        self.state_bytes = stream_state_bytes(order, stability_order)
        self.mem_budget, self.max_streams, self.max_piece = mem_budget, max_streams, max_piece
        self.results = {}        # rid -> frames (device tensor [T_out][H][W])
        self._cancel = set()
        self._lock = threading.Lock()

    def cancel(self, rid: int):
        """Cancel request rid (from any thread); it leaves at the loop's next tick."""
        with self._lock:
            self._cancel.add(rid)

    def mem_needed(self, r: Request) -> int:
        P = r.H * r.W
        T_out = (r.T + self.stride - 1) // self.stride
        return self.state_bytes * P + T_out * P * self.esz + self.max_piece * r.stream.shape[1]

    def run(self, requests, clock=time.perf_counter) -> ServeStats:
        torch = self.torch
        pending = sorted(requests, key=lambda r: (r.arrival, r.rid))
        for r in pending:
            if self.mem_needed(r) > self.mem_budget:
                raise ValueError(f"request {r.rid} alone exceeds the memory budget")
        active: list[_Live] = []
        used = 0
        launches = 0
        peak = 0
        waited = 0.0
        busy = 0.0
        lat_all = []
        pinned = {r.rid: torch.from_numpy(r.stream).pin_memory() for r in pending}  # camera buffers
        cancelled = 0
        t0 = clock()
        while pending or active:
            with self._lock:
                drop, self._cancel = self._cancel, set()
            if drop:
                for r in [p for p in pending if p.rid in drop]:
                    pending.remove(r)
                    pinned.pop(r.rid, None)
                    cancelled += 1
                for a in [x for x in active if x.req.rid in drop]:
                    a.s.close()                  # waits for its last launch, frees its state
                    used -= a.mem
                    active.remove(a)
                    cancelled += 1
            if not (pending or active):
                break
            now = clock() - t0
            # admission, first come first served, by memory and slots
            while (pending and pending[0].arrival <= now and len(active) < self.max_streams
                   and used + self.mem_needed(pending[0]) <= self.mem_budget):
                r = pending.pop(0)
                waited += now - r.arrival
                mem = self.mem_needed(r)
                used += mem
                live = _Live(r, Stream(self.rec, r.H, r.W, r.T, r.threshold), pinned.pop(r.rid),
                             torch.empty((self.max_piece, r.stream.shape[1]), dtype=torch.uint8,
                                         device=f"cuda:{self.rec.device}"), mem)
                active.append(live)
            peak = max(peak, len(active))
            # one launch over the pieces every active stream produced since the last tick
            jobs = []
            cs = self.rec.stream
            for a in active:
                produced = min(a.req.T, int((now - a.req.arrival) * a.req.rate))
                n = min(produced - a.s.steps, self.max_piece)
                if n <= 0:
                    continue
                with torch.cuda.stream(cs):
                    a.dev_buf[:n].copy_(a.staging[a.s.steps:a.s.steps + n], non_blocking=True)
                jobs.append((a, a.s.job(a.dev_buf, n)))
            if not jobs:
                nxt = [p.arrival for p in pending[:1]]
                time.sleep(min([1e-4] + [max(0.0, x - now) for x in nxt]))
                continue
            tb = clock()
            spk_run(self.rec.ctx, [j for _, j in jobs])
            launches += 1
            for a, _ in jobs:
                ready = a.s.ready()          # waits for the launch
                if ready > a.ready:
                    t_done = clock() - t0
                    k = np.arange(a.ready, ready)
                    produced_at = a.req.arrival + (k * self.stride + 1) / a.req.rate
                    a.latencies.append(t_done - produced_at)
                    a.ready = ready
            busy += clock() - tb
            # retire finished streams
            for a in [x for x in active if x.s.steps == x.req.T]:
                lat = np.concatenate(a.latencies) if a.latencies else np.zeros(0)
                lat_all.append(lat)
                self.results[a.req.rid] = a.s.frames
                a.s.close()
                used -= a.mem
                active.remove(a)
        wall = clock() - t0
        lat = np.concatenate(lat_all) if lat_all else np.zeros(1)
        frames = int(sum(v.shape[0] for v in self.results.values()))
        pf = int(sum(v.shape[0] * v.shape[1] * v.shape[2] for v in self.results.values()))
        return ServeStats(frames, pf, wall, busy, launches, float(np.percentile(lat, 50) * 1e3),
                          float(np.percentile(lat, 99) * 1e3), float(lat.max() * 1e3), peak, waited,
                          cancelled)

    def close(self):
        self.rec.close()
