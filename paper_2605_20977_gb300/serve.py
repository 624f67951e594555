"""Continuous-batching decode service over the C ABI.

A request is a sequence of 1..16 coded frames of one resolution (each frame a
container and its hyperlatents, already on the device).  The server keeps a
set of active requests, each with its own sequence state (the spatial and
temporal key/value caches stay on the device between frames).  Every
iteration decodes the next frame of every active request in one
psw_decode_batch call: their wavefront steps share launches (Sec. 3.2
parallelism across frames as well as along a wavefront).  A request that
arrives while an iteration runs is admitted before the next one, as soon as
a batch slot is free and its sequence state fits the HBM budget; finished
requests leave their slot and their (reset) sequence state, which the next
request of the same grid reuses; idle states of other grids are dropped when
a new one needs the memory.  Latency is completion minus arrival.

The decode engine defaults to the graph engine: the batch changes from
iteration to iteration, so a call often records its graphs first (the
context keeps the most recent batch shapes), and yet it served faster than
the persistent engine, which records nothing, on the measured trace.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import psw


@dataclass
class Request:
    rid: int
    arrival: float                     # seconds after the start of the run
    H: int
    W: int
    frames: list                       # [(container device tensor, length, hyperlatents device tensor)]
    outputs: list                      # device int16 [H][W][C] per frame (written by the server)
    mu: list | None = None             # optional float32 outputs per frame
    sigma: list | None = None
    admitted: float = -1.0
    done: float = -1.0
    seq: object = None
    next: int = 0
    status: list = field(default_factory=list)


class Server:
    """Admission by HBM budget and batch slots; one decode call per iteration."""

    def __init__(self, ctx: "psw.Context", hbm_budget: int, max_batch: int = 128,
                 engine: int = psw.ENGINE_GRAPH):
        self.ctx = ctx
        self.budget = int(hbm_budget)
        self.max_batch = int(max_batch)
        self.engine = engine

    def run(self, requests: list[Request], clock=time.perf_counter, sleep=time.sleep) -> dict:
        """Serve `requests` (arrival times relative to the start) until all
        are done.  A request whose sequence state alone exceeds the budget
        is rejected (done stays -1).  clock / sleep: the time source and the
        idle wait (replaceable for tests)."""
        ctx = self.ctx
        ctx.set_engine(self.engine)
        rejected = [r for r in requests if ctx.seq_bytes(r.H, r.W) > self.budget]
        pending = sorted((r for r in requests if ctx.seq_bytes(r.H, r.W) <= self.budget),
                         key=lambda r: (r.arrival, r.rid))
        served = list(pending)
        active: list[Request] = []
        idle: dict = {}            # (H, W) -> finished sequences kept for reuse (still counted in `used`)
        used = 0
        iters = batch_sum = frames = 0
        peak_active = peak_used = 0
        t0 = clock()
        pi = 0
        while pi < len(pending) or active:
            now = clock() - t0
            # admit everything that has arrived and fits
            while pi < len(pending) and pending[pi].arrival <= now and len(active) < self.max_batch:
                r = pending[pi]
                key = (r.H, r.W)
                if idle.get(key):
                    r.seq = idle[key].pop()                 # reuse: already counted
                else:
                    need = ctx.seq_bytes(r.H, r.W)
                    # make room by dropping idle sequences of other grids
                    for k in list(idle):
                        while idle[k] and used + need > self.budget:
                            idle[k].pop().close()
                            used -= ctx.seq_bytes(*k)
                    if used + need > self.budget:
                        break
                    r.seq = ctx.seq_create(r.H, r.W)
                    used += need
                r.admitted = now
                active.append(r)
                pi += 1
            peak_active = max(peak_active, len(active))
            peak_used = max(peak_used, used)
            if not active:
                # nothing to decode: wait for the next arrival
                sleep(max(pending[pi].arrival - (clock() - t0), 0.0))
                continue
            fds = [psw.frame_desc(r.H, r.W, psw.PSW_SCHED_WAVEFRONT) for r in active]
            st = ctx.decode_batch([r.seq for r in active], fds,
                                  [r.frames[r.next][0] for r in active], [r.frames[r.next][1] for r in active],
                                  [r.frames[r.next][2] for r in active], [r.outputs[r.next] for r in active],
                                  [r.mu[r.next] if r.mu else None for r in active],
                                  [r.sigma[r.next] if r.sigma else None for r in active], check=False)
            now = clock() - t0
            iters += 1
            batch_sum += len(active)
            frames += len(active)
            keep = []
            for r, s in zip(active, st):
                r.status.append(s)
                r.next += 1
                if r.next == len(r.frames):
                    r.done = now
                    r.seq.reset()
                    idle.setdefault((r.H, r.W), []).append(r.seq)
                    r.seq = None
                else:
                    keep.append(r)
            active = keep
        span = clock() - t0
        for k, v in idle.items():
            for q in v:
                q.close()
        lat = np.array([r.done - r.arrival for r in served]) if served else np.zeros(1)
        return {"requests": len(served), "rejected": len(rejected), "frames": frames, "makespan_s": span,
                "frames_per_s": frames / span if span > 0 else 0.0,
                "latency_p50_s": float(np.percentile(lat, 50)), "latency_p99_s": float(np.percentile(lat, 99)),
                "iterations": iters, "mean_batch": batch_sum / max(iters, 1),
                "peak_active": peak_active, "peak_hbm_bytes": peak_used}


def poisson_trace(rate: float, window: float, grids: list, max_frames: int = 16, seed: int = 1005):
    """Seeded arrivals over [0, window): exponential gaps at `rate` per
    second; each request picks a grid uniformly and 1..max_frames frames
    uniformly.  Returns [(arrival, grid index, frames)]."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= window:
            return out
        out.append((t, int(rng.integers(len(grids))), int(rng.integers(1, max_frames + 1))))
