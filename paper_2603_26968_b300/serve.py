"""Serving loop over the library's engine: Poisson arrivals, admission by free HBM,
round-level continuous batching, latency percentiles.

A request is a field to compress.  It waits in a FIFO queue until its device
memory fits in the HBM budget: its input, its per-field engine state and its output
buffer.  On admission its input is materialised on the device (on a generator
stream, standing in for the upload of the client's data) and submitted to the
engine.  The loop then alternates engine steps and polls.  A step runs one repair
round (compaction and reruns) over every field in repair and starts the new fields
beside it, so a request that arrives while others are on the GPU joins them at the
next round instead of waiting for them.  Latency is arrival to stream ready.

Everything that touches field values runs in the CUDA library; this module only
schedules, allocates and measures.
"""
from __future__ import annotations

import collections
import math
import time
from dataclasses import dataclass, field
from typing import Callable, Dict, List, Optional, Sequence

import numpy as np
import torch

from . import lopc
from .synth_gpu import ServeSpec, make_field


class Budget:
    """Bytes of device memory the server may hold for admitted requests."""

    def __init__(self, total: int):
        self.total = int(total)
        self.used = 0
        self.peak = 0

    def fits(self, n: int) -> bool:
        return self.used + n <= self.total

    def take(self, n: int) -> None:
        if not self.fits(n):
            raise ValueError("budget exceeded")
        self.used += n
        self.peak = max(self.peak, self.used)

    def give(self, n: int) -> None:
        self.used -= n
        if self.used < 0:
            raise ValueError("budget released twice")


def _align(n: int, a: int = 512) -> int:
    return (n + a - 1) // a * a


def request_bytes(spec: ServeSpec, mode: int = lopc.NOA) -> Dict[str, int]:
    """Device bytes a request holds while admitted (rounded to the allocator's 512 B)."""
    d = lopc.make_desc(spec.shape, spec.dtype, mode, spec.eb)
    return {"input": _align(spec.nbytes), "state": _align(lopc.engine_field_workspace_size(d)),
            "output": _align(lopc.compress_bound(d))}


@dataclass
class Served:
    spec: ServeSpec
    status: int
    size: int
    arrival: float
    admitted: float
    done: float
    stream: Optional[torch.Tensor] = None

    @property
    def latency(self) -> float:
        return self.done - self.arrival


@dataclass
class ServeReport:
    served: List[Served]
    wall: float
    in_flight_mean: float
    in_flight_max: int
    queue_max: int
    steps: int
    budget_bytes: int
    budget_peak: int
    joined_busy: int = 0          # requests submitted while other fields were in repair
    notes: Dict[str, float] = field(default_factory=dict)

    def latencies(self) -> np.ndarray:
        return np.array([s.latency for s in self.served if s.status == lopc.OK])

    def percentile(self, q: float) -> float:
        lat = self.latencies()
        return float(np.percentile(lat, q)) if lat.size else float("nan")

    def sustained_gbs(self) -> float:
        ok = [s for s in self.served if s.status == lopc.OK]
        if not ok:
            return 0.0
        t0 = min(s.arrival for s in ok)
        t1 = max(s.done for s in ok)
        return sum(s.spec.nbytes for s in ok) / max(1e-9, t1 - t0) / 1e9


class Server:
    """One engine on one GPU, driven by one host thread."""

    def __init__(self, budget_bytes: int, max_fields: int = 512, max_tiles: int = 1 << 23,
                 rounds_per_step: int = 1, device=None):
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else device
        self.engine = lopc.Engine(max_fields, max_tiles)
        self.max_fields = max_fields
        self.rounds = rounds_per_step
        self.budget = Budget(budget_bytes)
        self.gen_stream = torch.cuda.Stream(self.device)

    def close(self) -> None:
        self.engine.sync()
        self.engine.close()

    def run(self, specs: Sequence[ServeSpec], keep_streams: bool = False, mode: int = lopc.NOA,
            make_input: Callable[[ServeSpec, torch.Tensor], None] = None,
            clock: Callable[[], float] = time.perf_counter) -> ServeReport:
        """Serves `specs` (sorted by arrival) in real time; returns per-request results."""
        make_input = make_input or (lambda s, x: make_field(s, self.device, out=x))
        pending = collections.deque(sorted(specs, key=lambda s: s.arrival))
        queue: collections.deque = collections.deque()
        inflight: Dict[int, dict] = {}
        served: List[Served] = []
        steps = 0
        joined_busy = 0
        occ_sum = 0
        occ_max = 0
        q_max = 0
        t0 = clock()
        while pending or queue or inflight:
            now = clock() - t0
            while pending and pending[0].arrival <= now:
                queue.append(pending.popleft())
            q_max = max(q_max, len(queue))
            # admission: first come first served, while the head fits in the budget
            while queue and len(inflight) < self.max_fields:
                s = queue[0]
                need = request_bytes(s, mode)
                total = sum(need.values())
                if total > self.budget.total:
                    raise ValueError(f"request {s.index} needs {total} bytes, more than the whole budget")
                if not self.budget.fits(total):
                    break
                d = lopc.make_desc(s.shape, s.dtype, mode, s.eb)
                tdt = torch.float32 if s.dtype == "f32" else torch.float64
                with torch.cuda.stream(self.gen_stream):
                    x = torch.empty(s.shape, dtype=tdt, device=self.device)
                    out = torch.empty(need["output"], dtype=torch.uint8, device=self.device)
                    ws = torch.empty(need["state"], dtype=torch.uint8, device=self.device)
                    make_input(s, x)
                rc = self.engine.submit(x, d, out, ws, s.index, ready_stream=self.gen_stream)
                if rc == lopc.ERR_BUSY:
                    break
                self.budget.take(total)
                if any(r["submitted_step"] < steps for r in inflight.values()):
                    joined_busy += 1
                inflight[s.index] = {"spec": s, "x": x, "out": out, "ws": ws, "need": total,
                                     "admitted": clock() - t0, "submitted_step": steps}
                queue.popleft()
            if inflight:
                self.engine.step(self.rounds)
                steps += 1
                occ_sum += len(inflight)
                occ_max = max(occ_max, len(inflight))
                for tag, size, st in self.engine.poll():
                    r = inflight.pop(tag)
                    t = clock() - t0
                    stream = r["out"][:size].clone() if (keep_streams and st == lopc.OK) else None
                    served.append(Served(r["spec"], st, size, r["spec"].arrival, r["admitted"], t, stream))
                    self.budget.give(r["need"])
            elif pending and not queue:
                # idle until the next arrival
                wait = pending[0].arrival - (clock() - t0)
                if wait > 0:
                    time.sleep(min(wait, 0.002))
        wall = clock() - t0
        return ServeReport(served, wall, occ_sum / max(1, steps), occ_max, q_max, steps, self.budget.total,
                           self.budget.peak, joined_busy)


def default_budget(fraction: float = 0.6, reserve: int = 8 << 30) -> int:
    """A share of the device memory that is free now, minus a reserve."""
    free, _ = torch.cuda.mem_get_info()
    return max(1 << 30, int(min(free * fraction, free - reserve)))


def solo_stream(spec: ServeSpec, mode: int = lopc.NOA, device=None) -> torch.Tensor:
    """The request compressed alone with lopc_compress (the reference for serving)."""
    tdt = torch.float32 if spec.dtype == "f32" else torch.float64
    x = torch.empty(spec.shape, dtype=tdt, device=device or "cuda")
    make_field(spec, x.device, out=x)
    return lopc.compress(x, spec.eb, mode)


def summary(rep: ServeReport, offered_gbs: float) -> dict:
    ok = [s for s in rep.served if s.status == lopc.OK]
    return {
        "requests": len(rep.served), "ok": len(ok),
        "p50_ms": rep.percentile(50) * 1e3, "p99_ms": rep.percentile(99) * 1e3,
        "sustained_gbs": rep.sustained_gbs(), "offered_gbs": offered_gbs,
        "in_flight_mean": rep.in_flight_mean, "in_flight_max": rep.in_flight_max, "queue_max": rep.queue_max,
        "steps": rep.steps, "joined_while_busy": rep.joined_busy,
        "budget_gb": rep.budget_bytes / 1e9, "budget_peak_gb": rep.budget_peak / 1e9,
        "wall_s": rep.wall,
    }
