"""Launch autotuner for batched compression.

It searches the launch plan (``lopc_plan``) of a batch, per field class (f32 2D, f32
3D, f64 2D, f64 3D):
  - rerun_blocks_per_sm: how a repair round's tile list is spread over the GPU;
  - pass_order: the order in which the tile pass takes a field's tiles (by the
    field's sampled bin span, tile index, or ascending tile key), which decides how
    much chain work the pass does and how many repair rounds follow;
  - pass_budget16 and pass_dense16: when a tile's fixpoint leaves its frontier
    sweeps for the topological order.
The chunk geometry (the tile that is also the stream's chunk) is part of the format
and never tuned.  Output bytes do not depend on the plan (the repair's result is the
unique least fixpoint, Sec. III-E), so the tuner only times.

Search: coordinate descent over (knob, class) for the classes present, starting
from the library's default plan.  Each trial passes its plan to the batch
explicitly, runs once untimed (graph capture), then is timed with CUDA events
(median of ``reps``, L2 flushed before each).  Results are cached in a JSON file
keyed by device name and workload signature.
"""
from __future__ import annotations

import json
import os
from pathlib import Path
from typing import Callable, Dict, Iterable, List, Optional, Sequence

import numpy as np
import torch

from . import lopc

KNOBS = {
    "pass_order": (0, 1, 2),
    "rerun_blocks_per_sm": (1, 2, 3, 4, 6, 8),
    "pass_dense16": (4, 8, 12, 17),
    "pass_budget16": (16, 64, 256, 4096),
}
DEFAULT_CACHE = Path(__file__).resolve().parent / "tuned.json"


def signature(descs: Iterable) -> str:
    """Workload key: fields and tiles per class, in powers of two."""
    cnt = [0, 0, 0, 0]
    pts = [0, 0, 0, 0]
    for d in descs:
        c = (2 if d.dtype == lopc.F64 else 0) + (1 if d.ndim == 3 else 0)
        cnt[c] += 1
        pts[c] += int(np.prod([d.dims[k] for k in range(d.ndim)]))
    return ",".join(f"{n}:{int(np.log2(p)) if p else 0}" for n, p in zip(cnt, pts))


def classes_of(descs: Iterable) -> List[int]:
    return sorted({(2 if d.dtype == lopc.F64 else 0) + (1 if d.ndim == 3 else 0) for d in descs})


def time_ms(run: Callable[[], None], reps: int = 3, flush: Optional[torch.Tensor] = None) -> List[float]:
    """CUDA-event times of `reps` runs on the current stream, L2 flushed before each
    (a write of `flush`, a buffer larger than L2) when given."""
    st = torch.cuda.current_stream()
    out = []
    for _ in range(reps):
        if flush is not None:
            flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        run()
        b.record(st)
        b.synchronize()
        out.append(a.elapsed_time(b))
    return out


def tune(run: Callable[[lopc.Plan], None], classes: Sequence[int], reps: int = 3,
         flush: Optional[torch.Tensor] = None, knobs: Dict[str, Sequence[int]] = KNOBS,
         timer: Optional[Callable[[Callable[[], None]], List[float]]] = None) -> Dict:
    """Coordinate descent over the plan's knobs for the given classes.  `run(plan)`
    enqueues one batch with that plan; `timer(fn)` gives the times of `reps` runs of
    fn (CUDA events with L2 flushed by default).  Returns the best plan (as a dict),
    its time, the default plan's time and spread, and the trial log."""
    if timer is None:
        timer = lambda fn: time_ms(fn, reps, flush)  # noqa: E731

    def trial(d: dict) -> List[float]:
        pl = lopc.Plan.of(d)
        run(pl)                                     # graph capture, clocks up
        return timer(lambda: run(pl))

    best = lopc.plan_default().as_dict()
    t0 = trial(best)
    default_ms, best_ms = float(np.median(t0)), float(np.median(t0))
    trials = [{"plan": json.loads(json.dumps(best)), "ms": best_ms}]
    for knob, values in knobs.items():
        for c in classes:
            start = best[knob][c]  # measured already, with the other knobs as they are
            for v in values:
                if v == start or v == best[knob][c]:
                    continue
                cand = json.loads(json.dumps(best))
                cand[knob][c] = v
                ms = float(np.median(trial(cand)))
                trials.append({"knob": knob, "cls": c, "value": v, "ms": ms})
                if ms < best_ms:
                    best, best_ms = cand, ms
    # the default timed again beside the winner, for the noise level
    t1 = trial(lopc.plan_default().as_dict())
    return {"plan": best, "ms": best_ms, "default_ms": default_ms,
            "default_spread_ms": float(max(t0 + t1) - min(t0 + t1)), "trials": trials}


def apply(plan: dict) -> None:
    """Makes `plan` this thread's current plan (lopc_tune_*), which single-field calls
    and batches launched without a plan use."""
    lopc.tune_set(plan["rerun_blocks_per_sm"])
    lopc.tune_set_budget(plan["pass_budget16"])
    lopc.tune_set_dense(plan["pass_dense16"])
    lopc.tune_set_pass_order(plan["pass_order"])


def load(key: str, path: Optional[Path] = None) -> Optional[Dict]:
    p = Path(path or DEFAULT_CACHE)
    if not p.exists():
        return None
    try:
        v = json.loads(p.read_text()).get(key)
    except (OSError, ValueError):
        return None
    return v if isinstance(v, dict) and "plan" in v else None


def save(key: str, value: Dict, path: Optional[Path] = None) -> None:
    p = Path(path or DEFAULT_CACHE)
    data = {}
    if p.exists():
        try:
            data = json.loads(p.read_text())
        except (OSError, ValueError):
            data = {}
    data[key] = value
    tmp = p.with_suffix(f".{os.getpid()}.tmp")
    tmp.write_text(json.dumps(data, indent=1, sort_keys=True))
    os.replace(tmp, p)


def device_key(descs) -> str:
    return f"{torch.cuda.get_device_name()}|{signature(descs)}"
