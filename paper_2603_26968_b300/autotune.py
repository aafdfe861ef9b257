"""Launch autotuner for batched compression.

The tunable is the number of persistent rerun blocks per SM for each field class
(f32 2D, f32 3D, f64 2D, f64 3D): it sets how a repair round's tile list is spread
over the GPU, the round schedule of a batch.  The chunk geometry (the tile that is
also the stream's chunk) is part of the format and never tuned.  Output bytes do not
depend on the tunables, so the tuner only times.

Search: coordinate descent over the classes present in the workload, each trial
timed with CUDA events (median of `reps`); results are cached in a JSON file keyed
by device name and workload signature.
"""
from __future__ import annotations

import json
import os
from pathlib import Path
from typing import Callable, Dict, Iterable, List, Optional, Sequence

import numpy as np
import torch

from . import lopc

CANDIDATES = (1, 2, 3, 4, 6, 8)
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


def time_ms(run: Callable[[], None], reps: int = 3) -> float:
    st = torch.cuda.current_stream()
    out = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        run()
        b.record(st)
        b.synchronize()
        out.append(a.elapsed_time(b))
    return float(np.median(out))


def tune(run: Callable[[], None], classes: Sequence[int], candidates: Sequence[int] = CANDIDATES,
         reps: int = 3) -> Dict:
    """Coordinate descent over the rerun blocks per SM of the given classes; leaves
    the best setting active and returns it with the trial log."""
    best = list(lopc.tune_get())
    lopc.tune_set(best)
    run()                                          # warm: graphs captured, clocks up
    best_ms = time_ms(run, reps)
    trials = [{"setting": list(best), "ms": best_ms}]
    for c in classes:
        for v in candidates:
            if v == best[c]:
                continue
            cand = list(best)
            cand[c] = v
            lopc.tune_set(cand)
            run()
            ms = time_ms(run, reps)
            trials.append({"setting": cand, "ms": ms})
            if ms < best_ms:
                best, best_ms = cand, ms
    lopc.tune_set(best)
    return {"rerun_blocks_per_sm": best, "ms": best_ms, "trials": trials}


def load(key: str, path: Optional[Path] = None) -> Optional[Dict]:
    p = Path(path or DEFAULT_CACHE)
    if not p.exists():
        return None
    try:
        return json.loads(p.read_text()).get(key)
    except (OSError, ValueError):
        return None


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
