"""Seeded synthetic fields generated on the GPU, for the serving workload.

Serving offers up to ~200 fields per second of up to 1 GB each, far more than the
host generator in ``synth`` can produce, so these fields are made on the device.
A field is a sum of J separable Gaussian bumps (amplitude U[-1,1], centre uniform,
sigma log-uniform between side/64 and side/8 per axis) plus i.i.d. uniform noise of
amplitude 1e-4 in the field's dtype.  The bumps are a rank-J separable sum, so the
smooth part is one matrix product of per-axis profiles (no truncation at 4 sigma).
Bump parameters come from the counter-based streams of ``synth``; the noise comes
from a seeded torch generator on the device.  Nothing here touches the method's
arithmetic: this module only makes inputs.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import List, Sequence, Tuple

import numpy as np
import torch

from . import synth as S


@dataclass
class ServeSpec:
    """One request of the serving workload."""
    index: int
    arrival: float           # seconds after the start of serving
    shape: Tuple[int, ...]
    dtype: str               # "f32" or "f64"
    eb: float                # NOA bound (times the value range)
    seed: int

    @property
    def word(self) -> int:
        return 4 if self.dtype == "f32" else 8

    @property
    def nbytes(self) -> int:
        return int(np.prod(self.shape)) * self.word


def shape_for_bytes(nbytes: float, word: int, ndim: int) -> Tuple[int, ...]:
    """A near-cubic (or square) shape of about nbytes; 3D extents differ by a little
    so that no axis is special."""
    n = max(64.0, nbytes / word)
    if ndim == 2:
        side = max(8, int(round(math.sqrt(n))))
        return (side, max(8, int(round(n / side))))
    side = max(8, int(round(n ** (1.0 / 3.0))))
    return (side, side, max(8, int(round(n / (side * side)))))


def serve_requests(seed: int, rate: float, duration: float, min_bytes: float = 1e6,
                   max_bytes: float = 1e9, eb_lo: float = 1e-4, eb_hi: float = 1e-2) -> List[ServeSpec]:
    """Poisson arrivals at `rate` per second over `duration` seconds: exponential gaps,
    bytes log-uniform in [min_bytes, max_bytes], 2D or 3D and f32 or f64 with
    probability 1/2 each, NOA bound log-uniform in [eb_lo, eb_hi]."""
    out: List[ServeSpec] = []
    t = 0.0
    j = 0
    while True:
        u = S.uniform(seed, "serve", j * 6, 6)
        t += -math.log(max(u[0], 1e-300)) / rate
        if t >= duration:
            break
        nb = math.exp(math.log(min_bytes) + (math.log(max_bytes) - math.log(min_bytes)) * u[1])
        nd = 2 if u[2] < 0.5 else 3
        dt = "f32" if u[3] < 0.5 else "f64"
        eb = math.exp(math.log(eb_lo) + (math.log(eb_hi) - math.log(eb_lo)) * u[4])
        shape = shape_for_bytes(nb, 4 if dt == "f32" else 8, nd)
        out.append(ServeSpec(j, t, shape, dt, eb, seed * 1_000_003 + j))
        j += 1
    return out


def _profiles(n: int, centres: np.ndarray, sigmas: np.ndarray, device) -> torch.Tensor:
    """exp(-(i - c_j)^2 / (2 sigma_j^2)) for i in [0, n), one row per bump (float32)."""
    i = torch.arange(n, device=device, dtype=torch.float32)
    c = torch.from_numpy(centres.astype(np.float32)).to(device)[:, None]
    s = torch.from_numpy(sigmas.astype(np.float32)).to(device)[:, None]
    return torch.exp(-((i[None, :] - c) ** 2) / (2.0 * s * s))


def make_field(spec: ServeSpec, device="cuda", out: torch.Tensor = None) -> torch.Tensor:
    """The request's field on `device`, made on the current stream (into `out` if
    given: a contiguous tensor of the right shape and dtype)."""
    shape = spec.shape
    side = float(max(shape))
    nb = 8 + int(side) // 32
    u = S.uniform(spec.seed, "bumps", 0, nb * 8).reshape(nb, 8)
    amp = (2.0 * u[:, 0] - 1.0).astype(np.float32)
    lo, hi = math.log(side / 64.0), math.log(side / 8.0)
    sig = np.exp(lo + (hi - lo) * u[:, 1:4])
    cen = u[:, 4:7] * np.array([shape[0], shape[1], shape[-1]], dtype=np.float64)
    tdt = torch.float32 if spec.dtype == "f32" else torch.float64
    if out is None:
        out = torch.empty(shape, dtype=tdt, device=device)
    px = _profiles(shape[-1], cen[:, 2], sig[:, 2], device) * torch.from_numpy(amp).to(device)[:, None]
    if len(shape) == 2:
        a = _profiles(shape[0], cen[:, 0], sig[:, 0], device).t()              # (Y, J)
    else:
        pz = _profiles(shape[0], cen[:, 0], sig[:, 0], device)                  # (J, Z)
        py = _profiles(shape[1], cen[:, 1], sig[:, 1], device)                  # (J, Y)
        a = (pz[:, :, None] * py[:, None, :]).reshape(nb, -1).t()               # (Z*Y, J)
    flat = out.view(-1, shape[-1])
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        if tdt == torch.float32:
            torch.matmul(a.contiguous(), px, out=flat)
        else:
            flat.copy_(torch.matmul(a.contiguous(), px))
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    g = torch.Generator(device=out.device)
    g.manual_seed(int(spec.seed) & 0x7FFFFFFFFFFFFFFF)
    rows = max(1, (1 << 24) // shape[-1])           # noise in slabs of about 16 M values
    buf = torch.empty((min(rows, flat.shape[0]), shape[-1]), dtype=tdt, device=out.device)
    for r0 in range(0, flat.shape[0], rows):
        r1 = min(flat.shape[0], r0 + rows)
        nz = buf[: r1 - r0]
        torch.rand(nz.shape, generator=g, device=out.device, dtype=tdt, out=nz)
        flat[r0:r1].add_(nz.mul_(2e-4).sub_(1e-4))
    return out


def offered_load(specs: Sequence[ServeSpec], duration: float) -> float:
    """Offered bytes per second of a request list."""
    return sum(s.nbytes for s in specs) / duration
