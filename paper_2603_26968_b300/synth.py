"""Seeded synthetic scalar fields shaped like the paper's workloads (Table II).

The paper's inputs (Isabel, NYX, Miranda, S3D, ...) are SDRBench-style simulation
fields that are not available here.  These generators stand in for them: smooth
fields built from Gaussian bumps, optional value noise, optional snapping to a grid
(plateaus and exact ties) and sparse spikes.

Randomness is counter based: value ``i`` of a named stream is SplitMix64's output
for counter ``i + 1`` (Steele, Lea, Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014), mapped to ``[0, 1)`` with its top 53 bits.  Every draw is
therefore addressable and the fields are reproducible bit for bit with numpy on any
machine.  This module holds none of the compressor's arithmetic; the CPU oracle and
the CUDA path both read the bytes it returns.
"""
from __future__ import annotations

import hashlib
import math
from dataclasses import dataclass, field
from typing import List, Sequence, Tuple

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix64(z: np.ndarray) -> np.ndarray:
    z = z.copy()
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


def stream_seed(seed: int, name: str) -> int:
    """64-bit key of the stream ``name`` under ``seed``."""
    h = int.from_bytes(hashlib.sha256(f"{seed}:{name}".encode()).digest()[:8], "little")
    return h


def uniform(seed: int, name: str, start: int, count: int) -> np.ndarray:
    """Draws ``start .. start+count-1`` of stream ``name`` as float64 in [0, 1)."""
    with np.errstate(over="ignore"):
        ctr = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        z = np.uint64(stream_seed(seed, name)) + ctr * _GAMMA
        z = _mix64(z)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


# --------------------------------------------------------------------------- bumps

def _profile(n: int, c: float, sigma: float) -> Tuple[int, np.ndarray]:
    """exp(-(i-c)^2 / (2 sigma^2)) on the integer points within 4 sigma of c."""
    lo = max(0, int(math.ceil(c - 4.0 * sigma)))
    hi = min(n - 1, int(math.floor(c + 4.0 * sigma)))
    if hi < lo:
        return 0, np.zeros(0)
    i = np.arange(lo, hi + 1, dtype=np.float64)
    return lo, np.exp(-((i - c) ** 2) / (2.0 * sigma * sigma))


def add_bumps(f: np.ndarray, n_bumps: int, sigma_lo: float, sigma_hi: float,
              seed: int, name: str = "bumps") -> None:
    """Adds ``n_bumps`` truncated Gaussian bumps to the float64 array ``f`` in place.

    Bump ``j`` draws (amplitude, sigma, centre per axis) from stream ``name`` at
    counters ``j*(2+ndim) ...``: amplitude U[-1,1], sigma U[sigma_lo, sigma_hi],
    centre uniform over the domain in continuous coordinates.
    """
    nd = f.ndim
    per = 2 + nd
    u = uniform(seed, name, 0, n_bumps * per).reshape(n_bumps, per)
    for j in range(n_bumps):
        amp = 2.0 * u[j, 0] - 1.0
        sig = sigma_lo + (sigma_hi - sigma_lo) * u[j, 1]
        profs = [_profile(f.shape[d], u[j, 2 + d] * f.shape[d], sig) for d in range(nd)]
        if any(p[1].size == 0 for p in profs):
            continue
        if nd == 2:
            (y0, gy), (x0, gx) = profs
            box = f[y0:y0 + gy.size, x0:x0 + gx.size]
            box += np.multiply.outer(amp * gy, gx)
        else:
            (z0, gz), (y0, gy), (x0, gx) = profs
            gyx = None
            step = 16
            for zz in range(0, gz.size, step):
                gzs = gz[zz:zz + step]
                if gyx is None:
                    gyx = np.multiply.outer(gy, gx)
                box = f[z0 + zz:z0 + zz + gzs.size, y0:y0 + gy.size, x0:x0 + gx.size]
                box += (amp * gzs)[:, None, None] * gyx[None, :, :]


# ---------------------------------------------------------------------- value noise

def _smooth_axis(n: int, spacing: int) -> Tuple[np.ndarray, np.ndarray]:
    i = np.arange(n)
    cell = i // spacing
    t = (i % spacing) / float(spacing)
    return cell, t * t * (3.0 - 2.0 * t)


def add_value_noise(f: np.ndarray, spacings: Sequence[int], amps: Sequence[float],
                    seed: int, name: str = "vnoise") -> None:
    """Adds octaves of lattice value noise (values U[-1,1] on a lattice of the given
    spacing, tensor-product interpolation with smoothstep weights)."""
    for o, (sp, a) in enumerate(zip(spacings, amps)):
        lat_shape = tuple(n // sp + 2 for n in f.shape)
        lat = 2.0 * uniform(seed, f"{name}{o}", 0, int(np.prod(lat_shape))).reshape(lat_shape) - 1.0
        g = lat
        # interpolate one axis at a time, last axis first
        for ax in reversed(range(f.ndim)):
            cell, w = _smooth_axis(f.shape[ax], sp)
            g0 = np.take(g, cell, axis=ax)
            g1 = np.take(g, cell + 1, axis=ax)
            shp = [1] * f.ndim
            shp[ax] = -1
            wv = w.reshape(shp)
            g = g0 * (1.0 - wv) + g1 * wv
        f += a * g


def add_uniform_noise(f: np.ndarray, amp: float, seed: int, name: str = "noise") -> None:
    u = uniform(seed, name, 0, f.size).reshape(f.shape)
    f += amp * (2.0 * u - 1.0)


def snap_and_spike(f: np.ndarray, grid: float, spike_frac: float, seed: int) -> None:
    """Snaps ``f`` to multiples of ``grid`` (plateaus, exact ties) and adds sparse
    spikes of magnitude U[0.1, 0.5] x range with a random sign."""
    np.multiply(np.rint(f / grid), grid, out=f)
    rng = float(f.max() - f.min())
    n = f.size
    flat = f.reshape(-1)
    chunk = 1 << 24
    for s0 in range(0, n, chunk):
        m = min(chunk, n - s0)
        pick = uniform(seed, "spike_pick", s0, m) < spike_frac
        idx = np.nonzero(pick)[0]
        if idx.size == 0:
            continue
        mag = 0.1 + 0.4 * uniform(seed, "spike_mag", s0, m)[idx]
        sgn = np.where(uniform(seed, "spike_sign", s0, m)[idx] < 0.5, -1.0, 1.0)
        flat[s0 + idx] += sgn * mag * rng


# ------------------------------------------------------------------------ recipes

@dataclass
class FieldSpec:
    """One synthetic field: its shape, dtype, recipe and error bound."""
    name: str
    shape: Tuple[int, ...]
    dtype: str                      # "f32" or "f64"
    recipe: str                     # "bumps", "bumps_vnoise", "snapped"
    n_bumps: int
    sigma: Tuple[float, float]
    seed: int
    eb: float                       # NOA bound (fraction of the value range)
    noise: float = 0.0
    extra: dict = field(default_factory=dict)

    @property
    def nbytes(self) -> int:
        return int(np.prod(self.shape)) * (4 if self.dtype == "f32" else 8)


def make_field(spec: FieldSpec) -> np.ndarray:
    """Generates the field described by ``spec`` (C order, slowest axis first)."""
    f = np.zeros(spec.shape, dtype=np.float64)
    add_bumps(f, spec.n_bumps, spec.sigma[0], spec.sigma[1], spec.seed)
    if spec.recipe == "bumps_vnoise":
        sp = spec.extra.get("spacings", (64, 32, 16))
        am = spec.extra.get("amps", (0.05, 0.025, 0.0125))
        add_value_noise(f, sp, am, spec.seed)
    if spec.noise > 0.0:
        add_uniform_noise(f, spec.noise, spec.seed)
    if spec.recipe == "snapped":
        snap_and_spike(f, spec.extra.get("grid", 1e-3), spec.extra.get("spike_frac", 0.01), spec.seed)
    return f.astype(np.float32 if spec.dtype == "f32" else np.float64)


def field_sha256(x: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(x).tobytes()).hexdigest()


# Workloads of the paper's evaluation, synthesised.  The shapes follow the configs:
# a 2D image, NYX-sized 512^3 f32 and Miranda-sized 256x384x384 f64 (Table II).

def spec_2d_small(seed: int = 1, shape=(256, 256), eb: float = 1e-3) -> FieldSpec:
    """2D f32 256x256: 32 bumps (sigma U[4,40] px) + uniform noise 1e-4, NOA 1e-3."""
    return FieldSpec("2d_f32_bumps", tuple(shape), "f32", "bumps", 32, (4.0, 40.0), seed, eb, noise=1e-4)


def spec_3d_f32(seed: int = 1, n: int = 512, eb: float = 1e-3) -> FieldSpec:
    """3D f32 n^3: 256 bumps (sigma U[8,64] voxels at n=512, scaled with n) plus
    3-octave value noise (lattice spacing 64/32/16, amplitudes 0.05/0.025/0.0125)."""
    k = n / 512.0
    sp = tuple(max(2, int(round(s * k))) for s in (64, 32, 16))
    return FieldSpec(f"3d_f32_{n}", (n, n, n), "f32", "bumps_vnoise", 256, (8.0 * k, 64.0 * k), seed, eb,
                     extra={"spacings": sp, "amps": (0.05, 0.025, 0.0125)})


def spec_3d_f64_ties(seed: int = 1, shape=(256, 384, 384), eb: float = 5e-4) -> FieldSpec:
    """3D f64 (Miranda shape): 64 bumps (sigma U[16,96] at full size, scaled), snapped to
    a 1e-3 grid, 1 % spikes of U[0.1,0.5] x range."""
    k = shape[0] / 256.0
    return FieldSpec("3d_f64_ties", tuple(shape), "f64", "snapped", 64, (16.0 * k, 96.0 * k), seed, eb,
                     extra={"grid": 1e-3, "spike_frac": 0.01})


def spec_batch(seed: int = 1, count: int = 64, max_2d: int = 4096, max_3d: int = 384,
               min_2d: int = 128, min_3d: int = 64) -> List[FieldSpec]:
    """Mixed batch: ndim 2/3 with p=1/2; 2D side log-uniform [min_2d, max_2d], 3D side
    log-uniform [min_3d, max_3d] (1 in 10 anisotropic), f32/f64 with p=1/2, 16+side/8
    bumps plus 1e-4 uniform noise, NOA bound log-uniform in [1e-4, 1e-2]."""
    u = uniform(seed, "batch", 0, count * 8).reshape(count, 8)
    out = []
    for j in range(count):
        nd = 2 if u[j, 0] < 0.5 else 3
        dt = "f32" if u[j, 1] < 0.5 else "f64"
        eb = 10.0 ** (-4.0 + 2.0 * u[j, 2])
        if nd == 2:
            side = int(round(math.exp(math.log(min_2d) + (math.log(max_2d) - math.log(min_2d)) * u[j, 3])))
            shape = (side, side)
        else:
            side = int(round(math.exp(math.log(min_3d) + (math.log(max_3d) - math.log(min_3d)) * u[j, 3])))
            if u[j, 4] < 0.1:
                shape = (max(2, side // 2), side, side + side // 4)
            else:
                shape = (side, side, side)
        nb = 16 + side // 8
        sig = (side / 64.0, side / 8.0)
        out.append(FieldSpec(f"batch{j}", shape, dt, "bumps", nb, sig, seed * 1000 + j, eb, noise=1e-4))
    return out
