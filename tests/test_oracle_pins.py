"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: the paper's worked
example, hand-derived fixtures, exact rational arithmetic, brute force over tiny
fields, closed forms, or invariants the paper proves (Sec. III-E).
"""
import itertools
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

# The Freudenthal offsets of the grid triangulation (Sec. II), written out here
# independently of the oracle: all non-zero 0/1 vectors and their negatives.
OFFS3 = [d for d in itertools.product((0, 1), repeat=3) if any(d)]
OFFS3 = OFFS3 + [tuple(-c for c in d) for d in OFFS3]


def neighbours(shape, i):
    sh = (1,) + tuple(shape) if len(shape) == 2 else tuple(shape)
    z, rem = divmod(i, sh[1] * sh[2])
    y, x = divmod(rem, sh[2])
    out = []
    for dz, dy, dx in OFFS3:
        zz, yy, xx = z + dz, y + dy, x + dx
        if 0 <= zz < sh[0] and 0 <= yy < sh[1] and 0 <= xx < sh[2]:
            out.append((zz * sh[1] + yy) * sh[2] + xx)
    return out


def sos_less(xf, a, b):
    """a precedes b: lower value, ties broken by the lower index (Sec. II)."""
    return xf[a] < xf[b] or (xf[a] == xf[b] and a < b)


def rint_half_even(fr: Fraction) -> int:
    return round(fr)  # Python rounds a Fraction half to even


# ----------------------------------------------------------------- quantizer

def test_worked_example_bin_10(orc):
    g = json.load(open(os.path.join(GOLDEN, "quantizer_worked_example.json")))
    x = np.array(g["inside"] + g["outside_below"] + g["outside_above"], np.float64)
    e = orc.resolve_eps(x.reshape(1, -1), 0, g["eb"])
    assert e["eps"] == g["eb"]
    b = orc.quantize(x, e["inv"])
    ni = len(g["inside"])
    nb = len(g["outside_below"])
    assert (b[:ni] == g["bin"]).all()
    assert (b[ni:ni + nb] < g["bin"]).all()
    assert (b[ni + nb:] > g["bin"]).all()
    # subbin 0 of bin 10 is the lowest double of the bin: just above 0.95
    lo = orc.lowest_in_bin(1, g["bin"], e["inv"])
    assert 0.9499 < lo <= 0.95 + 1e-12
    assert orc.q1(1, np.nextafter(lo, -np.inf), e["inv"]) == g["bin"] - 1


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_quantizer_matches_exact_rational(orc, dtype):
    rng = np.random.default_rng(7)
    for eb in (1e-2, 3.7e-4, 0.25, 1e-6):
        x = (rng.standard_normal(2000) * rng.choice([1e-3, 1.0, 50.0], 2000)).astype(dtype)
        x[:3] = [0.0, -0.0, np.finfo(dtype).tiny / 4]
        e = orc.resolve_eps(x.reshape(1, -1), 0, eb)
        b = orc.quantize(x, e["inv"])
        inv = Fraction(e["inv"])
        for xi, bi in zip(x[:500], b[:500]):
            assert bi == rint_half_even(Fraction(float(xi)) * inv)
        # eps_q = eps (1 - 2^-16), inv = 1/eps_q, both single IEEE roundings
        assert Fraction(e["eps_q"]) == Fraction(eb * (1.0 - 2.0 ** -16))


def test_quantizer_ties_round_to_even(orc):
    # inv = 1: the product is the value itself, so half-integers are exact ties
    for v, want in [(2.5, 2), (3.5, 4), (-2.5, -2), (-3.5, -4), (0.5, 0), (1.5, 2), (2.4999999, 2)]:
        assert orc.q1(1, v, 1.0) == want


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_quantizer_monotone(orc, dtype):
    rng = np.random.default_rng(3)
    x = np.sort(np.concatenate([rng.standard_normal(20000), [0.0, -0.0, 1e-40, -1e-40]]).astype(dtype))
    e = orc.resolve_eps(x.reshape(1, -1), 0, 1e-3)
    b = orc.quantize(x, e["inv"])
    assert (np.diff(b) >= 0).all()


def test_range_limit(orc):
    x = np.array([[1.0, 2.0]], np.float32)
    assert orc.compress_status(x, 0, 1e-12) == orc.RANGE           # 2e12 bins > 2^30
    assert orc.compress_status(x.astype(np.float64), 0, 1e-12) == 0  # f64 bins up to 2^52


@pytest.mark.parametrize("dtype_c", [0, 1])
def test_bin_span_below_eps(orc, dtype_c):
    """Sec. III-A/III-E: every value of a bin lies within eps of every other, which
    the shrink eps_q = eps (1 - 2^-16) guarantees; lo(b) is the bin's minimum."""
    rng = np.random.default_rng(11)
    for eps in (1e-3, 0.37, 1e-6):
        e = orc.resolve_eps(np.zeros((1, 2)), 0, eps)
        for b in rng.integers(-10**5, 10**5, 60):
            lo = orc.lowest_in_bin(dtype_c, int(b), e["inv"])
            lo_next = orc.lowest_in_bin(dtype_c, int(b) + 1, e["inv"])
            hi = orc.succ_k(dtype_c, lo_next, 0)
            hi = np.nextafter(np.float32(hi), np.float32(-np.inf)) if dtype_c == 0 else np.nextafter(hi, -np.inf)
            assert orc.q1(dtype_c, float(lo), e["inv"]) == b
            assert orc.q1(dtype_c, float(hi), e["inv"]) == b
            below = np.nextafter(np.float32(lo), np.float32(-np.inf)) if dtype_c == 0 else np.nextafter(lo, -np.inf)
            assert orc.q1(dtype_c, float(below), e["inv"]) == b - 1
            assert Fraction(float(hi)) - Fraction(float(lo)) < Fraction(eps)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_succ_k_walks_representable_values(orc, dtype):
    dc = 0 if dtype == np.float32 else 1
    for v0 in [dtype(1.0), dtype(-1.0), dtype(-np.finfo(dtype).tiny), dtype(0.0), dtype(-3 * np.finfo(dtype).smallest_subnormal)]:
        v = v0
        for k in range(8):
            got = orc.succ_k(dc, float(v0), k)
            want = v if v != 0 else dtype(0.0)
            assert dtype(got) == want and not (got == 0 and math.copysign(1, got) < 0)
            v = np.nextafter(v, dtype(np.inf))   # passes -0 then +0: one position


def test_resolve_eps_modes(orc):
    x = np.array([[3.0, -1.5], [2.0, 0.25]], np.float32)
    assert orc.resolve_eps(x, 0, 0.01)["eps"] == 0.01
    e = orc.resolve_eps(x, 1, 0.01)
    assert e["eps"] == 0.01 * (3.0 - (-1.5))
    c = orc.resolve_eps(np.full((3, 3), -0.0, np.float64), 1, 0.01)
    assert c["constant"] and c["const_value"] == 0.0 and math.copysign(1, c["const_value"]) > 0
    bad = x.copy()
    bad[0, 0] = np.nan
    assert orc.compress_status(bad, 1, 0.01) == orc.NONFINITE
    bad[0, 0] = np.inf
    assert orc.compress_status(bad, 0, 0.01) == orc.NONFINITE
    assert orc.compress_status(x, 0, 0.0) == orc.INVALID_ARG
    assert orc.compress_status(x, 0, -1.0) == orc.INVALID_ARG
    assert orc.compress_status(x, 0, float("nan")) == orc.INVALID_ARG


# ----------------------------------------------------------------- repair

def test_repair_hand_chains(orc):
    g = json.load(open(os.path.join(GOLDEN, "repair_chains.json")))
    for c in g["cases"]:
        x = np.array([c["x"]], np.float64)
        b = orc.quantize(x, orc.resolve_eps(x, 0, 10.0)["inv"])
        assert (b == 0).all()
        assert orc.repair_lfp(x, b).ravel().tolist() == c["s"], c["why"]
        s2, _ = orc.repair_alg2(x, b)
        assert s2.ravel().tolist() == c["s"]


def constraints(x, b):
    xf = x.ravel().tolist()
    bf = b.ravel().tolist()
    out = []
    for p in range(len(xf)):
        for n in neighbours(x.shape, p):
            if bf[n] == bf[p] and sos_less(xf, n, p):
                out.append((n, p, 1 if n > p else 0))
    return out


def brute_least(n, cons, kmax):
    grid = np.array(list(itertools.product(range(kmax + 1), repeat=n)), np.int64)
    ok = np.ones(len(grid), bool)
    for (a, p, t) in cons:
        ok &= grid[:, p] >= grid[:, a] + t
    valid = grid[ok]
    if len(valid) == 0:
        return None
    least = valid.min(axis=0)
    return least


def tiny_fields():
    for shape, vals in [((2, 2), (0, 1, 2)), ((2, 3), (0, 1, 2)), ((1, 5), (0, 1, 2)), ((2, 2, 2), (0, 1))]:
        n = int(np.prod(shape))
        for combo in itertools.product(vals, repeat=n):
            yield np.array(combo, np.float64).reshape(shape)


def test_repair_three_way_exhaustive(orc):
    """Sort-based least fixpoint == the paper's Alg. 2 iteration == brute-force
    least solution, on every field of a few tiny shapes (heavy ties)."""
    count = 0
    for x in tiny_fields():
        b = np.zeros(x.shape, np.int64)          # one bin: every neighbour constrains
        s = orc.repair_lfp(x, b).ravel()
        s2, _ = orc.repair_alg2(x, b)
        assert (s == s2.ravel()).all()
        cons = constraints(x, b)
        kmax = min(x.size - 1, 4)
        if s.max() <= kmax and x.size <= 8:
            least = brute_least(x.size, cons, kmax)
            assert least is not None and (least == s).all()
        # the solution is valid
        for (a, p, t) in cons:
            assert s[p] >= s[a] + t
        count += 1
    assert count > 500


def test_repair_bounds_on_random_fields(orc):
    """Sec. III-E: same-bin local minima stay 0; no point exceeds its highest same-bin
    neighbour + 1; subbins lie in [0, n-1] for a same-bin component of n points."""
    rng = np.random.default_rng(5)
    for shape in [(9, 11), (5, 6, 7)]:
        x = np.round(rng.standard_normal(shape), 1)
        e = orc.resolve_eps(x, 1, 0.2)
        b = orc.quantize(x, e["inv"])
        s = orc.repair_lfp(x, b).ravel()
        s2, iters = orc.repair_alg2(x, b)
        assert (s == s2.ravel()).all() and iters >= 1
        xf, bf = x.ravel().tolist(), b.ravel().tolist()
        # components of same-bin neighbours
        comp = list(range(x.size))

        def find(i):
            while comp[i] != i:
                comp[i] = comp[comp[i]]
                i = comp[i]
            return i
        for p in range(x.size):
            for n in neighbours(shape, p):
                if bf[n] == bf[p]:
                    comp[find(n)] = find(p)
        size = {}
        for p in range(x.size):
            size[find(p)] = size.get(find(p), 0) + 1
        for p in range(x.size):
            same = [n for n in neighbours(shape, p) if bf[n] == bf[p]]
            lower = [n for n in same if sos_less(xf, n, p)]
            if not lower:
                assert s[p] == 0
            if same:
                assert s[p] <= max(s[n] for n in same) + 1
            assert s[p] <= size[find(p)] - 1


def test_constraint_masks_brute_force(orc):
    rng = np.random.default_rng(2)
    x = np.round(rng.standard_normal((3, 4, 5)), 1)
    b = orc.quantize(x, orc.resolve_eps(x, 1, 0.3)["inv"])
    m = orc.constraint_masks(x, b).ravel()
    want = {}
    for (n, p, t) in constraints(x, b):
        want.setdefault(p, set()).add(n)
    for p in range(x.size):
        assert bin(int(m[p])).count("1") == len(want.get(p, ()))


# ----------------------------------------------------------------- decode, whole method

@pytest.mark.parametrize("shape,dtype,eb", [((37, 53), np.float32, 1e-2), ((37, 53), np.float64, 1e-3),
                                            ((9, 21, 19), np.float32, 3e-2), ((9, 21, 19), np.float64, 1e-4)])
def test_roundtrip_invariants(orc, shape, dtype, eb):
    rng = np.random.default_rng(13)
    x = (np.cumsum(rng.standard_normal(shape), axis=-1) * 0.1).astype(dtype)
    x.ravel()[::17] = x.ravel()[::13][: x.ravel()[::17].size]       # plant exact ties
    st = orc.compress(x, 1, eb)
    y = orc.decompress(st)
    e = orc.resolve_eps(x, 1, eb)
    b = orc.quantize(x, e["inv"])
    s = orc.repair_lfp(x, b)
    assert (orc.reconstruct(0 if dtype == np.float32 else 1, b, s, e["inv"]) == y).all()
    xd, yd = x.astype(np.float64), y.astype(np.float64)
    assert (yd <= xd).all()                                            # x_hat <= x
    assert np.abs(xd - yd).max() < e["eps"]                            # |x - x_hat| < eps
    assert (orc.quantize(y, e["inv"]) == b).all()                      # q(x_hat) = b
    assert orc.order_violations(x, y) == 0                             # local order kept
    lx, ux = orc.critical_types(x)
    ly, uy = orc.critical_types(y)
    assert (lx == ly).all() and (ux == uy).all()                       # Table III: 0/0/0


def test_exhaustive_tiny_fields_roundtrip(orc):
    for x in tiny_fields():
        for eb in (0.9, 0.3):
            st = orc.compress(x, 1, eb) if x.max() > x.min() else orc.compress(x, 0, eb)
            y = orc.decompress(st)
            assert orc.order_violations(x, y) == 0
            lx, ux = orc.critical_types(x)
            ly, uy = orc.critical_types(y)
            assert (lx == ly).all() and (ux == uy).all()


def test_order_checker_detects_a_planted_flip(orc):
    rng = np.random.default_rng(1)
    x = rng.standard_normal((8, 8)).astype(np.float32)
    y = orc.decompress(orc.compress(x, 1, 1e-2))
    assert orc.order_violations(x, y) == 0
    i = int(np.argmax(x))
    y2 = y.copy()
    y2.ravel()[i] = y.min() - 1.0                 # the maximum becomes a minimum
    assert orc.order_violations(x, y2) > 0
    l2, u2 = orc.critical_types(y2)
    lx, ux = orc.critical_types(x)
    assert not ((lx == l2).all() and (ux == u2).all())


def test_critical_types_hand_examples(orc):
    # single peak in the middle of a 3x3 image: a maximum (upper link empty)
    x = np.array([[0, 1, 0], [1, 5, 1], [0, 1, 0]], np.float64)
    lo, up = orc.critical_types(x)
    assert up[1, 1] == 0 and lo[1, 1] == 1
    # the link of the centre is the hexagon (0,1),(1,1),(1,0),(0,-1),(-1,-1),(-1,0);
    # alternate high/low around it: a saddle with 3 lower and 3 upper pieces
    x = np.zeros((3, 3))
    ring = [(1, 2), (2, 2), (2, 1), (1, 0), (0, 0), (0, 1)]
    for k, (r, c) in enumerate(ring):
        x[r, c] = 1.0 if k % 2 == 0 else -1.0
    x[0, 2] = x[2, 0] = 0.5
    lo, up = orc.critical_types(x)
    assert lo[1, 1] == 3 and up[1, 1] == 3
    # a monotone ramp: the centre is regular (1, 1)
    x = np.add.outer(np.arange(3.0), np.arange(3.0) * 0.1)
    lo, up = orc.critical_types(x)
    assert lo[1, 1] == 1 and up[1, 1] == 1
