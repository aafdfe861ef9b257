"""Pins of the oracle's verification summary: critical-point types (Sec. II),
Table III's false positives / negatives / types, local order, the error bound
(Sec. III-A) and PSNR.

The link structure is pinned against the triangulation itself: the tests build the
Kuhn (Freudenthal) simplices of the grid explicitly (two triangles per square, six
tetrahedra per cube, all along the main diagonal) and take links from them, which
shares nothing with the oracle's neighbour-offset rule.  Summary counts are pinned
by closed forms (a negated field, a constant field, a shifted field) and by the
Euler characteristic of a 2D grid.
"""
import itertools

import numpy as np
import pytest

import oracle as O


# ---------------------------------------------------------------- explicit complex

def kuhn_simplices(shape):
    """Top simplices of the Kuhn triangulation of a grid of `shape` (2D or 3D), as
    tuples of vertex coordinates: each unit cell is cut along its main diagonal into
    the chains corner -> corner + e_a -> ... -> corner + (1, ..., 1)."""
    axes = [a for a, n in enumerate(shape) if n > 1]  # a grid one point thick along an
    out = []                                           # axis is triangulated over the others
    if not axes:
        return [(tuple(0 for _ in shape),)]
    for corner in itertools.product(*[range(n - 1) if n > 1 else [0] for n in shape]):
        for perm in itertools.permutations(axes):
            v = list(corner)
            chain = [tuple(v)]
            for a in perm:
                v[a] += 1
                chain.append(tuple(v))
            out.append(tuple(chain))
    return out


def links_from_simplices(shape):
    """For every vertex: its link vertices and link edges (pairs of other vertices of
    a simplex containing it)."""
    verts = {}
    edges = {}
    for s in kuhn_simplices(shape):
        for v in s:
            others = [u for u in s if u != v]
            verts.setdefault(v, set()).update(others)
            es = edges.setdefault(v, set())
            for a, b in itertools.combinations(others, 2):
                es.add((min(a, b), max(a, b)))
    return verts, edges


def components(nodes, edges):
    par = {v: v for v in nodes}

    def find(v):
        while par[v] != v:
            v = par[v]
        return v

    for a, b in edges:
        if a in par and b in par:
            ra, rb = find(a), find(b)
            if ra != rb:
                par[ra] = rb
    return sum(1 for v in nodes if find(v) == v)


def brute_types(x):
    """(lower, upper) link component counts of every point from the explicit complex,
    with the order 'value, then flat index' (Simulation of Simplicity)."""
    shape = x.shape
    verts, edges = links_from_simplices(shape)
    flat = lambda v: int(np.ravel_multi_index(v, shape))
    lo = np.zeros(shape, np.uint8)
    up = np.zeros(shape, np.uint8)
    for v in itertools.product(*[range(n) for n in shape]):
        lk = verts.get(v, set())
        below = {u for u in lk if (x[u], flat(u)) < (x[v], flat(v))}
        above = lk - below
        es = edges.get(v, set())
        lo[v] = components(below, [e for e in es if e[0] in below and e[1] in below])
        up[v] = components(above, [e for e in es if e[0] in above and e[1] in above])
    return lo, up


@pytest.mark.parametrize("shape", [(5, 6), (1, 7), (6, 1), (2, 2), (4, 5, 3), (3, 3, 3), (1, 4, 5), (2, 3, 1)])
@pytest.mark.parametrize("levels", [3, 1000])
def test_critical_types_match_explicit_triangulation(shape, levels):
    rng = np.random.default_rng(hash((shape, levels)) % 2**32)
    for _ in range(4):
        x = rng.integers(0, levels, shape).astype(np.float64)  # few levels: many ties
        lo, up = O.critical_types(x)
        blo, bup = brute_types(x)
        assert (lo == blo).all() and (up == bup).all()


def test_explicit_complex_is_a_triangulated_square_and_cube():
    # sanity of the test's own complex: Euler characteristic 1 (a disc, a ball)
    for shape in [(3, 4), (3, 3, 4)]:
        simp = kuhn_simplices(shape)
        faces = set()
        for s in simp:
            for k in range(1, len(s) + 1):
                faces.update(itertools.combinations(sorted(s), k))
        chi = sum((-1) ** (len(f) - 1) for f in faces)
        assert chi == 1


# ---------------------------------------------------------------- hand cases (3D)

def quad3(a, b, c):
    """a z^2 + b y^2 + c x^2 on the 3x3x3 grid centred at the origin."""
    z, y, x = np.meshgrid(*[np.arange(-1.0, 2.0)] * 3, indexing="ij")
    return a * z * z + b * y * y + c * x * x


def test_critical_types_3d_saddles_by_hand():
    # f = z^2 + y^2 - 3 x^2 at the centre: the lower neighbours are +-(0,0,1),
    # +-(0,1,1), +-(1,0,1), +-(1,1,1) -- the four positive offsets are pairwise
    # adjacent, the four negative ones too, and no positive one is adjacent to a
    # negative one: two lower pieces; the upper ones form the hexagon
    # (0,1,0),(1,1,0),(1,0,0),(0,-1,0),(-1,-1,0),(-1,0,0): one piece.
    lo, up = O.critical_types(quad3(1, 1, -3))
    assert (lo[1, 1, 1], up[1, 1, 1]) == (2, 1)
    lo, up = O.critical_types(-quad3(1, 1, -3))          # negated: the other saddle
    assert (lo[1, 1, 1], up[1, 1, 1]) == (1, 2)
    lo, up = O.critical_types(quad3(1, 1, 1))            # bowl: a minimum
    assert (lo[1, 1, 1], up[1, 1, 1]) == (0, 1)
    lo, up = O.critical_types(-quad3(1, 1, 1))           # cap: a maximum
    assert (lo[1, 1, 1], up[1, 1, 1]) == (1, 0)
    z, y, x = np.meshgrid(*[np.arange(3.0)] * 3, indexing="ij")
    lo, up = O.critical_types(x + 0.1 * y + 0.01 * z)    # a generic linear ramp
    assert (lo[1, 1, 1], up[1, 1, 1]) == (1, 1)


# ---------------------------------------------------------------- Euler characteristic (2D)

@pytest.mark.parametrize("shape", [(7, 9), (1, 5), (2, 2), (12, 3)])
def test_euler_characteristic_2d(shape):
    """Summing 1 - chi(lower link) over the vertices gives the Euler characteristic
    of the square, 1 (each simplex counted at its highest vertex).  In 2D a lower
    link is a union of paths (chi = its component count) except the full hexagon of
    an interior maximum (chi = 0)."""
    rng = np.random.default_rng(sum(shape))
    for levels in (2, 5, 10**6):
        x = rng.integers(0, levels, shape).astype(np.float64)
        lo, up = O.critical_types(x)
        interior = np.zeros(shape, bool)
        interior[1:-1, 1:-1] = True
        total = int((1 - lo.astype(np.int64)).sum()) + int((interior & (up == 0)).sum())
        assert total == 1


# ---------------------------------------------------------------- summary closed forms

def neighbour_pairs(shape):
    """Edges of the triangulation: for every positive offset d in {0,1}^n \\ 0, the
    points p with p + d inside the grid."""
    nd = len(shape)
    tot = 0
    for d in itertools.product([0, 1], repeat=nd):
        if any(d):
            tot += int(np.prod([n - k for n, k in zip(shape, d)]))
    return tot


@pytest.mark.parametrize("shape", [(13, 11), (5, 6, 7)])
def test_verify_negated_field(shape):
    # distinct values: negation reverses every neighbour pair; minima and maxima swap
    # (false types), saddles stay saddles, regular points stay regular
    rng = np.random.default_rng(3)
    x = rng.permutation(int(np.prod(shape))).reshape(shape).astype(np.float64)
    r = O.verify(x, -x, 0, 1e9)
    lo, up = O.critical_types(x)
    assert r["order_violations"] == neighbour_pairs(shape)
    assert r["cp_y"] == [r["cp_x"][1], r["cp_x"][0], r["cp_x"][2], r["cp_x"][3]]
    assert r["false_positives"] == 0 and r["false_negatives"] == 0
    assert r["false_types"] == r["cp_x"][0] + r["cp_x"][1]
    assert r["link_mismatches"] == int((lo != up).sum())


@pytest.mark.parametrize("shape", [(9, 8), (4, 5, 6)])
def test_verify_constant_reconstruction(shape):
    # a constant y orders points by index alone: a linear function on a convex grid,
    # so one minimum (the first point), one maximum (the last) and no saddle
    rng = np.random.default_rng(4)
    x = rng.standard_normal(shape)
    y = np.zeros(shape)
    r = O.verify(x, y, 0, 10.0)
    n = x.size
    assert r["cp_y"] == [1, 1, 0, n - 2]
    cx = O.classify(*O.critical_types(x)).ravel()
    crit = cx != O.CP_REGULAR
    ends = np.zeros(n, bool)
    ends[[0, n - 1]] = True
    assert r["false_negatives"] == int((crit & ~ends).sum())
    assert r["false_positives"] == int((~crit & ends).sum())
    assert r["false_types"] == int(crit[0] and cx[0] != O.CP_MIN) + int(crit[-1] and cx[-1] != O.CP_MAX)


def test_verify_shifted_field_error_terms():
    # dyadic values and shift: every difference and square is exact
    rng = np.random.default_rng(5)
    x = rng.integers(-64, 64, (6, 7, 8)).astype(np.float64) / 8.0
    c = 0.25
    for dt in (np.float64, np.float32):
        xs = x.astype(dt)
        r = O.verify(xs, xs + dt(c), 1, 0.01)
        assert r["order_violations"] == 0 and r["link_mismatches"] == 0
        assert r["false_positives"] == r["false_negatives"] == r["false_types"] == 0
        assert r["max_abs_err"] == c and r["mse"] == c * c
        rng_ = float(x.max() - x.min())
        assert r["x_min"] == float(x.min()) and r["x_max"] == float(x.max())
        assert r["psnr"] == pytest.approx(20 * np.log10(rng_ / c), abs=1e-12)
        assert r["eps"] == pytest.approx(0.01 * rng_, rel=1e-15)
        assert r["bound_ok"] == (c <= 0.01 * rng_)
    r = O.verify(x, x, 0, 1e-3)
    assert r["psnr"] == float("inf") and r["max_abs_err"] == 0.0 and r["bound_ok"]


def test_verify_roundtrip_has_table_iii_zeros():
    # Table III: LOPC's reconstructions have 0 false positives / negatives / types
    from paper_2603_26968_b300 import synth
    x = synth.make_field(synth.FieldSpec("t", (24, 40, 33), "f32", "bumps", 12, (3.0, 12.0), 7, 1e-3, noise=1e-3))
    for eb in (1e-2, 1e-3):
        y = O.decompress(O.compress(x, 1, eb))
        r = O.verify(x, y, 1, eb)
        assert r["order_violations"] == 0 and r["link_mismatches"] == 0
        assert r["false_positives"] == r["false_negatives"] == r["false_types"] == 0
        assert r["cp_x"] == r["cp_y"] and r["bound_ok"] and r["max_abs_err"] > 0


def test_verify_rejects_nonfinite():
    x = np.zeros((3, 3))
    y = x.copy()
    y[1, 1] = np.nan
    with pytest.raises(O.OracleError):
        O.verify(x, y)


def brute_class(lo, up):
    """Sec. II's rule, point by point: empty lower link -> minimum (0); empty upper
    link -> maximum (1); one piece each -> regular (3); otherwise saddle (2)."""
    out = np.empty(lo.shape, np.uint8)
    for i in np.ndindex(lo.shape):
        l, u = int(lo[i]), int(up[i])
        out[i] = 0 if l == 0 else 1 if u == 0 else 3 if (l == 1 and u == 1) else 2
    return out


@pytest.mark.parametrize("shape", [(6, 7), (4, 4, 5)])
def test_verify_counts_brute_force(shape):
    # y = x with a few points moved: every count of the summary against the explicit
    # complex and Table III's definitions, point by point
    rng = np.random.default_rng(11)
    for trial in range(6):
        x = rng.integers(0, 6, shape).astype(np.float64)
        y = x.copy()
        idx = rng.choice(x.size, size=1 + trial, replace=False)
        y.ravel()[idx] = rng.integers(-3, 9, idx.size)
        r = O.verify(x, y, 0, 100.0)
        lx, ux = brute_types(x)
        ly, uy = brute_types(y)
        cx, cy = brute_class(lx, ux), brute_class(ly, uy)
        fp = fn = ft = 0
        for i in np.ndindex(shape):
            kx, ky = cx[i] != 3, cy[i] != 3
            fp += (not kx) and ky
            fn += kx and not ky
            ft += kx and ky and cx[i] != cy[i]
        assert r["cp_x"] == [int((cx == k).sum()) for k in range(4)]
        assert r["cp_y"] == [int((cy == k).sum()) for k in range(4)]
        assert (r["false_positives"], r["false_negatives"], r["false_types"]) == (fp, fn, ft)
        assert r["link_mismatches"] == int(((lx != ly) | (ux != uy)).sum())
        flat = lambda v: int(np.ravel_multi_index(v, shape))
        bad = 0
        edges = set()                              # every edge of the complex, once
        for s in kuhn_simplices(shape):
            for a, b in itertools.combinations(s, 2):
                edges.add((min(a, b), max(a, b)))
        for a, b in edges:
            bad += ((x[a], flat(a)) < (x[b], flat(b))) != ((y[a], flat(a)) < (y[b], flat(b)))
        assert r["order_violations"] == bad


def test_isolated_point_is_a_minimum():
    # a point without neighbours has both links empty; the minimum test comes first
    r = O.verify(np.ones((1, 1)), np.ones((1, 1)), 0, 1.0)
    assert r["cp_x"] == [1, 0, 0, 0] and r["order_violations"] == 0
