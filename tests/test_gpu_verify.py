"""GPU parity of the verifier (lopc_verify): per-point link piece counts of x and y
equal the oracle's critical_types element by element, and the report equals the
oracle's verification summary (counts and the range / largest error exactly, MSE and
PSNR within the tolerance of their summation order), on fields that span several
tiles with ragged edges, degenerate shapes, heavy ties, and reconstructions that
keep or break the local order.  At the full benchmark sizes: per-point types on
sampled sub-boxes against the oracle, and the report against plain PyTorch."""
import zlib

import numpy as np
import pytest
import torch

from paper_2603_26968_b300 import synth as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_2603_26968_b300 import build, lopc
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return lopc


def packed(lo, up):
    return (lo.astype(np.uint8) | (up.astype(np.uint8) << 4)).astype(np.uint8)


def gpu_verify(L, x, y, mode, eb, types=True):
    xt = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    yt = torch.from_numpy(np.ascontiguousarray(y)).cuda()
    tx = torch.empty(x.shape, dtype=torch.uint8, device="cuda") if types else None
    ty = torch.empty(x.shape, dtype=torch.uint8, device="cuda") if types else None
    r = L.verify(xt, yt, eb, mode, types_x=tx, types_y=ty)
    torch.cuda.synchronize()
    return r, (tx.cpu().numpy() if types else None), (ty.cpu().numpy() if types else None)


def assert_report(r, o, dtype):
    exact = ["points", "order_violations", "cp_x", "cp_y", "false_positives", "false_negatives",
             "false_types", "link_mismatches", "x_min", "x_max", "max_abs_err", "bound_ok"]
    for k in exact:
        assert r[k] == o[k], (k, r[k], o[k])
    # float32 squares are summed in float32 over at most 16 points first
    rtol = 2e-6 if dtype == np.float32 else 1e-12
    assert r["mse"] == pytest.approx(o["mse"], rel=rtol, abs=0.0)
    if np.isfinite(o["psnr"]):
        assert abs(r["psnr"] - o["psnr"]) <= 10 * np.log10(1 + 2 * rtol) + 1e-12
    else:
        assert r["psnr"] == o["psnr"]
    assert r["eps"] == o["eps"]


def perturbed(x, rng, frac=0.01):
    y = x.copy()
    idx = rng.choice(x.size, size=max(1, int(frac * x.size)), replace=False)
    y.ravel()[idx] = y.ravel()[rng.permutation(idx)]
    return y


CASES = [
    # name, shape, dtype
    ("2d_f32_ragged", (150, 197), np.float32),
    ("2d_f64_ragged", (70, 131), np.float64),
    ("3d_f32_ragged", (21, 35, 40), np.float32),
    ("3d_f64_ragged", (17, 33, 21), np.float64),
    ("3d_f32_thin", (1, 5, 37), np.float32),
    ("2d_row", (1, 300), np.float32),
    ("2d_col", (77, 1), np.float64),
    ("3d_col", (9, 1, 1), np.float32),
    ("single", (1, 1), np.float32),
]


@pytest.mark.parametrize("name,shape,dtype", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("kind", ["roundtrip", "ties", "perturbed", "negated", "constant"])
def test_verify_parity(L, orc, name, shape, dtype, kind):
    rng = np.random.default_rng(zlib.crc32(f"{name}/{kind}".encode()))
    if kind == "ties":
        x = rng.integers(0, 4, shape).astype(dtype)
    else:
        x = np.cumsum(rng.standard_normal(shape), axis=-1).astype(dtype)
    if kind == "roundtrip":
        xt = torch.from_numpy(x).cuda()
        y = L.decompress(L.compress(xt, 1e-2, L.NOA)).cpu().numpy()
    elif kind in ("ties", "perturbed"):
        y = perturbed(x, rng)
    elif kind == "negated":
        y = -x
    else:
        y = np.zeros_like(x)
    reports = {}
    for mode, eb in ((L.NOA, 1e-2), (L.ABS, 0.05)):
        r, tx, ty = gpu_verify(L, x, y, mode, eb)
        o = orc.verify(x, y, mode, eb)
        assert_report(r, o, dtype)
        assert (tx == packed(*orc.critical_types(x))).all()
        assert (ty == packed(*orc.critical_types(y))).all()
        reports[mode] = r
    if kind == "roundtrip":  # compressed at NOA 1e-2: the guarantees under that bound
        r = reports[L.NOA]
        assert r["order_violations"] == 0 and r["false_positives"] == r["false_negatives"] == r["false_types"] == 0
        assert r["link_mismatches"] == 0 and r["bound_ok"]


def test_verify_without_types_gives_the_same_report(L, orc):
    x = np.cumsum(np.random.default_rng(1).standard_normal((40, 50, 33)), axis=0).astype(np.float32)
    y = perturbed(x, np.random.default_rng(2))
    a, _, _ = gpu_verify(L, x, y, L.NOA, 1e-3, types=True)
    b, _, _ = gpu_verify(L, x, y, L.NOA, 1e-3, types=False)
    assert a == b


def test_verify_is_deterministic(L):
    x = torch.randn(64, 96, 80, device="cuda")
    y = x + 1e-3 * torch.randn_like(x)
    r = [L.verify(x, y, 1e-3, L.NOA) for _ in range(3)]
    assert r[0] == r[1] == r[2]


def test_verify_nonfinite(L):
    x = torch.zeros(20, 30, device="cuda")
    y = x.clone()
    y[3, 4] = float("nan")
    with pytest.raises(L.LopcError) as e:
        L.verify(x, y, 1e-3, L.NOA)
    assert e.value.code == -2


def test_verify_bad_arguments(L):
    x = torch.zeros(8, 8, device="cuda")
    with pytest.raises(ValueError):
        L.verify(x, torch.zeros(8, 9, device="cuda"))
    d = L.make_desc((8, 8), "f32", L.NOA, 1e-3)
    ws = torch.empty(16, dtype=torch.uint8, device="cuda")
    r = L.VerifyReport()
    import ctypes as C
    rc = L.lib().lopc_verify(C.byref(d), C.c_void_p(x.data_ptr()), C.c_void_p(x.data_ptr()), None, None,
                             C.byref(r), C.c_void_p(ws.data_ptr()), ws.numel(), None)
    assert rc == -8


# ------------------------------------------------------------ full-size configs

def order_mismatches(x: torch.Tensor, y: torch.Tensor) -> int:
    if x.dim() == 2:
        x, y = x[None], y[None]
    nz, ny, nx = x.shape
    bad = 0
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                if dz == dy == dx == 0:
                    continue
                a = (slice(0, nz - dz), slice(0, ny - dy), slice(0, nx - dx))
                c = (slice(dz, nz), slice(dy, ny), slice(dx, nx))
                bad += int(((x[c] < x[a]) != (y[c] < y[a])).sum().item())
    return bad


FULL = [
    ("c2_f32_512", lambda: S.make_field(S.spec_3d_f32(n=512)), 1e-3),
    ("c3_f64_ties", lambda: S.make_field(S.spec_3d_f64_ties()), 5e-4),
]


@pytest.mark.parametrize("name,make,eb", FULL, ids=[f[0] for f in FULL])
def test_full_size_verify(L, orc, name, make, eb):
    x = make()
    xt = torch.from_numpy(x).cuda()
    y = L.decompress(L.compress(xt, eb, L.NOA))
    tx = torch.empty(x.shape, dtype=torch.uint8, device="cuda")
    ty = torch.empty(x.shape, dtype=torch.uint8, device="cuda")
    r = L.verify(xt, y, eb, L.NOA, types_x=tx, types_y=ty)
    # the paper's guarantee (Table III's 0/0/0, local order, bound)
    assert r["order_violations"] == 0 and r["link_mismatches"] == 0
    assert r["false_positives"] == r["false_negatives"] == r["false_types"] == 0
    assert r["cp_x"] == r["cp_y"] and sum(r["cp_x"]) == x.size and r["bound_ok"]
    assert bool((tx == ty).all())
    # range, largest error and MSE against plain PyTorch in binary64
    xd, yd = xt.double(), y.double()
    d = (xd - yd).abs()
    assert r["x_min"] == float(xd.min()) and r["x_max"] == float(xd.max())
    assert r["max_abs_err"] == float(d.max())
    rtol = 2e-6 if x.dtype == np.float32 else 1e-12
    assert r["mse"] == pytest.approx(float((d * d).mean()), rel=rtol)
    # per-point link pieces on sampled sub-boxes against the oracle (a one-point halo
    # inside the field; none where the box meets the field's boundary)
    rng = np.random.default_rng(0)
    tn = tx.cpu().numpy()
    for k in range(12):
        lo = [0 if k == 0 else int(rng.integers(0, n - 20)) for n in x.shape]
        if k == 1:
            lo = [n - 20 for n in x.shape]
        hi = [a + 20 for a in lo]
        glo = [max(0, a - 1) for a in lo]
        ghi = [min(n, b + 1) for n, b in zip(x.shape, hi)]
        sub = np.ascontiguousarray(x[glo[0]:ghi[0], glo[1]:ghi[1], glo[2]:ghi[2]])
        want = packed(*orc.critical_types(sub))
        inner = tuple(slice(a - g, b - g) for a, b, g in zip(lo, hi, glo))
        got = tn[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]]
        assert (got == want[inner]).all()
    # class counts are those of the per-point types
    lo_t, up_t = (tx & 15).long(), (tx >> 4).long()
    cls = torch.where(lo_t == 0, 0, torch.where(up_t == 0, 1, torch.where((lo_t == 1) & (up_t == 1), 3, 2)))
    assert torch.bincount(cls.view(-1), minlength=4).tolist() == r["cp_x"]
    # a broken reconstruction at full size: order violations against plain PyTorch
    y2 = y.clone().view(-1)
    idx = torch.from_numpy(rng.choice(x.size, 100000, replace=False)).cuda()
    y2[idx] = y2[idx.flip(0)]
    y2 = y2.view(x.shape)
    r2 = L.verify(xt, y2, eb, L.NOA)
    assert r2["order_violations"] == order_mismatches(xd, y2.double()) > 0
    assert r2["false_positives"] + r2["false_negatives"] + r2["false_types"] > 0
