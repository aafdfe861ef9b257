"""GPU parity: the CUDA library's streams and reconstructions are byte-identical to
the CPU oracle's (the paper's bit-for-bit claim, Sec. I and V), on fields that span
several tiles with ragged edges, degenerate shapes, heavy ties and deep repair
chains; plus the error paths.  All calls go through the C ABI."""
import numpy as np
import pytest
import torch

from paper_2603_26968_b300 import synth as S
from gpu_cases import CASES, bumps  # noqa: F401

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_2603_26968_b300 import build, lopc
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return lopc


def gpu_roundtrip(L, x: np.ndarray, mode: int, eb: float):
    xt = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    st = L.compress(xt, eb, mode)
    y = L.decompress(st)
    torch.cuda.synchronize()
    return bytes(st.cpu().numpy().tobytes()), y.cpu().numpy()


def assert_parity(L, orc, x, mode, eb):
    st_g, y_g = gpu_roundtrip(L, x, mode, eb)
    st_o = orc.compress(x, mode, eb)
    assert len(st_g) == len(st_o), (len(st_g), len(st_o))
    if st_g != st_o:
        diff = next(i for i in range(len(st_o)) if st_g[i] != st_o[i])
        raise AssertionError(f"stream differs at byte {diff} of {len(st_o)}")
    y_o = orc.decompress(st_o)
    assert y_g.dtype == y_o.dtype and y_g.shape == y_o.shape
    assert y_g.tobytes() == y_o.tobytes()
    # the GPU decoder reads the oracle's stream too (same bytes, so same output)
    return st_o, y_o


@pytest.mark.parametrize("name,make,mode,eb", CASES, ids=[c[0] for c in CASES])
def test_stream_and_reconstruction_parity(L, orc, name, make, mode, eb):
    x = make()
    assert_parity(L, orc, x, mode, eb)


@pytest.mark.parametrize("name,make,mode,eb", CASES[:12], ids=[c[0] for c in CASES[:12]])
def test_stage_parity_bins_and_subbins(L, orc, name, make, mode, eb):
    x = make()
    xt = torch.from_numpy(x).cuda()
    b_g, s_g = L.quantize_repair(xt, eb, mode)
    e = orc.resolve_eps(x, mode, eb)
    b_o = orc.quantize(x, e["inv"])
    s_o = orc.repair_lfp(x, b_o)
    assert (b_g.cpu().numpy() == b_o).all()
    assert (s_g.cpu().numpy().astype(np.uint64) == s_o).all()


@pytest.mark.parametrize("shape,dtype", [((17, 17, 17), np.float32), ((33, 65), np.float64), ((65, 66), np.float32),
                                         ((9, 18, 33), np.float64)])
def test_stale_buffer_bytes_never_reach_the_stream(L, orc, shape, dtype):
    """Fields whose edge chunks hold a point count that is not a multiple of 4, so a raw
    record ends inside its last 16-byte unit: the padding must be zeros (as the oracle
    writes them) even when the output and workspace hold stale bytes from earlier use."""
    x = bumps(shape, dtype, seed=11)
    xt = torch.from_numpy(x).cuda()
    d = L.make_desc(tuple(x.shape), xt.dtype, L.NOA, 1e-3)
    out = torch.full((L.compress_bound(d),), 0xCD, dtype=torch.uint8, device="cuda")
    ws = torch.full((L.compress_workspace_size(d),), 0xAB, dtype=torch.uint8, device="cuda")
    want = orc.compress(x, 1, 1e-3)
    for _ in range(2):
        st = L.compress(xt, 1e-3, L.NOA, out=out, workspace=ws)
        assert bytes(st.cpu().numpy().tobytes()) == want
        ws.fill_(0x5A)
        out.fill_(0xFF)


def test_decoder_reads_oracle_streams_after_gpu_compress(L, orc):
    x = bumps((90, 110), np.float32, seed=3)
    st = orc.compress(x, 1, 1e-3)
    t = torch.frombuffer(bytearray(st), dtype=torch.uint8).cuda()
    y = L.decompress(t).cpu().numpy()
    assert y.tobytes() == orc.decompress(st).tobytes()


def test_deep_chain_needs_many_rounds(L, orc):
    x = np.linspace(1.0, 0.0, 2000, dtype=np.float32).reshape(1, 2000)
    assert_parity(L, orc, x, 0, 10.0)
    rounds, runs = L.last_stats()  # stats of the last compress (the round trip above)
    assert rounds >= 10


# ------------------------------------------------------------------ error paths

def test_nonfinite(L):
    x = torch.zeros(40, 50, device="cuda")
    x[3, 7] = float("nan")
    assert L.compress_status(x, 1e-3, L.NOA) == -2
    assert L.compress_status(x, 1e-3, L.ABS) == -2
    x[3, 7] = float("inf")
    assert L.compress_status(x.double(), 1e-3, L.ABS) == -2


def test_range(L):
    x = torch.linspace(-1, 1, 4096, device="cuda").reshape(64, 64)
    assert L.compress_status(x, 1e-12, L.ABS) == -3
    assert L.compress_status(x.double(), 1e-12, L.ABS) == 0


def test_capacity_and_workspace(L, orc):
    x = bumps((64, 80), np.float32)
    st = orc.compress(x, 1, 1e-3)
    xt = torch.from_numpy(x).cuda()
    assert L.compress_status(xt, 1e-3, L.NOA, out_cap=len(st)) == 0
    assert L.compress_status(xt, 1e-3, L.NOA, out_cap=len(st) - 1) == -4
    d = L.make_desc(x.shape, "f32", L.NOA, 1e-3)
    assert L.compress_status(xt, 1e-3, L.NOA, ws_bytes=L.compress_workspace_size(d) - 1) == -8


def test_round_cap_not_converged(L):
    x = torch.linspace(1.0, 0.0, 2000, device="cuda").reshape(1, 2000)
    old = L.set_round_cap(2)
    try:
        assert L.compress_status(x, 10.0, L.ABS) == -6
    finally:
        L.set_round_cap(old)
    assert L.compress_status(x, 10.0, L.ABS) == 0


def test_corrupt_streams_never_fault(L, orc):
    x = bumps((70, 90), np.float32, seed=9)
    st = orc.compress(x, 1, 1e-3)
    rng = np.random.default_rng(0)
    dev = torch.device("cuda")
    # truncated
    for cut in (len(st) - 16, 200, 100):
        t = torch.frombuffer(bytearray(st[:cut]), dtype=torch.uint8).to(dev)
        assert L.decompress_status(t, x.shape, torch.float32) == -5
    # bit flips past the header
    outcomes = set()
    for k in range(60):
        b = bytearray(st)
        pos = 128 + int(rng.integers(0, len(st) - 128))
        b[pos] ^= 1 << int(rng.integers(0, 8))
        t = torch.frombuffer(b, dtype=torch.uint8).to(dev)
        rc = L.decompress_status(t, x.shape, torch.float32)
        assert rc in (0, -5)
        outcomes.add(rc)
        rc_o = orc.decompress_status(bytes(b), x.shape, x.dtype)
        if rc_o == orc.CORRUPT:
            assert rc == -5
    assert -5 in outcomes
    torch.cuda.synchronize()


def test_gpu_decodes_format1_fixtures(L):
    import pathlib
    g = pathlib.Path(__file__).resolve().parent / "golden"
    for name in ("v1_2d_f32", "v1_3d_f64", "v1_3d_f32_abs"):
        st = (g / f"{name}.lopc").read_bytes()
        want = np.load(g / f"{name}_xhat.npy")
        t = torch.frombuffer(bytearray(st), dtype=torch.uint8).cuda()
        y = L.decompress(t)
        assert y.cpu().numpy().tobytes() == want.tobytes()


def test_predictor_flag_corruptions_gpu(L, orc):
    import pathlib
    g = pathlib.Path(__file__).resolve().parent / "golden"
    b = bytearray((g / "v1_2d_f32.lopc").read_bytes())
    b[128 + 3] |= 0x40  # the format-2 predictor flag in a format-1 stream
    t = torch.frombuffer(b, dtype=torch.uint8).cuda()
    assert L.decompress_status(t, (70, 90), torch.float32) == -5
    rng = np.random.default_rng(1)
    x = rng.uniform(-1.0, 1.0, (64, 64)).astype(np.float32)
    b = bytearray(orc.compress(x, 0, 1e-9))
    assert int.from_bytes(b[128:132], "little") & 0x80000000
    b[128 + 3] |= 0x40  # the predictor flag on a raw record
    t = torch.frombuffer(b, dtype=torch.uint8).cuda()
    assert L.decompress_status(t, (64, 64), torch.float32) == -5
    torch.cuda.synchronize()


def test_both_bin_predictors_occur(L, orc):
    # a smooth field takes the Lorenzo residual; rows constant along x take the 1D
    # difference; streams equal the oracle's either way
    rng = np.random.default_rng(2)
    rows = rng.integers(-2**20, 2**20, (32, 32)).astype(np.float64)
    x = np.repeat(rows[:, :, None], 32, axis=2).astype(np.float32)
    st = assert_parity(L, orc, x, 0, 1.0)[0]
    nch = int.from_bytes(st[80:88], "little")
    tab = np.frombuffer(st[128:128 + 4 * nch], np.uint32)
    assert (tab & 0x40000000).any()
    x = bumps((40, 50, 60), np.float32)
    st = assert_parity(L, orc, x, 1, 1e-3)[0]
    nch = int.from_bytes(st[80:88], "little")
    tab = np.frombuffer(st[128:128 + 4 * nch], np.uint32)
    assert ((tab & 0xC0000000) == 0).any()


# ------------------------------------------------------------ full-size configs

def lfp_local_equality(x: torch.Tensor, b: torch.Tensor, s: torch.Tensor) -> int:
    """Counts points where s(p) != max(0, max over same-bin lower neighbours n of
    s(n) + [idx_n > idx_p]).  On the acyclic constraint graph this equation has one
    solution, the least fixpoint, so zero mismatches pins s exactly."""
    if x.dim() == 2:
        x, b, s = x[None], b[None], s[None]
    need = torch.zeros_like(s)
    nz, ny, nx = x.shape
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                if dz == dy == dx == 0:
                    continue
                for sign in (-1, 1):
                    oz, oy, ox = sign * dz, sign * dy, sign * dx
                    zp = slice(max(0, -oz), nz - max(0, oz))
                    yp = slice(max(0, -oy), ny - max(0, oy))
                    xp = slice(max(0, -ox), nx - max(0, ox))
                    zn = slice(max(0, oz), nz - max(0, -oz))
                    yn = slice(max(0, oy), ny - max(0, -oy))
                    xn = slice(max(0, ox), nx - max(0, -ox))
                    xv, nv = x[zp, yp, xp], x[zn, yn, xn]
                    same = b[zp, yp, xp] == b[zn, yn, xn]
                    # neighbour index is higher for sign > 0: it precedes only if strictly lower
                    lower = (nv < xv) if sign > 0 else (nv <= xv)
                    cand = torch.where(same & lower, s[zn, yn, xn] + (1 if sign > 0 else 0), torch.zeros_like(s[zn, yn, xn]))
                    torch.maximum(need[zp, yp, xp], cand, out=need[zp, yp, xp])
    return int((need != s).sum().item())


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
                # the neighbour c has the higher index: it is below a only if strictly lower
                bad += int(((x[c] < x[a]) != (y[c] < y[a])).sum().item())
    return bad


def split_stream(st: bytes):
    nch = int.from_bytes(st[80:88], "little")
    tab = np.frombuffer(st[128:128 + 8 * nch], np.uint32)
    o = 128 + (8 * nch + 15) // 16 * 16
    offs = []
    for v in tab:
        offs.append(o)
        o += ((int(v) & 0x3FFFFFFF) + 15) // 16 * 16
    return tab, offs


def tile_points(shape, tile, tid):
    """Flat indices of chunk tid's points in chunk order, and the clipped chunk shape."""
    sh = (1,) + tuple(shape) if len(shape) == 2 else tuple(shape)
    nt = [-(-sh[k] // tile[k]) for k in range(3)]
    tz, rem = divmod(tid, nt[1] * nt[2])
    ty, tx = divmod(rem, nt[2])
    z0, y0, x0 = tz * tile[0], ty * tile[1], tx * tile[2]
    z1, y1, x1 = min(z0 + tile[0], sh[0]), min(y0 + tile[1], sh[1]), min(x0 + tile[2], sh[2])
    zz, yy, xx = np.meshgrid(np.arange(z0, z1), np.arange(y0, y1), np.arange(x0, x1), indexing="ij")
    return ((zz * sh[1] + yy) * sh[2] + xx).ravel(), (z1 - z0, y1 - y0, x1 - x0)


FULL = [  # name, field, mode, bound, chunk tile, whether the tile pass takes tile-key order
    ("c2_f32_512", lambda: S.make_field(S.spec_3d_f32(n=512)), 1, 1e-3, (16, 16, 16), 0),
    ("c2_f32_512_loose", lambda: S.make_field(S.spec_3d_f32(n=512)), 1, 1e-2, (16, 16, 16), 1),
    ("c3_f64_ties", lambda: S.make_field(S.spec_3d_f64_ties()), 1, 5e-4, (8, 16, 16), 0),
]


@pytest.mark.parametrize("name,make,mode,eb,tile,ordered", FULL, ids=[f[0] for f in FULL])
def test_full_size_sampled_parity(L, orc, name, make, mode, eb, tile, ordered):
    x = make()
    dc = 0 if x.dtype == np.float32 else 1
    xt = torch.from_numpy(x).cuda()
    st_t = L.compress(xt, eb, mode)
    assert L.last_fixpoint_work()["pass_ordered"] == ordered
    st = bytes(st_t.cpu().numpy().tobytes())
    b_t, s_t = L.quantize_repair(xt, eb, mode)
    e = orc.resolve_eps(x, mode, eb)
    rng = np.random.default_rng(0)
    # bins at sampled points against the oracle's exact quantizer
    idx = rng.integers(0, x.size, 20000)
    xf = x.ravel()
    bf = b_t.view(-1)[torch.from_numpy(idx).cuda()].cpu().numpy()
    assert all(orc.q1(dc, float(xf[i]), e["inv"]) == int(bf[k]) for k, i in enumerate(idx))
    # subbins: the least-fixpoint equation holds at every point
    xd = xt.double() if dc == 0 else xt
    assert lfp_local_equality(xd, b_t, s_t) == 0
    # sampled chunks: the oracle encodes the same records from these bins/subbins
    tab, offs = split_stream(st)
    nch = len(tab) // 2
    bn, sn = b_t.view(-1).cpu().numpy(), s_t.view(-1).cpu().numpy().astype(np.uint64)
    for tid in list(rng.integers(0, nch, 40)) + [0, nch - 1]:
        pts, cshape = tile_points(x.shape, tile, int(tid))
        sb, rb, ss, rs = orc.encode_chunk(dc, bn[pts], sn[pts], cshape)
        assert int(tab[tid]) == sb and st[offs[tid]:offs[tid] + (sb & 0x3FFFFFFF)] == rb
        assert int(tab[nch + tid]) == ss and st[offs[nch + tid]:offs[nch + tid] + (ss & 0x3FFFFFFF)] == rs
    # decompression: error bound, x_hat <= x, neighbour order, sampled values
    y = L.decompress(st_t)
    yd = y.double()
    assert bool((yd <= xd).all()) and float((xd - yd).max()) < e["eps"]
    assert order_mismatches(xd, yd) == 0
    ys = y.view(-1)[torch.from_numpy(idx[:2000]).cuda()].cpu().numpy()
    want = orc.reconstruct(dc, bf[:2000], sn[idx[:2000]], e["inv"])
    assert ys.tobytes() == want.tobytes()


@pytest.mark.parametrize("shape,dtype,other", [
    ((32, 16, 48), np.float32, (16, 32, 48)),   # 2 x 1 x 3 and 1 x 2 x 3 tiles
    ((128, 64), np.float32, (64, 128)),         # 2 x 1 and 1 x 2 tiles
    ((16, 32, 40), np.float64, (8, 64, 40)),    # 2 x 2 x 3 and 1 x 4 x 3 tiles
])
def test_decompress_with_descriptor(L, orc, shape, dtype, other):
    """lopc.decompress with the field's descriptor (one batch call checked on the
    device) gives the oracle's reconstruction; a descriptor with other dims but as many
    tiles is CORRUPT, and an output too small is CAPACITY, both before any write."""
    x = bumps(shape, dtype, seed=4)
    st = orc.compress(x, 1, 1e-3)
    t = torch.frombuffer(bytearray(st), dtype=torch.uint8).cuda()
    d = L.peek(t)
    assert tuple(d.shape) == shape
    y = L.decompress(t, desc=d)
    assert y.cpu().numpy().tobytes() == orc.decompress(st).tobytes()
    assert torch.equal(y, L.decompress(t))
    bad = L.make_desc(other, "f32" if dtype == np.float32 else "f64", L.NOA, 1e-3)
    with pytest.raises(L.LopcError) as e:
        L.decompress(t, desc=bad)
    assert e.value.code == -5
    small = torch.empty(int(np.prod(shape)) - 1, dtype=y.dtype, device="cuda")
    with pytest.raises(L.LopcError) as e:
        L.decompress(t, out=small, desc=d)
    assert e.value.code == -4
