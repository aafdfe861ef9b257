"""Pins of the oracle's lossless stages (Sec. III-C) and stream format.

DIFFNB, BIT and RZE are checked against hand-derived outputs and against properties
that follow from their definitions (negabinary value, closed-form sizes, inverses).
"""
import numpy as np
import pytest


def negabinary_value(u: int, bits: int) -> int:
    return sum(((u >> k) & 1) * (-2) ** k for k in range(bits))


def test_diffnb_hand_example(orc):
    # v = [0, 1, -1, 2]: deltas 0, 1, -2, 3; in negabinary 0, 1, "10", "111"
    got = np.frombuffer(orc.diffnb(4, np.array([0, 1, -1, 2])), np.uint32).tolist()
    assert got == [0, 1, 2, 7]


@pytest.mark.parametrize("w", [4, 8])
def test_diffnb_is_delta_in_negabinary(orc, w):
    rng = np.random.default_rng(0)
    lim = 2 ** 29 if w == 4 else 2 ** 50
    v = rng.integers(-lim, lim, 300)
    u = np.frombuffer(orc.diffnb(w, v), np.uint32 if w == 4 else np.uint64)
    prev = 0
    for vi, ui in zip(v.tolist(), u.tolist()):
        assert negabinary_value(int(ui), 8 * w) == vi - prev
        prev = vi
    assert (orc.undiffnb(w, orc.diffnb(w, v), v.size) == v).all()


def test_bit_hand_example(orc):
    # one word with value 1: plane 0, group 0, bit 0 set; n pads to 32 words
    out = orc.bit(4, np.array([1], np.uint32).tobytes(), 1)
    assert len(out) == 4 * 32
    assert out[:4] == bytes([1, 0, 0, 0]) and not any(out[4:])
    # word 33 with bit 5: plane 5, group 1, bit 1 (G = 2 groups for 64 words)
    w = np.zeros(64, np.uint32)
    w[33] = 1 << 5
    out = np.frombuffer(orc.bit(4, w.tobytes(), 64), np.uint32)
    G = 2
    assert out[5 * G + 1] == 1 << 1 and out.sum() == 1 << 1


@pytest.mark.parametrize("w", [4, 8])
def test_bit_inverse(orc, w):
    rng = np.random.default_rng(1)
    for n in (1, 31, 32, 33, 2048, 4095):
        words = rng.integers(0, 256, n * w, dtype=np.uint8).tobytes()
        b = orc.bit(w, words, n)
        n32 = (n + 31) // 32 * 32
        assert len(b) == w * n32
        back = orc.unbit(w, b, n32)
        assert back[: n * w] == words and not any(back[n * w:])


def test_rze_all_zero_closed_form(orc):
    # L bytes of zeros: bitmaps of ceil(L/8), ceil(./8), ceil(./8) bytes; only the
    # last level is stored and nothing else is kept
    for L, g in [(16384, 1), (16384, 4), (16384, 8), (1, 1), (100, 1)]:
        U = L // g
        l0 = -(-U // 8)
        l1 = -(-l0 // 8)
        l2 = -(-l1 // 8)
        out = orc.rze(g, bytes(L))
        assert out == bytes(l2)
        assert orc.unrze(g, out, L) == bytes(L)


def test_rze_single_byte_hand_example(orc):
    # one non-zero byte 0x55 at position 0 of 16384:
    # M0 = 01 00 .. (2048 B) -> repeat bits 0,1 -> M1 = 03 00 .. (256 B), K0 = [01, 00]
    # M1 -> M2 = 03 00 .. (32 B), K1 = [03, 00]; payload [55]
    data = bytearray(16384)
    data[0] = 0x55
    out = orc.rze(1, bytes(data))
    want = bytes([3]) + bytes(31) + bytes([3, 0]) + bytes([1, 0]) + bytes([0x55])
    assert out == want
    assert orc.unrze(1, out, 16384) == bytes(data)


@pytest.mark.parametrize("g", [1, 4, 8])
def test_rze_inverse(orc, g):
    rng = np.random.default_rng(2)
    for L in (g * 8, g * 100, 16384):
        for density in (0.0, 0.01, 0.3, 1.0):
            a = rng.integers(1, 256, L, dtype=np.uint8)
            a[rng.random(L) >= density] = 0
            out = orc.rze(g, a.tobytes())
            assert orc.unrze(g, out, L) == a.tobytes()


def test_rze_rejects_wrong_lengths(orc):
    data = bytearray(4096)
    data[7] = 9
    out = orc.rze(1, bytes(data))
    with pytest.raises(orc.OracleError):
        orc.unrze(1, out[:-1], 4096)
    with pytest.raises(orc.OracleError):
        orc.unrze(1, out + b"\0", 4096)


def test_stream_header_fields(orc):
    x = np.linspace(0, 1, 70 * 90, dtype=np.float32).reshape(70, 90)
    st = orc.compress(x, 1, 1e-2)
    h = np.frombuffer(st[:128], np.uint8)
    assert st[:4] == b"LOPC"
    assert int.from_bytes(st[4:6], "little") == 2  # format 2: Lorenzo or 1D-difference bin records
    assert h[6] == 0 and h[7] == 2
    assert int.from_bytes(st[8:16], "little") == 70 and int.from_bytes(st[16:24], "little") == 90
    tiles = -(-70 // 64) * -(-90 // 64)
    assert int.from_bytes(st[80:88], "little") == tiles
    assert int.from_bytes(st[88:96], "little") == len(st)
    assert len(st) % 16 == 0
    d = orc.peek(st)
    assert d.ndim == 2 and d.dims[0] == 70 and d.dims[1] == 90 and d.mode == 1


def test_constant_field_stream(orc):
    x = np.full((5, 6, 7), 2.5, np.float64)
    st = orc.compress(x, 1, 1e-3)
    assert len(st) == 128 and st[33] == 1
    y = orc.decompress(st)
    assert (y == 2.5).all()


def _rebuild(st, records, sizes):
    """Stream with the given record list (format: header, u32 size table, records
    padded to 16 bytes)."""
    pad = lambda n: (n + 15) // 16 * 16
    table = b"".join(int(v).to_bytes(4, "little") for v in sizes)
    table += bytes(pad(len(table)) - len(table))
    body = b"".join(r + bytes(pad(len(r)) - len(r)) for r in records)
    total = 128 + len(table) + len(body)
    hdr = bytearray(st[:128])
    hdr[88:96] = total.to_bytes(8, "little")
    return bytes(hdr) + table + body


def _split(st):
    nch = int.from_bytes(st[80:88], "little")
    sizes = [int.from_bytes(st[128 + 4 * k:132 + 4 * k], "little") for k in range(2 * nch)]
    o = 128 + (8 * nch + 15) // 16 * 16
    recs = []
    for v in sizes:
        n = v & 0x7FFFFFFF
        recs.append(st[o:o + n])
        o += (n + 15) // 16 * 16
    return sizes, recs


def test_raw_records_decode(orc):
    """A record whose size entry carries bit 31 holds the chunk's words verbatim."""
    rng = np.random.default_rng(4)
    x = np.cumsum(rng.standard_normal((64, 64)), axis=1).astype(np.float32)
    st = orc.compress(x, 1, 1e-3)
    y = orc.decompress(st)
    e = orc.resolve_eps(x, 1, 1e-3)
    b = orc.quantize(x, e["inv"]).astype(np.int32)
    s = orc.repair_lfp(x, b.astype(np.int64)).astype(np.uint32)
    sizes, recs = _split(st)
    assert len(sizes) == 2
    st2 = _rebuild(st, [b.tobytes(), s.tobytes()], [0x80000000 | 16384, 0x80000000 | 16384])
    assert (orc.decompress(st2) == y).all()
    bad = _rebuild(st, [b.tobytes()[:-4], recs[1]], [0x80000000 | 16380, sizes[1]])
    assert orc.decompress_status(bad, x.shape, x.dtype) == orc.CORRUPT


def test_capacity_and_corrupt(orc):
    rng = np.random.default_rng(5)
    x = np.cumsum(rng.standard_normal((40, 50)), axis=1).astype(np.float32)
    st = orc.compress(x, 1, 1e-3)
    assert orc.compress_status(x, 1, 1e-3, cap=len(st) - 1) == orc.CAPACITY
    assert orc.decompress_status(st[:-16], x.shape, x.dtype) == orc.CORRUPT
    assert orc.decompress_status(st[:100], x.shape, x.dtype) == orc.CORRUPT
    bad = bytearray(st)
    bad[0] ^= 1
    assert orc.decompress_status(bytes(bad), x.shape, x.dtype) == orc.CORRUPT
    # random bit flips past the header: never a crash; either corrupt or a value
    for k in range(200):
        b = bytearray(st)
        pos = 128 + int(rng.integers(0, len(st) - 128))
        b[pos] ^= 1 << int(rng.integers(0, 8))
        rc = orc.decompress_status(bytes(b), x.shape, x.dtype)
        assert rc in (0, orc.CORRUPT)


# ------------------------------------------------------------ format 2 bin records

M32 = np.uint64(0xAAAAAAAA)


def nb_words(r, w=4):
    mask = (1 << (8 * w)) - 1
    m = 0xAAAAAAAAAAAAAAAA & mask
    return np.array([((int(v) + m) ^ m) & mask for v in r.ravel()], np.uint64 if w == 8 else np.uint32)


def record_of(orc, words, w=4):
    """Bin record built from given mapped words with the separately pinned stages."""
    return orc.rze(1, orc.bit(w, words.tobytes(), words.size))


@pytest.mark.parametrize("shape", [(16, 16, 16), (5, 7, 9), (1, 64, 64), (1, 13, 30)])
def test_lorenzo_residual_of_a_linear_ramp(orc, shape):
    # b = c0 + cx x + cy y + cz z: the Lorenzo residual is c0 at the origin, cx / cy /
    # cz along the three axis lines through it, and 0 everywhere else (a closed form)
    c0, cx, cy, cz = 7, 3, -5, 11
    z, y, x = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    b = (c0 + cx * x + cy * y + cz * z).astype(np.int64)
    r = np.zeros(shape, np.int64)
    r[0, 0, 0] = c0
    r[0, 0, 1:] = cx
    r[0, 1:, 0] = cy
    r[1:, 0, 0] = cz
    sb, rb, _, _ = orc.encode_chunk(0, b.ravel(), np.zeros(b.size, np.uint64), shape)
    assert not (sb & orc.DIFF_FLAG) and not (sb & orc.RAW_FLAG)
    assert rb == record_of(orc, nb_words(r))


def test_rows_constant_along_x_take_the_1d_difference(orc):
    # bins constant along x with random row values: the 1D difference is nonzero only
    # at row starts (one row against the previous); the Lorenzo residual there is a
    # second difference of four random rows, with more one bits: the 1D difference wins
    rng = np.random.default_rng(0)
    shape = (16, 16, 16)
    rows = rng.integers(-2**20, 2**20, shape[:2])
    b = np.repeat(rows[:, :, None], shape[2], axis=2).astype(np.int64)
    sb, rb, _, _ = orc.encode_chunk(0, b.ravel(), np.zeros(b.size, np.uint64), shape)
    assert sb & orc.DIFF_FLAG
    d = np.diff(np.concatenate([[0], b.ravel()]))
    assert rb == record_of(orc, nb_words(d))


@pytest.mark.parametrize("shape,dt", [((20, 37, 33), np.float32), ((9, 40, 45), np.float64), ((130, 70), np.float32),
                                      ((1, 3, 200), np.float64)])
def test_format2_roundtrip_and_both_predictors(orc, shape, dt):
    rng = np.random.default_rng(len(shape))
    smooth = np.cumsum(np.cumsum(rng.standard_normal(shape), axis=-1), axis=0)
    x = (smooth + (rng.random(shape) < 0.02) * 50.0).astype(dt)
    for eb in (1e-2, 1e-4):
        st = orc.compress(x, 1, eb)
        y = orc.decompress(st)
        assert orc.order_violations(x, y) == 0
        assert np.abs(x.astype(np.float64) - y).max() <= orc.resolve_eps(x, 1, eb)["eps"]


def test_format1_fixtures_still_decode(orc):
    import pathlib
    g = pathlib.Path(__file__).resolve().parent / "golden"
    for name in ("v1_2d_f32", "v1_3d_f64", "v1_3d_f32_abs"):
        st = (g / f"{name}.lopc").read_bytes()
        assert int.from_bytes(st[4:6], "little") == 1
        y = orc.decompress(st)
        assert y.tobytes() == np.load(g / f"{name}_xhat.npy").tobytes()


def test_predictor_flag_corruptions(orc):
    import pathlib
    g = pathlib.Path(__file__).resolve().parent / "golden"
    st = bytearray((g / "v1_2d_f32.lopc").read_bytes())
    st[128 + 3] |= 0x40                       # bit 30 of chunk 0's bin size in a format-1 stream
    with pytest.raises(orc.OracleError):
        orc.decompress(bytes(st))
    rng = np.random.default_rng(1)
    x = rng.uniform(-1.0, 1.0, (64, 64)).astype(np.float32)
    st = bytearray(orc.compress(x, 0, 1e-9))  # bins of +-1e9 at random: stored raw
    size = int.from_bytes(st[128:132], "little")
    assert size & orc.RAW_FLAG
    st[128 + 3] |= 0x40                       # a raw record with the predictor flag
    with pytest.raises(orc.OracleError):
        orc.decompress(bytes(st))
