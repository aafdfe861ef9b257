"""ctypes wrapper of the plain C oracle (``lopc_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may use it; the library's product path never does.
The oracle shares no code with the CUDA library.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from pathlib import Path

import numpy as np

HERE = Path(__file__).resolve().parent
SRC = HERE / "lopc_oracle.c"
LIB = HERE / "_liboracle.so"
LIB_OMP = HERE / "_liboracle_omp.so"

OK, INVALID_ARG, NONFINITE, RANGE, CAPACITY, CORRUPT = 0, -1, -2, -3, -4, -5


def build(force: bool = False, openmp: bool = False) -> Path:
    """Compiles the oracle with gcc (IEEE binary64 on SSE2, no FMA contraction).

    ``openmp=True`` builds the same source a second time with -fopenmp
    (``_liboracle_omp.so``): the quantizer's points and the coder's and decoder's
    chunks are then split over threads; the output bytes are the same."""
    out = LIB_OMP if openmp else LIB
    if out.exists() and not force and out.stat().st_mtime >= max(SRC.stat().st_mtime,
                                                               (HERE / "lopc_oracle.h").stat().st_mtime):
        return out
    tmp = out.with_suffix(f".{os.getpid()}.tmp")
    cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-Wno-unknown-pragmas",
           "-shared", "-fPIC", *(["-fopenmp"] if openmp else []), str(SRC), "-o", str(tmp),
           "-lquadmath", "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


class Desc(C.Structure):
    _fields_ = [("dtype", C.c_int32), ("ndim", C.c_int32), ("dims", C.c_int64 * 3),
                ("mode", C.c_int32), ("pad_", C.c_int32), ("eb", C.c_double)]


_libs = {}


def lib(openmp: bool = False):
    """The single-threaded oracle, or (openmp=True) its OpenMP build."""
    if openmp not in _libs:
        L = C.CDLL(str(build(openmp=openmp)))
        P = C.c_void_p
        L.orc_resolve_eps.argtypes = [C.POINTER(Desc), P, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                      C.POINTER(C.c_double), C.POINTER(C.c_int), C.POINTER(C.c_double)]
        L.orc_quantize.argtypes = [C.c_int, P, C.c_int64, C.c_double, P]
        L.orc_q1.argtypes = [C.c_int, C.c_double, C.c_double]
        L.orc_q1.restype = C.c_int64
        L.orc_lowest_in_bin.argtypes = [C.c_int, C.c_int64, C.c_double, C.POINTER(C.c_double)]
        L.orc_succ_k.argtypes = [C.c_int, C.c_double, C.c_uint64]
        L.orc_succ_k.restype = C.c_double
        L.orc_constraint_masks.argtypes = [C.POINTER(Desc), P, P, P]
        L.orc_repair_lfp.argtypes = [C.POINTER(Desc), P, P, P]
        L.orc_repair_alg2.argtypes = [C.POINTER(Desc), P, P, P]
        L.orc_repair_alg2.restype = C.c_int64
        L.orc_reconstruct.argtypes = [C.c_int, C.c_int64, P, P, C.c_double, P]
        L.orc_diffnb.argtypes = [C.c_int, P, C.c_int64, P]
        L.orc_diffnb.restype = C.c_size_t
        L.orc_undiffnb.argtypes = [C.c_int, P, C.c_int64, P]
        L.orc_bit.argtypes = [C.c_int, P, C.c_int64, P]
        L.orc_bit.restype = C.c_size_t
        L.orc_unbit.argtypes = [C.c_int, P, C.c_int64, P]
        L.orc_rze.argtypes = [C.c_int, P, C.c_size_t, P]
        L.orc_rze.restype = C.c_size_t
        L.orc_unrze.argtypes = [C.c_int, P, C.c_size_t, C.c_size_t, P]
        L.orc_encode_chunk.argtypes = [C.c_int, P, P, P, P, P, P, P]
        L.orc_compress_bound.argtypes = [C.POINTER(Desc)]
        L.orc_compress_bound.restype = C.c_size_t
        L.orc_compress.argtypes = [C.POINTER(Desc), P, P, C.c_size_t, C.POINTER(C.c_size_t)]
        L.orc_peek.argtypes = [P, C.c_size_t, C.POINTER(Desc)]
        L.orc_decompress.argtypes = [P, C.c_size_t, P, C.c_size_t]
        L.orc_order_violations.argtypes = [C.POINTER(Desc), P, P]
        L.orc_order_violations.restype = C.c_int64
        L.orc_critical_types.argtypes = [C.POINTER(Desc), P, P, P]
        _libs[openmp] = L
    return _libs[openmp]


def omp_threads() -> int:
    """Threads the OpenMP build uses (OMP_NUM_THREADS, else every core it sees)."""
    n = os.environ.get("OMP_NUM_THREADS")
    return int(n) if n and n.isdigit() and int(n) > 0 else (os.cpu_count() or 1)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def dtype_code(x: np.ndarray) -> int:
    if x.dtype == np.float32:
        return 0
    if x.dtype == np.float64:
        return 1
    raise TypeError(x.dtype)


def make_desc(shape, dtype_c: int, mode: int = 1, eb: float = 1e-3) -> Desc:
    d = Desc()
    d.dtype = dtype_c
    d.ndim = len(shape)
    for k, n in enumerate(shape):
        d.dims[k] = int(n)
    d.mode = mode
    d.eb = float(eb)
    return d


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: status {code}")
        self.code = code


def _c(x: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(x)


def resolve_eps(x: np.ndarray, mode: int, eb: float):
    x = _c(x)
    d = make_desc(x.shape, dtype_code(x), mode, eb)
    e, eq, iv, cv = C.c_double(), C.c_double(), C.c_double(), C.c_double()
    const = C.c_int()
    rc = lib().orc_resolve_eps(C.byref(d), _ptr(x), C.byref(e), C.byref(eq), C.byref(iv), C.byref(const),
                               C.byref(cv))
    if rc:
        raise OracleError(rc, "resolve_eps")
    return dict(eps=e.value, eps_q=eq.value, inv=iv.value, constant=bool(const.value), const_value=cv.value)


def quantize(x: np.ndarray, inv: float) -> np.ndarray:
    x = _c(x)
    b = np.empty(x.shape, np.int64)
    rc = lib().orc_quantize(dtype_code(x), _ptr(x), x.size, inv, _ptr(b))
    if rc:
        raise OracleError(rc, "quantize")
    return b


def q1(dtype_c: int, v: float, inv: float) -> int:
    return lib().orc_q1(dtype_c, v, inv)


def lowest_in_bin(dtype_c: int, b: int, inv: float) -> float:
    v = C.c_double()
    rc = lib().orc_lowest_in_bin(dtype_c, int(b), inv, C.byref(v))
    if rc:
        raise OracleError(rc, "lowest_in_bin")
    return v.value


def succ_k(dtype_c: int, v: float, k: int) -> float:
    return lib().orc_succ_k(dtype_c, v, int(k))


def constraint_masks(x: np.ndarray, b: np.ndarray) -> np.ndarray:
    x = _c(x)
    b = _c(b.astype(np.int64))
    m = np.empty(x.shape, np.uint16)
    d = make_desc(x.shape, dtype_code(x))
    lib().orc_constraint_masks(C.byref(d), _ptr(x), _ptr(b), _ptr(m))
    return m


def repair_lfp(x: np.ndarray, b: np.ndarray) -> np.ndarray:
    x = _c(x)
    b = _c(b.astype(np.int64))
    s = np.zeros(x.shape, np.uint64)
    d = make_desc(x.shape, dtype_code(x))
    rc = lib().orc_repair_lfp(C.byref(d), _ptr(x), _ptr(b), _ptr(s))
    if rc:
        raise OracleError(rc, "repair_lfp")
    return s


def repair_alg2(x: np.ndarray, b: np.ndarray):
    x = _c(x)
    b = _c(b.astype(np.int64))
    s = np.zeros(x.shape, np.uint64)
    d = make_desc(x.shape, dtype_code(x))
    it = lib().orc_repair_alg2(C.byref(d), _ptr(x), _ptr(b), _ptr(s))
    return s, int(it)


def reconstruct(dtype_c: int, b: np.ndarray, s: np.ndarray, inv: float) -> np.ndarray:
    b = _c(b.astype(np.int64))
    s = _c(s.astype(np.uint64))
    out = np.empty(b.shape, np.float32 if dtype_c == 0 else np.float64)
    rc = lib().orc_reconstruct(dtype_c, b.size, _ptr(b), _ptr(s), inv, _ptr(out))
    if rc:
        raise OracleError(rc, "reconstruct")
    return out


# codec stages ----------------------------------------------------------------

def diffnb(w: int, v: np.ndarray) -> bytes:
    v = _c(v.astype(np.int64))
    out = np.zeros(v.size * w, np.uint8)
    lib().orc_diffnb(w, _ptr(v), v.size, _ptr(out))
    return out.tobytes()


def undiffnb(w: int, data: bytes, n: int) -> np.ndarray:
    a = np.frombuffer(data, np.uint8).copy()
    v = np.empty(n, np.int64)
    lib().orc_undiffnb(w, _ptr(a), n, _ptr(v))
    return v


def bit(w: int, words: bytes, n: int) -> bytes:
    a = np.frombuffer(words, np.uint8).copy()
    n32 = (n + 31) // 32 * 32
    out = np.zeros(n32 * w, np.uint8)
    L = lib().orc_bit(w, _ptr(a), n, _ptr(out))
    return out[:L].tobytes()


def unbit(w: int, data: bytes, n32: int) -> bytes:
    a = np.frombuffer(data, np.uint8).copy()
    out = np.zeros(n32 * w, np.uint8)
    lib().orc_unbit(w, _ptr(a), n32, _ptr(out))
    return out.tobytes()


def rze(g: int, data: bytes) -> bytes:
    a = np.frombuffer(data, np.uint8).copy() if len(data) else np.zeros(1, np.uint8)
    out = np.zeros(2 * len(data) + 64, np.uint8)
    n = lib().orc_rze(g, _ptr(a), len(data), _ptr(out))
    return out[:n].tobytes()


def unrze(g: int, data: bytes, L: int) -> bytes:
    a = np.frombuffer(data, np.uint8).copy() if len(data) else np.zeros(1, np.uint8)
    out = np.zeros(max(L, 1), np.uint8)
    rc = lib().orc_unrze(g, _ptr(a), len(data), L, _ptr(out))
    if rc:
        raise OracleError(rc, "unrze")
    return out[:L].tobytes()


SIZE_MASK, DIFF_FLAG, RAW_FLAG = 0x3FFFFFFF, 0x40000000, 0x80000000


def encode_chunk(dtype_c: int, b: np.ndarray, s: np.ndarray, shape):
    """Records of one chunk of `shape` (cz, cy, cx; 2D: cz = 1), points in chunk
    order: (bin_size, bin_record, subbin_size, subbin_record)."""
    b = _c(b.astype(np.int64))
    s = _c(s.astype(np.uint64))
    dims = np.array(list(shape), np.int64)
    assert dims.size == 3 and int(np.prod(dims)) == b.size
    w = 4 if dtype_c == 0 else 8
    rb = np.zeros(b.size * w + 64, np.uint8)
    rs = np.zeros(b.size * w + 64, np.uint8)
    sb, ss = C.c_uint32(), C.c_uint32()
    lib().orc_encode_chunk(dtype_c, _ptr(b), _ptr(s), _ptr(dims), _ptr(rb), C.byref(sb), _ptr(rs), C.byref(ss))
    return sb.value, rb[: sb.value & SIZE_MASK].tobytes(), ss.value, rs[: ss.value & SIZE_MASK].tobytes()


# whole stream ------------------------------------------------------------------

def compress(x: np.ndarray, mode: int = 1, eb: float = 1e-3, openmp: bool = False) -> bytes:
    x = _c(x)
    L = lib(openmp)
    d = make_desc(x.shape, dtype_code(x), mode, eb)
    cap = L.orc_compress_bound(C.byref(d))
    if cap == 0:
        raise OracleError(INVALID_ARG, "compress_bound")
    out = np.zeros(cap, np.uint8)
    sz = C.c_size_t()
    rc = L.orc_compress(C.byref(d), _ptr(x), _ptr(out), cap, C.byref(sz))
    if rc:
        raise OracleError(rc, "compress")
    return out[:sz.value].tobytes()


def compress_status(x: np.ndarray, mode: int, eb: float, cap: int | None = None) -> int:
    x = _c(x)
    d = make_desc(x.shape, dtype_code(x), mode, eb)
    bound = lib().orc_compress_bound(C.byref(d))
    if cap is None:
        cap = bound
    out = np.zeros(max(cap, 1), np.uint8)
    sz = C.c_size_t()
    return lib().orc_compress(C.byref(d), _ptr(x), _ptr(out), cap, C.byref(sz))


def peek(stream: bytes) -> Desc:
    a = np.frombuffer(stream, np.uint8).copy()
    d = Desc()
    rc = lib().orc_peek(_ptr(a), a.size, C.byref(d))
    if rc:
        raise OracleError(rc, "peek")
    return d


def decompress(stream: bytes, openmp: bool = False) -> np.ndarray:
    a = np.frombuffer(stream, np.uint8).copy()
    d = peek(stream)
    shape = tuple(int(d.dims[k]) for k in range(d.ndim))
    out = np.empty(shape, np.float32 if d.dtype == 0 else np.float64)
    rc = lib(openmp).orc_decompress(_ptr(a), a.size, _ptr(out), out.nbytes)
    if rc:
        raise OracleError(rc, "decompress")
    return out


def decompress_status(stream: bytes, shape, dtype) -> int:
    a = np.frombuffer(stream, np.uint8).copy() if len(stream) else np.zeros(1, np.uint8)
    out = np.empty(shape, dtype)
    return lib().orc_decompress(_ptr(a), len(stream), _ptr(out), out.nbytes)


# checkers ------------------------------------------------------------------------

def order_violations(x: np.ndarray, y: np.ndarray) -> int:
    x, y = _c(x), _c(y)
    assert x.dtype == y.dtype and x.shape == y.shape
    d = make_desc(x.shape, dtype_code(x))
    return int(lib().orc_order_violations(C.byref(d), _ptr(x), _ptr(y)))


def critical_types(x: np.ndarray):
    x = _c(x)
    d = make_desc(x.shape, dtype_code(x))
    lo = np.empty(x.shape, np.uint8)
    up = np.empty(x.shape, np.uint8)
    lib().orc_critical_types(C.byref(d), _ptr(x), _ptr(lo), _ptr(up))
    return lo, up


# verification summary (Sec. II critical points, Table III, Sec. III-A bound, PSNR) --

CP_MIN, CP_MAX, CP_SADDLE, CP_REGULAR = 0, 1, 2, 3


def classify(lower_cc: np.ndarray, upper_cc: np.ndarray) -> np.ndarray:
    """Sec. II: a point with an empty lower link is a minimum, one with an empty upper
    link a maximum, one whose lower and upper links are one piece each is regular,
    any other point a saddle.  (The minimum test comes first, so a point without
    neighbours counts as a minimum.)"""
    c = np.full(lower_cc.shape, CP_SADDLE, np.uint8)
    c[(lower_cc == 1) & (upper_cc == 1)] = CP_REGULAR
    c[upper_cc == 0] = CP_MAX
    c[lower_cc == 0] = CP_MIN
    return c


def verify(x: np.ndarray, y: np.ndarray, mode: int = 1, eb: float = 1e-3) -> dict:
    """What a reconstruction y keeps of x:
      - order_violations: neighbour pairs whose order (with the index tie-break of
        Sec. II) differs between x and y, each pair once;
      - cp_x, cp_y: minima, maxima, saddles, regular points (Sec. II);
      - false_positives / false_negatives / false_types (Table III): critical in y
        only / in x only / in both with another type;
      - link_mismatches: points whose (lower, upper) link component counts differ;
      - x_min, x_max, max_abs_err = max |x - y|, mse = mean (x - y)^2, all in
        binary64; psnr = 20 log10(x_max - x_min) - 10 log10(mse) (+inf when mse = 0);
      - eps: the bound of Sec. III-A (eb, or eb (x_max - x_min) for NOA) and
        bound_ok = max_abs_err <= eps."""
    x, y = _c(x), _c(y)
    assert x.dtype == y.dtype and x.shape == y.shape
    if not (np.isfinite(x).all() and np.isfinite(y).all()):
        raise OracleError(NONFINITE, "verify")
    lx, ux = critical_types(x)
    ly, uy = critical_types(y)
    cx, cy = classify(lx, ux), classify(ly, uy)
    crit_x, crit_y = cx != CP_REGULAR, cy != CP_REGULAR
    xd, yd = x.astype(np.float64), y.astype(np.float64)
    d = np.abs(xd - yd)
    x_min, x_max = float(xd.min()), float(xd.max())
    mse = float(np.mean(d * d))
    r = x_max - x_min
    if mse == 0.0:
        psnr = float("inf")
    elif r == 0.0:
        psnr = float("-inf")
    else:
        psnr = 20.0 * np.log10(r) - 10.0 * np.log10(mse)
    eps = eb if mode == 0 else eb * r
    max_err = float(d.max())
    return {
        "points": int(x.size),
        "order_violations": order_violations(x, y),
        "cp_x": [int((cx == k).sum()) for k in range(4)],
        "cp_y": [int((cy == k).sum()) for k in range(4)],
        "false_positives": int((~crit_x & crit_y).sum()),
        "false_negatives": int((crit_x & ~crit_y).sum()),
        "false_types": int((crit_x & crit_y & (cx != cy)).sum()),
        "link_mismatches": int(((lx != ly) | (ux != uy)).sum()),
        "x_min": x_min, "x_max": x_max, "max_abs_err": max_err, "mse": mse, "psnr": float(psnr),
        "eps": float(eps), "bound_ok": bool(max_err <= eps),
    }
