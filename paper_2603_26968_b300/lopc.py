"""Python binding of the C ABI in ``include/lopc.h`` (ctypes; marshalling only).

Every step of compression and decompression runs in the CUDA library
``liblopc.so``; this module passes device pointers of torch tensors, sizes and the
current CUDA stream.  There is no fallback: if the library is missing, importing
the binding's functions raises.
"""
from __future__ import annotations

import ctypes as C
from pathlib import Path
from typing import Optional, Tuple

import torch

PKG = Path(__file__).resolve().parent
LIB_PATH = PKG / "liblopc.so"

OK = 0
ERRORS = {-1: "INVALID_ARG", -2: "NONFINITE", -3: "RANGE", -4: "CAPACITY", -5: "CORRUPT",
          -6: "NOT_CONVERGED", -7: "CUDA", -8: "WORKSPACE", -9: "BUSY"}
ERR_CAPACITY, ERR_BUSY = -4, -9
ERRORS_INV = {v: k for k, v in ERRORS.items()}
F32, F64 = 0, 1
ABS, NOA = 0, 1
REPAIR_TILES, REPAIR_WORKLIST = 0, 1


class LopcError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {ERRORS.get(code, code)} ({lib().lopc_strerror(code).decode()})")
        self.code = code


class FieldDesc(C.Structure):
    _fields_ = [("dtype", C.c_int32), ("ndim", C.c_int32), ("dims", C.c_int64 * 3),
                ("mode", C.c_int32), ("reserved", C.c_int32), ("eb", C.c_double)]

    @property
    def shape(self) -> Tuple[int, ...]:
        return tuple(int(self.dims[k]) for k in range(self.ndim))

    @property
    def torch_dtype(self):
        return torch.float32 if self.dtype == F32 else torch.float64


_lib = None


class VerifyReport(C.Structure):
    """lopc_verify_report (include/lopc.h)."""
    _fields_ = [("points", C.c_int64), ("order_violations", C.c_int64), ("cp_x", C.c_int64 * 4),
                ("cp_y", C.c_int64 * 4), ("false_positives", C.c_int64), ("false_negatives", C.c_int64),
                ("false_types", C.c_int64), ("link_mismatches", C.c_int64), ("nonfinite", C.c_int64),
                ("x_min", C.c_double), ("x_max", C.c_double), ("max_abs_err", C.c_double), ("mse", C.c_double),
                ("psnr", C.c_double), ("eps", C.c_double), ("bound_ok", C.c_int32), ("reserved", C.c_int32)]


class Plan(C.Structure):
    """lopc_plan: launch settings of a batched compression, per field class (0 f32 2D,
    1 f32 3D, 2 f64 2D, 3 f64 3D).  Output bytes never depend on them."""
    _fields_ = [("rerun_blocks_per_sm", C.c_int32 * 4), ("pass_budget16", C.c_int32 * 4),
                ("pass_dense16", C.c_int32 * 4), ("pass_order", C.c_int32 * 4)]

    def as_dict(self) -> dict:
        return {k: list(getattr(self, k)) for k, _ in self._fields_}

    @classmethod
    def of(cls, d: dict) -> "Plan":
        p = cls()
        for k, _ in cls._fields_:
            setattr(p, k, (C.c_int32 * 4)(*[int(v) for v in d[k]]))
        return p


def plan_default() -> Plan:
    p = Plan()
    lib().lopc_plan_default(C.byref(p))
    return p


def plan_get() -> Plan:
    """This thread's current plan (the lopc_tune_* settings)."""
    p = Plan()
    lib().lopc_plan_get(C.byref(p))
    return p


def lib():
    """Loads ``liblopc.so`` (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not LIB_PATH.exists():
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2603_26968_b300.build")
        L = C.CDLL(str(LIB_PATH))
        P, D = C.c_void_p, C.POINTER(FieldDesc)
        L.lopc_compress_bound.argtypes = [D]
        L.lopc_compress_bound.restype = C.c_size_t
        L.lopc_compress_workspace_size.argtypes = [D]
        L.lopc_compress_workspace_size.restype = C.c_size_t
        L.lopc_decompress_workspace_size.argtypes = [D]
        L.lopc_decompress_workspace_size.restype = C.c_size_t
        L.lopc_compress.argtypes = [D, P, P, C.c_size_t, C.POINTER(C.c_size_t), P, C.c_size_t, P]
        L.lopc_peek.argtypes = [P, C.c_size_t, D]
        L.lopc_decompress.argtypes = [P, C.c_size_t, P, C.c_size_t, P, C.c_size_t, P]
        L.lopc_decompress_noalloc.argtypes = [P, C.c_size_t, P, C.c_size_t, P]
        L.lopc_noalloc_max_chunks.restype = C.c_int64
        L.lopc_batch_compress_workspace_size.argtypes = [C.c_int, D]
        L.lopc_batch_compress_workspace_size.restype = C.c_size_t
        L.lopc_batch_compress.argtypes = [C.c_int, D, P, P, P, P, P, C.POINTER(Plan), P, C.c_size_t, P]
        L.lopc_plan_default.argtypes = [C.POINTER(Plan)]
        L.lopc_plan_default.restype = None
        L.lopc_plan_get.argtypes = [C.POINTER(Plan)]
        L.lopc_plan_get.restype = None
        L.lopc_batch_decompress_workspace_size.argtypes = [C.c_int, D]
        L.lopc_batch_decompress_workspace_size.restype = C.c_size_t
        L.lopc_batch_decompress.argtypes = [C.c_int, D, P, P, P, P, P, C.c_size_t, P]
        L.lopc_quantize_repair.argtypes = [D, P, P, P, P, C.c_size_t, P]
        L.lopc_set_round_cap.argtypes = [C.c_int64]
        L.lopc_set_round_cap.restype = C.c_int64
        L.lopc_last_stats.argtypes = [C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
        L.lopc_last_fixpoint_stats.argtypes = [C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
        L.lopc_last_phase_cycles.argtypes = [C.POINTER(C.c_int64), C.c_int]
        L.lopc_last_fixpoint_work.argtypes = [C.POINTER(C.c_int64), C.c_int]
        L.lopc_last_round_tiles.argtypes = [C.POINTER(C.c_int64), C.c_int]
        L.lopc_decode_phase_enable.argtypes = [C.c_int]
        L.lopc_decode_phase_read.argtypes = [C.POINTER(C.c_int64), C.c_int]
        L.lopc_profile_enable.argtypes = [C.c_int]
        L.lopc_profile_reset.argtypes = []
        L.lopc_profile_read.argtypes = [C.POINTER(C.c_char_p), C.POINTER(C.c_int64), C.POINTER(C.c_double), C.c_int]
        L.lopc_profile_read.restype = C.c_int
        L.lopc_profile_read_launches.argtypes = [C.c_char_p, C.POINTER(C.c_double), C.c_int]
        L.lopc_profile_read_launches.restype = C.c_int
        E = C.c_void_p
        L.lopc_engine_create.argtypes = [C.c_int, C.c_int64, C.POINTER(E)]
        L.lopc_engine_destroy.argtypes = [E]
        L.lopc_engine_destroy.restype = None
        L.lopc_engine_field_workspace_size.argtypes = [D]
        L.lopc_engine_field_workspace_size.restype = C.c_size_t
        L.lopc_engine_submit.argtypes = [E, D, P, P, C.c_size_t, P, C.c_size_t, C.c_uint64, P]
        L.lopc_engine_step.argtypes = [E, C.c_int, C.POINTER(C.c_int)]
        L.lopc_engine_poll.argtypes = [E, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64), C.POINTER(C.c_int), C.c_int]
        L.lopc_engine_sync.argtypes = [E]
        L.lopc_tune_set.argtypes = [C.POINTER(C.c_int)]
        L.lopc_tune_set.restype = None
        L.lopc_tune_get.argtypes = [C.POINTER(C.c_int)]
        L.lopc_tune_get.restype = None
        L.lopc_tune_set_budget.argtypes = [C.POINTER(C.c_int)]
        L.lopc_tune_set_budget.restype = None
        L.lopc_tune_get_budget.argtypes = [C.POINTER(C.c_int)]
        L.lopc_tune_get_budget.restype = None
        L.lopc_tune_set_dense.argtypes = [C.POINTER(C.c_int)]
        L.lopc_tune_set_dense.restype = None
        L.lopc_tune_set_pass_order.argtypes = [C.POINTER(C.c_int)]
        L.lopc_tune_set_pass_order.restype = None
        L.lopc_tune_get_pass_order.argtypes = [C.POINTER(C.c_int)]
        L.lopc_tune_get_pass_order.restype = None
        L.lopc_tune_get_dense.argtypes = [C.POINTER(C.c_int)]
        L.lopc_tune_get_dense.restype = None
        L.lopc_verify_workspace_size.argtypes = [D]
        L.lopc_verify_workspace_size.restype = C.c_size_t
        L.lopc_verify.argtypes = [D, P, P, P, P, C.POINTER(VerifyReport), P, C.c_size_t, P]
        L.lopc_set_repair_mode.argtypes = [C.c_int]
        L.lopc_set_repair_mode.restype = C.c_int
        L.lopc_strerror.argtypes = [C.c_int]
        L.lopc_strerror.restype = C.c_char_p
        _lib = L
    return _lib


def make_desc(shape, dtype, mode: int = NOA, eb: float = 1e-3) -> FieldDesc:
    d = FieldDesc()
    if dtype in (torch.float32, F32, "f32"):
        d.dtype = F32
    elif dtype in (torch.float64, F64, "f64"):
        d.dtype = F64
    else:
        raise TypeError(dtype)
    d.ndim = len(shape)
    for k, n in enumerate(shape):
        d.dims[k] = int(n)
    d.mode = int(mode)
    d.eb = float(eb)
    return d


def _stream(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def _check(rc: int, what: str):
    if rc != OK:
        raise LopcError(rc, what)


def compress_bound(desc: FieldDesc) -> int:
    return int(lib().lopc_compress_bound(C.byref(desc)))


def compress_workspace_size(desc: FieldDesc) -> int:
    return int(lib().lopc_compress_workspace_size(C.byref(desc)))


def decompress_workspace_size(desc: FieldDesc) -> int:
    return int(lib().lopc_decompress_workspace_size(C.byref(desc)))


def _field_desc(x: torch.Tensor, mode: int, eb: float) -> FieldDesc:
    if not x.is_cuda or not x.is_contiguous():
        raise ValueError("field must be a contiguous CUDA tensor")
    return make_desc(tuple(x.shape), x.dtype, mode, eb)


def compress(x: torch.Tensor, eb: float, mode: int = NOA, out: Optional[torch.Tensor] = None,
             workspace: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """Compresses a CUDA field; returns the stream as a uint8 CUDA tensor (a view of
    ``out`` when given)."""
    d = _field_desc(x, mode, eb)
    if out is None:
        out = torch.empty(compress_bound(d), dtype=torch.uint8, device=x.device)
    if workspace is None:
        workspace = torch.empty(compress_workspace_size(d), dtype=torch.uint8, device=x.device)
    size = C.c_size_t()
    rc = lib().lopc_compress(C.byref(d), C.c_void_p(x.data_ptr()), C.c_void_p(out.data_ptr()), out.numel(),
                             C.byref(size), C.c_void_p(workspace.data_ptr()), workspace.numel(),
                             C.c_void_p(_stream(stream)))
    _check(rc, "lopc_compress")
    return out[: size.value]


def peek(stream_bytes) -> FieldDesc:
    b = bytes(stream_bytes[:128]) if not isinstance(stream_bytes, torch.Tensor) else \
        bytes(stream_bytes[:128].cpu().numpy().tobytes())
    buf = C.create_string_buffer(b, len(b))
    d = FieldDesc()
    _check(lib().lopc_peek(buf, len(b), C.byref(d)), "lopc_peek")
    return d


def decompress(stream_t: torch.Tensor, out: Optional[torch.Tensor] = None, desc: Optional[FieldDesc] = None,
               workspace: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """Decompresses a stream held in a uint8 CUDA tensor.  Without `desc`, through
    lopc_decompress, which reads the header to the host first.  With the field's
    descriptor (what lopc_peek gives), through lopc_batch_decompress of one stream,
    which checks the header against it on the device: one status read instead of two
    round trips."""
    if not stream_t.is_cuda:
        raise ValueError("stream must be a CUDA tensor")
    if desc is None:
        d = peek(stream_t)
        if out is None:
            out = torch.empty(d.shape, dtype=d.torch_dtype, device=stream_t.device)
        if workspace is None:
            workspace = torch.empty(decompress_workspace_size(d), dtype=torch.uint8, device=stream_t.device)
        rc = lib().lopc_decompress(C.c_void_p(stream_t.data_ptr()), stream_t.numel(), C.c_void_p(out.data_ptr()),
                                   out.numel() * out.element_size(), C.c_void_p(workspace.data_ptr()),
                                   workspace.numel(), C.c_void_p(_stream(stream)))
        _check(rc, "lopc_decompress")
        return out
    if out is None:
        out = torch.empty(desc.shape, dtype=desc.torch_dtype, device=stream_t.device)
    need = (4 if desc.dtype == F32 else 8)
    for n in desc.shape:
        need *= int(n)
    if out.device != stream_t.device or not out.is_contiguous() or out.numel() * out.element_size() < need:
        raise LopcError(ERR_CAPACITY, "lopc_decompress")
    if workspace is None:
        workspace = torch.empty(decompress_workspace_size(desc), dtype=torch.uint8, device=stream_t.device)
    status = torch.empty(1, dtype=torch.int32, device=stream_t.device)
    rc = lib().lopc_batch_decompress(1, C.byref(desc), (C.c_void_p * 1)(stream_t.data_ptr()),
                                     (C.c_size_t * 1)(stream_t.numel()), (C.c_void_p * 1)(out.data_ptr()),
                                     C.c_void_p(status.data_ptr()), C.c_void_p(workspace.data_ptr()),
                                     workspace.numel(), C.c_void_p(_stream(stream)))
    _check(rc, "lopc_decompress")
    if stream is not None:
        stream.synchronize()
    _check(int(status.item()), "lopc_decompress")
    return out


def decompress_noalloc(stream_t: torch.Tensor, out: torch.Tensor, stream=None) -> int:
    """Status of lopc_decompress_noalloc: decompression into ``out`` with the
    library's fixed scratch instead of a workspace (for callers that cannot
    allocate device memory; see include/lopc.h)."""
    return lib().lopc_decompress_noalloc(C.c_void_p(stream_t.data_ptr()), stream_t.numel(),
                                         C.c_void_p(out.data_ptr()), out.numel() * out.element_size(),
                                         C.c_void_p(_stream(stream)))


def quantize_repair(x: torch.Tensor, eb: float, mode: int = NOA) -> Tuple[torch.Tensor, torch.Tensor]:
    """Bins (int64) and subbins (uint64 bits in an int64 tensor) of a CUDA field."""
    d = _field_desc(x, mode, eb)
    ws = torch.empty(compress_workspace_size(d), dtype=torch.uint8, device=x.device)
    b = torch.empty(x.shape, dtype=torch.int64, device=x.device)
    s = torch.empty(x.shape, dtype=torch.int64, device=x.device)
    rc = lib().lopc_quantize_repair(C.byref(d), C.c_void_p(x.data_ptr()), C.c_void_p(b.data_ptr()),
                                    C.c_void_p(s.data_ptr()), C.c_void_p(ws.data_ptr()), ws.numel(),
                                    C.c_void_p(_stream(None)))
    _check(rc, "lopc_quantize_repair")
    return b, s


def verify_workspace_size(desc: FieldDesc) -> int:
    return int(lib().lopc_verify_workspace_size(C.byref(desc)))


def verify(x: torch.Tensor, y: torch.Tensor, eb: float = 1e-3, mode: int = NOA,
           types_x: Optional[torch.Tensor] = None, types_y: Optional[torch.Tensor] = None,
           workspace: Optional[torch.Tensor] = None, stream=None) -> dict:
    """What the reconstruction ``y`` keeps of ``x`` (lopc_verify): order violations,
    critical-point classes of both, false positives / negatives / types, link
    mismatches, range, max |x - y|, MSE, PSNR and the bound of (mode, eb).  Given
    uint8 CUDA tensors of x's shape, ``types_x`` / ``types_y`` receive each point's
    lower-link pieces | upper-link pieces << 4."""
    if y.shape != x.shape or y.dtype != x.dtype or not y.is_cuda or not y.is_contiguous():
        raise ValueError("y must be a contiguous CUDA tensor like x")
    d = _field_desc(x, mode, eb)
    if workspace is None:
        workspace = torch.empty(verify_workspace_size(d), dtype=torch.uint8, device=x.device)
    for t in (types_x, types_y):
        if t is not None and (t.dtype != torch.uint8 or t.shape != x.shape or not t.is_cuda or not t.is_contiguous()):
            raise ValueError("types must be contiguous uint8 CUDA tensors of the field's shape")
    tx = C.c_void_p(types_x.data_ptr()) if types_x is not None else None
    ty = C.c_void_p(types_y.data_ptr()) if types_y is not None else None
    r = VerifyReport()
    rc = lib().lopc_verify(C.byref(d), C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()), tx, ty, C.byref(r),
                           C.c_void_p(workspace.data_ptr()), workspace.numel(), C.c_void_p(_stream(stream)))
    _check(rc, "lopc_verify")
    return {
        "points": r.points, "order_violations": r.order_violations, "cp_x": list(r.cp_x), "cp_y": list(r.cp_y),
        "false_positives": r.false_positives, "false_negatives": r.false_negatives,
        "false_types": r.false_types, "link_mismatches": r.link_mismatches,
        "x_min": r.x_min, "x_max": r.x_max, "max_abs_err": r.max_abs_err, "mse": r.mse, "psnr": r.psnr,
        "eps": r.eps, "bound_ok": bool(r.bound_ok),
    }


def set_repair_mode(mode: int) -> int:
    """Repair schedule of single-field calls on this thread (REPAIR_TILES or
    REPAIR_WORKLIST); returns the previous one.  Query workspace sizes after it."""
    rc = lib().lopc_set_repair_mode(int(mode))
    if rc < 0:
        raise LopcError(rc, "lopc_set_repair_mode")
    return rc


def set_round_cap(cap: int) -> int:
    return int(lib().lopc_set_round_cap(int(cap)))


def last_stats() -> Tuple[int, int]:
    r, t = C.c_int64(), C.c_int64()
    lib().lopc_last_stats(C.byref(r), C.byref(t))
    return r.value, t.value


def last_fixpoint_stats() -> Tuple[int, int]:
    """(sweeps summed over tile runs, most sweeps of one run) of the last compression."""
    a, b = C.c_int64(), C.c_int64()
    lib().lopc_last_fixpoint_stats(C.byref(a), C.byref(b))
    return a.value, b.value


def last_phase_cycles() -> list:
    """SM cycles per kernel phase of the last compression (see include/lopc.h)."""
    a = (C.c_int64 * 9)()
    lib().lopc_last_phase_cycles(a, 9)
    return [int(v) for v in a]


def last_fixpoint_work() -> dict:
    """Fixpoint point evaluations and raises of the last compression (pass, reruns),
    rerun tiles loaded and idle, and whether the tile pass ran in tile-key order."""
    v = (C.c_int64 * 7)()
    lib().lopc_last_fixpoint_work(v, 7)
    return {"pass_evals": v[0], "pass_raises": v[1], "rerun_evals": v[2], "rerun_raises": v[3],
            "rerun_tiles": v[4], "rerun_idle": v[5], "pass_ordered": v[6]}


def last_round_tiles() -> list:
    """Tiles listed per repair round of the last profiled compression."""
    v = (C.c_int64 * 4096)()
    n = lib().lopc_last_round_tiles(v, 4096)
    return [int(v[k]) for k in range(min(n, 4096))]


def decode_phase_enable(on: bool = True) -> None:
    _check(lib().lopc_decode_phase_enable(1 if on else 0), "lopc_decode_phase_enable")


def decode_phase_read() -> dict:
    """SM cycles per decode phase since the last read (summed over blocks)."""
    v = (C.c_int64 * 8)()
    rc = lib().lopc_decode_phase_read(v, 8)
    if rc < 0:
        _check(rc, "lopc_decode_phase_read")
    names = ["bin_rze", "bin_planes_scan", "bin_range_cache", "sub_rze1", "sub_rzew", "sub_planes_values"]
    return dict(zip(names, [int(a) for a in v[:6]]))


def compress_status(x: torch.Tensor, eb: float, mode: int = NOA, out_cap: Optional[int] = None,
                    ws_bytes: Optional[int] = None) -> int:
    """Raw status of lopc_compress (for error-path tests)."""
    d = _field_desc(x, mode, eb)
    cap = compress_bound(d) if out_cap is None else out_cap
    out = torch.empty(max(cap, 1), dtype=torch.uint8, device=x.device)
    wsz = compress_workspace_size(d) if ws_bytes is None else ws_bytes
    ws = torch.empty(max(wsz, 1), dtype=torch.uint8, device=x.device)
    size = C.c_size_t()
    return lib().lopc_compress(C.byref(d), C.c_void_p(x.data_ptr()), C.c_void_p(out.data_ptr()), cap,
                               C.byref(size), C.c_void_p(ws.data_ptr()), wsz, C.c_void_p(_stream(None)))


def decompress_status(stream_t: torch.Tensor, shape, dtype) -> int:
    out = torch.empty(shape, dtype=dtype, device=stream_t.device)
    d = make_desc(shape, dtype)
    ws = torch.empty(decompress_workspace_size(d), dtype=torch.uint8, device=stream_t.device)
    return lib().lopc_decompress(C.c_void_p(stream_t.data_ptr()), stream_t.numel(), C.c_void_p(out.data_ptr()),
                                 out.numel() * out.element_size(), C.c_void_p(ws.data_ptr()), ws.numel(),
                                 C.c_void_p(_stream(None)))


def profile_enable(on: bool = True) -> None:
    """Per-kernel CUDA-event timing inside the library (see include/lopc.h)."""
    lib().lopc_profile_enable(1 if on else 0)


def profile_reset() -> None:
    lib().lopc_profile_reset()


def profile_read() -> dict:
    """{kernel name: (launches, total milliseconds)} since the last reset."""
    cap = 64
    names = (C.c_char_p * cap)()
    launches = (C.c_int64 * cap)()
    ms = (C.c_double * cap)()
    n = lib().lopc_profile_read(names, launches, ms, cap)
    return {names[i].decode(): (int(launches[i]), float(ms[i])) for i in range(min(n, cap))}


# ------------------------------------------------------------------------ batches

def profile_read_launches(name: str) -> list:
    """Times (ms) of every timed launch of one kernel, in launch order."""
    cap = 100000
    v = (C.c_double * cap)()
    n = lib().lopc_profile_read_launches(name.encode(), v, cap)
    return [float(v[k]) for k in range(min(n, cap))]


def _descs(items):
    arr = (FieldDesc * len(items))()
    for i, d in enumerate(items):
        arr[i] = d
    return arr


def batch_compress_workspace_size(descs) -> int:
    return int(lib().lopc_batch_compress_workspace_size(len(descs), _descs(descs)))


def batch_decompress_workspace_size(descs) -> int:
    return int(lib().lopc_batch_decompress_workspace_size(len(descs), _descs(descs)))


class BatchCompress:
    """A reusable batched compression of fixed fields (inputs, outputs, workspace
    and result arrays stay allocated, so repeated launches replay one cached graph)."""

    def __init__(self, fields, ebs, modes=None, device=None, plan: Optional[Plan] = None):
        self.plan = plan
        self.fields = [f.contiguous() for f in fields]
        n = len(self.fields)
        modes = modes if modes is not None else [NOA] * n
        self.descs = [make_desc(tuple(f.shape), f.dtype, m, e) for f, m, e in zip(self.fields, modes, ebs)]
        dev = self.fields[0].device if device is None else device
        self.caps = [compress_bound(d) for d in self.descs]
        self.outs = [torch.empty(c, dtype=torch.uint8, device=dev) for c in self.caps]
        self.ws = torch.empty(batch_compress_workspace_size(self.descs), dtype=torch.uint8, device=dev)
        self.sizes = torch.zeros(n, dtype=torch.int64, device=dev)
        self.status = torch.zeros(n, dtype=torch.int32, device=dev)
        self._d = _descs(self.descs)
        self._x = (C.c_void_p * n)(*[f.data_ptr() for f in self.fields])
        self._o = (C.c_void_p * n)(*[o.data_ptr() for o in self.outs])
        self._c = (C.c_size_t * n)(*self.caps)

    def launch(self, stream=None, plan: Optional[Plan] = None) -> None:
        """Enqueues the batch on the stream (asynchronous).  ``plan`` (else the one
        given at construction, else this thread's current plan) sets the launches."""
        pl = plan if plan is not None else self.plan
        rc = lib().lopc_batch_compress(len(self.fields), self._d, self._x, self._o, self._c,
                                       C.c_void_p(self.sizes.data_ptr()), C.c_void_p(self.status.data_ptr()),
                                       C.byref(pl) if pl is not None else None,
                                       C.c_void_p(self.ws.data_ptr()), self.ws.numel(), C.c_void_p(_stream(stream)))
        _check(rc, "lopc_batch_compress")

    def results(self):
        """(list of stream tensors, list of status codes) after the launch finished."""
        sizes = self.sizes.cpu().tolist()
        st = self.status.cpu().tolist()
        return [o[:n] for o, n in zip(self.outs, sizes)], st


def batch_compress(fields, ebs, modes=None, stream=None, plan: Optional[Plan] = None):
    b = BatchCompress(fields, ebs, modes, plan=plan)
    b.launch(stream)
    torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()
    return b.results()


def batch_decompress(streams, outs=None, stream=None):
    """Decompresses a list of uint8 CUDA stream tensors; returns (fields, statuses)."""
    descs = [peek(s) for s in streams]
    n = len(streams)
    dev = streams[0].device
    if outs is None:
        outs = [torch.empty(d.shape, dtype=d.torch_dtype, device=dev) for d in descs]
    ws = torch.empty(batch_decompress_workspace_size(descs), dtype=torch.uint8, device=dev)
    status = torch.zeros(n, dtype=torch.int32, device=dev)
    ins = (C.c_void_p * n)(*[s.data_ptr() for s in streams])
    sizes = (C.c_size_t * n)(*[s.numel() for s in streams])
    xs = (C.c_void_p * n)(*[o.data_ptr() for o in outs])
    rc = lib().lopc_batch_decompress(n, _descs(descs), ins, sizes, xs, C.c_void_p(status.data_ptr()),
                                     C.c_void_p(ws.data_ptr()), ws.numel(), C.c_void_p(_stream(stream)))
    _check(rc, "lopc_batch_decompress")
    torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()
    return outs, status.cpu().tolist()


def tune_set(rerun_blocks_per_sm) -> None:
    """Persistent rerun blocks per SM for classes (f32 2D, f32 3D, f64 2D, f64 3D)."""
    lib().lopc_tune_set((C.c_int * 4)(*[int(v) for v in rerun_blocks_per_sm]))


def tune_get() -> Tuple[int, int, int, int]:
    v = (C.c_int * 4)()
    lib().lopc_tune_get(v)
    return tuple(int(a) for a in v)


def tune_set_budget(sixteenths) -> None:
    """Pass frontier-evaluation budget per class, in sixteenths of a tile's points."""
    lib().lopc_tune_set_budget((C.c_int * 4)(*[int(v) for v in sixteenths]))


def tune_get_budget() -> Tuple[int, int, int, int]:
    v = (C.c_int * 4)()
    lib().lopc_tune_get_budget(v)
    return tuple(int(a) for a in v)


def tune_set_dense(sixteenths) -> None:
    """Same-bin pair density (sixteenths) above which a tile pass goes topological."""
    lib().lopc_tune_set_dense((C.c_int * 4)(*[int(v) for v in sixteenths]))


def tune_get_dense() -> Tuple[int, int, int, int]:
    v = (C.c_int * 4)()
    lib().lopc_tune_get_dense(v)
    return tuple(int(a) for a in v)


PASS_ORDER_AUTO, PASS_ORDER_INDEX, PASS_ORDER_KEY = 0, 1, 2


def tune_set_pass_order(modes) -> None:
    """Tile-pass order per class: PASS_ORDER_AUTO, PASS_ORDER_INDEX or PASS_ORDER_KEY."""
    lib().lopc_tune_set_pass_order((C.c_int * 4)(*[int(v) for v in modes]))


def tune_get_pass_order() -> Tuple[int, int, int, int]:
    v = (C.c_int * 4)()
    lib().lopc_tune_get_pass_order(v)
    return tuple(int(a) for a in v)


def engine_field_workspace_size(desc: FieldDesc) -> int:
    return int(lib().lopc_engine_field_workspace_size(C.byref(desc)))


class Engine:
    """The library's serving engine (round-level continuous batching).  Buffers
    passed to submit() must stay alive until poll() reports their tag."""

    def __init__(self, max_fields: int = 1024, max_tiles: int = 1 << 22):
        self._e = C.c_void_p()
        _check(lib().lopc_engine_create(int(max_fields), int(max_tiles), C.byref(self._e)), "lopc_engine_create")
        self.max_fields = max_fields
        self._tags = (C.c_uint64 * max_fields)()
        self._sizes = (C.c_uint64 * max_fields)()
        self._stat = (C.c_int * max_fields)()

    def submit(self, x: torch.Tensor, desc: FieldDesc, out: torch.Tensor, ws: torch.Tensor, tag: int,
               ready_stream=None) -> int:
        """Queues a field; returns OK or ERR_BUSY (other errors raise)."""
        rc = lib().lopc_engine_submit(self._e, C.byref(desc), C.c_void_p(x.data_ptr()), C.c_void_p(out.data_ptr()),
                                      out.numel(), C.c_void_p(ws.data_ptr()), ws.numel(), C.c_uint64(tag),
                                      C.c_void_p(_stream(ready_stream)))
        if rc not in (OK, ERR_BUSY):
            _check(rc, "lopc_engine_submit")
        return rc

    def step(self, rounds: int = 1) -> int:
        active = C.c_int(0)
        _check(lib().lopc_engine_step(self._e, int(rounds), C.byref(active)), "lopc_engine_step")
        return int(active.value)

    def poll(self):
        """[(tag, stream length, status)] of the fields finished since the last poll."""
        n = lib().lopc_engine_poll(self._e, self._tags, self._sizes, self._stat, self.max_fields)
        if n < 0:
            _check(n, "lopc_engine_poll")
        return [(int(self._tags[k]), int(self._sizes[k]), int(self._stat[k])) for k in range(n)]

    def sync(self) -> None:
        _check(lib().lopc_engine_sync(self._e), "lopc_engine_sync")

    def close(self) -> None:
        if self._e:
            lib().lopc_engine_destroy(self._e)
            self._e = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
