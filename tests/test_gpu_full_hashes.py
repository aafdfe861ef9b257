"""Whole-stream bit identity with the oracle at full size.

For every full-size workload (the 2D image, the 512^3 float32 field at NOA 1e-2,
1e-3 and 1e-4, the 256x384x384 float64 field with ties, and each of the 64 fields of
the mixed batch), the SHA-256 of the CUDA path's stream and of its reconstruction
must equal the oracle's, stored in tests/golden/full_hashes.json by
tests/golden/make_full_hashes.py (the paper's claim that CPU and GPU give the same
bytes, Sec. I and Sec. V).  The field's own hash is checked first, so that a
generator difference shows up as one and not as a compressor bug.  The sampled
diagnostics in test_gpu_parity.py say where a difference lies.
"""
import hashlib
import json
from pathlib import Path

import numpy as np
import pytest
import torch

from full_cases import cases, field_key
from paper_2603_26968_b300 import synth as S

pytestmark = pytest.mark.gpu

GOLD = json.loads((Path(__file__).resolve().parent / "golden" / "full_hashes.json").read_text())["cases"]
CASES = cases()
SINGLE = [c for c in CASES if c[1] == "single"]
BATCH = [c for c in CASES if c[1] == "batch"]


@pytest.fixture(scope="module")
def L():
    from paper_2603_26968_b300 import build, lopc
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return lopc


_fields = {}


def host_field(spec):
    k = field_key(spec)
    if k not in _fields:
        _fields.clear()  # one full-size field at a time
        _fields[k] = S.make_field(spec)
    return _fields[k]


def sha(t) -> str:
    a = t.cpu().numpy() if isinstance(t, torch.Tensor) else t
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def test_golden_table_covers_every_case():
    assert set(GOLD) == {c[0] for c in CASES}


@pytest.mark.parametrize("mode_name", ["tiles", "worklist"])
@pytest.mark.parametrize("name,group,spec", SINGLE, ids=[c[0] for c in SINGLE])
def test_full_size_stream_and_xhat_hash(L, name, group, spec, mode_name):
    want = GOLD[name]
    x = host_field(spec)
    assert sha(x) == want["field_sha256"], "the generator made another field"
    xt = torch.from_numpy(x).cuda()
    prev = L.set_repair_mode(L.REPAIR_WORKLIST if mode_name == "worklist" else L.REPAIR_TILES)
    try:
        st = L.compress(xt, spec.eb, L.NOA)
    finally:
        L.set_repair_mode(prev)
    assert st.numel() == want["stream_bytes"]
    assert sha(st) == want["stream_sha256"]
    y = L.decompress(st)
    assert sha(y) == want["xhat_sha256"]


def test_full_size_batch_hashes(L):
    xs = [torch.from_numpy(S.make_field(sp)).cuda() for _, _, sp in BATCH]
    for (name, _, _), x in zip(BATCH, xs):
        assert sha(x) == GOLD[name]["field_sha256"], name
    streams, status = L.batch_compress(xs, [sp.eb for _, _, sp in BATCH])
    assert status == [0] * len(BATCH)
    for (name, _, _), st in zip(BATCH, streams):
        assert st.numel() == GOLD[name]["stream_bytes"], name
        assert sha(st) == GOLD[name]["stream_sha256"], name
    outs, dstat = L.batch_decompress(streams)
    assert dstat == [0] * len(BATCH)
    for (name, _, _), y in zip(BATCH, outs):
        assert sha(y) == GOLD[name]["xhat_sha256"], name
    # one call per field gives the same bytes
    for (name, _, sp), x in zip(BATCH, xs):
        assert sha(L.compress(x, sp.eb, L.NOA)) == GOLD[name]["stream_sha256"], name
