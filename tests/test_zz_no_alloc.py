"""lopc_decompress_noalloc: decompression for callers that cannot allocate device
memory (allocator callbacks, hosts that reserve all memory up front).  Its output
must equal lopc_decompress's, bit for bit (the tolerance of every decompression test
here), on calls made back to back that share the library's fixed scratch array.

This file is collected last on purpose; it also passes on its own in a fresh process.
"""
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


def _field(shape, dtype, seed):
    f = np.zeros(shape, np.float64)
    S.add_bumps(f, 20, max(shape) / 30.0, max(shape) / 5.0, seed)
    S.add_uniform_noise(f, 1e-4, seed)
    return torch.from_numpy(f.astype(dtype)).cuda()


def test_noalloc_matches_workspace_decompress_on_consecutive_calls(L):
    fields = [_field((96, 80, 72), np.float32, 1), _field((130, 200), np.float64, 2)]
    streams = [L.compress(x, 1e-3, L.NOA) for x in fields]
    refs = [L.decompress(st) for st in streams]
    # two calls in a row on different streams (the second reuses the scratch the
    # first left behind), then the first stream again
    for st, ref, x in list(zip(streams, refs, fields)) + [(streams[0], refs[0], fields[0])]:
        out = torch.full_like(x, float("nan"))
        assert L.decompress_noalloc(st, out) == 0
        torch.cuda.synchronize()
        assert out.cpu().numpy().tobytes() == ref.cpu().numpy().tobytes()


def test_noalloc_rejects_streams_beyond_its_scratch(L):
    x = _field((64, 64), np.float32, 3)
    st = L.compress(x, 1e-3, L.NOA)
    hdr = bytearray(st[:128].cpu().numpy().tobytes())
    max_chunks = L.lib().lopc_noalloc_max_chunks()
    nx = 64 * (max_chunks + 1)                      # one chunk more than the scratch holds
    hdr[16:24] = nx.to_bytes(8, "little")
    hdr[80:88] = (max_chunks + 1).to_bytes(8, "little")
    out = torch.empty(16, dtype=torch.float32, device="cuda")
    # the header declares more bytes than the 128 passed: a truncated stream is
    # reported as corrupt before its chunk count is looked at
    dev = torch.frombuffer(bytearray(hdr), dtype=torch.uint8).cuda()
    assert L.decompress_noalloc(dev, out) == -5     # LOPC_ERR_CORRUPT
    hdr[88:96] = (128).to_bytes(8, "little")        # a stream that claims to be whole
    dev = torch.frombuffer(hdr, dtype=torch.uint8).cuda()
    assert L.decompress_noalloc(dev, out) == -8     # LOPC_ERR_WORKSPACE
    # the scratch is idle after a failed call: a good stream decodes right after
    ok = torch.empty_like(x)
    assert L.decompress_noalloc(st, ok) == 0
    torch.cuda.synchronize()
    assert ok.cpu().numpy().tobytes() == L.decompress(st).cpu().numpy().tobytes()
