"""Batches: many fields of uneven sizes, ranks and dtypes in one launch sequence.
Every field's stream must be byte-identical alone and in the batch (and to the
oracle's), and its reconstruction likewise; a failing field fails alone."""
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


def mixed_specs(seed=3):
    # the mixed-batch recipe at small sizes: 2D sides 16..200, 3D sides 8..48
    return S.spec_batch(seed=seed, count=14, max_2d=200, min_2d=16, max_3d=48, min_3d=8)


def test_batch_equals_single_and_oracle(L, orc):
    specs = mixed_specs()
    xs = [S.make_field(sp) for sp in specs]
    fields = [torch.from_numpy(x).cuda() for x in xs]
    ebs = [sp.eb for sp in specs]
    streams, status = L.batch_compress(fields, ebs)
    assert status == [0] * len(specs)
    for x, t, st, eb in zip(xs, fields, streams, ebs):
        single = L.compress(t, eb, L.NOA)
        got = bytes(st.cpu().numpy().tobytes())
        assert got == bytes(single.cpu().numpy().tobytes())
        assert got == orc.compress(x, 1, eb)
    outs, dstat = L.batch_decompress(streams)
    assert dstat == [0] * len(specs)
    for x, y, st in zip(xs, outs, streams):
        assert y.cpu().numpy().tobytes() == orc.decompress(bytes(st.cpu().numpy().tobytes())).tobytes()


def test_batch_repeated_launches_replay_identically(L):
    specs = mixed_specs(seed=5)
    fields = [torch.from_numpy(S.make_field(sp)).cuda() for sp in specs]
    b = L.BatchCompress(fields, [sp.eb for sp in specs])
    b.launch()
    first, st1 = b.results()
    first = [bytes(s.cpu().numpy().tobytes()) for s in first]
    for _ in range(3):
        b.launch()
        again, st2 = b.results()
        assert st2 == st1 and [bytes(s.cpu().numpy().tobytes()) for s in again] == first


def test_batch_fields_fail_alone(L, orc):
    good = torch.from_numpy(S.make_field(S.spec_2d_small(shape=(40, 50)))).cuda()
    bad = good.clone()
    bad[3, 4] = float("nan")
    const = torch.full((9, 10, 11), 2.0, dtype=torch.float64, device="cuda")
    tiny = torch.linspace(-1, 1, 64 * 64, device="cuda").reshape(64, 64)
    streams, status = L.batch_compress([good, bad, const, tiny], [1e-3, 1e-3, 1e-3, 1e-12],
                                       [L.NOA, L.NOA, L.NOA, L.ABS])
    assert status == [0, -2, 0, -3]
    assert bytes(streams[0].cpu().numpy().tobytes()) == orc.compress(good.cpu().numpy(), 1, 1e-3)
    assert bytes(streams[2].cpu().numpy().tobytes()) == orc.compress(const.cpu().numpy(), 1, 1e-3)


def test_batch_decompress_reports_corrupt_streams_alone(L):
    a = torch.from_numpy(S.make_field(S.spec_2d_small(shape=(70, 80)))).cuda()
    b = torch.from_numpy(S.make_field(S.spec_3d_f32(n=24))).cuda()
    sa = L.compress(a, 1e-3, L.NOA).clone()
    sb = L.compress(b, 1e-3, L.NOA).clone()
    sb[-20] ^= 0xFF  # inside the last record
    outs, st = L.batch_decompress([sa, sb])
    assert st[0] == 0 and st[1] in (0, -5)
    assert torch.equal(outs[0], L.decompress(sa))
