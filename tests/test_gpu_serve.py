"""Serving engine and request loop on the GPU: each served stream is byte-identical
to the same field compressed alone and to the oracle's stream of that field, fields
admitted while others are in repair join them between rounds, and a failing field
fails alone."""
import numpy as np
import pytest
import torch

from paper_2603_26968_b300 import synth_gpu as SG

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_2603_26968_b300 import build, lopc
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return lopc


def _mixed_specs(n, seed, rate=3000.0):
    specs = SG.serve_requests(seed, rate, 10.0, min_bytes=64e3, max_bytes=8e6)[:n]
    assert len(specs) == n
    return specs


def test_served_streams_equal_solo_streams(L, orc):
    """Each served stream equals the same field compressed alone and, byte for byte,
    the oracle's stream of that field (copied to the host)."""
    from paper_2603_26968_b300 import serve
    specs = _mixed_specs(24, seed=5)
    assert {(len(s.shape), s.dtype) for s in specs} == {(2, "f32"), (3, "f32"), (2, "f64"), (3, "f64")}
    srv = serve.Server(budget_bytes=2 << 30, max_fields=64)
    rep = srv.run(specs, keep_streams=True)
    srv.close()
    assert len(rep.served) == len(specs)
    assert rep.in_flight_max >= 2
    assert rep.joined_busy >= 1            # some fields joined a repair already under way
    for r in rep.served:
        assert r.status == L.OK, (r.spec, r.status)
        solo = serve.solo_stream(r.spec)
        assert r.size == solo.numel()
        assert torch.equal(r.stream, solo), r.spec
        x = SG.make_field(r.spec).cpu().numpy()   # the field the server compressed
        want = orc.compress(x, 1, r.spec.eb, openmp=True)
        assert bytes(r.stream.cpu().numpy().tobytes()) == want, r.spec


def test_tight_budget_serialises_but_still_matches(L, orc):
    from paper_2603_26968_b300 import serve
    specs = _mixed_specs(8, seed=6)
    need = max(sum(serve.request_bytes(s).values()) for s in specs)
    srv = serve.Server(budget_bytes=need, max_fields=8)     # room for the largest request only
    rep = srv.run(specs, keep_streams=True)
    srv.close()
    assert rep.budget_peak <= need
    for r in rep.served:
        assert r.status == L.OK
        assert torch.equal(r.stream, serve.solo_stream(r.spec))
        want = orc.compress(SG.make_field(r.spec).cpu().numpy(), 1, r.spec.eb, openmp=True)
        assert bytes(r.stream.cpu().numpy().tobytes()) == want, r.spec


def test_several_rounds_per_step_match_solo(L, orc):
    from paper_2603_26968_b300 import serve
    specs = _mixed_specs(10, seed=11)
    srv = serve.Server(budget_bytes=2 << 30, max_fields=32, rounds_per_step=3)
    rep = srv.run(specs, keep_streams=True)
    srv.close()
    for r in rep.served:
        assert r.status == L.OK
        assert torch.equal(r.stream, serve.solo_stream(r.spec))
        want = orc.compress(SG.make_field(r.spec).cpu().numpy(), 1, r.spec.eb, openmp=True)
        assert bytes(r.stream.cpu().numpy().tobytes()) == want, r.spec


def _engine_submit(L, E, x, eb, tag, cap=None):
    d = L.make_desc(tuple(x.shape), x.dtype, L.NOA, eb)
    out = torch.empty(cap if cap is not None else L.compress_bound(d), dtype=torch.uint8, device=x.device)
    ws = torch.empty(L.engine_field_workspace_size(d), dtype=torch.uint8, device=x.device)
    assert E.submit(x, d, out, ws, tag) == L.OK
    return out, ws


def _drain(E, want):
    got = {}
    for _ in range(100000):
        E.step(1)
        for tag, size, st in E.poll():
            got[tag] = (size, st)
        if len(got) == want:
            return got
    raise AssertionError("engine did not finish")


def test_engine_failing_fields_fail_alone(L):
    E = L.Engine(max_fields=8, max_tiles=1 << 16)
    good = [SG.make_field(s) for s in _mixed_specs(3, seed=7)]
    bad = good[0].clone()
    bad.view(-1)[123] = float("nan")
    keep = [_engine_submit(L, E, x, 1e-3, k) for k, x in enumerate(good)]
    keep.append(_engine_submit(L, E, bad, 1e-3, 10))
    keep.append(_engine_submit(L, E, good[1], 1e-3, 11, cap=200))      # output too small
    got = _drain(E, 5)
    E.close()
    assert got[10][1] == L.ERRORS_INV["NONFINITE"]
    assert got[11][1] == L.ERRORS_INV["CAPACITY"]
    for k, x in enumerate(good):
        size, st = got[k]
        assert st == L.OK
        assert torch.equal(keep[k][0][:size], L.compress(x, 1e-3, L.NOA))


def test_engine_reports_busy_when_full(L):
    E = L.Engine(max_fields=2, max_tiles=1 << 16)
    xs = [SG.make_field(s) for s in _mixed_specs(3, seed=8)]
    d = [L.make_desc(tuple(x.shape), x.dtype, L.NOA, 1e-3) for x in xs]
    bufs = [(torch.empty(L.compress_bound(a), dtype=torch.uint8, device="cuda"),
             torch.empty(L.engine_field_workspace_size(a), dtype=torch.uint8, device="cuda")) for a in d]
    assert E.submit(xs[0], d[0], *bufs[0], 0) == L.OK
    assert E.submit(xs[1], d[1], *bufs[1], 1) == L.OK
    assert E.submit(xs[2], d[2], *bufs[2], 2) == L.ERR_BUSY
    got = _drain(E, 2)
    assert E.submit(xs[2], d[2], *bufs[2], 2) == L.OK             # slots are free again after the poll
    got.update(_drain(E, 1))
    E.close()
    assert all(st == L.OK for _, st in got.values())


def test_gpu_generator_is_deterministic(L):
    s = _mixed_specs(2, seed=9)[1]
    a = SG.make_field(s)
    b = SG.make_field(s)
    assert torch.equal(a, b)
    assert torch.isfinite(a).all()
