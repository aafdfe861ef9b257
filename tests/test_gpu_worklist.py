"""The paper's worklist repair schedule (Sec. III-D, Alg. 2) as an alternate GPU
mode: from subbins 0, one thread per worklist point, atomicMax raises, deduplicated
worklists.  It reaches the same least fixpoint as the tile schedule, so its streams
are byte-identical to the oracle's and to the tile mode's, on every parity case and
at the full benchmark size; plus its round cap and error paths."""
import numpy as np
import pytest
import torch

from gpu_cases import CASES, bumps
from paper_2603_26968_b300 import synth as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_2603_26968_b300 import build, lopc
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return lopc


class worklist_mode:
    def __init__(self, L):
        self.L = L

    def __enter__(self):
        self.prev = self.L.set_repair_mode(self.L.REPAIR_WORKLIST)

    def __exit__(self, *a):
        self.L.set_repair_mode(self.prev)


@pytest.mark.parametrize("name,make,mode,eb", CASES, ids=[c[0] for c in CASES])
def test_worklist_stream_parity(L, orc, name, make, mode, eb):
    x = make()
    xt = torch.from_numpy(x).cuda()
    with worklist_mode(L):
        st = bytes(L.compress(xt, eb, mode).cpu().numpy().tobytes())
        rounds, runs = L.last_stats()
    assert st == orc.compress(x, mode, eb)
    # the tile mode on the same field: the same bytes
    assert bytes(L.compress(xt, eb, mode).cpu().numpy().tobytes()) == st


@pytest.mark.parametrize("name,make,mode,eb", CASES[:12], ids=[c[0] for c in CASES[:12]])
def test_worklist_subbins_equal_the_least_fixpoint(L, orc, name, make, mode, eb):
    x = make()
    xt = torch.from_numpy(x).cuda()
    with worklist_mode(L):
        b_g, s_g = L.quantize_repair(xt, eb, mode)
        work = L.last_fixpoint_work()
        rounds, _ = L.last_stats()
    e = orc.resolve_eps(x, mode, eb)
    s_o = orc.repair_lfp(x, orc.quantize(x, e["inv"]))
    assert (s_g.cpu().numpy().astype(np.uint64) == s_o).all()
    # every raise of the first iteration evaluated a point; rounds count iterations
    assert rounds >= 1 and work["rerun_raises"] <= work["rerun_evals"]


def test_worklist_iterations_follow_the_longest_chain(L, orc):
    # a decreasing ramp in one bin: point i needs i raises, one per iteration at most
    # along a chain read in order; the schedule still ends and is exact
    x = np.linspace(1.0, 0.0, 2000, dtype=np.float32).reshape(1, 2000)
    xt = torch.from_numpy(x).cuda()
    with worklist_mode(L):
        st = bytes(L.compress(xt, 10.0, L.ABS).cpu().numpy().tobytes())
        rounds, _ = L.last_stats()
    assert st == orc.compress(x, 0, 10.0)
    assert rounds >= 2


def test_worklist_round_cap(L):
    x = torch.from_numpy(np.linspace(1.0, 0.0, 2000, dtype=np.float32).reshape(1, 2000)).cuda()
    old = L.set_round_cap(3)
    try:
        with worklist_mode(L):
            assert L.compress_status(x, 10.0, L.ABS) == -6
    finally:
        L.set_round_cap(old)
    with worklist_mode(L):
        assert L.compress_status(x, 10.0, L.ABS) == 0


def test_worklist_errors(L):
    x = torch.zeros(40, 50, device="cuda")
    x[3, 7] = float("nan")
    with worklist_mode(L):
        assert L.compress_status(x, 1e-3, L.NOA) == -2
        d = L.make_desc((40, 50), "f32", L.NOA, 1e-3)
        ws_wl = L.compress_workspace_size(d)
    ws_tiles = L.compress_workspace_size(d)
    assert ws_wl >= ws_tiles + 12 * 40 * 50
    # a workspace sized for the tile mode is too small for the worklist mode
    y = torch.from_numpy(bumps((40, 50), np.float32)).cuda()
    out = torch.empty(L.compress_bound(d), dtype=torch.uint8, device="cuda")
    ws = torch.empty(ws_tiles, dtype=torch.uint8, device="cuda")
    with worklist_mode(L):
        with pytest.raises(L.LopcError) as e:
            L.compress(y, 1e-3, L.NOA, out=out, workspace=ws)
    assert e.value.code == -8


def test_worklist_full_size_equals_tiles(L):
    x = S.make_field(S.spec_3d_f32(n=512))
    xt = torch.from_numpy(x).cuda()
    a = L.compress(xt, 1e-3, L.NOA).cpu().numpy().tobytes()
    with worklist_mode(L):
        b = L.compress(xt, 1e-3, L.NOA).cpu().numpy().tobytes()
        rounds, _ = L.last_stats()
    assert a == b and rounds > 1
