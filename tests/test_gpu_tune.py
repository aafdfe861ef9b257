"""Launch tuning never changes output bytes: the repair's result is the unique least
fixpoint whatever the schedule (Sec. III-E), so the rerun grid, the tile pass's
frontier budget, its switch to the topological order and the order in which it takes
the tiles only move time."""
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


@pytest.fixture
def restore(L):
    saved = (L.tune_get(), L.tune_get_budget(), L.tune_get_dense(), L.tune_get_pass_order())
    yield
    L.tune_set(saved[0])
    L.tune_set_budget(saved[1])
    L.tune_set_dense(saved[2])
    L.tune_set_pass_order(saved[3])


SETTINGS = [  # (rerun blocks per SM, frontier budget in 16ths, dense threshold in 16ths, pass order)
    ([4, 4, 6, 6], [64] * 4, [8] * 4, [0] * 4),      # defaults
    ([1, 1, 1, 1], [1] * 4, [17] * 4, [2] * 4),      # tiny grid; topological at once; tile-key order
    ([8, 8, 8, 8], [4096] * 4, [17] * 4, [1] * 4),   # frontier sweeps only, index order
    ([2, 5, 3, 7], [16] * 4, [0] * 4, [2, 1, 2, 1]), # every tile in topological order
]


@pytest.mark.parametrize("eb", [1e-2, 1e-3])
def test_streams_do_not_depend_on_tuning(L, restore, eb):
    fields = [
        torch.from_numpy(S.make_field(S.spec_3d_f32(seed=3, n=96, eb=eb))).cuda(),
        torch.from_numpy(S.make_field(S.spec_2d_small(seed=4, shape=(300, 260), eb=eb))).cuda(),
        torch.from_numpy(S.make_field(S.spec_3d_f64_ties(seed=5, shape=(40, 56, 48), eb=eb))).cuda(),
    ]
    ref = None
    for rerun, budget, dense, order in SETTINGS:
        L.tune_set(rerun)
        L.tune_set_budget(budget)
        L.tune_set_dense(dense)
        L.tune_set_pass_order(order)
        got = [L.compress(x, eb, L.NOA).cpu().numpy().tobytes() for x in fields]
        streams, status = L.batch_compress(fields, [eb] * len(fields))
        assert status == [0] * len(fields)
        assert [s.cpu().numpy().tobytes() for s in streams] == got
        if ref is None:
            ref = got
        assert got == ref, (rerun, budget, dense, order)


def test_pass_order_follows_the_sample_span(L, restore):
    """By default the pass takes tile-key order only where a field's tiles span few
    bins (long same-bin chains across tile faces); forcing either order gives the same
    bytes and reports the order taken."""
    x = torch.from_numpy(S.make_field(S.spec_3d_f32(seed=7, n=96))).cuda()
    for eb, want in ((0.1, 1), (1e-4, 0)):
        L.tune_set_pass_order([L.PASS_ORDER_AUTO] * 4)
        auto = L.compress(x, eb, L.NOA).cpu().numpy().tobytes()
        assert L.last_fixpoint_work()["pass_ordered"] == want, eb
        for mode, flag in ((L.PASS_ORDER_INDEX, 0), (L.PASS_ORDER_KEY, 1)):
            L.tune_set_pass_order([mode] * 4)
            assert L.compress(x, eb, L.NOA).cpu().numpy().tobytes() == auto
            assert L.last_fixpoint_work()["pass_ordered"] == flag
