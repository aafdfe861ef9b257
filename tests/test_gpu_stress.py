"""Stress of the repair's concurrency: reruns take tiles appended to the round in
progress, two blocks can hold the same tile, a tile pass in tile-key order reads the
subbins its neighbours are writing, and the order in which tiles are taken depends on
timing.  Whatever the schedule, the subbins must be the least fixpoint (checked at
every point by its defining equation) and repeated compressions, single or batched,
in either pass order, must give the same bytes."""
import numpy as np
import pytest
import torch

from gpu_cases import bumps
from paper_2603_26968_b300 import synth as S
from test_gpu_parity import lfp_local_equality

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_2603_26968_b300 import build, lopc
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return lopc


FIELDS = [
    # shape, dtype, NOA bound, seed
    ((96, 112, 128), np.float32, 1e-2, 1),
    ((96, 112, 128), np.float32, 3e-3, 2),
    ((80, 96, 104), np.float64, 1e-2, 3),
    ((1000, 1200), np.float32, 1e-2, 4),
    ((600, 900), np.float64, 3e-3, 5),
    ((128, 128, 128), np.float32, 1e-3, 6),
]


def smooth(shape, dtype, seed):
    f = np.zeros(shape, np.float64)
    S.add_bumps(f, 16, max(shape) / 12.0, max(shape) / 3.0, seed)
    S.add_uniform_noise(f, 1e-4, seed)
    return f.astype(dtype)


@pytest.fixture
def auto_order(L):
    saved = L.tune_get_pass_order()
    yield
    L.tune_set_pass_order(saved)


@pytest.mark.parametrize("shape,dtype,eb,seed", FIELDS, ids=[f"{len(f[0])}d_{np.dtype(f[1]).name}_{f[2]:g}" for f in FIELDS])
def test_least_fixpoint_and_identical_bytes_under_any_schedule(L, auto_order, shape, dtype, eb, seed):
    x = smooth(shape, dtype, seed)
    xt = torch.from_numpy(x).cuda()
    first = None
    for rep in range(6):
        # alternate the pass order: index / tile key / by the field
        L.tune_set_pass_order([(L.PASS_ORDER_INDEX, L.PASS_ORDER_KEY, L.PASS_ORDER_AUTO)[rep % 3]] * 4)
        b, s = L.quantize_repair(xt, eb, L.NOA)
        xd = xt.double() if dtype == np.float32 else xt
        assert lfp_local_equality(xd, b, s) == 0, f"repetition {rep}"
        st = bytes(L.compress(xt, eb, L.NOA).cpu().numpy().tobytes())
        if first is None:
            first = st
        assert st == first, f"repetition {rep}"


def test_batch_of_loose_fields_equals_single_calls(L, auto_order):
    xs = [smooth(sh, dt, sd) for sh, dt, _, sd in FIELDS] + [bumps((40, 50, 60), np.float32, seed=9)]
    ebs = [eb for _, _, eb, _ in FIELDS] + [1e-2]
    fields = [torch.from_numpy(x).cuda() for x in xs]
    singles = [bytes(L.compress(t, eb, L.NOA).cpu().numpy().tobytes()) for t, eb in zip(fields, ebs)]
    b = L.BatchCompress(fields, ebs)
    for rep in range(3):
        L.tune_set_pass_order([(L.PASS_ORDER_AUTO, L.PASS_ORDER_KEY, L.PASS_ORDER_INDEX)[rep]] * 4)
        b.launch()
        streams, status = b.results()
        assert status == [0] * len(fields)
        assert [bytes(s.cpu().numpy().tobytes()) for s in streams] == singles
