"""The launch-plan autotuner's host logic, on the CPU: coordinate descent over the
plan's knobs (with a synthetic timer standing in for CUDA events), the workload
signature, and the JSON cache."""
import json
from types import SimpleNamespace

import pytest


@pytest.fixture(scope="module")
def T():
    from paper_2603_26968_b300 import autotune, build
    build.build()   # the default plan comes from the library (no GPU call)
    return autotune


def test_coordinate_descent_finds_each_knobs_best_value(T):
    default = T.lopc.plan_default().as_dict()
    cls = 1

    def cost(p):  # a separable cost with a known best value per knob for class 1
        return (10.0 + abs(p["rerun_blocks_per_sm"][cls] - 2) + (0.0 if p["pass_order"][cls] == 2 else 0.5)
                + 0.1 * abs(p["pass_dense16"][cls] - 12) + (0.0 if p["pass_budget16"][cls] == 256 else 0.3))

    seen = []
    timed = []

    def run(pl):
        seen.append(pl.as_dict())

    def timer(fn):
        fn()
        c = cost(seen[-1])
        timed.append(seen[-1])
        return [c - 0.01, c, c + 0.01]

    out = T.tune(run, [cls], reps=3, timer=timer)
    best = out["plan"]
    assert best["rerun_blocks_per_sm"][cls] == 2 and best["pass_order"][cls] == 2
    assert best["pass_dense16"][cls] == 12 and best["pass_budget16"][cls] == 256
    for k in T.KNOBS:  # other classes keep the default
        assert [v for c, v in enumerate(best[k]) if c != cls] == [v for c, v in enumerate(default[k]) if c != cls]
    assert out["ms"] == pytest.approx(10.0)
    assert out["default_ms"] == pytest.approx(cost(default))
    assert out["default_spread_ms"] == pytest.approx(0.02)
    # one trial of the default, one per other value of every knob, the default again
    assert len(out["trials"]) == 1 + sum(len(v) - 1 for v in T.KNOBS.values())
    assert len(timed) == len(out["trials"]) + 1
    # every trial ran once untimed (capture) before it was timed
    assert len(seen) == 2 * len(timed)


def test_ties_keep_the_earlier_plan(T):
    default = T.lopc.plan_default().as_dict()
    out = T.tune(lambda pl: None, [0, 3], timer=lambda fn: [5.0, 5.0, 5.0])
    assert out["plan"] == default and out["ms"] == 5.0 and out["default_spread_ms"] == 0.0


def test_signature_and_classes(T):
    L = T.lopc
    d = [SimpleNamespace(dtype=L.F32, ndim=2, dims=[256, 256, 0]),
         SimpleNamespace(dtype=L.F64, ndim=3, dims=[64, 64, 64]),
         SimpleNamespace(dtype=L.F64, ndim=3, dims=[32, 64, 64])]
    assert T.classes_of(d) == [0, 3]
    assert T.signature(d) == "1:16,0:0,0:0,2:18"


def test_cache_round_trip(T, tmp_path):
    p = tmp_path / "tuned.json"
    assert T.load("k", p) is None
    v = {"plan": {"pass_order": [0, 1, 2, 0]}, "ms": 1.5}
    T.save("k", v, p)
    T.save("other", {"plan": {}, "ms": 2.0}, p)
    assert T.load("k", p) == v and T.load("other", p)["ms"] == 2.0
    assert set(json.loads(p.read_text())) == {"k", "other"}
    p.write_text("{broken")
    assert T.load("k", p) is None
    T.save("k", v, p)  # a broken cache is replaced
    assert T.load("k", p) == v
