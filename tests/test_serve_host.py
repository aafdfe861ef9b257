"""Host logic of the serving workload and loop (no GPU): the Poisson request
generator and the HBM budget."""
import math

import numpy as np
import pytest

from paper_2603_26968_b300 import synth_gpu as SG


def test_requests_are_seeded_and_deterministic():
    a = SG.serve_requests(1, 200.0, 5.0)
    b = SG.serve_requests(1, 200.0, 5.0)
    c = SG.serve_requests(2, 200.0, 5.0)
    assert [(s.arrival, s.shape, s.dtype, s.eb) for s in a] == [(s.arrival, s.shape, s.dtype, s.eb) for s in b]
    assert [s.arrival for s in a] != [s.arrival for s in c]


def test_requests_follow_the_workload_distribution():
    rate, dur = 200.0, 60.0
    specs = SG.serve_requests(1, rate, dur)
    n = len(specs)
    # Poisson count: mean = var = rate * dur; 5 sigma
    assert abs(n - rate * dur) < 5 * math.sqrt(rate * dur)
    gaps = np.diff([0.0] + [s.arrival for s in specs])
    assert abs(gaps.mean() - 1 / rate) < 5 * (1 / rate) / math.sqrt(n)
    assert all(0 <= s.arrival < dur for s in specs)
    assert all(np.diff([s.arrival for s in specs]) > 0)
    # bytes log-uniform on [1 MB, 1 GB] (shape rounding moves a size by a few percent)
    lb = np.log10([s.nbytes for s in specs])
    assert lb.min() > 6 - 0.05 and lb.max() < 9 + 0.05
    assert abs(lb.mean() - 7.5) < 0.05
    ebs = np.log10([s.eb for s in specs])
    assert ebs.min() >= -4 and ebs.max() <= -2 and abs(ebs.mean() + 3) < 0.05
    f64 = np.mean([s.dtype == "f64" for s in specs])
    d3 = np.mean([len(s.shape) == 3 for s in specs])
    assert abs(f64 - 0.5) < 0.03 and abs(d3 - 0.5) < 0.03


@pytest.mark.parametrize("nb", [1e6, 3.3e7, 1e9])
@pytest.mark.parametrize("word", [4, 8])
@pytest.mark.parametrize("nd", [2, 3])
def test_shape_for_bytes_is_close(nb, word, nd):
    sh = SG.shape_for_bytes(nb, word, nd)
    assert len(sh) == nd
    got = np.prod(sh) * word
    assert abs(got / nb - 1) < 0.05


def test_budget_accounting():
    from paper_2603_26968_b300.serve import Budget
    b = Budget(100)
    assert b.fits(100) and not b.fits(101)
    b.take(60)
    assert not b.fits(41) and b.fits(40)
    with pytest.raises(ValueError):
        b.take(41)
    b.take(40)
    b.give(60)
    assert b.used == 40 and b.peak == 100
    with pytest.raises(ValueError):
        b.give(50)
