"""Equal-width and run-time-balanced windows (paper_1407_5140_gb300/windows.py)."""
import numpy as np
import pytest

import oracle as O
from paper_1407_5140_gb300 import windows as WN


@pytest.mark.parametrize("B,h,o", [(65, 4, 0.75), (4609, 15, 0.75), (2049, 32, 0.75), (257, 5, 0.5), (8193, 64, 0.75)])
def test_equal_windows_match_the_library_rule(B, h, o):
    w, lo = O.windows(B, h, o)
    elo, ehi = WN.equal_windows(B, h, o)
    assert list(elo) == list(lo) and np.all(ehi - elo + 1 == w)


def test_uniform_costs_keep_the_windows_balanced_and_valid():
    B, h, o = 4609, 15, 0.75
    lo, hi = WN.equal_windows(B, h, o)
    nlo, nhi = WN.balanced_windows(lo, hi, np.full(h, 1e5), B, o, 9)
    assert WN.valid_windows(nlo, nhi, B, 9)
    widths = nhi - nlo + 1
    assert widths[:-1].max() - widths[:-1].min() <= 2


def test_slow_windows_get_narrower():
    B, h, o = 4609, 15, 0.75
    lo, hi = WN.equal_windows(B, h, o)
    t = np.linspace(1.0, 9.0, h) * 1e4          # higher windows four times slower at the top
    nlo, nhi = WN.balanced_windows(lo, hi, t, B, o, 9)
    assert WN.valid_windows(nlo, nhi, B, 9)
    w = (nhi - nlo + 1).astype(float)
    assert w[0] > 2.0 * w[-2]                     # ~ sqrt(9 / 1) = 3 times wider
    # predicted sweeps t_i (w_i' / w_i)^2 are far more even than before
    pred = t * (w / (hi - lo + 1)) ** 2
    assert pred[:-1].max() / pred[:-1].min() < 0.25 * t.max() / t.min()


def test_width_cap():
    """A cap keeps the widest window (and so every walker's shared-memory row)
    bounded; the set still covers the range and stays valid."""
    B, h, o = 16385, 64, 0.75                     # Ising L = 128, 64 windows
    lo, hi = WN.equal_windows(B, h, o)
    t = 1.0 + 100.0 * np.abs(np.linspace(-1, 1, h)) ** 2  # slow at both ends, fast in the middle
    free_lo, free_hi = WN.balanced_windows(lo, hi, t, B, o, 5)
    cap = 2 * int((hi - lo + 1)[0])
    c_lo, c_hi = WN.balanced_windows(lo, hi, t, B, o, 5, max_width=cap)
    assert (free_hi - free_lo + 1).max() > cap
    assert WN.valid_windows(c_lo, c_hi, B, 5) and (c_hi - c_lo + 1).max() <= cap
    with pytest.raises(ValueError):
        WN.balanced_windows(lo, hi, t, B, o, 5, max_width=20)


def test_invalid_sets_are_detected():
    assert not WN.valid_windows([0, 10, 20], [15, 25, 40], 42, 5)      # does not end at B - 1
    assert not WN.valid_windows([0, 16, 20], [15, 25, 41], 42, 5)      # gap
    assert not WN.valid_windows([0, 10, 38], [15, 25, 41], 42, 5)      # last window too narrow
    assert WN.valid_windows([0, 10, 20], [15, 25, 41], 42, 5)
