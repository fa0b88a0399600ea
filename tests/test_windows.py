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


def test_stage_durations_from_stage_sweeps():
    ss = np.full((3, 33), -1, np.int64)
    ss[:, 0] = [100, 300, 200]
    ss[:, 1] = [250, 900, 260]
    assert list(WN.stage_durations(ss, 0)) == [100, 300, 200]
    assert list(WN.stage_durations(ss, 1)) == [150, 600, 60]
    assert WN.stage_durations(ss, 2) is None
    ws = ss.copy()
    ws[:, 0] = -1                                 # a warm start that began at stage 1
    assert list(WN.stage_durations(ws, 1)) == [250, 900, 260]


class _FakeBatch:
    """Stands in for a Rewl batch on windows (lo, hi): a window's stage k takes
    cost * width^2 sweeps, cost rising tenfold from the lowest window to the
    highest; the DOS is ln g = 0.01 b on every bin."""

    made = []

    def __init__(self, lo, hi, n_inst, B):
        self.lo, self.hi, self.n, self.B = np.asarray(lo), np.asarray(hi), n_inst, B
        self.t = 0
        self.k0 = 0
        self.init = {}
        self.closed = False
        _FakeBatch.made.append(self)

    def _dur(self):
        w = (self.hi - self.lo + 1).astype(float)
        cost = np.linspace(1.0, 10.0, len(w)) * 1e-3
        return np.ceil(cost * w * w)

    def stage_sweeps(self, inst):
        d = self._dur()
        ss = np.full((len(d), 33), -1, np.int64)
        end = np.zeros_like(d)
        for k in range(self.k0, 21):
            end = end + d
            ss[:, k] = np.where(end <= self.t, end, -1)
        return ss

    def run_cycles(self, n, x):
        self.t += n * x

    def status(self, inst):
        return {"all_converged": bool(np.all(self.stage_sweeps(inst)[:, 20] >= 0)), "sweeps": self.t}

    def get_dos(self, inst):
        return 0.01 * np.arange(self.B, dtype=float), None

    def set_initial_lng(self, inst, g, ln_f):
        self.init[inst] = (np.asarray(g).copy(), ln_f)
        self.k0 = int(round(-np.log2(ln_f)))

    def run_to_convergence(self, x, max_sweeps, poll_cycles=1):
        self.t += max_sweeps
        return self.status(0)["all_converged"]

    def close(self):
        self.closed = True


def test_self_tuning_run_resizes_uneven_windows_and_continues_from_the_joined_dos():
    B, h, o = 4609, 15, 0.75
    lo, hi = WN.equal_windows(B, h, o)
    _FakeBatch.made = []
    ctx, (flo, fhi), resizes, sweeps = WN.self_tuning_run(
        lambda a, b: _FakeBatch(a, b, 2, B), (lo, hi), B, o, 9, 100, n_inst=2, tune_at=(0, 1, 2))
    assert resizes and resizes[0]["after_stage"] == 0
    assert WN.valid_windows(flo, fhi, B, 9)
    first, last = _FakeBatch.made[0], _FakeBatch.made[-1]
    assert first.closed and not last.closed and last is ctx
    # each instance restarts from its own joined DOS, shifted to start at 0, at ln f = 2^-(k+1)
    k = resizes[-1]["after_stage"]
    for i in range(2):
        g, lnf = last.init[i]
        assert lnf == 2.0 ** -(k + 1) and g[0] == 0.0 and np.allclose(np.diff(g), 0.01)
    # the resized windows are more even in predicted stage time than the equal set
    d0, d1 = first._dur(), last._dur()
    assert d1.max() / d1.mean() < d0.max() / d0.mean()
    assert sweeps >= last.t


def test_self_tuning_run_keeps_even_windows():
    B, h, o = 4609, 15, 0.75
    lo, hi = WN.equal_windows(B, h, o)

    class Even(_FakeBatch):
        def _dur(self):
            return np.full(len(self.lo), 500.0)

    made = []
    ctx, (flo, fhi), resizes, _ = WN.self_tuning_run(
        lambda a, b: made.append(Even(a, b, 1, B)) or made[-1], (lo, hi), B, o, 9, 100, n_inst=1)
    assert resizes == [] and len(made) == 1 and list(flo) == list(lo)


def test_site_division_by_multiply_high_is_exact_up_to_the_largest_lattice():
    """The kernels split a site index into (row, column) with a multiply-high
    by ceil(2^32 / L); that is exact for every site of every even L up to the
    largest accepted lattice side, 512 (the error term site * e / 2^32, with
    e = ceil(2^32 / L) L - 2^32 < L, stays below 1 / L while L^3 < 2^32)."""
    for L in range(4, 513, 2):
        m = np.uint64(-(-(1 << 32) // L))
        site = np.arange(L * L, dtype=np.uint64)
        y = (site * m) >> np.uint64(32)
        assert np.array_equal(y, site // np.uint64(L)), L


def test_self_tuning_run_averages_stages_on_the_current_windows():
    """A resize after stage 4 with tune_avg = 3 uses stages 2..4, all run on
    the starting windows; the continuation starts at ln f = 2^-5."""
    B, h, o = 4609, 15, 0.75
    lo, hi = WN.equal_windows(B, h, o)
    _FakeBatch.made = []
    ctx, _, resizes, _ = WN.self_tuning_run(
        lambda a, b: _FakeBatch(a, b, 1, B), (lo, hi), B, o, 9, 100, n_inst=1, tune_at=(4,), tune_avg=3)
    assert [r["after_stage"] for r in resizes] == [4] and resizes[0]["stages_averaged"] == 3
    assert ctx.init[0][1] == 2.0 ** -5 and ctx.k0 == 5
