"""Thermodynamics from a DOS (paper_1407_5140_gb300/thermo.py) against
independent routes: Kaufman's exact ln Z(K) differentiated in multiprecision,
the Potts q = 2 / Ising mapping, and synthetic data with known answers."""
import math
import os

import numpy as np
import pytest

from oracle import exact_dos as ed
from paper_1407_5140_gb300 import thermo as TH

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(L):
    rows = np.loadtxt(os.path.join(GOLDEN, f"ising_L{L}_exact_lng.txt"), usecols=(0, 1))
    return rows[:, 1], rows[:, 0]


def _kaufman_cu(L, T):
    """Exact U and C of the L x L Ising model at temperature T from
    d/dK and d^2/dK^2 of ln Z(K) = ln P(K) + 2NK (K = 1/T), multiprecision."""
    import mpmath
    N = L * L
    with mpmath.workdps(60 + N):
        def lnz(K):
            return mpmath.log(ed.kaufman_polynomial_value(L, K, mpmath.mp).real) + 2 * N * K
        K = mpmath.mpf(1) / T
        d1 = mpmath.diff(lnz, K, 1)
        d2 = mpmath.diff(lnz, K, 2)
        return float(-d1), float(K * K * d2)


@pytest.mark.parametrize("L", [16, 32])
def test_canonical_matches_kaufman_derivatives(L):
    lg, E = _golden(L)
    Ts = [1.5, 2.0, 2.269, 2.4, 3.5]
    u, c = TH.canonical(lg, E, Ts)
    for T, uu, cc in zip(Ts, u, c):
        ue, ce = _kaufman_cu(L, T)
        assert abs(uu - ue) <= 1e-9 * L * L, (T, uu, ue)
        assert abs(cc - ce) <= 1e-8 * ce, (T, cc, ce)


def test_limits_and_log_z():
    lg, E = _golden(16)
    N = 256
    u, c = TH.canonical(lg, E, [1e6, 0.05])
    assert abs(u[0]) < 1e-2 and abs(u[1] + 2 * N) < 1e-6
    # ln Z at infinite temperature is ln sum g = N ln 2
    assert abs(TH.log_z(lg, E, 1e12)[0] - N * math.log(2)) < 1e-6


def test_cv_peak_against_kaufman_and_known_shift():
    """The L = 16 peak from the exact DOS sits where the exact C(T) is flat, and
    above the infinite-lattice T_c = 2 / ln(1 + sqrt 2) by the known O(1/L)
    finite-size shift."""
    lg, E = _golden(16)
    t, cmax = TH.cv_peak(lg, E, 2.0, 2.6)
    ce = [_kaufman_cu(16, t + dt)[1] for dt in (-1e-4, 0.0, 1e-4)]
    assert ce[1] >= ce[0] and ce[1] >= ce[2]
    assert abs(cmax - ce[1]) <= 1e-8 * ce[1]
    tc = 2.0 / math.log(1.0 + math.sqrt(2.0))
    assert 0.0 < t - tc < 0.1


def test_potts_q2_peak_is_half_the_ising_peak():
    """E_Ising = 2 E_Potts + 2N for q = 2, so the Potts specific heat is the Ising
    one at T_Ising = 2 T_Potts, with the same height (exact DOS, L = 6)."""
    L, N = 6, 36
    gi = ed.ising_transfer(L)
    gp = ed.potts_transfer(2, L)
    ti, ci = TH.cv_peak(np.log(list(gi.values())), np.array(list(gi.keys()), float), 1.5, 3.5)
    tp, cp = TH.cv_peak(np.log(list(gp.values())), np.array(list(gp.keys()), float), 0.75, 1.75)
    assert abs(2 * tp - ti) < 1e-8 and abs(cp - ci) < 1e-8 * ci


def test_bootstrap_standard_error_of_the_mean():
    x = np.random.default_rng(5).normal(0.0, 1.0, 64)
    m, se = TH.bootstrap(x, n_resamples=2000, seed=1)
    assert m == pytest.approx(x.mean())
    assert se == pytest.approx(x.std(ddof=1) / 8.0, rel=0.12)


def test_extrapolation_recovers_a_known_limit():
    L = np.array([16, 24, 32, 48, 64])
    tc, se, a = TH.extrapolate_tc(L, 0.7012316 + 0.83 / L ** 2)
    assert abs(tc - 0.7012316) < 1e-12 and abs(a - 0.83) < 1e-9
    tc, se, a = TH.extrapolate_tc(L, 0.7012316 + 0.83 / L ** 2 + np.array([1, -1, 1, -1, 1]) * 1e-4,
                                  err=np.full(5, 1e-4))
    assert abs(tc - 0.7012316) < 3 * se and 0.0 < se < 1e-3


def test_bootstrap_dos_matches_the_spread_of_independent_experiments():
    """Sec. II B error analysis on synthetic pieces with a known spread: the
    exact Ising L = 8 DOS cut into 4 windows at 75 % overlap, every run's piece
    shifted by its own arbitrary constant (as WL leaves it) plus independent
    noise of sigma per bin.  The bootstrap standard error of the joined ln g
    from one experiment of n runs must match the spread of the joined mean DOS
    over many independent experiments, and the mean DOS must sit on the exact
    one within that spread.  Runs through the library's host-only joining."""
    from paper_1407_5140_gb300 import thermo as TH
    from paper_1407_5140_gb300 import windows as WN
    rows = np.loadtxt(os.path.join(GOLDEN, "ising_L8_exact_lng.txt"), usecols=(0, 1))
    N, B = 64, 65
    exact = np.full(B, np.nan)
    exact[((rows[:, 0] + 2 * N) // 4).astype(int)] = rows[:, 1]
    reach = np.isfinite(exact).astype(np.uint8)
    lo, hi = WN.equal_windows(B, 4, 0.75)
    w = int(hi[0] - lo[0] + 1)
    base = np.nan_to_num(exact)
    rng = np.random.default_rng(3)
    n, sigma = 16, 0.02

    def experiment():
        P = np.empty((n, 4, w))
        for r in range(n):
            for i in range(4):
                P[r, i] = base[lo[i]:lo[i] + w] + rng.uniform(-50, 50) + rng.normal(0, sigma, w)
        return P

    mean, std, obs = TH.bootstrap_dos(experiment(), lo, w, reach, 4.0, math.log(2), n_resamples=200, seed=1,
                                      observables={"lnZ(T=3)": lambda lg: TH.log_z(lg, -2 * N + 4 * np.arange(B), 3.0)[0]})
    from paper_1407_5140_gb300 import rewl as R
    means = np.array([R.join_pieces(experiment().mean(axis=0), lo, w, reach, 4.0, math.log(2)) for _ in range(300)])
    emp = np.std(means, axis=0, ddof=1)
    ok = reach.astype(bool)
    ok[0] = False                                   # fixed by the normalisation
    ratio = std[ok] / emp[ok]
    assert 0.7 < np.median(ratio) < 1.4, np.median(ratio)
    assert np.all((ratio > 0.3) & (ratio < 3.0)), ratio
    # the mean DOS is unbiased: within a few standard errors of the exact one
    z = (mean[ok] - exact[ok]) / emp[ok]
    assert np.max(np.abs(z)) < 5.0 and abs(np.mean(z)) < 1.0, (np.max(np.abs(z)), np.mean(z))
    # an observable's error follows too
    val, err = obs["lnZ(T=3)"]
    assert err > 0 and np.isfinite(val)


@pytest.mark.parametrize("dE", [2800.0, 28000.0, 112000.0])
def test_cv_peak_resolves_narrow_first_order_peaks(dE):
    """At a first-order transition the C_v peak of an L x L lattice is about
    T^2 / (N de) wide (2e-5 at L = 200, 4e-6 at L = 400), far below the
    coarse grid's spacing: a two-level system with the levels' weights equal
    at T0 (its C(T) = dE^2 p (1 - p) / T^2 peaks within a few 1e-6 of T0)
    must be located to 1e-8, against a dense scan of the closed form."""
    T0 = 0.70123 + 1e-5 * (dE / 28000)
    E = np.array([-dE, 0.0])
    lg = np.array([0.0, dE / T0])
    t, _ = TH.cv_peak(lg, E, 0.66, 0.76)
    w = T0 * T0 / dE
    Ts = np.linspace(T0 - 40 * w, T0 + 40 * w, 400001)
    p = 1.0 / (1.0 + np.exp(-(lg[1] - lg[0] - (E[1] - E[0]) / Ts)))
    C = dE * dE * p * (1 - p) / Ts ** 2
    assert abs(t - Ts[np.argmax(C)]) < 1e-8
