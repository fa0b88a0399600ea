"""Canonical thermodynamics from a density of states, peak finding, bootstrap
errors over independent runs (of a scalar, and of the joined DOS by
resampling the pieces of every window, Sec. II B) and the finite-size
extrapolation of a
transition temperature (Sec. III and Sec. IV A: the q = 10 Potts transition
located from the specific-heat maxima of L x L lattices).

Host-side analysis of the ln g that ``Rewl.get_dos`` returns (k_B = J = 1):

    Z(T)   = sum_E g(E) exp(-E / T)
    U(T)   = <E>,   C(T) = (<E^2> - <E>^2) / T^2

evaluated with a shift by the largest exponent, so ln g up to ~10^5 is safe in
double precision.
"""
import math

import numpy as np


def _finite(ln_g, E):
    ln_g = np.asarray(ln_g, np.float64)
    E = np.asarray(E, np.float64)
    ok = np.isfinite(ln_g)
    return ln_g[ok], E[ok]


def log_z(ln_g, E, T):
    """ln Z at each temperature of T (array or scalar)."""
    lg, e = _finite(ln_g, E)
    T = np.atleast_1d(np.asarray(T, np.float64))
    a = lg[None, :] - e[None, :] / T[:, None]
    m = a.max(axis=1, keepdims=True)
    return (m[:, 0] + np.log(np.exp(a - m).sum(axis=1)))


def canonical(ln_g, E, T):
    """(U, C) at each temperature of T: internal energy and specific heat of the
    whole lattice (divide by N for per-site values)."""
    lg, e = _finite(ln_g, E)
    T = np.atleast_1d(np.asarray(T, np.float64))
    a = lg[None, :] - e[None, :] / T[:, None]
    a -= a.max(axis=1, keepdims=True)
    w = np.exp(a)
    z = w.sum(axis=1)
    # moments about a reference energy keep the variance free of cancellation
    u = (w * e[None, :]).sum(axis=1) / z
    d = e[None, :] - u[:, None]
    var = (w * d * d).sum(axis=1) / z - ((w * d).sum(axis=1) / z) ** 2
    return u, var / (T * T)


def cv_peak(ln_g, E, T_lo, T_hi, n_grid=400, tol=1e-10):
    """Temperature and height of the specific-heat maximum in [T_lo, T_hi]:
    a grid scan, then golden-section refinement around the best grid point."""
    Ts = np.linspace(T_lo, T_hi, n_grid)
    _, c = canonical(ln_g, E, Ts)
    i = int(np.argmax(c))
    a, b = Ts[max(i - 1, 0)], Ts[min(i + 1, n_grid - 1)]
    g = (math.sqrt(5.0) - 1.0) / 2.0

    def f(t):
        return -canonical(ln_g, E, t)[1][0]

    x1, x2 = b - g * (b - a), a + g * (b - a)
    f1, f2 = f(x1), f(x2)
    while b - a > tol:
        if f1 < f2:
            b, x2, f2 = x2, x1, f1
            x1 = b - g * (b - a)
            f1 = f(x1)
        else:
            a, x1, f1 = x1, x2, f2
            x2 = a + g * (b - a)
            f2 = f(x2)
    t = 0.5 * (a + b)
    return t, -f(t)


def bootstrap(samples, stat=np.mean, n_resamples=200, seed=0):
    """(statistic of the samples, bootstrap standard error): resample the
    independent runs with replacement n_resamples times."""
    x = np.asarray(samples)
    rng = np.random.default_rng(seed)
    n = x.shape[0]
    reps = np.array([stat(x[rng.integers(0, n, n)]) for _ in range(n_resamples)])
    return stat(x), float(np.std(reps, ddof=1))


def bootstrap_dos(pieces, lo, ww, reach, bin_width, ln_g_first, n_resamples=200, seed=0, observables=None):
    """Error analysis of Sec. II B (last paragraph) over n independent runs of
    one instance.  pieces: (n, h, w) per-window ln g of every run.  The mean of
    the n pieces of each window, joined, is the mean global DOS; each bootstrap
    resample draws n pieces with replacement for every window separately,
    averages them and joins the result, so the join points differ between
    resamples.  Returns (mean_ln_g, std_ln_g over the resamples, and for each
    observables[name](ln_g) the value on the mean DOS with its standard error).
    The joining is the library's (rewl_join_pieces)."""
    from . import rewl as R
    P = np.asarray(pieces, np.float64)
    n, h, w = P.shape
    mean = R.join_pieces(P.mean(axis=0), lo, ww, reach, bin_width, ln_g_first)
    rng = np.random.default_rng(seed)
    reps = np.empty((n_resamples, mean.size))
    obs = {k: [] for k in (observables or {})}
    for r in range(n_resamples):
        pick = rng.integers(0, n, size=(h, n))                  # n runs per window, with repetition
        res = P[pick, np.arange(h)[:, None], :].mean(axis=1)    # (h, w)
        reps[r] = R.join_pieces(res, lo, ww, reach, bin_width, ln_g_first)
        for k, f in (observables or {}).items():
            obs[k].append(f(reps[r]))
    std = np.std(reps, axis=0, ddof=1)
    out_obs = {k: (f(mean), np.std(np.asarray(obs[k]), axis=0, ddof=1)) for k, f in (observables or {}).items()}
    return mean, std, out_obs


def extrapolate_tc(L, Tc, err=None, power=2):
    """Weighted least-squares fit Tc(L) = Tc(inf) + a / L^power; returns
    (Tc(inf), its standard error, a).  power = d = 2 for a first-order
    transition in two dimensions."""
    L = np.asarray(L, np.float64)
    y = np.asarray(Tc, np.float64)
    w = np.ones_like(y) if err is None else 1.0 / np.maximum(np.asarray(err, np.float64), 1e-300) ** 2
    X = np.stack([np.ones_like(L), L ** -power], axis=1)
    A = X.T @ (w[:, None] * X)
    coef = np.linalg.solve(A, X.T @ (w * y))
    cov = np.linalg.inv(A)
    if err is None:
        r = y - X @ coef
        dof = max(1, len(y) - 2)
        cov = cov * float(r @ r) / dof
    return float(coef[0]), float(math.sqrt(max(cov[0, 0], 0.0))), float(coef[1])
