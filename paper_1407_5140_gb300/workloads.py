"""Seeded workload descriptions shared by the tests, the benchmark and the oracle
side of the parity checks.  Holds sizes, seeds and instance lists only -- none of
the method's arithmetic.

Each workload is a list of instance dicts with the fields of ``rewl_instance``
(model 0 = Ising, 1 = Potts).
"""
import numpy as np

ISING, POTTS = 0, 1


def _inst(model, L, q, h, m, seed, instance_id=0, overlap=0.75, flatness=0.8, ln_f_final=2.0 ** -20,
          flat_rule=0):
    N = L * L
    return dict(model=model, L=L, q=q, e_min=-2 * N, e_max=(2 * N if model == ISING else 0), n_windows=h,
                overlap=overlap, walkers_per_window=m, flatness=flatness, ln_f_final=ln_f_final, seed=seed,
                instance_id=instance_id, flat_rule=flat_rule)


def config0():
    """2D Ising L=8, E in [-128, 128], 4 windows at 75 % overlap, 1 walker per
    window, exchange every 1000 sweeps, Philox seed 0."""
    return [_inst(ISING, 8, 2, 4, 1, 0)]


def config1(sizes=(32, 64), seeds=32):
    """Batched 2D Ising: L = 32 and 64, 16 windows at 75 %, 4 walkers per window,
    32 independent seeds (0..31) per size, exchange every 10^4 sweeps."""
    return [_inst(ISING, L, 2, 16, 4, s) for L in sizes for s in range(seeds)]


def config2(seeds=1):
    """2D q=10 Potts, L = 32, E in [-2048, 0], 32 windows at 75 %, 8 walkers per
    window."""
    return [_inst(POTTS, 32, 10, 32, 8, s) for s in range(seeds)]


def config3(seed=3):
    """Uneven batch: 64 Ising instances with L drawn from {16, 24, 32, 48, 64}
    and 32 q=10 Potts instances with L from {16, 24, 32}; windows scale with the
    energy range (h = clamp(round(N/128), 4, 32)) at 75 %; m = 8 (L <= 24), 4
    (L = 32), 2 (L >= 48)."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(64):
        L = int(rng.choice([16, 24, 32, 48, 64]))
        out.append(_inst(ISING, L, 2, _h(L), _m(L), 1000 + k))
    for k in range(32):
        L = int(rng.choice([16, 24, 32]))
        out.append(_inst(POTTS, L, 10, _h(L), _m(L), 2000 + k))
    return out


def config4_training(seeds=2):
    """Plain-REWL runs the warm-start network learns from: Ising and q=10 Potts
    at L = 8, 16, 24, 32, 48 (windows and walkers as in the uneven batch), run
    to ln f = 2^-14."""
    out = []
    for L in (8, 16, 24, 32, 48):
        for s in range(seeds):
            out.append(_inst(ISING, L, 2, _h(L), _m(L), 4000 + 10 * L + s, ln_f_final=2.0 ** -14))
            out.append(_inst(POTTS, L, 10, _h(L), _m(L), 5000 + 10 * L + s, ln_f_final=2.0 ** -14))
    return out


def config4_targets():
    """Warm-start targets: 2D Ising L = 128 and q=10 Potts L = 64, each 64
    windows x 4 walkers at 75 % overlap, ln f_final = 2^-20."""
    return [_inst(ISING, 128, 2, 64, 4, 6128), _inst(POTTS, 64, 10, 64, 4, 7064)]


def potts_fss(sizes=(16, 24, 32, 48, 64), seeds=4, q=10, width=490, walkers=4, seed0=8000, e_range=None):
    """q-state Potts instances for locating the transition from specific-heat
    maxima (Sec. IV A): windows of about `width` bins at 75 % overlap,
    `walkers` walkers each, `seeds` independent runs per size.  e_range =
    (a, b) restricts the energies to [a N, b N] (default: all, [-2N, 0])."""
    out = []
    for L in sizes:
        N = L * L
        e_min, e_max = (-2 * N, 0) if e_range is None else (int(round(e_range[0] * N)), int(round(e_range[1] * N)))
        B = e_max - e_min + 1
        h = max(4, int(round((B / width - 1.0) / 0.25 + 1.0)))
        for s in range(seeds):
            d = _inst(POTTS, L, q, h, walkers, seed0 + 100 * L + s)
            d.update(e_min=e_min, e_max=e_max)
            out.append(d)
    return out


def exchange_study(seeds=8, L=48, q=10, h=15):
    """q-state Potts L x L with h windows at 75 % overlap and one walker per
    window, run through the first WL iteration (ln f_final = 1) and through
    the first eight (ln f_final = 2^-7): the exchange-frequency experiment of
    Sec. IV B."""
    out = []
    for s in range(seeds):
        out.append(_inst(POTTS, L, q, h, 1, 9000 + s, ln_f_final=1.0))
        out.append(_inst(POTTS, L, q, h, 1, 9100 + s, ln_f_final=2.0 ** -7))
    return out


def _h(L):
    return int(min(32, max(4, round(L * L / 128))))


def _m(L):
    return 8 if L <= 24 else (4 if L == 32 else 2)


def attempts_per_sweep(instances):
    """Single-spin trials in one sweep of every walker of the batch."""
    return sum(d["n_windows"] * d["walkers_per_window"] * d["L"] * d["L"] for d in instances)
