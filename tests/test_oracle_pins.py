"""Pins of the CPU oracle against things the paper and the mathematics fix.

Nothing here compares the oracle with itself: every expected value is either
printed in the paper, a textbook closed form, a brute-force enumeration, an
independent library routine, or a statistical property of the exact method.
"""
import json
import math
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle as O
from oracle import concat as cc
from oracle import exact_dos as ed

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------
# windows (Sec. II A, Fig. 1; widths quoted in Sec. IV A)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("L,h", [(100, 77), (200, 317), (300, 717), (400, 1277)])
def test_windows_reproduce_potts_piece_counts(L, h):
    # Sec. IV A / Fig. 5: q=10 Potts, windows of Delta E = 1000 at 75 % overlap
    # give 77 / 317 / 717 / 1277 pieces for L = 100 ... 400 (E in [-2N, 0]).
    B = 2 * L * L + 1
    w, lo = O.windows(B, h, 0.75)
    assert w == 1001                      # 1000 energy units, inclusive
    assert lo[0] == 0 and lo[-1] + w - 1 == B - 1
    assert set(np.diff(lo)) == {250}      # (1 - o) * 1000


@pytest.mark.parametrize("o,frac", [(0.5, 1 / 5), (0.625, 1 / 4), (0.75, 1 / 3), (0.875, 1 / 2)])
def test_window_widths_h9(o, frac):
    # Sec. IV A: for h = 9 the window widths are 1/5, 1/4, 1/3, 1/2 of the range
    B = 360001
    w, lo = O.windows(B, 9, o)
    assert abs(w / B - frac) < 1e-4
    ov = (lo[0] + w - lo[1]) / w           # overlap with the next window
    assert abs(ov - o) < 1e-3


def test_windows_config0():
    w, lo = O.windows(65, 4, 0.75)
    assert w == 38 and list(lo) == [0, 9, 18, 27]
    w1, lo1 = O.windows(65, 1, 0.75)
    assert w1 == 65 and list(lo1) == [0]


# ---------------------------------------------------------------------------
# exact densities of states
# ---------------------------------------------------------------------------
ISING_L4 = {-32: 2, -24: 32, -20: 64, -16: 424, -12: 1728, -8: 6688, -4: 13568, 0: 20524,
            4: 13568, 8: 6688, 12: 1728, 16: 424, 20: 64, 24: 32, 32: 2}


def test_ising_l4_bruteforce_and_kaufman():
    bf = ed.ising_bruteforce(4)
    assert bf == ISING_L4
    assert ed.ising_kaufman(4) == bf
    assert {k: int(v) for k, v in ed.ising_transfer(4).items()} == bf


def test_ising_l6_kaufman_equals_transfer_matrix():
    tm = ed.ising_transfer(6)
    ka = ed.ising_kaufman(6)
    assert {k: int(round(v)) for k, v in tm.items()} == ka


@pytest.mark.parametrize("L", [8, 16])
def test_ising_kaufman_invariants(L):
    g = ed.ising_kaufman(L)
    N = L * L
    assert sum(g.values()) == 2 ** N                          # sum g = 2^N
    assert all(g[E] == g.get(-E) for E in g)                  # g(E) = g(-E), even L
    assert sum(c * E for E, c in g.items()) == 0              # <E> = 0 at beta = 0
    assert sum(c * E * E for E, c in g.items()) == 2 * N * 2 ** N   # Var E = 2N
    assert g[-2 * N] == 2 and -2 * N + 4 not in g             # ground states, gap
    assert g[-2 * N + 8] == 2 * N and g[-2 * N + 12] == 4 * N  # one / two flipped spins


def test_prime_field_kaufman_matches_multiprecision_and_brute_force():
    """The prime-field evaluation (exact integers by NTT + CRT) of the same closed
    form agrees with brute force at L = 4 and with the multiprecision DFT at
    L = 6..16 -- two independent ways of reading the coefficients off."""
    assert ed.ising_kaufman_modular(4) == ed.ising_bruteforce(4)
    for L in (6, 8, 10, 12, 16):
        assert ed.ising_kaufman_modular(L) == ed.ising_kaufman(L), L


@pytest.mark.parametrize("L", [32, 64])
def test_prime_field_kaufman_invariants_large(L):
    g = ed.ising_kaufman_modular(L)
    N = L * L
    assert sum(g.values()) == 2 ** N
    assert all(g[E] == g.get(-E) for E in g)
    assert sum(c * E * E for E, c in g.items()) == 2 * N * 2 ** N
    assert g[-2 * N] == 2 and -2 * N + 4 not in g
    assert g[-2 * N + 8] == 2 * N and g[-2 * N + 12] == 4 * N
    # the fixture written for this size agrees (L = 32 from the multiprecision path)
    rows = np.loadtxt(os.path.join(GOLDEN, f"ising_L{L}_exact_lng.txt"), usecols=(0, 1))
    assert len(rows) == len(g)
    assert max(abs(math.log(g[int(E)]) - lg) / max(1.0, lg) for E, lg in rows) < 1e-12   # 13 digits stored


def test_golden_l8_is_kaufman():
    rows = np.loadtxt(os.path.join(GOLDEN, "ising_L8_exact_lng.txt"), dtype=object)
    g = ed.ising_kaufman(8)
    assert {int(r[0]): int(r[2]) for r in rows} == g


def test_potts_q3_bruteforce_pins():
    q, L = 3, 4
    N = L * L
    bf = ed.potts_bruteforce(q, L)
    assert {k: int(round(v)) for k, v in ed.potts_transfer(q, L).items()} == bf
    assert sum(bf.values()) == q ** N
    E0 = -2 * N
    # low-energy counts: all equal; one odd spin; a domino; a two-colour domino
    assert bf[E0] == q
    assert bf[E0 + 4] == N * q * (q - 1)
    assert bf[E0 + 6] == 2 * N * q * (q - 1)
    assert bf[E0 + 7] == 2 * N * q * (q - 1) * (q - 2)
    for off in (1, 2, 3, 5):
        assert E0 + off not in bf
    # infinite-temperature moments: bonds are independent, P(equal) = 1/q
    tot = q ** N
    mean = sum(c * E for E, c in bf.items()) / tot
    var = sum(c * E * E for E, c in bf.items()) / tot - mean ** 2
    assert abs(mean - (-2 * N / q)) < 1e-9
    assert abs(var - 2 * N * (q - 1) / q ** 2) < 1e-9


def test_potts_q2_is_ising():
    # E_Ising = 2 E_Potts + 2N for q = 2
    N = 16
    p2 = ed.potts_transfer(2, 4)
    assert {2 * E + 2 * N: int(round(c)) for E, c in p2.items()} == ISING_L4


# ---------------------------------------------------------------------------
# Philox4x32-10 against a library implementation (Triton's, run on the CPU
# through its interpreter), on random keys and counters
# ---------------------------------------------------------------------------
_TRITON_SCRIPT = r"""
import json, os, sys
os.environ["TRITON_INTERPRET"] = "1"
import numpy as np, torch, triton, triton.language as tl

@triton.jit
def k(out, c0p, c1p, c2p, c3p, seed, n: tl.constexpr):
    i = tl.arange(0, n)
    a, b, c, d = tl.philox(seed, tl.load(c0p + i), tl.load(c1p + i), tl.load(c2p + i), tl.load(c3p + i))
    tl.store(out + 4 * i + 0, a); tl.store(out + 4 * i + 1, b)
    tl.store(out + 4 * i + 2, c); tl.store(out + 4 * i + 3, d)

req = json.loads(sys.stdin.read())
res = []
for seed, ctrs in req:
    c = torch.tensor(np.array(ctrs, dtype=np.uint32).view(np.int32))
    out = torch.zeros(4 * c.shape[0], dtype=torch.int32)
    k[(1,)](out, c[:, 0].contiguous(), c[:, 1].contiguous(), c[:, 2].contiguous(), c[:, 3].contiguous(), seed, n=c.shape[0])
    res.append((out.numpy().view(np.uint32).reshape(-1, 4)).tolist())
print(json.dumps(res))
"""


def test_philox_matches_triton_library():
    pytest.importorskip("triton")
    rng = np.random.default_rng(1234)
    req = []
    for seed in [0, 1, 0xDEADBEEF12345678, int(rng.integers(0, 2 ** 63))]:
        ctrs = rng.integers(0, 2 ** 32, size=(16, 4), dtype=np.uint64)
        ctrs[0] = 0
        req.append((int(seed), ctrs.astype(np.uint32).tolist()))
    env = dict(os.environ, TRITON_INTERPRET="1")
    p = subprocess.run([sys.executable, "-c", _TRITON_SCRIPT], input=json.dumps(req),
                       capture_output=True, text=True, env=env, timeout=600)
    if p.returncode != 0:
        pytest.skip("triton interpreter unavailable: " + p.stderr[-300:])
    lib_out = json.loads(p.stdout.strip().splitlines()[-1])
    for (seed, ctrs), expect in zip(req, lib_out):
        key = (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
        got = O.philox(key, np.array(ctrs, dtype=np.uint32))
        assert got.tolist() == expect


def test_philox_output_is_uniform():
    ctr = np.zeros((1 << 16, 4), np.uint32)
    ctr[:, 0] = np.arange(1 << 16)
    ctr[:, 2] = 7
    out = O.philox((3, 4), ctr).astype(np.uint64)
    for word in range(4):
        hist = np.bincount((out[:, word] >> 28).astype(np.int64), minlength=16)
        chi2 = ((hist - hist.mean()) ** 2 / hist.mean()).sum()
        assert chi2 < 50                       # 15 dof, p ~ 1e-5
    assert len(np.unique(out[:, 0])) > 65000


# ---------------------------------------------------------------------------
# acceptance threshold lam = -ln u
# ---------------------------------------------------------------------------
def test_lam_threshold_against_libm_all_k():
    k = np.arange(1 << 24, dtype=np.uint32)
    lam = O.lam_fix(k).astype(np.float64)
    exact = -np.log((k.astype(np.float64) + 1.0) / 2.0 ** 24) * 2.0 ** 32
    # a few binary32 ulp of lam, plus the truncation to the 2^-32 grid
    assert np.all(np.abs(lam - exact) <= 4 * 2.0 ** -24 * exact + 1.0)
    assert np.all(lam >= 1)
    assert np.all(np.diff(lam) <= 0)            # monotone in u: a valid CDF
    assert lam[-1] == 1                         # u = 1: accept only downhill or level
    assert abs(lam[0] - 24 * math.log(2) * 2 ** 32) / lam[0] < 1e-7


def test_lam_threshold_gives_metropolis_probabilities():
    # P(lam > c) over all 2^24 k must equal exp(-c) up to the 2^-24 grid
    k = np.arange(1 << 24, dtype=np.uint32)
    lam = np.sort(O.lam_fix(k).astype(np.float64)) / 2.0 ** 32
    for c in [1e-6, 0.01, 0.5, 1.0, 2.5, 7.0, 15.0]:
        p = (lam > c).sum() / 2.0 ** 24
        assert abs(p - math.exp(-c)) < 3 * 2.0 ** -24 + 1e-6 * math.exp(-c)


# ---------------------------------------------------------------------------
# the oracle's REWL
# ---------------------------------------------------------------------------
def _ising(L, h, m, seed=0, **kw):
    N = L * L
    return O.Oracle(O.ISING, L, 2, -2 * N, 2 * N, h, 0.75, m, seed=seed, **kw)


def _exact_ising_lng(L, B):
    return ed.log_dos_on_bins(ed.ising_kaufman(L), -2 * L * L, 4, B)


def test_energy_bookkeeping_and_windows():
    for model, q in [(O.ISING, 2), (O.POTTS, 10)]:
        L = 8
        N = L * L
        emax = 2 * N if model == O.ISING else 0
        o = O.Oracle(model, L, q, -2 * N, emax, 4, 0.75, 2, seed=3)
        o.init()
        for _ in range(3):
            o.run(5)
            o.exchange()
            s = o.state()
            for k in range(o.n_walkers):
                assert s["E"][k] == o.energy_of(k)                     # incremental == full sum
                b = s["bin"][k]
                assert (s["E"][k] + 2 * N) == b * o.step
                win = k // o.m
                assert o.lo[win] <= b <= o.lo[win] + o.w - 1           # inside the window
                assert o.reach[b]
            if model == O.POTTS:
                assert s["spins"].min() >= 0 and s["spins"].max() < q


def test_reachable_mask_matches_bruteforce():
    o = _ising(4, 1, 1)
    assert set(np.nonzero(o.reach)[0]) == {(E + 32) // 4 for E in ISING_L4}
    p = O.Oracle(O.POTTS, 4, 3, -32, 0, 1, 0.75, 1)
    assert set(np.nonzero(p.reach)[0]) == {E + 32 for E in ed.potts_bruteforce(3, 4)}


def test_sampler_with_exact_weights_is_flat():
    # detailed balance of the single-spin update with weights 1/g(E) (Sec. II A):
    # with ln g frozen at the exact values, every energy is visited equally often
    L, S = 4, 128
    o = _ising(L, 1, S, seed=11, threads=0)
    o.init()
    o.set_lng(np.nan_to_num(_exact_ising_lng(L, o.B)), -1)
    o.run(2000)
    H0 = o.state()["H"].astype(float)
    o.run(10000)
    H = o.state()["H"].astype(float) - H0
    r = o.reach.astype(bool)
    R = H[:, r] / H[:, r].mean(axis=1, keepdims=True)
    t = (R.mean(0) - 1) / (R.std(0) / math.sqrt(S))
    assert np.abs(t).max() < 4.0
    # a biased sampler, e.g. plain Metropolis at beta = 0, would not be flat
    assert np.abs(R.mean(0) - 1).max() < 0.02


def test_exchange_acceptance_follows_eq1():
    # two windows, one walker each, frozen hand-made weights; the number of
    # accepted swaps must match sum_t min(1, g_a(X)/g_a(Y) * g_b(Y)/g_b(X))
    L = 4
    o = _ising(L, 2, 1, seed=5)
    o.init()
    rng = np.random.default_rng(0)
    o.set_lng(np.zeros(o.B), -1)
    ga = rng.uniform(0, 2.0, o.w)
    gb = rng.uniform(0, 2.0, o.w)
    o.set_walker_lng(0, ga)
    o.set_walker_lng(1, gb)
    expected, var = 0.0, 0.0
    acc0 = 0
    for _ in range(3000):
        o.run(1)
        s = o.state()
        if o.counters()["t_exch"] % 2 == 0:
            X, Y = s["bin"][0], s["bin"][1]
            lo_a, lo_b, w = o.lo[0], o.lo[1], o.w
            if lo_b <= X < lo_b + w and lo_a <= Y < lo_a + w:
                ratio = (math.exp(ga[X - lo_a]) / math.exp(ga[Y - lo_a])) * \
                        (math.exp(gb[Y - lo_b]) / math.exp(gb[X - lo_b]))
                # weights are 1/g: new/old weight = g_a(X) g_b(Y) / (g_a(Y) g_b(X))
                p = min(1.0, ratio)
                expected += p
                var += p * (1 - p)
        o.exchange()
    acc = int(o.counters()["ex_acc"][0]) - acc0
    assert var > 50
    assert abs(acc - expected) < 4.5 * math.sqrt(var)


def test_wl_l4_single_walker_converges():
    L = 4
    errs = []
    for seed in range(8):
        o = _ising(L, 1, 1, seed=seed)
        o.init()
        assert o.run_to_convergence(1000, 10 ** 7)
        lg, _ = cc.concatenate(o.pieces(), o.lo, o.w, o.reach, 4.0, math.log(2))
        errs.append(cc.mean_relative_error(lg, _exact_ising_lng(L, o.B)))
        st = o.state()
        assert np.all(st["conv"] == 1) and np.all(st["stage"] == 20)
    assert np.mean(errs) < 0.05


def test_wl_config0_converges_and_more_walkers_help():
    # Config-0 shape: L = 8, 4 windows at 75 % overlap, exchange every 1000 sweeps.
    L = 8
    ex = _exact_ising_lng(L, 65)
    e1, e4 = [], []
    for seed in range(4):
        for m, acc in [(1, e1), (4, e4)]:
            o = _ising(L, 4, m, seed=seed, threads=0)
            o.init()
            assert o.run_to_convergence(1000, 10 ** 7)
            lg, joins = cc.concatenate(o.pieces(), o.lo, o.w, o.reach, 4.0, math.log(2))
            acc.append(cc.mean_relative_error(lg, ex))
            c = o.counters()
            assert np.all(c["ex_acc"][:3] > 0)            # every window pair exchanged
    assert np.mean(e1) < 0.03
    # averaging m walkers per window reduces the error (Sec. IV B, ~ 1/sqrt(m))
    assert np.mean(e4) < np.mean(e1)


def test_wl_potts_small_lattices_converge():
    for q in (2, 3):
        L = 4
        N = L * L
        ex_g = ed.potts_bruteforce(q, L) if q == 3 else ed.potts_transfer(q, L)
        o = O.Oracle(O.POTTS, L, q, -2 * N, 0, 2, 0.75, 2, seed=1)
        o.init()
        assert o.run_to_convergence(1000, 10 ** 7)
        lg, _ = cc.concatenate(o.pieces(), o.lo, o.w, o.reach, 1.0, math.log(q))
        ex = ed.log_dos_on_bins({E: int(round(c)) for E, c in ex_g.items()}, -2 * N, 1, o.B)
        assert set(np.nonzero(np.isfinite(ex))[0]) == set(np.nonzero(o.reach)[0])
        assert cc.mean_relative_error(lg, ex) < 0.05


def test_concatenate_reassembles_exact_pieces():
    # pieces cut from an exact curve with arbitrary offsets join back exactly
    L = 8
    ex = _exact_ising_lng(L, 65)
    w, lo = O.windows(65, 4, 0.75)
    reach = np.isfinite(ex).astype(np.uint8)
    pieces = np.array([np.nan_to_num(ex[l:l + w]) + 17.0 * i for i, l in enumerate(lo)])
    lg, joins = cc.concatenate(pieces, lo, w, reach, 4.0, math.log(2))
    assert np.allclose(lg[reach.astype(bool)], ex[reach.astype(bool)], atol=1e-9)
    assert np.all(np.diff(joins) > 0)


UNEVEN_LO, UNEVEN_HI = [0, 14, 30, 44], [24, 38, 52, 64]     # Ising L = 8, B = 65: widths 25, 25, 23, 21


def test_uneven_windows_rejected_when_invalid():
    bad = [([1, 14, 30, 44], [24, 38, 52, 64]),     # does not start at bin 0
           ([0, 14, 30, 44], [24, 38, 52, 63]),     # does not end at bin B - 1
           ([0, 25, 30, 44], [24, 38, 52, 64]),     # gap between windows 0 and 1
           ([0, 14, 14, 44], [24, 38, 52, 64]),     # lower ends not increasing
           ([0, 14, 30, 44], [24, 38, 38, 64])]     # upper ends not increasing
    for lo, hi in bad:
        with pytest.raises(ValueError):
            O.Oracle(0, 8, 2, -128, 128, 4, 0.75, 1, windows=(lo, hi))


def test_concatenate_reassembles_uneven_pieces():
    L, B = 8, 65
    ex = _exact_ising_lng(L, B)
    reach = np.isfinite(ex).astype(np.uint8)
    ww = np.array(UNEVEN_HI) - np.array(UNEVEN_LO) + 1
    pieces = np.zeros((4, ww.max()))
    for i, (l, n) in enumerate(zip(UNEVEN_LO, ww)):
        pieces[i, :n] = np.nan_to_num(ex[l:l + n]) - 5.0 * i
    lg, joins = cc.concatenate(pieces, UNEVEN_LO, ww, reach, 4.0, math.log(2))
    assert np.allclose(lg[reach.astype(bool)], ex[reach.astype(bool)], atol=1e-9)


def test_wl_with_uneven_windows_converges():
    """Windows of different widths (Sec. V: run-time-balanced windows) change
    nothing in the method; the joined DOS converges to the exact one."""
    ex = _exact_ising_lng(8, 65)
    eps = []
    for seed in range(4):
        o = O.Oracle(0, 8, 2, -128, 128, 4, 0.75, 2, seed=seed, windows=(UNEVEN_LO, UNEVEN_HI))
        assert list(o.lo) == UNEVEN_LO and list(o.ww) == [25, 25, 23, 21] and o.w == 25
        o.init()
        assert o.run_to_convergence(1000, 3_000_000)
        lg, _ = cc.concatenate(o.pieces(), o.lo, o.ww, o.reach, 4.0, math.log(2))
        eps.append(cc.mean_relative_error(lg, ex))
    assert np.mean(eps) < 0.02, eps


# ---------------------------------------------------------------------------
# warm-start network reference: chain-rule gradient against finite differences
# ---------------------------------------------------------------------------
def test_zhou_bhatt_decision_is_exact():
    """Eq. (8): flat iff H >= a / sqrt(ln f) = a 2^(k/2) at ln f = 2^-k, i.e.
    H^2 >= a^2 2^k -- checked in exact rational arithmetic around the
    threshold for exactly representable a (ties included where a^2 2^k is a
    perfect square)."""
    from fractions import Fraction
    for a in (1.0, 0.5, 2.5, 10.0, 0.1, 3.0):
        for k in range(0, 33):
            x = Fraction(a) ** 2 * 2 ** k
            h0 = math.isqrt(int(math.ceil(x)))
            for h in range(max(0, h0 - 2), h0 + 3):
                assert O.zb_flat(h, a, k) == (h * h >= x), (a, k, h)


def test_zhou_bhatt_rule_converges_faster_than_80_percent():
    """Sec. IV B: with m walkers per window the Zhou-Bhatt minimum (a = 1)
    ends WL iterations much sooner than the 80 % rule; the joined DOS still
    converges to the exact one (Config-0 shape with m = 4)."""
    ex = ed.log_dos_on_bins(ed.ising_kaufman(8), -128, 4, 65)
    sweeps, eps = {}, {}
    for rule, a in ((0, 0.8), (1, 1.0)):
        sw, er = [], []
        for seed in range(3):
            o = O.Oracle(0, 8, 2, -128, 128, 4, 0.75, 4, flatness=a, seed=seed, flat_rule=rule)
            o.init()
            assert o.run_to_convergence(1000, 3_000_000)
            sw.append(int(np.max(o.counters()["conv_sweep"])))
            lg, _ = cc.concatenate(o.pieces(), o.lo, o.w, o.reach, 4.0, math.log(2))
            er.append(cc.mean_relative_error(lg, ex))
        sweeps[rule], eps[rule] = np.mean(sw), np.mean(er)
    assert sweeps[1] < 0.4 * sweeps[0], sweeps
    assert eps[1] < 0.05 and eps[0] < 0.02, eps


def test_mlp_reference_gradient_matches_finite_differences():
    from oracle import mlp as M
    rng = np.random.default_rng(0)
    p = M.init_params(1)
    x = rng.normal(size=(7, 5))
    t = rng.normal(size=7)
    g = M.gradient(p, x, t)
    idx = rng.choice(M.N_PARAMS, 60, replace=False)
    idx = np.concatenate([idx, [0, 639, 640, 767, M.N_PARAMS - 129, M.N_PARAMS - 1]])
    for i in idx:
        h = 1e-6
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (M.loss(pp, x, t) - M.loss(pm, x, t)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 + 1e-5 * abs(fd), (i, fd, g[i])


@pytest.mark.parametrize("model,L,q,h,m", [(O.ISING, 8, 2, 4, 1), (O.ISING, 6, 2, 2, 3), (O.POTTS, 4, 3, 2, 2)])
def test_lowering_a_window_by_a_constant_leaves_the_run_unchanged(model, L, q, h, m):
    """ln g of a window is defined up to a constant: lowering a running
    window's ln g by 2^s once all of it reached 2^s (here s = 3, so it happens
    many times) must leave every decision of the run unchanged -- the same
    configurations, energies, histograms, stages, exchanges and convergence
    sweeps as with the default s = 20 (never reached at these sizes) -- and
    each window's ln g must differ from the default run's by one multiple of
    2^3 on its realisable bins, so the joined DOS is the same."""
    N = L * L
    runs = []
    for s in (20, 3):
        o = O.Oracle(model, L, q, -2 * N, 2 * N if model == O.ISING else 0, h, 0.75, m, seed=7)
        o.set_shift_exp(s)
        o.init()
        for _ in range(400):
            o.run(1000)
            o.exchange()
            if o.all_converged():
                break
        assert o.all_converged()
        runs.append(o)
    a, b = runs[0].state(), runs[1].state()
    for key in ("spins", "E", "bin", "H", "stage", "conv", "latch", "replica"):
        assert np.array_equal(a[key], b[key]), key
    ca, cb = runs[0].counters(), runs[1].counters()
    for key in ("ex_prop", "ex_acc", "n_acc", "conv_sweep"):
        assert np.array_equal(ca[key], cb[key]), key
    o = runs[0]
    lowered = 0
    for win in range(h):
        rb = o.reach[o.lo[win]:o.lo[win] + o.ww[win]].astype(bool)
        d = a["lng"][win * m:(win + 1) * m, :o.ww[win]][:, rb] - b["lng"][win * m:(win + 1) * m, :o.ww[win]][:, rb]
        assert np.all(d == d.flat[0]) and d.flat[0] % 8 == 0, win
        lowered += d.flat[0] > 0
    assert lowered == h                    # every window was lowered at least once
    bw, lf = (4.0, math.log(2)) if model == O.ISING else (1.0, math.log(q))
    ga, _ = cc.concatenate(runs[0].pieces(), o.lo, o.w, o.reach, bw, lf)
    gb, _ = cc.concatenate(runs[1].pieces(), o.lo, o.w, o.reach, bw, lf)
    assert np.allclose(ga, gb, rtol=0, atol=1e-9, equal_nan=True)


@pytest.mark.parametrize("m,sums", [
    (2, [3, 5, -3, -5, 7, 1, -1, 2 ** 53 + 1]),
    (3, [1, 2, -1, -2, 4, 5, -4, -5]),
    (4, [2, 6, 10, -2, -6, -10, 3, 5]),
])
def test_merge_rounds_the_mean_to_nearest_ties_to_even(m, sums):
    """The merge (Sec. II A) sets every walker of the window to the mean of
    their ln g, on the 2^-32 grid: nearest multiple, exact halves to the even
    one (Python's round of the exact fraction is that rule)."""
    from fractions import Fraction
    o = O.Oracle(O.ISING, 4, 2, -32, 32, 1, 0.75, m, seed=3)
    o.init()
    w = o.w
    rows = np.zeros((m, w), np.int64)
    for b, total in enumerate(sums):
        # split the sum unevenly over the walkers (all on the 2^-32 grid)
        part = [total // m + (j - m // 2) * 7 for j in range(m)]
        part[-1] += total - sum(part)
        rows[:, b] = part
    for j in range(m):
        o.set_walker_lng(j, rows[j].astype(np.float64) * 2.0 ** -32)
    o.average_window(0)
    got = o.state()["lng"]
    for b, total in enumerate(sums):
        want = round(Fraction(total, m))
        for j in range(m):
            assert got[j, b] * 2.0 ** 32 == want, (m, total, got[j, b] * 2.0 ** 32, want)


def test_eighty_percent_rule_is_min_at_least_four_fifths_of_the_mean_inclusive():
    """flat iff min H >= 0.8 <H> over the n reachable bins (Sec. II A), exact
    80 % counting as flat: the oracle's IEEE evaluation agrees with exact
    rational arithmetic on random cases and on constructed boundaries."""
    rng = np.random.default_rng(5)
    cases = []
    for _ in range(20000):
        n = int(rng.integers(1, 5000))
        mean = int(rng.integers(1, 10 ** 7))
        s = mean * n + int(rng.integers(0, n))
        cases.append((int(rng.integers(0, 2 * mean)), s, n))
    for _ in range(5000):                  # exactly 80 %: 5 min n = 4 sum
        n = int(rng.integers(1, 5000))
        k = int(rng.integers(1, 10 ** 8))
        s = 5 * k * n                       # sum with 4 sum / (5 n) = 4 k
        cases += [(4 * k, s, n), (4 * k - 1, s, n)]
    for mn, s, n in cases:
        exact = 5 * mn * n >= 4 * s
        assert O.pct_flat(mn, s, n, 0.8) == exact, (mn, s, n)
