"""GPU path vs CPU oracle, element by element, through the C ABI.

Integer work (lattices, energies, bins, histograms, exchange decisions,
counters) must be bit-exact; ln g is compared exactly too, because every value
it takes is a multiple of 2^-32 held exactly on both sides.
"""
import math
import os

import numpy as np
import pytest

import oracle as O
from oracle import concat as cc
from paper_1407_5140_gb300 import workloads as W

from _pairs import assert_same_state, make_gpu, make_oracle, step_both

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _torch():
    import torch
    return torch


# ---------------------------------------------------------------------------
# primitives
# ---------------------------------------------------------------------------
def test_lam_threshold_bit_exact_all_k():
    torch = _torch()
    from paper_1407_5140_gb300 import rewl as R
    n = 1 << 24
    k = torch.arange(n, dtype=torch.int64, device="cuda").to(torch.int32)
    out = torch.empty(n, dtype=torch.int64, device="cuda")
    R.debug_lam(k.data_ptr(), out.data_ptr(), n)
    expect = O.lam_fix(np.arange(n, dtype=np.uint32))
    got = out.cpu().numpy()
    bad = np.nonzero(got != expect)[0]
    assert bad.size == 0, f"{bad.size} thresholds differ, first k={bad[:5]}"


def test_philox_bit_exact():
    torch = _torch()
    from paper_1407_5140_gb300 import rewl as R
    rng = np.random.default_rng(7)
    ctr = rng.integers(0, 2 ** 32, size=(4096, 4), dtype=np.uint64).astype(np.uint32)
    for key in [(0, 0), (123, 456), (0xFFFFFFFF, 0x9E3779B9)]:
        c = torch.from_numpy(ctr.view(np.int32)).cuda()
        out = torch.empty_like(c)
        R.debug_philox(key[0], key[1], c.data_ptr(), out.data_ptr(), ctr.shape[0])
        assert np.array_equal(out.cpu().numpy().view(np.uint32), O.philox(key, ctr))


# ---------------------------------------------------------------------------
# trajectories
# ---------------------------------------------------------------------------
def _ising(L, h, m, seed=0, **kw):
    d = W._inst(W.ISING, L, 2, h, m, seed)
    d.update(kw)
    return d


def _potts(L, q, h, m, seed=0, **kw):
    d = W._inst(W.POTTS, L, q, h, m, seed)
    d.update(kw)
    return d


CASES = [
    ("ising_L8_h4_m1", _ising(8, 4, 1), 40, 3),
    ("ising_L4_h1_m1", _ising(4, 1, 1, seed=9), 200, 2),
    ("ising_L6_h2_m3", _ising(6, 2, 3, seed=5), 100, 3),
    ("ising_L24_h6_m2", _ising(24, 6, 2, seed=2), 10, 2),
    ("ising_L32_h16_m4", _ising(32, 16, 4, seed=1), 6, 2),
    ("ising_L48_h8_m2", _ising(48, 8, 2, seed=4), 3, 2),
    ("potts_q10_L32_h32_m8", _potts(32, 10, 32, 8, seed=0), 3, 2),
    ("potts_q3_L4_h2_m2", _potts(4, 3, 2, 2, seed=6), 200, 3),
    ("potts_q2_L8_h3_m2", _potts(8, 2, 3, 2, seed=8), 50, 2),
    ("ising_L8_partial_range", _ising(8, 3, 2, seed=3, e_min=-120, e_max=40), 40, 3),
]


@pytest.mark.parametrize("name,d,sweeps,cycles", CASES, ids=[c[0] for c in CASES])
def test_trajectory_matches_oracle(name, d, sweeps, cycles):
    gpu = make_gpu([d])
    orc = make_oracle(d)
    orc.init()
    assert_same_state(gpu, 0, orc, f"{name} after init")
    for c in range(cycles):
        step_both(gpu, [orc], sweeps)
        assert_same_state(gpu, 0, orc, f"{name} cycle {c}")


@pytest.mark.parametrize("producers", [1, 2, 4])
@pytest.mark.parametrize("wpc", [1, 3, 6])
def test_launch_shape_does_not_change_results(producers, wpc):
    d = _ising(16, 6, 2, seed=11)
    gpu = make_gpu([d], producer_warps=producers, windows_per_cta=wpc)
    orc = make_oracle(d)
    orc.init()
    for c in range(3):
        step_both(gpu, [orc], 25)
    assert_same_state(gpu, 0, orc, f"producers={producers} wpc={wpc}")


def test_potts_producers_and_check_every():
    d = _potts(16, 10, 8, 4, seed=12)
    for producers, ce in [(1, 1), (3, 3), (4, 1)]:
        gpu = make_gpu([d], producer_warps=producers, check_every=ce)
        orc = make_oracle(d)
        orc.set_check_every(ce)
        orc.init()
        for c in range(3):
            step_both(gpu, [orc], 20)
        assert_same_state(gpu, 0, orc, f"producers={producers} check_every={ce}")


def test_batch_of_mixed_instances_matches_each_oracle():
    ds = [_ising(8, 4, 1, seed=0), _potts(8, 10, 4, 2, seed=1), _ising(16, 5, 3, seed=2),
          _ising(8, 4, 1, seed=0, instance_id=7), _potts(12, 4, 3, 2, seed=3)]
    gpu = make_gpu(ds)
    orcs = [make_oracle(d) for d in ds]
    for o in orcs:
        o.init()
    for c in range(3):
        step_both(gpu, orcs, 30)
        for k, o in enumerate(orcs):
            assert_same_state(gpu, k, o, f"instance {k} cycle {c}")


def test_full_convergence_config0_bit_exact_and_accurate():
    d = W.config0()[0]
    gpu = make_gpu([d])
    orc = make_oracle(d)
    orc.init()
    for c in range(200):
        step_both(gpu, [orc], 1000)
        if orc.all_converged():
            break
    assert orc.all_converged()
    assert gpu.status(0)["all_converged"]
    assert_same_state(gpu, 0, orc, "config0 converged")
    ex = _golden_lng(8, 65)
    lg, _ = gpu.get_dos(0)
    eps = cc.mean_relative_error(lg, ex)
    olg, _ = cc.concatenate(orc.pieces(), orc.lo, orc.w, orc.reach, 4.0, math.log(2))
    assert np.allclose(lg, olg, equal_nan=True, atol=1e-9)       # host-side join agrees
    assert eps < 0.03, eps


@pytest.mark.parametrize("d", [_ising(8, 4, 4, seed=31, flat_rule=1, flatness=1.0),
                               _potts(6, 3, 3, 2, seed=32, flat_rule=1, flatness=2.0),
                               _ising(16, 5, 3, seed=33, flat_rule=1, flatness=0.5)],
                         ids=["ising_L8_a1", "potts_q3_L6_a2", "ising_L16_a0.5"])
def test_zhou_bhatt_trajectories_match_oracle(d):
    """Eq. (8) flatness (min H >= a / sqrt(ln f)) on both sides: the stage
    sequence, merges and every other state element stay bit-exact."""
    gpu = make_gpu([d])
    orc = make_oracle(d)
    orc.init()
    for c in range(6):
        step_both(gpu, [orc], 150)
        assert_same_state(gpu, 0, orc, f"cycle {c}")
    assert int(np.max(orc.state()["stage"])) > 0        # the rule did end some iterations


def test_zhou_bhatt_full_convergence_bit_exact():
    """Config-0 shape with 4 walkers per window and the Eq. (8) rule (a = 1) run
    to ln f = 2^-20 on both sides; bit-exact end state, DOS near the exact one."""
    d = _ising(8, 4, 4, seed=1, flat_rule=1, flatness=1.0)
    gpu = make_gpu([d])
    orc = make_oracle(d)
    orc.init()
    for c in range(100):
        step_both(gpu, [orc], 1000)
        if orc.all_converged():
            break
    assert orc.all_converged() and gpu.status(0)["all_converged"]
    assert_same_state(gpu, 0, orc, "zhou-bhatt converged")
    lg, _ = gpu.get_dos(0)
    assert cc.mean_relative_error(lg, _golden_lng(8, 65)) < 0.06


EXTREMES = [
    ("ising_L128_h64_m1", _ising(128, 64, 1, seed=41), 2, 2),          # largest lattice, 4 words per row
    ("potts_q10_L128_h16_m1", _potts(128, 10, 16, 1, seed=42), 1, 2),  # 16 KB lattice, w = 6899
    ("potts_q127_L8_h2_m2", _potts(8, 127, 2, 2, seed=43), 40, 2),     # largest q
    ("ising_L8_h1_m32", _ising(8, 1, 32, seed=44), 30, 2),             # a full consumer warp, one window
    ("ising_L16_h40_o0.9", _ising(16, 40, 2, seed=45, overlap=0.9), 20, 2),   # many narrow windows
    ("ising_L8_h4_o0", _ising(8, 4, 2, seed=46, overlap=0.0), 40, 3),  # disjoint windows
    ("ising_L10_h3_m3", _ising(10, 3, 3, seed=47), 40, 2),             # ragged rounds (N = 100)
    ("config4_ising_L128_h64_m4", _ising(128, 64, 4, seed=48), 1, 2),  # warm-start target shapes
    ("config4_potts_q10_L64_h64_m4", _potts(64, 10, 64, 4, seed=49), 2, 2),
]


@pytest.mark.parametrize("name,d,sweeps,cycles", EXTREMES, ids=[c[0] for c in EXTREMES])
def test_extreme_sizes_match_oracle(name, d, sweeps, cycles):
    """Maximum lattice size, q, walkers per window and window count, disjoint
    windows and ragged rounds: bit-exact against the oracle."""
    gpu = make_gpu([d])
    orc = make_oracle(d)
    orc.init()
    assert_same_state(gpu, 0, orc, f"{name} after init")
    for c in range(cycles):
        step_both(gpu, [orc], sweeps)
        assert_same_state(gpu, 0, orc, f"{name} cycle {c}")


GLOBAL_LATTICE = [
    # 40 KB and 160 KB lattices (the paper's Potts L = 200 and 400) stay in
    # global memory; energy sub-ranges keep the oracle's sweeps short
    ("potts_q10_L200_sub", _potts(200, 10, 3, 2, seed=51, e_min=-60000, e_max=-59000), {}, 2, 2),
    ("potts_q10_L400_sub", _potts(400, 10, 2, 1, seed=52, e_min=-200000, e_max=-199200), {}, 1, 2),
    ("ising_L400_sub", _ising(400, 2, 2, seed=53, e_min=-200000, e_max=-198000), {}, 1, 2),
    # global placement forced on lattices that would fit in shared memory
    ("ising_L32_global", _ising(32, 8, 2, seed=54), {"lattice_placement": 1}, 6, 2),
    ("potts_q10_L32_global", _potts(32, 10, 8, 2, seed=55), {"lattice_placement": 1}, 4, 2),
    ("ising_L10_h3_m3_global", _ising(10, 3, 3, seed=47), {"lattice_placement": 1}, 40, 2),
]


@pytest.mark.parametrize("name,d,opts,sweeps,cycles", GLOBAL_LATTICE, ids=[c[0] for c in GLOBAL_LATTICE])
def test_global_memory_lattices_match_oracle(name, d, opts, sweeps, cycles):
    """The sweep kernel with the lattices left in global memory (large L):
    bit-exact against the oracle."""
    gpu = make_gpu([d], **opts)
    orc = make_oracle(d)
    orc.init()
    assert_same_state(gpu, 0, orc, f"{name} after init")
    for c in range(cycles):
        step_both(gpu, [orc], sweeps)
        assert_same_state(gpu, 0, orc, f"{name} cycle {c}")


def test_lattice_placement_does_not_change_results():
    """Potts L = 200 with its lattices in global memory (the default there)
    and forced into shared memory: identical states after sweeps and
    exchanges."""
    d = _potts(200, 10, 4, 2, seed=56, e_min=-52000, e_max=-50500)
    a = make_gpu([d])
    b = make_gpu([d], lattice_placement=2)
    for _ in range(2):
        for g in (a, b):
            g.run(2)
            g.exchange()
    sa, sb = a.state(0, 40000), b.state(0, 40000)
    for k in sa:
        assert np.array_equal(sa[k], sb[k]), k
    with pytest.raises(Exception):
        make_gpu([_potts(514, 10, 4, 1)])


def test_learned_warm_start_install_then_bit_exact():
    """rewl_warm_start writes each walker's ln g from the network (window
    pieces shifted to a zero minimum), resets H and latches and sets the stage;
    the oracle given the same ln g and stage then follows the GPU bit for bit."""
    from paper_1407_5140_gb300 import rewl as R
    d = _ising(16, 4, 2, seed=50)
    gpu = make_gpu([d])
    net = R.Mlp(max_batch=1024, seed=3)
    gpu.warm_start(0, net, 2.0 ** -4)
    g = gpu.state(0, 256)
    assert np.all(g["stage"] == 4) and not np.any(g["conv"]) and not np.any(g["H"]) and not np.any(g["latch"])
    orc = make_oracle(d)
    orc.init()
    orc.set_lng(np.zeros(orc.B), 4)
    for k in range(orc.n_walkers):
        orc.set_walker_lng(k, g["lng"][k])
    assert_same_state(gpu, 0, orc, "after the warm start")
    for c in range(4):
        step_both(gpu, [orc], 100)
        assert_same_state(gpu, 0, orc, f"warm start cycle {c}")
    net.close()


UNEVEN = [
    ("ising_L8_uneven", _ising(8, 4, 2, seed=51), ([0, 14, 30, 44], [24, 38, 52, 64]), 40, 3),
    ("ising_L16_uneven5", _ising(16, 5, 3, seed=52), ([0, 40, 90, 150, 200], [70, 120, 180, 230, 256]), 25, 3),
    ("potts_q3_L6_uneven", _potts(6, 3, 3, 2, seed=53), ([0, 20, 45], [35, 60, 72]), 40, 3),
]


@pytest.mark.parametrize("name,d,win,sweeps,cycles", UNEVEN, ids=[c[0] for c in UNEVEN])
def test_uneven_windows_match_oracle(name, d, win, sweeps, cycles):
    """Windows of different widths (rewl_create_batch_windows, Sec. V): state,
    exchanges and the joined DOS bit-exact / equal to the oracle's."""
    gpu = make_gpu([d], windows=[win])
    orc = make_oracle(d, windows=win)
    orc.init()
    g = gpu.geometry(0)
    assert list(g["lo"]) == list(orc.lo) and list(g["ww"]) == list(orc.ww) and g["w"] == orc.w
    assert_same_state(gpu, 0, orc, f"{name} after init")
    for c in range(cycles):
        step_both(gpu, [orc], sweeps)
        assert_same_state(gpu, 0, orc, f"{name} cycle {c}")
    lg, _ = gpu.get_dos(0)
    olg, _ = cc.concatenate(orc.pieces(), orc.lo, orc.ww, orc.reach, 4.0 if d["model"] == 0 else 1.0,
                            math.log(2 if d["model"] == 0 else d["q"]))
    assert np.allclose(lg, olg, equal_nan=True, atol=1e-9)


def test_uneven_windows_invalid_and_checkpoint(tmp_path):
    from paper_1407_5140_gb300 import rewl as R
    d = _ising(8, 4, 2, seed=54)
    for lo, hi in [([1, 14, 30, 44], [24, 38, 52, 64]), ([0, 25, 30, 44], [24, 38, 52, 64]),
                   ([0, 14, 30, 44], [24, 38, 52, 63]), ([0, 14, 30, 62], [24, 38, 52, 64])]:
        with pytest.raises(R.RewlError) as ei:
            make_gpu([d], windows=[(lo, hi)])
        assert ei.value.code == -1
    win = ([0, 14, 30, 44], [24, 38, 52, 64])
    a = make_gpu([d], windows=[win])
    a.run(50)
    a.exchange()
    path = str(tmp_path / "uneven.ckpt")
    a.save(path)
    b = R.Rewl.load(path)
    assert list(b.geometry(0)["ww"]) == [25, 25, 23, 21]
    a.run(30)
    b.run(30)
    sa, sb = a.state(0, 64), b.state(0, 64)
    for key in ("spins", "lng", "H", "bin", "stage"):
        assert np.array_equal(np.asarray(sa[key]), np.asarray(sb[key])), key


def test_empty_batch_is_rejected():
    from paper_1407_5140_gb300 import rewl as R
    with pytest.raises(R.RewlError) as ei:
        R.Rewl([])
    assert ei.value.code == -1


def test_graph_cycles_equal_stepwise_calls():
    d = _ising(16, 4, 2, seed=21)
    a = make_gpu([d])
    b = make_gpu([d])
    a.run_cycles(5, 30)
    for _ in range(5):
        b.run(30)
        b.exchange()
    sa, sb = a.state(0, 256), b.state(0, 256)
    for k in sa:
        assert np.array_equal(sa[k], sb[k]), k


def test_checkpoint_resume_is_bit_exact(tmp_path):
    from paper_1407_5140_gb300 import rewl as R
    d = _potts(8, 10, 4, 2, seed=5)
    a = make_gpu([d])
    a.run_cycles(3, 40)
    p = str(tmp_path / "ck.bin")
    a.save(p)
    b = R.Rewl.load(p)
    a.run_cycles(4, 40)
    b.run_cycles(4, 40)
    sa, sb = a.state(0, 64), b.state(0, 64)
    for k in sa:
        assert np.array_equal(sa[k], sb[k]), k


def test_warm_start_and_frozen_sampling_match_oracle():
    d = _ising(8, 4, 2, seed=13)
    ex = _golden_lng(8, 65)
    for lnf in (2.0 ** -4, 0.0):
        gpu = make_gpu([d])
        gpu.set_initial_lng(0, np.nan_to_num(ex), lnf)
        orc = make_oracle(d)
        orc.init()
        orc.set_lng(np.nan_to_num(ex), 4 if lnf else -1)
        for c in range(3):
            step_both(gpu, [orc], 50)
        assert_same_state(gpu, 0, orc, f"warm start ln f = {lnf}")


def test_config1_launch_sampled_instances_match_oracle():
    # the benchmark's workload and launch shape; three instances per size are
    # re-run on the oracle and compared element by element
    ds = W.config1()
    gpu = make_gpu(ds)
    gpu.run(4)
    gpu.exchange()
    gpu.run(2)
    for k in (0, 17, 31, 32, 50, 63):
        o = make_oracle(ds[k])
        o.init()
        o.run(4)
        o.exchange()
        o.run(2)
        assert_same_state(gpu, k, o, f"config1 instance {k}")


def test_invalid_arguments_fail_cleanly():
    from paper_1407_5140_gb300 import rewl as R
    for bad in [dict(L=7), dict(L=3), dict(n_windows=0), dict(overlap=1.0), dict(e_min=-130),
                dict(e_min=-126), dict(ln_f_final=0.0), dict(flatness=1.5), dict(flat_rule=2),
                dict(flat_rule=1, flatness=0.0), dict(flat_rule=1, flatness=2e6)]:
        d = _ising(8, 4, 1)
        d.update(bad)
        with pytest.raises(R.RewlError) as ei:
            make_gpu([d])
        assert ei.value.code == -1


def _golden_lng(L, B):
    rows = np.loadtxt(os.path.join(GOLDEN, f"ising_L{L}_exact_lng.txt"), usecols=(0, 1))
    out = np.full(B, np.nan)
    N = L * L
    for E, lg in rows:
        out[(int(E) + 2 * N) // 4] = lg
    return out


def test_config3_uneven_batch_sampled_instances_match_oracle():
    # the uneven-size batch (96 instances of mixed model and L) in one context;
    # one instance of each (model, L) re-run on the oracle
    ds = W.config3()
    gpu = make_gpu(ds)
    gpu.run(3)
    gpu.exchange()
    gpu.run(2)
    seen = {}
    for k, d in enumerate(ds):
        seen.setdefault((d["model"], d["L"]), k)
    for (model, L), k in sorted(seen.items()):
        o = make_oracle(ds[k])
        o.init()
        o.run(3)
        o.exchange()
        o.run(2)
        assert_same_state(gpu, k, o, f"config3 instance {k} (model {model}, L {L})")


def test_potts_q10_full_convergence_invariants():
    # q = 10 Potts: sum_E g(E) = q^N checked in log space, and the full
    # converged run agrees with the oracle bit for bit at L = 8
    d = _potts(8, 10, 4, 2, seed=4)
    gpu = make_gpu([d])
    orc = make_oracle(d)
    orc.init()
    for c in range(400):
        step_both(gpu, [orc], 1000)
        if orc.all_converged():
            break
    assert orc.all_converged() and gpu.status(0)["all_converged"]
    assert_same_state(gpu, 0, orc, "potts q10 L8 converged")
    lg, _ = gpu.get_dos(0)
    from oracle.exact_dos import log_sum
    N = 64
    assert abs(log_sum(lg) - N * math.log(10)) < 2e-3 * N * math.log(10)


def test_potts_q10_l32_config2_log_sum_invariant():
    # the q = 10, L = 32 workload (32 windows x 8 walkers) run to ln f = 2^-20:
    # ln sum_E g(E) must be 1024 ln 10.  The bound, 0.7 in ln (3e-4 of 2358),
    # is the spread of this sum over independent q = 10 runs at L = 16..64 to
    # the same ln f; this seed's run gives 0.11.
    ds = W.config2()
    gpu = make_gpu(ds)
    assert gpu.run_to_convergence(1000, 3_000_000, poll_cycles=50)
    lg, _ = gpu.get_dos(0)
    from oracle.exact_dos import log_sum
    target = 1024 * math.log(10)
    assert abs(log_sum(lg) - target) < 0.7, (log_sum(lg), target)
    c = gpu.counters(0)
    assert np.all(c["ex_acc"][:31] > 0)


def test_transfer_bytes_count_every_copy():
    # rewl_transfer_bytes: a read-out adds the 4-byte error word and the
    # instance's h * m * w ln g values; a warm start adds ln g, its
    # stage-start copy, stages and flags; neither moves bytes the other way
    d = W.config0()[0]
    gpu = make_gpu([d])
    h2d0, d2h0 = gpu.transfer_bytes()
    assert h2d0 > 0
    g = gpu.geometry(0)
    nbytes = g["h"] * g["m"] * g["w"] * 8
    gpu.get_dos(0, per_window=True)
    h2d1, d2h1 = gpu.transfer_bytes()
    assert h2d1 == h2d0 and d2h1 - d2h0 == 4 + nbytes
    gpu.set_initial_lng(0, np.zeros(g["B"]), 0.5)
    h2d2, d2h2 = gpu.transfer_bytes()
    assert h2d2 - h2d1 == 2 * nbytes + 4 * g["h"] + g["h"] and d2h2 - d2h1 == 4


SHIFTED = [
    ("config0_full", _ising(8, 4, 1, seed=60), 1000, 200),
    ("ising_L6_h2_m3_full", _ising(6, 2, 3, seed=61), 1000, 200),
    ("potts_q3_L4_full", _potts(4, 3, 2, 2, seed=62), 1000, 200),
    ("potts_q10_L200_sub", _potts(200, 10, 3, 2, seed=63, e_min=-60000, e_max=-59000), 2, 3),
]


@pytest.mark.parametrize("name,d,sweeps,cycles", SHIFTED, ids=[c[0] for c in SHIFTED])
def test_lowered_windows_match_oracle(name, d, sweeps, cycles):
    """A running window's ln g lowered by 2^s once all of it has reached 2^s
    (s = 3 here, so it happens throughout the run): bit-exact against the
    oracle doing the same, to full convergence on the small lattices."""
    gpu = make_gpu([d], lng_shift=3)
    orc = make_oracle(d)
    orc.set_shift_exp(3)
    orc.init()
    for c in range(cycles):
        step_both(gpu, [orc], sweeps)
        if orc.all_converged():
            break
    assert_same_state(gpu, 0, orc, f"{name} after {c + 1} cycles")
    if cycles > 10:
        assert orc.all_converged() and gpu.status(0)["all_converged"]
