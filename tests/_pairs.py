"""Helpers that build the same seeded instance on the GPU library and on the CPU
oracle and compare their states element by element."""
import numpy as np

import oracle as O


def make_oracle(d, threads=0, windows=None):
    return O.Oracle(d["model"], d["L"], d["q"], d["e_min"], d["e_max"], d["n_windows"], d["overlap"],
                    d["walkers_per_window"], d["flatness"], d["ln_f_final"], seed=d["seed"],
                    instance=d["instance_id"], threads=threads, flat_rule=d.get("flat_rule", 0),
                    windows=windows)


def make_gpu(ds, windows=None, **opts):
    from paper_1407_5140_gb300 import rewl as R
    ctx = R.Rewl([R.instance(**d) for d in ds], windows=windows)
    for k, v in opts.items():
        ctx.set_option(getattr(R, "OPT_" + k.upper()), v)
    return ctx


def assert_same_state(gpu, inst, orc, what=""):
    g = gpu.state(inst, orc.N)
    o = orc.state()
    for key in ("spins", "E", "bin", "stage", "conv", "latch", "replica"):
        a, b = np.asarray(g[key]), np.asarray(o[key])
        assert a.shape == b.shape, (what, key, a.shape, b.shape)
        bad = np.nonzero(a.reshape(a.shape[0], -1) != b.reshape(b.shape[0], -1))
        assert bad[0].size == 0, f"{what}: {key} differs at {bad[0][:5]} gpu={a.ravel()[:8]} oracle={b.ravel()[:8]}"
    assert np.array_equal(g["lng"], o["lng"]), f"{what}: ln g differs (max |d| = {np.abs(g['lng'] - o['lng']).max()})"
    assert np.array_equal(g["H"].astype(np.uint64), o["H"] & np.uint64(0xFFFFFFFF)), f"{what}: H differs"
    gc = gpu.counters(inst)
    oc = orc.counters()
    assert np.array_equal(gc["ex_prop"], oc["ex_prop"]), f"{what}: exchange proposals differ"
    assert np.array_equal(gc["ex_acc"], oc["ex_acc"]), f"{what}: exchange acceptances differ"
    assert np.array_equal(gc["n_acc"], oc["n_acc"]), f"{what}: accepted-move counts differ"
    assert np.array_equal(gc["conv_sweep"], oc["conv_sweep"]), f"{what}: convergence sweeps differ"


def step_both(gpu, orcs, sweeps, exchange=True):
    gpu.run(sweeps)
    for o in orcs:
        o.run(sweeps)
    if exchange:
        gpu.exchange()
        for o in orcs:
            o.exchange()
