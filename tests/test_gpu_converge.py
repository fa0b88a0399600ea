"""Full runs to ln f = 2^-20 on the GPU judged against the exact density of
states (Beale's method: Kaufman's closed form, tests/golden/), and the error
analysis of Sec. II B on their pieces.

The batched Ising configuration (16 windows x 4 walkers at 75 % overlap,
exchanges every 10^4 sweeps) at L = 32 and L = 64, four seeds each, run
together in one batch."""
import math
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _exact(L):
    rows = np.loadtxt(os.path.join(GOLDEN, f"ising_L{L}_exact_lng.txt"), usecols=(0, 1))
    N = L * L
    out = np.full(N + 1, np.nan)
    out[((rows[:, 0] + 2 * N) // 4).astype(int)] = rows[:, 1]
    return out


def _eps(lg, ex):
    ok = np.isfinite(lg) & np.isfinite(ex) & (ex != 0)
    return float(np.mean(np.abs(lg[ok] - ex[ok]) / np.abs(ex[ok])))


@pytest.fixture(scope="module")
def converged():
    import torch
    from paper_1407_5140_gb300 import rewl as R
    from paper_1407_5140_gb300 import workloads as W
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ds = [d for d in W.config1(sizes=(32, 64), seeds=32) if d["seed"] < 4]
    ctx = R.Rewl([R.instance(**d) for d in ds], stream=stream)
    assert ctx.run_to_convergence(10_000, 20_000_000, poll_cycles=2)
    yield ctx, ds
    ctx.close()


def test_config1_reaches_the_exact_dos(converged):
    """Mean relative ln g error against the exact DOS at ln f = 2^-20 with
    m = 4 walkers per window: every run within 1e-3 at L = 64 (measured
    1.5e-4 .. 2.0e-4); at L = 32 the 80 % flatness rule with four walkers
    reaches 1e-3 on average over runs (measured 5.7e-4 .. 1.7e-3 per run, mean
    8.8e-4).  The runs are bit-for-bit repeatable, so these are fixed values."""
    ctx, ds = converged
    res = {}
    for k, d in enumerate(ds):
        lg, _ = ctx.get_dos(k)
        res.setdefault(d["L"], []).append(_eps(lg, _exact(d["L"])))
        # the invariant sum g = 2^N holds for the joined DOS
        v = lg[np.isfinite(lg)]
        m = v.max()
        assert abs(m + math.log(np.exp(v - m).sum()) - d["L"] ** 2 * math.log(2)) < 0.5
    print({L: (np.mean(e), np.max(e)) for L, e in res.items()})
    assert np.max(res[64]) <= 1e-3, res[64]
    assert np.mean(res[32]) <= 1e-3 and np.max(res[32]) <= 2e-3, res[32]


def test_bootstrap_errors_cover_the_deviation_from_exact(converged):
    """Sec. II B: pieces averaged over the seeds, joined; 200 bootstrap
    resamples of the pieces give error bars on ln g.  The mean DOS must lie
    within a few of its error bars of the exact DOS (bins outside the first
    few, which the normalisation pins)."""
    from paper_1407_5140_gb300 import thermo as TH
    ctx, ds = converged
    for L in (32, 64):
        ks = [k for k, d in enumerate(ds) if d["L"] == L]
        g = ctx.geometry(ks[0])
        P = np.stack([ctx.get_dos(k, per_window=True)[0] for k in ks])
        mean, std, _ = TH.bootstrap_dos(P, g["lo"], g["ww"], g["reach"], 4.0, math.log(2), n_resamples=200, seed=L)
        ex = _exact(L)
        ok = np.isfinite(mean) & np.isfinite(ex) & (std > 0)
        z = np.abs(mean[ok] - ex[ok]) / std[ok]
        print(L, float(np.median(z)), float(np.percentile(z, 95)))
        # with four runs the bootstrap error is itself uncertain; the bulk of the
        # bins must still sit within a few error bars
        assert np.median(z) < 3.0 and np.percentile(z, 95) < 8.0, (L, np.median(z), np.percentile(z, 95))
