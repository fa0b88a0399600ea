"""Energy windows: the equal-width rule and run-time-balanced windows.

The paper's outlook (Sec. V) notes that equal-size windows do not proceed
through the WL scheme at equal pace, above all in the first iterations, and
proposes sizing them so that every window meets its flatness criterion after
about the same number of MC steps.  ``balanced_windows`` does that from a
pilot run: a walker's random walk over w bins takes ~w^2 steps to visit them,
so a window whose first WL iteration took t sweeps is resized by
(t_mean / t)^(1/2), and the windows are laid out again over the B bins with
the same fractional overlap.  The result goes to ``Rewl(..., windows=...)``
(rewl_create_batch_windows).

``stage_durations`` reads, from rewl_get_stage_sweeps, how long each window
took for one WL stage; ``self_tuning_run`` repeats the resizing during the
run (the paper's "self-tuning" windows): after each of the first stages it
resizes the windows from the measured stage durations when they are
uneven, and continues from the joined ln g at the current ln f.
"""
import math

import numpy as np


def equal_windows(B, h, overlap):
    """(lo, hi) of the equal-width rule: w = ceil(B / (1 + (h-1)(1-o))),
    lo_i = floor(i (B - w) / (h - 1)) (the windows rewl_create builds)."""
    w = min(B, int(math.ceil(B / (1.0 + (h - 1) * (1.0 - overlap)))))
    lo = np.array([0 if h == 1 else (i * (B - w)) // (h - 1) for i in range(h)], np.int64)
    return lo, lo + w - 1


def _layout(widths, overlap, B):
    """Place windows of the given (float) widths from bin 0 upward, each
    overlapping its lower neighbour by `overlap` times the narrower width;
    returns (lo, hi) and the upper end reached."""
    lo, hi = [], []
    start = 0
    for i, wf in enumerate(widths):
        w = max(1, int(round(wf)))
        if i > 0:
            ov = max(1, int(math.ceil(overlap * min(w, hi[-1] - lo[-1] + 1))))
            start = hi[-1] + 1 - ov
        lo.append(start)
        hi.append(start + w - 1)
    return np.array(lo, np.int64), np.array(hi, np.int64), hi[-1]


def balanced_windows(lo, hi, t, B, overlap, min_width, max_width=None):
    """Windows sized so that each should finish a WL iteration in about the
    same number of sweeps: widths w_i (t_mean / t_i)^(1/2), same overlap rule,
    scaled to cover bins 0..B-1 exactly; every window at least min_width
    wide and, if max_width is given, at most that wide (each walker's ln g row
    in shared memory is as long as the widest window, so very wide windows
    cost occupancy).  t: sweeps of each window's slowest walker in a pilot
    run."""
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    t = np.asarray(t, np.float64)
    rel = (hi - lo + 1.0) * np.sqrt(t.mean() / np.maximum(t, 1.0))
    cap = np.inf if max_width is None else float(max_width)

    def widths(scale):
        return np.minimum(np.maximum(rel * scale, min_width), cap)

    a, b = 1e-6, 4.0 * B / rel.sum() + 1.0        # scale factors bracketing the span
    if max_width is not None and _layout(widths(1e9), overlap, B)[2] < B - 1:
        raise ValueError("max_width too small to cover the range with this many windows")
    while _layout(widths(b), overlap, B)[2] < B - 1:
        b *= 2.0
    for _ in range(200):
        s = 0.5 * (a + b)
        _, _, top = _layout(widths(s), overlap, B)
        if top >= B - 1:
            b = s
        else:
            a = s
    nlo, nhi, _ = _layout(widths(b), overlap, B)
    nhi[-1] = B - 1                              # the last window ends at the last bin
    if nhi[-1] - nlo[-1] + 1 < min_width:
        nlo[-1] = B - min_width
    for i in range(len(nlo) - 1):                # keep both ends increasing and overlapping
        nhi[i] = min(nhi[i], B - 2)
    return nlo, nhi


def valid_windows(lo, hi, B, min_width):
    """The conditions rewl_create_batch_windows checks."""
    lo = np.asarray(lo)
    hi = np.asarray(hi)
    if lo[0] != 0 or hi[-1] != B - 1:
        return False
    if np.any(hi - lo + 1 < min_width) or np.any(hi >= B):
        return False
    return bool(np.all(np.diff(lo) > 0) and np.all(np.diff(hi) > 0) and np.all(lo[1:] <= hi[:-1]))


def stage_durations(stage_sweeps, k):
    """Sweeps each window took for WL stage k (ln f = 2^-k), from the
    (h, 33) array of rewl_get_stage_sweeps; None if some window has not
    ended stage k."""
    ss = np.asarray(stage_sweeps)
    end = ss[:, k]
    if np.any(end < 0):
        return None
    start = ss[:, k - 1] if k > 0 else np.zeros_like(end)
    start = np.where(start < 0, 0, start)
    return (end - start).astype(np.float64)


def self_tuning_run(make_ctx, windows, B, overlap, min_width, exchange_interval, n_inst=1,
                    tune_at=(0, 1, 2, 3, 4, 5), tune_avg=1, imbalance=1.2, max_width=None, poll_cycles=5,
                    log=None):
    """Run a batch of n_inst instances that share one window set to the end
    of the WL scheme on self-tuning windows.  make_ctx(lo, hi) builds the
    batch on those windows.  After each stage k in tune_at, once every window
    of every instance has ended it, the sweeps per window of stages
    k - tune_avg + 1 .. k (summed, mean over the instances; only stages run on
    the current windows) are compared: if the slowest window took more than
    `imbalance` times the mean, the windows are resized from those durations
    (balanced_windows) and a new batch continues on them, each instance from
    its own joined ln g at ln f = 2^-(k+1).  Returns (context, (lo, hi),
    resize log, sweeps run summed over the contexts)."""
    lo, hi = windows
    ctx = make_ctx(lo, hi)
    first = 0                      # first stage run on the current windows
    resizes, sweeps_total = [], 0
    for k in sorted(tune_at):
        while True:
            ss = [ctx.stage_sweeps(i) for i in range(n_inst)]
            if all(np.all(s[:, k] >= 0) for s in ss) or ctx.status(0)["all_converged"]:
                break
            ctx.run_cycles(poll_cycles, exchange_interval)
        span = range(max(first, k - tune_avg + 1), k + 1)
        durs = [[stage_durations(s, j) for j in span] for s in ss]
        if not len(span) or any(d is None for per in durs for d in per):
            break
        d = np.mean([np.sum(per, axis=0) for per in durs], axis=0)
        if d.max() <= imbalance * d.mean():
            continue
        nlo, nhi = balanced_windows(lo, hi, d, B, overlap, min_width, max_width)
        if not valid_windows(nlo, nhi, B, min_width):
            continue
        lng = [ctx.get_dos(i)[0] for i in range(n_inst)]
        sweeps_total += int(ctx.status(0)["sweeps"])
        ctx.close()
        lo, hi = nlo, nhi
        ctx = make_ctx(lo, hi)
        for i in range(n_inst):
            g = lng[i]
            ctx.set_initial_lng(i, np.where(np.isfinite(g), g - np.nanmin(g), 0.0), 2.0 ** -(k + 1))
        first = k + 1
        resizes.append({"after_stage": k, "stages_averaged": len(span), "slowest_over_mean": float(d.max() / d.mean()),
                        "widths_min_max": [int((hi - lo + 1).min()), int((hi - lo + 1).max())]})
        if log:
            log(f"after stage {k}: slowest window {d.max() / d.mean():.2f} x mean, resized")
    while not ctx.run_to_convergence(exchange_interval, 50 * exchange_interval, poll_cycles=poll_cycles):
        pass
    sweeps_total += int(ctx.status(0)["sweeps"])
    return ctx, (lo, hi), resizes, sweeps_total
