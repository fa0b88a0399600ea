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
