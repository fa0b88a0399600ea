"""Joining per-window ln g pieces into one global ln g (Sec. II B of Vogel, Li,
Wuest, Landau, arXiv:1407.5140).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper's two steps, written as plain loops:
 (i)  in the overlap of windows i and i+1, estimate d ln g / dE of each piece
      with the five-point stencil
          beta(b) = [f(b-2s) - 8 f(b-s) + 8 f(b+s) - f(b+2s)] / (12 s dE),
      dE = energy per bin (the step width s is "up to ~10"; default s = 1);
 (ii) join at the bin where the two inverse temperatures agree best, cutting
      the overhanging tails: piece i below the join, piece i+1 from it on,
      piece i+1 shifted so that both agree at the join.
Readings (the paper is silent): candidate bins are those above the previous
join whose whole stencil lies inside both windows on realisable energies; ties
go to the lowest bin; if no candidate exists the join is the first realisable
bin of the overlap above the previous join.  The result is normalised so that
ln g(E_min) = ln 2 (Ising) or ln q (Potts).
"""
import math

import numpy as np


def stencil_beta(f, b, s, dE):
    return (f(b - 2 * s) - 8.0 * f(b - s) + 8.0 * f(b + s) - f(b + 2 * s)) / (12.0 * s * dE)


def concatenate(pieces, lo, w, reach, dE, ln_g_min, s=1):
    """pieces: (h, >= w) ln g per window on window-local bins; lo: first global
    bin of each window; w: bins per window (one number, or one per window);
    reach: (B,) realisable-energy mask.  Returns (ln_g (B,), joins (h-1,))
    with ln_g = nan on unrealisable bins."""
    h = len(pieces)
    ws = np.broadcast_to(np.asarray(w), (h,))
    B = len(reach)
    glob = np.full(B, np.nan)
    joins = []
    shift = 0.0                  # offset that maps piece i onto the global curve
    start = lo[0]                # first bin taken from piece i
    for i in range(h - 1):
        a_lo, b_lo = lo[i], lo[i + 1]
        ov_lo, ov_hi = max(a_lo, b_lo), min(a_lo + ws[i] - 1, b_lo + ws[i + 1] - 1)
        fa = lambda b, i=i: pieces[i][b - lo[i]]
        fb = lambda b, i=i: pieces[i + 1][b - lo[i + 1]]
        best, best_d = None, None
        for b in range(max(ov_lo, start + 1), ov_hi + 1):
            pts = [b - 2 * s, b - s, b, b + s, b + 2 * s]
            if pts[0] < ov_lo or pts[-1] > ov_hi or not all(reach[p] for p in pts):
                continue
            d = abs(stencil_beta(fa, b, s, dE) - stencil_beta(fb, b, s, dE))
            if best_d is None or d < best_d:
                best, best_d = b, d
        if best is None:
            best = max(ov_lo, start + 1)
            while best < ov_hi and not reach[best]:
                best += 1
        joins.append(best)
        for b in range(start, best):
            glob[b] = fa(b) + shift
        shift = fa(best) + shift - fb(best)
        start = best
    for b in range(start, lo[h - 1] + ws[h - 1]):
        glob[b] = pieces[h - 1][b - lo[h - 1]] + shift
    glob[~reach.astype(bool)] = np.nan
    first = int(np.argmax(reach))
    glob += ln_g_min - glob[first]
    return glob, np.array(joins, dtype=np.int64)


def ising_ln_g_min():
    return math.log(2.0)


def potts_ln_g_min(q):
    return math.log(float(q))


def mean_relative_error(ln_g, ln_g_exact):
    """epsilon = mean over realisable bins of |ln g - ln g_exact| / ln g_exact."""
    m = np.isfinite(ln_g_exact) & np.isfinite(ln_g)
    return float(np.mean(np.abs(ln_g[m] - ln_g_exact[m]) / ln_g_exact[m]))
