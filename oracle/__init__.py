"""CPU oracle of replica-exchange Wang-Landau sampling (REWL).

TEST INFRASTRUCTURE ONLY.  Nothing in the product package imports this module;
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` use it.  It shares no code with the
CUDA library in ``paper_1407_5140_gb300/``.

Contents
--------
- ``rewl_oracle.c``  : the REWL algorithm in plain C with FP64 ln g
  (Sec. II A of Vogel, Li, Wuest, Landau, arXiv:1407.5140; Eq. (1); Fig. 2).
- ``exact_dos.py``   : exact densities of states (brute force, transfer
  matrix, Kaufman's closed form as used by Beale) -- the pins.
- ``concat.py``      : joining the per-window DOS pieces (Sec. II B).

This module is a thin ctypes view of the C oracle.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

ISING, POTTS = 0, 1

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        vp, i32, i64, u32, u64, f64 = C.c_void_p, C.c_int, C.c_long, C.c_uint32, C.c_uint64, C.c_double
        L.oracle_create.restype = vp
        L.oracle_create.argtypes = [i32, i32, i32, i64, i64, i32, f64, i32, f64, f64, u64, u32]
        L.oracle_destroy.argtypes = [vp]
        L.oracle_init.argtypes = [vp]
        L.oracle_run.argtypes = [vp, i64, i32]
        L.oracle_exchange.argtypes = [vp]
        L.oracle_set_lng.argtypes = [vp, vp, i32]
        L.oracle_set_walker_lng.argtypes = [vp, i32, vp]
        L.oracle_geometry.argtypes = [vp, vp, vp, vp, vp]
        L.oracle_get_state.argtypes = [vp] * 10
        L.oracle_get_counters.argtypes = [vp] * 7
        L.oracle_all_converged.argtypes = [vp]
        L.oracle_set_check_every.argtypes = [vp, i64]
        L.oracle_set_shift_exp.argtypes = [vp, C.c_int]
        L.oracle_pct_flat.argtypes = [C.c_uint64, C.c_uint64, C.c_int, C.c_double]
        L.oracle_pct_flat.restype = C.c_int
        L.oracle_average_window.argtypes = [vp, C.c_int]
        L.oracle_average_window.restype = None
        L.oracle_set_flat_rule.argtypes = [vp, C.c_int]
        L.oracle_set_windows.argtypes = [vp, vp, vp]
        L.oracle_set_windows.restype = C.c_int
        L.oracle_window_widths.argtypes = [vp, vp]
        L.oracle_zb_flat.argtypes = [C.c_uint64, C.c_double, C.c_int]
        L.oracle_zb_flat.restype = C.c_int
        L.oracle_error.argtypes = [vp]
        L.oracle_energy_of.argtypes = [vp, i32]
        L.oracle_energy_of.restype = i64
        L.oracle_philox.argtypes = [u32, u32, vp, i64, vp]
        L.oracle_lam.argtypes = [vp, i64, vp]
        L.oracle_windows.argtypes = [i32, i32, f64, vp, vp]
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def windows(B, h, overlap):
    """(w, lo[]) of the equal-width window partition with overlap o."""
    lo = np.zeros(h, np.int32)
    w = np.zeros(1, np.int32)
    if lib().oracle_windows(B, h, overlap, _p(lo), _p(w)):
        raise ValueError("invalid window parameters")
    return int(w[0]), lo


def philox(key, counters):
    """Philox4x32-10 blocks for an (n, 4) array of counters."""
    ctr = np.ascontiguousarray(counters, dtype=np.uint32).reshape(-1, 4)
    out = np.zeros_like(ctr)
    lib().oracle_philox(int(key[0]), int(key[1]), _p(ctr), ctr.shape[0], _p(out))
    return out


def zb_flat(min_h, a, stage):
    """The oracle's Zhou-Bhatt decision (Eq. (8)) for one walker."""
    return bool(lib().oracle_zb_flat(int(min_h), float(a), int(stage)))


def lam_fix(k):
    """Acceptance threshold max(1, trunc(2^32 * -ln((k+1) 2^-24))) of the oracle."""
    k = np.ascontiguousarray(k, dtype=np.uint32)
    out = np.zeros(k.shape, np.int64)
    lib().oracle_lam(_p(k), k.size, _p(out))
    return out


def pct_flat(min_h, sum_h, n_reach, p):
    """The 80 % flatness predicate as the oracle evaluates it."""
    return bool(lib().oracle_pct_flat(min_h, sum_h, n_reach, p))


class Oracle:
    """One REWL instance: h windows x m walkers on an L x L lattice."""

    def __init__(self, model, L, q, e_min, e_max, n_windows, overlap, walkers_per_window,
                 flatness=0.8, ln_f_final=2.0 ** -20, seed=0, instance=0, threads=0, flat_rule=0,
                 windows=None):
        self.model, self.L, self.q = model, L, (2 if model == ISING else q)
        self.N = L * L
        self.h, self.m = n_windows, walkers_per_window
        self.threads = threads
        self._o = lib().oracle_create(model, L, q, e_min, e_max, n_windows, overlap,
                                      walkers_per_window, flatness, ln_f_final, seed, instance)
        if not self._o:
            raise ValueError("oracle_create rejected the parameters")
        lib().oracle_set_flat_rule(self._o, flat_rule)
        if windows is not None:
            lo = np.ascontiguousarray(windows[0], dtype=np.int32)
            hi = np.ascontiguousarray(windows[1], dtype=np.int32)
            assert lo.size == n_windows and hi.size == n_windows
            if lib().oracle_set_windows(self._o, _p(lo), _p(hi)):
                raise ValueError("oracle_set_windows rejected the windows")
        B = np.zeros(1, np.int32)
        w = np.zeros(1, np.int32)
        lib().oracle_geometry(self._o, _p(B), _p(w), None, None)
        self.B, self.w = int(B[0]), int(w[0])
        self.lo = np.zeros(self.h, np.int32)
        self.reach = np.zeros(self.B, np.uint8)
        lib().oracle_geometry(self._o, _p(B), _p(w), _p(self.lo), _p(self.reach))
        self.ww = np.zeros(self.h, np.int32)             # bins of each window (w: the widest)
        lib().oracle_window_widths(self._o, _p(self.ww))
        self.step = 4 if model == ISING else 1
        self.e_min, self.e_max = e_min, e_max

    def __del__(self):
        if getattr(self, "_o", None):
            lib().oracle_destroy(self._o)
            self._o = None

    @property
    def n_walkers(self):
        return self.h * self.m

    def init(self):
        err = lib().oracle_init(self._o)
        if err:
            raise RuntimeError(f"oracle init error {err}")

    def run(self, n_sweeps):
        err = lib().oracle_run(self._o, n_sweeps, self.threads)
        if err:
            raise RuntimeError(f"oracle run error {err}")

    def exchange(self):
        lib().oracle_exchange(self._o)

    def set_lng(self, ln_g_global, stage0):
        a = np.ascontiguousarray(ln_g_global, dtype=np.float64)
        assert a.size == self.B
        if lib().oracle_set_lng(self._o, _p(a), stage0):
            raise RuntimeError("ln g out of the exact range")

    def set_walker_lng(self, k, local):
        a = np.ascontiguousarray(local, dtype=np.float64)
        assert a.size == self.w
        if lib().oracle_set_walker_lng(self._o, k, _p(a)):
            raise RuntimeError("ln g out of the exact range")

    def state(self):
        nw, w = self.n_walkers, self.w
        s = {
            "spins": np.zeros((nw, self.N), np.int8),
            "E": np.zeros(nw, np.int64),
            "bin": np.zeros(nw, np.int32),
            "lng": np.zeros((nw, w), np.float64),
            "H": np.zeros((nw, w), np.uint64),
            "stage": np.zeros(self.h, np.int32),
            "conv": np.zeros(self.h, np.uint8),
            "latch": np.zeros(nw, np.uint8),
            "replica": np.zeros(nw, np.int64),
        }
        lib().oracle_get_state(self._o, *[_p(s[k]) for k in
                                          ("spins", "E", "bin", "lng", "H", "stage", "conv", "latch", "replica")])
        return s

    def counters(self):
        c = {
            "sweeps": np.zeros(1, np.int64),
            "t_exch": np.zeros(1, np.uint64),
            "ex_prop": np.zeros(self.h, np.uint64),
            "ex_acc": np.zeros(self.h, np.uint64),
            "n_acc": np.zeros(self.n_walkers, np.uint64),
            "conv_sweep": np.zeros(self.h, np.int64),
        }
        lib().oracle_get_counters(self._o, *[_p(c[k]) for k in
                                             ("sweeps", "t_exch", "ex_prop", "ex_acc", "n_acc", "conv_sweep")])
        c["sweeps"] = int(c["sweeps"][0])
        c["t_exch"] = int(c["t_exch"][0])
        return c

    def set_check_every(self, c):
        lib().oracle_set_check_every(self._o, c)

    def set_shift_exp(self, e):
        """ln g of a running window is lowered by 2^e once every realisable
        bin of every walker has reached 2^e (1 <= e <= 20; 20 by default)."""
        lib().oracle_set_shift_exp(self._o, e)

    def average_window(self, win):
        """The merge alone (Sec. II A): window win's walkers take the mean of
        their ln g, nearest multiple of 2^-32, ties to even."""
        lib().oracle_average_window(self._o, win)

    def all_converged(self):
        return bool(lib().oracle_all_converged(self._o))

    def energy_of(self, k):
        return int(lib().oracle_energy_of(self._o, k))

    def pieces(self):
        """Per-window ln g: walker-mean of each window (identical after a merge)."""
        s = self.state()
        return s["lng"].reshape(self.h, self.m, self.w).mean(axis=1)

    def run_to_convergence(self, exchange_interval, max_sweeps):
        """Alternate `exchange_interval` sweeps with one exchange phase until
        every window has converged (Sec. II A: the run ends when every walker
        reached ln f_final)."""
        done = 0
        while not self.all_converged():
            if done >= max_sweeps:
                return False
            n = min(exchange_interval, max_sweeps - done)
            self.run(n)
            done += n
            if self.h > 1:
                self.exchange()
        return True
