"""Python binding of the REWL C ABI (``include/rewl.h``): argument marshalling only.

Every step of the sampling runs in the CUDA library ``_build/librewl.so``; this
module converts arguments, allocates host arrays for results and raises on
error codes.  PyTorch is used only to hand the library a CUDA stream and device
buffers.  There is no CPU fallback: importing the binding without the built
library raises.
"""
import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "librewl.so")

ISING, POTTS = 0, 1
OPT_CHECK_EVERY, OPT_PRODUCER_WARPS, OPT_WINDOWS_PER_CTA, OPT_MAX_SWEEPS_PER_LAUNCH, OPT_AUTOTUNE = 1, 2, 3, 4, 5
OPT_LATTICE_PLACEMENT, OPT_LNG_SHIFT = 6, 7
STATUS = {0: "REWL_OK", -1: "REWL_EINVAL", -2: "REWL_ENOMEM", -3: "REWL_ECUDA", -4: "REWL_ETIMEOUT",
          -5: "REWL_ESTATE", -6: "REWL_EDEVICE"}


class RewlError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class rewl_instance(C.Structure):
    _fields_ = [("model", C.c_int32), ("L", C.c_int32), ("q", C.c_int32), ("n_windows", C.c_int32),
                ("e_min", C.c_int64), ("e_max", C.c_int64), ("overlap", C.c_double),
                ("walkers_per_window", C.c_int32), ("flat_rule", C.c_int32), ("flatness", C.c_double),
                ("ln_f_final", C.c_double), ("seed", C.c_uint64), ("instance_id", C.c_uint32),
                ("reserved2", C.c_uint32)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"REWL CUDA library not built ({LIB_PATH}); run "
                              "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = C.CDLL(LIB_PATH)
        vp, i32, i64, u32, u64, f64 = C.c_void_p, C.c_int, C.c_long, C.c_uint32, C.c_uint64, C.c_double
        L.rewl_create.argtypes = [C.POINTER(vp), i32, i32, i32, i64, i64, i32, f64, i32, f64, f64, u64, vp]
        L.rewl_create_batch.argtypes = [C.POINTER(vp), C.POINTER(rewl_instance), i32, vp]
        L.rewl_create_batch_windows.argtypes = [C.POINTER(vp), C.POINTER(rewl_instance), i32, vp, vp, vp]
        L.rewl_window_widths.argtypes = [vp, i32, vp]
        L.rewl_run.argtypes = [vp, i64]
        L.rewl_exchange.argtypes = [vp]
        L.rewl_run_cycles.argtypes = [vp, i64, i64]
        L.rewl_run_to_convergence.argtypes = [vp, i64, i64, i64, vp]
        L.rewl_get_dos.argtypes = [vp, i32, vp, i64, vp, vp, i32]
        L.rewl_status_query.argtypes = [vp, i32, vp, vp, vp]
        L.rewl_set_initial_lng.argtypes = [vp, i32, vp, f64]
        L.rewl_geometry.argtypes = [vp, i32, vp, vp, vp, vp, vp, vp]
        L.rewl_get_state.argtypes = [vp, i32] + [vp] * 9
        L.rewl_get_counters.argtypes = [vp, i32, vp, vp, vp, vp]
        L.rewl_set_option.argtypes = [vp, i32, i64]
        L.rewl_launch_count.argtypes = [vp]
        L.rewl_launch_count.restype = i64
        L.rewl_transfer_bytes.argtypes = [vp, vp, vp]
        L.rewl_save.argtypes = [vp, C.c_char_p]
        L.rewl_load.argtypes = [C.POINTER(vp), C.c_char_p, vp]
        L.rewl_last_error.argtypes = [vp]
        L.rewl_last_error.restype = C.c_char_p
        L.rewl_destroy.argtypes = [vp]
        L.rewl_destroy.restype = None
        L.rewl_mlp_create.argtypes = [C.POINTER(vp), i32, u64, vp]
        L.rewl_mlp_set_params.argtypes = [vp, vp, i64]
        L.rewl_mlp_get_params.argtypes = [vp, vp, i64]
        L.rewl_mlp_forward.argtypes = [vp, vp, vp, i32]
        L.rewl_mlp_gradient.argtypes = [vp, vp, vp, i32, vp, vp]
        L.rewl_mlp_train_step.argtypes = [vp, vp, vp, i32, C.c_float, vp]
        L.rewl_mlp_launch_count.argtypes = [vp]
        L.rewl_mlp_launch_count.restype = i64
        L.rewl_mlp_last_error.argtypes = [vp]
        L.rewl_mlp_last_error.restype = C.c_char_p
        L.rewl_mlp_destroy.argtypes = [vp]
        L.rewl_mlp_destroy.restype = None
        L.rewl_warm_start.argtypes = [vp, i32, vp, f64]
        L.rewl_mlp_forward_noalloc.argtypes = [vp, vp, vp, i32, vp]
        L.rewl_join_pieces.argtypes = [i32, i32, i32, vp, vp, vp, f64, f64, vp, vp]
        L.rewl_get_stage_sweeps.argtypes = [vp, i32, vp]
        L.rewl_debug_lam.argtypes = [vp, vp, i64]
        L.rewl_debug_philox.argtypes = [u32, u32, vp, vp, i64]
        for name in ("rewl_create", "rewl_create_batch", "rewl_run", "rewl_exchange", "rewl_run_cycles",
                     "rewl_run_to_convergence", "rewl_get_dos", "rewl_status_query", "rewl_set_initial_lng",
                     "rewl_geometry", "rewl_get_state", "rewl_get_counters", "rewl_set_option", "rewl_save",
                     "rewl_load", "rewl_debug_lam", "rewl_debug_philox", "rewl_mlp_create", "rewl_mlp_set_params",
                     "rewl_mlp_get_params", "rewl_mlp_forward", "rewl_mlp_gradient", "rewl_mlp_train_step",
                     "rewl_warm_start", "rewl_mlp_forward_noalloc", "rewl_join_pieces",
                     "rewl_get_stage_sweeps"):
            getattr(L, name).restype = i32
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _check(code, ctx=None):
    if code != 0:
        raise RewlError(code, lib().rewl_last_error(ctx).decode())


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)       # torch.cuda.Stream


def instance(model, L, q=2, e_min=None, e_max=None, n_windows=1, overlap=0.75, walkers_per_window=1,
             flatness=0.8, ln_f_final=2.0 ** -20, seed=0, instance_id=0, flat_rule=0):
    N = L * L
    if e_min is None:
        e_min = -2 * N
    if e_max is None:
        e_max = 2 * N if model == ISING else 0
    return rewl_instance(model, L, q, n_windows, e_min, e_max, overlap, walkers_per_window, flat_rule, flatness,
                         ln_f_final, seed, instance_id, 0)


class Rewl:
    """A REWL context: one or more independent instances sampled together."""

    def __init__(self, instances, stream=None, _handle=None, windows=None):
        """windows: None (equal-width windows from each instance's overlap) or one
        (lo, hi) pair of bin-index arrays per instance (rewl_create_batch_windows)."""
        self._h = C.c_void_p()
        if _handle is not None:
            self._h = _handle
        else:
            if isinstance(instances, rewl_instance):
                instances = [instances]
            arr = (rewl_instance * len(instances))(*instances)
            if windows is None:
                code = lib().rewl_create_batch(C.byref(self._h), arr, len(instances), _stream_ptr(stream))
            else:
                lo = np.ascontiguousarray(np.concatenate([np.asarray(w[0]) for w in windows]), dtype=np.int32)
                hi = np.ascontiguousarray(np.concatenate([np.asarray(w[1]) for w in windows]), dtype=np.int32)
                code = lib().rewl_create_batch_windows(C.byref(self._h), arr, len(instances), _p(lo), _p(hi),
                                                       _stream_ptr(stream))
            if code != 0:
                msg = lib().rewl_last_error(self._h if self._h else None).decode()
                if self._h:
                    lib().rewl_destroy(self._h)
                    self._h = C.c_void_p()
                raise RewlError(code, msg)
        self.n_inst = len(instances) if instances is not None else None
        self._geom = {}

    @classmethod
    def create(cls, model, L, q, e_min, e_max, n_windows, overlap, walkers_per_window, flatness=0.8,
               ln_f_final=2.0 ** -20, seed=0, stream=None):
        """rewl_create: one instance."""
        h = C.c_void_p()
        code = lib().rewl_create(C.byref(h), model, L, q, e_min, e_max, n_windows, overlap, walkers_per_window,
                                 flatness, ln_f_final, seed, _stream_ptr(stream))
        if code != 0:
            msg = lib().rewl_last_error(h if h else None).decode()
            if h:
                lib().rewl_destroy(h)
            raise RewlError(code, msg)
        obj = cls(None, _handle=h)
        obj.n_inst = 1
        return obj

    @classmethod
    def load(cls, path, stream=None):
        h = C.c_void_p()
        code = lib().rewl_load(C.byref(h), path.encode(), _stream_ptr(stream))
        if code != 0:
            msg = lib().rewl_last_error(h if h else None).decode()
            if h:
                lib().rewl_destroy(h)
            raise RewlError(code, msg)
        return cls(None, _handle=h)

    def close(self):
        if self._h:
            lib().rewl_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- running
    def run(self, n_sweeps):
        _check(lib().rewl_run(self._h, n_sweeps), self._h)

    def exchange(self):
        _check(lib().rewl_exchange(self._h), self._h)

    def run_cycles(self, n_cycles, sweeps_per_cycle):
        _check(lib().rewl_run_cycles(self._h, n_cycles, sweeps_per_cycle), self._h)

    def run_to_convergence(self, exchange_interval, max_sweeps, poll_cycles=1):
        c = C.c_int(0)
        _check(lib().rewl_run_to_convergence(self._h, exchange_interval, max_sweeps, poll_cycles,
                                             C.byref(c)), self._h)
        return bool(c.value)

    def set_option(self, option, value):
        _check(lib().rewl_set_option(self._h, option, value), self._h)

    def set_initial_lng(self, inst, ln_g0, ln_f_start):
        a = np.ascontiguousarray(ln_g0, dtype=np.float64)
        _check(lib().rewl_set_initial_lng(self._h, inst, _p(a), ln_f_start), self._h)

    def launch_count(self):
        return int(lib().rewl_launch_count(self._h))

    def transfer_bytes(self):
        """(host->device, device->host) bytes the library copied for this context."""
        a, b = C.c_int64(), C.c_int64()
        _check(lib().rewl_transfer_bytes(self._h, C.byref(a), C.byref(b)), self._h)
        return a.value, b.value

    def warm_start(self, inst, net, ln_f_start):
        """rewl_warm_start: ln g of every walker from the network, ln f = ln_f_start."""
        _check(lib().rewl_warm_start(self._h, inst, net._h, ln_f_start), self._h)

    def save(self, path):
        _check(lib().rewl_save(self._h, path.encode()), self._h)

    # -- read-out
    def geometry(self, inst=0):
        if inst not in self._geom:
            h, m, B, w = C.c_int(), C.c_int(), C.c_int(), C.c_int()
            _check(lib().rewl_geometry(self._h, inst, C.byref(h), C.byref(m), C.byref(B), C.byref(w), None, None),
                   self._h)
            lo = np.zeros(h.value, np.int32)
            reach = np.zeros(B.value, np.uint8)
            _check(lib().rewl_geometry(self._h, inst, None, None, None, None, _p(lo), _p(reach)), self._h)
            ww = np.zeros(h.value, np.int32)
            _check(lib().rewl_window_widths(self._h, inst, _p(ww)), self._h)
            self._geom[inst] = dict(h=h.value, m=m.value, B=B.value, w=w.value, lo=lo, reach=reach, ww=ww)
        return self._geom[inst]

    def status(self, inst=0):
        allc = C.c_int()
        sw = C.c_long()
        lnf = np.zeros(self.geometry(inst)["h"], np.float64)
        _check(lib().rewl_status_query(self._h, inst, C.byref(allc), _p(lnf), C.byref(sw)), self._h)
        return {"all_converged": bool(allc.value), "ln_f": lnf, "sweeps": sw.value}

    def state(self, inst, N):
        g = self.geometry(inst)
        n_windows, m, w = g["h"], g["m"], g["w"]
        nw = n_windows * m
        s = {
            "spins": np.zeros((nw, N), np.int8),
            "E": np.zeros(nw, np.int64),
            "bin": np.zeros(nw, np.int32),
            "lng": np.zeros((nw, w), np.float64),
            "H": np.zeros((nw, w), np.uint32),
            "stage": np.zeros(n_windows, np.int32),
            "conv": np.zeros(n_windows, np.uint8),
            "latch": np.zeros(nw, np.uint8),
            "replica": np.zeros(nw, np.int64),
        }
        _check(lib().rewl_get_state(self._h, inst, *[_p(s[k]) for k in
                                                     ("spins", "E", "bin", "lng", "H", "stage", "conv", "latch",
                                                      "replica")]), self._h)
        return s

    def counters(self, inst=0):
        g = self.geometry(inst)
        n_windows, m = g["h"], g["m"]
        c = {"ex_prop": np.zeros(n_windows, np.uint64), "ex_acc": np.zeros(n_windows, np.uint64),
             "n_acc": np.zeros(n_windows * m, np.uint64), "conv_sweep": np.zeros(n_windows, np.int64)}
        _check(lib().rewl_get_counters(self._h, inst, *[_p(c[k]) for k in ("ex_prop", "ex_acc", "n_acc",
                                                                           "conv_sweep")]), self._h)
        return c

    def stage_sweeps(self, inst=0):
        """(h, 33) sweep counts at which each window ended each WL stage
        (ln f = 2^-k), -1 where it has not."""
        g = self.geometry(inst)
        out = np.zeros(g["h"] * 33, np.int64)
        _check(lib().rewl_get_stage_sweeps(self._h, inst, _p(out)), self._h)
        return out.reshape(g["h"], 33)

    def get_dos(self, inst=0, per_window=False):
        g = self.geometry(inst)
        cap = g["h"] * g["w"] if per_window else g["B"]
        out = np.zeros(cap, np.float64)
        e = np.zeros(cap, np.int64)
        n = C.c_long()
        _check(lib().rewl_get_dos(self._h, inst, _p(out), cap, C.byref(n), _p(e), 1 if per_window else 0), self._h)
        if per_window:
            return out.reshape(g["h"], g["w"]), e.reshape(g["h"], g["w"])
        return out, e


def join_pieces(pieces, lo, ww, reach, bin_width, ln_g_first):
    """rewl_join_pieces: join per-window ln g pieces (h x w array, window i's
    bins lo[i] .. lo[i] + ww[i] - 1 first in row i) as rewl_get_dos does
    (Sec. II B); host only.  Returns B values, NaN on unrealisable bins."""
    P = np.ascontiguousarray(pieces, np.float64)
    h, w = P.shape
    lo = np.ascontiguousarray(lo, np.int32)
    ww = np.ascontiguousarray(np.broadcast_to(np.asarray(ww, np.int32), (h,)), np.int32)
    reach = np.ascontiguousarray(reach, np.uint8)
    out = np.zeros(reach.size, np.float64)
    code = lib().rewl_join_pieces(h, w, reach.size, _p(lo), _p(ww), _p(reach), float(bin_width), float(ln_g_first),
                                  _p(P), _p(out))
    if code != 0:
        raise RewlError(code, lib().rewl_last_error(None).decode())
    return out


# -- primitive checks (device pointers from torch tensors)
def debug_lam(k_dev, out_dev, n):
    _check(lib().rewl_debug_lam(C.c_void_p(k_dev), C.c_void_p(out_dev), n))


def debug_philox(key0, key1, ctr_dev, out_dev, n):
    _check(lib().rewl_debug_philox(key0, key1, C.c_void_p(ctr_dev), C.c_void_p(out_dev), n))


N_PARAMS = 33921


def _mcheck(code, h):
    if code != 0:
        raise RewlError(code, lib().rewl_mlp_last_error(h).decode())


class Mlp:
    """The warm-start network (``rewl_mlp_*``).  x, t, y are torch CUDA tensors
    (float32, contiguous); batches are multiples of 64."""

    def __init__(self, max_batch=8192, seed=0, stream=None):
        self._h = C.c_void_p()
        code = lib().rewl_mlp_create(C.byref(self._h), max_batch, seed, _stream_ptr(stream))
        if code != 0:
            msg = lib().rewl_mlp_last_error(self._h if self._h else None).decode()
            if self._h:
                lib().rewl_mlp_destroy(self._h)
                self._h = C.c_void_p()
            raise RewlError(code, msg)
        self.max_batch = max_batch

    def close(self):
        if self._h:
            lib().rewl_mlp_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, p):
        a = np.ascontiguousarray(p, dtype=np.float32)
        _mcheck(lib().rewl_mlp_set_params(self._h, _p(a), a.size), self._h)

    def get_params(self):
        a = np.zeros(N_PARAMS, np.float32)
        _mcheck(lib().rewl_mlp_get_params(self._h, _p(a), a.size), self._h)
        return a

    def forward(self, x, y):
        n = _check_rows(x, 5, "x")
        _check_vec(y, n, "y")
        _mcheck(lib().rewl_mlp_forward(self._h, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()), n), self._h)

    def gradient(self, x, t):
        n = _check_rows(x, 5, "x")
        _check_vec(t, n, "t")
        g = np.zeros(N_PARAMS, np.float32)
        loss = np.zeros(1, np.float32)
        _mcheck(lib().rewl_mlp_gradient(self._h, C.c_void_p(x.data_ptr()), C.c_void_p(t.data_ptr()), n,
                                        _p(g), _p(loss)), self._h)
        return g, float(loss[0])

    def train_step(self, x, t, lr, want_loss=False):
        n = _check_rows(x, 5, "x")
        _check_vec(t, n, "t")
        loss = np.zeros(1, np.float32)
        _mcheck(lib().rewl_mlp_train_step(self._h, C.c_void_p(x.data_ptr()), C.c_void_p(t.data_ptr()), n,
                                          lr, _p(loss) if want_loss else None), self._h)
        return float(loss[0]) if want_loss else None

    def launch_count(self):
        return int(lib().rewl_mlp_launch_count(self._h))


def _check_dev_f32(a, name):
    """a must be a contiguous float32 CUDA tensor on the current device: the
    kernels read and write it through its raw pointer."""
    import torch
    if not isinstance(a, torch.Tensor):
        raise ValueError(f"{name} must be a torch tensor")
    if a.dtype != torch.float32 or not a.is_cuda or not a.is_contiguous():
        raise ValueError(f"{name} must be a contiguous float32 CUDA tensor")
    if a.device.index != torch.cuda.current_device():
        raise ValueError(f"{name} is on cuda:{a.device.index}, the current device is cuda:{torch.cuda.current_device()}")


def _check_rows(x, cols, name):
    _check_dev_f32(x, name)
    if x.dim() != 2 or x.shape[1] != cols:
        raise ValueError(f"{name} must have shape [n, {cols}]")
    return int(x.shape[0])


def _check_vec(v, n, name):
    _check_dev_f32(v, name)
    if v.numel() < n:
        raise ValueError(f"{name} holds {v.numel()} values, {n} needed")


def mlp_forward_noalloc(params, x, y, stream=None):
    """rewl_mlp_forward_noalloc: network output without any device allocation.
    params (33921 floats), x ([n, 5]) and y ([n]) are contiguous float32 CUDA
    tensors on the current device; anything else raises ValueError before the
    library is called."""
    n = _check_rows(x, 5, "x")
    _check_vec(y, n, "y")
    _check_dev_f32(params, "params")
    if params.numel() != N_PARAMS:
        raise ValueError(f"params must hold {N_PARAMS} values")
    code = lib().rewl_mlp_forward_noalloc(C.c_void_p(params.data_ptr()), C.c_void_p(x.data_ptr()),
                                          C.c_void_p(y.data_ptr()), n, _stream_ptr(stream))
    if code != 0:
        raise RewlError(code, lib().rewl_mlp_last_error(None).decode())
