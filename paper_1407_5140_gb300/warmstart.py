"""Training-set assembly and the training loop of the learned warm start.

The network (``rewl.Mlp``, kernels in ``csrc/rewl_mlp.cu``) maps
x = (model, 16/L, log10 q, E/N, window / (h-1)) to the entropy density
s = ln g(E) / N.  Training data are ln g curves that plain REWL produced at
small L (joined with ``Rewl.get_dos``, normalised to ln g(E_min) = ln 2 or
ln q); every realisable bin of every window gives one sample.  The loop draws
seeded mini-batches on the host and runs every forward, backward and Adam step
in the library's kernels.
"""
import math

import numpy as np

from . import rewl as R


def curve_samples(model, L, q, e_min, step, ln_g, lo, w):
    """(x, t) samples of one joined ln g curve: one per (window, realisable bin);
    w: bins per window (one number, or one per window)."""
    N = L * L
    h = len(lo)
    ws = np.broadcast_to(np.asarray(w), (h,))
    xs, ts = [], []
    for i, l0 in enumerate(lo):
        for b in range(l0, l0 + int(ws[i])):
            v = ln_g[b]
            if not np.isfinite(v):
                continue
            E = e_min + b * step
            xs.append((float(model), 16.0 / L, math.log10(q), E / N, i / (h - 1) if h > 1 else 0.0))
            ts.append(v / N)
    return np.asarray(xs, np.float32), np.asarray(ts, np.float32)


def training_set(ctx, instances):
    """Samples of every instance of a finished plain-REWL context."""
    X, T = [], []
    for k, d in enumerate(instances):
        g = ctx.geometry(k)
        ln_g, _ = ctx.get_dos(k)
        step = 4 if d["model"] == R.ISING else 1
        q = 2 if d["model"] == R.ISING else d["q"]
        x, t = curve_samples(d["model"], d["L"], q, d["e_min"], step, ln_g, g["lo"], g["ww"])
        X.append(x)
        T.append(t)
    return np.concatenate(X), np.concatenate(T)


def train(net, X, T, steps=3000, batch=4096, lr=2e-3, seed=0, log_every=0, lr_end=None):
    """Adam on seeded mini-batches; returns the loss history (every log_every
    steps).  With lr_end the step size follows a cosine from lr down to lr_end
    over the run, which settles the last steps' mini-batch noise."""
    import torch

    rng = np.random.default_rng(seed)
    batch = min(batch, net.max_batch)
    batch -= batch % 64
    X = np.ascontiguousarray(X, np.float32)
    T = np.ascontiguousarray(T, np.float32)
    # mini-batches are gathered on the host into pinned buffers and copied in
    xh = torch.empty((batch, 5), dtype=torch.float32).pin_memory()
    th = torch.empty(batch, dtype=torch.float32).pin_memory()
    xb = torch.empty((batch, 5), dtype=torch.float32, device="cuda")
    tb = torch.empty(batch, dtype=torch.float32, device="cuda")
    hist = []
    for it in range(steps):
        idx = rng.integers(0, X.shape[0], batch)
        # the previous step (on the network's stream) is done with xb, tb and
        # its copies have left the pinned buffers
        torch.cuda.synchronize()
        np.take(X, idx, axis=0, out=xh.numpy())
        np.take(T, idx, out=th.numpy())
        xb.copy_(xh, non_blocking=True)
        tb.copy_(th, non_blocking=True)
        want = bool(log_every) and (it % log_every == 0 or it == steps - 1)
        step_lr = lr if lr_end is None else lr_end + 0.5 * (lr - lr_end) * (1.0 + math.cos(math.pi * it / max(1, steps - 1)))
        loss = net.train_step(xb, tb, step_lr, want_loss=want)
        if want:
            hist.append((it, loss))
    return hist


def predict(net, X):
    """Network output for host features X (padded to a multiple of 64)."""
    import torch

    n = X.shape[0]
    n_pad = (n + 63) // 64 * 64
    out = np.zeros(n, np.float32)
    for s in range(0, n_pad, net.max_batch):
        chunk = X[s:s + net.max_batch]
        m = chunk.shape[0]
        mp = (m + 63) // 64 * 64
        xb = np.zeros((mp, 5), np.float32)
        xb[:m] = chunk
        xd = torch.from_numpy(xb).cuda()
        yd = torch.empty(mp, dtype=torch.float32, device="cuda")
        net.forward(xd, yd)
        out[s:s + m] = yd.cpu().numpy()[:m]
    return out
