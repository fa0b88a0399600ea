"""FP64 reference of the warm-start network: a 5 -> 128 -> 128 -> 128 -> 1
perceptron with tanh hidden units, trained on the mean squared error with Adam.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  The learned warm start
is not in the paper; it predicts an initial ln g(E) per window from
(model, L, q, E, window) features.  This module is the plain statement of the
forward pass, the gradients (written out by the chain rule) and one Adam step
(Kingma & Ba, 2015), against which the GPU kernels are checked.

Parameter order (flat vector): W1 [128x5], b1 [128], W2 [128x128], b2 [128],
W3 [128x128], b3 [128], W4 [1x128], b4 [1]; W[out][in], y = W x + b.
"""
import numpy as np

SIZES = [(128, 5), (128, 128), (128, 128), (1, 128)]
N_PARAMS = sum(o * i + o for o, i in SIZES)


def unflatten(p):
    out, k = [], 0
    for o, i in SIZES:
        W = p[k:k + o * i].reshape(o, i)
        k += o * i
        b = p[k:k + o]
        k += o
        out.append((W, b))
    return out


def forward(p, x):
    """x: (n, 5) -> (y (n,), hidden activations [h1, h2, h3])."""
    layers = unflatten(np.asarray(p, np.float64))
    a = np.asarray(x, np.float64)
    hs = []
    for li, (W, b) in enumerate(layers):
        z = a @ W.T + b
        if li < 3:
            a = np.tanh(z)
            hs.append(a)
        else:
            a = z
    return a[:, 0], hs


def loss(p, x, t):
    y, _ = forward(p, x)
    return 0.5 * np.mean((y - np.asarray(t, np.float64)) ** 2)


def gradient(p, x, t):
    """d loss / d p by the chain rule (loss = mean over samples of (y-t)^2 / 2)."""
    layers = unflatten(np.asarray(p, np.float64))
    x = np.asarray(x, np.float64)
    y, hs = forward(p, x)
    n = x.shape[0]
    dz = ((y - np.asarray(t, np.float64)) / n)[:, None]          # (n, 1)
    inputs = [x] + hs                                              # input of each layer
    grads = [None] * 4
    for li in range(3, -1, -1):
        W, b = layers[li]
        grads[li] = (dz.T @ inputs[li], dz.sum(axis=0))
        if li > 0:
            dh = dz @ W
            dz = dh * (1.0 - hs[li - 1] ** 2)                     # tanh' = 1 - tanh^2
    flat = []
    for dW, db in grads:
        flat.append(dW.ravel())
        flat.append(db.ravel())
    return np.concatenate(flat)


def adam_step(p, m, v, g, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (bias-corrected moments); returns new (p, m, v)."""
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    mh = m / (1 - beta1 ** step)
    vh = v / (1 - beta2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def init_params(seed):
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights and biases."""
    rng = np.random.default_rng(seed)
    flat = []
    for o, i in SIZES:
        a = 1.0 / np.sqrt(i)
        flat.append(rng.uniform(-a, a, o * i))
        flat.append(rng.uniform(-a, a, o))
    return np.concatenate(flat)
