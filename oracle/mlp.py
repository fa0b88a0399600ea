"""FP64 reference of the warm-start network: a 5 -> 128 -> 128 -> 128 -> 1
perceptron with tanh hidden units, trained on the mean squared error with Adam.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  The learned warm start
is not in the paper; it predicts an initial ln g(E) per window from
(model, L, q, E, window) features.  This module is the plain statement of the
forward pass, the gradients (written out by the chain rule) and one Adam step
(Kingma & Ba, 2015), against which the GPU kernels are checked.

Parameter order (flat vector): W1 [128x5], b1 [128], W2 [128x128], b2 [128],
W3 [128x128], b3 [128], W4 [1x128], b4 [1]; W[out][in], y = W x + b.

``forward_bf16`` / ``gradient_bf16`` state the same network with the operands
of its two 128 x 128 products (forward, and both backward products of each)
rounded to bfloat16, the precision the library promises for them; everything
else stays FP64.  They give the value a BF16-operand implementation must
reproduce up to its FP32 accumulation, together with the sum of absolute terms
of every output, from which a per-element tolerance follows.  Parity unpinned
in the strict sense: bfloat16 rounding is pinned against a library conversion,
and the result against the FP64 network within the BF16 error bound.
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


def round_bf16(a):
    """Nearest bfloat16 (8-bit significand, ties to even) of every element of
    a, via its float32 value; returned as float64."""
    u = np.ascontiguousarray(a, np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def forward_bf16(p, x):
    """Forward pass with the operands of the two 128 x 128 products rounded to
    bfloat16: h1 = tanh(W1 x + b1); h2 = tanh(bf(h1) bf(W2)^T + b2);
    h3 = tanh(bf(h2) bf(W3)^T + b3); y = W4 h3 + b4.  Returns (y, [h1, h2, h3],
    |y| bound terms: sum of |W4| |h3| + |b4| per sample)."""
    (W1, b1), (W2, b2), (W3, b3), (W4, b4) = unflatten(np.asarray(p, np.float64))
    x = np.asarray(x, np.float64)
    h1 = np.tanh(x @ W1.T + b1)
    h2 = np.tanh(round_bf16(h1) @ round_bf16(W2).T + b2)
    h3 = np.tanh(round_bf16(h2) @ round_bf16(W3).T + b3)
    y = (h3 @ W4.T + b4)[:, 0]
    ya = (np.abs(h3) @ np.abs(W4).T + np.abs(b4))[:, 0]
    return y, [h1, h2, h3], ya


def gradient_bf16(p, x, t):
    """Gradient of the loss with bfloat16 operands in the 128 x 128 products:
    dW3 = bf(dz3)^T bf(h2), dz2 = (bf(dz3) bf(W3)) (1 - h2^2),
    dW2 = bf(dz2)^T bf(h1), dz1 = (bf(dz2) bf(W2)) (1 - h1^2); the other sums
    (dW4, db4, dz3, the biases, dW1) in FP64.  Returns (g, a): a is the same
    chain with every factor replaced by its absolute value (the sum of absolute
    terms of each gradient element, with |y| + |b4| standing in for |y - t| where
larger)."""
    layers = unflatten(np.asarray(p, np.float64))
    (W1, _), (W2, _), (W3, _), (W4, _) = layers
    x = np.asarray(x, np.float64)
    y, (h1, h2, h3), _ = forward_bf16(p, x)
    n = x.shape[0]
    bf = round_bf16
    dy = (y - np.asarray(t, np.float64)) / n
    dz3 = dy[:, None] * W4[0][None, :] * (1.0 - h3 ** 2)
    dz2 = (bf(dz3) @ bf(W3)) * (1.0 - h2 ** 2)
    dz1 = (bf(dz2) @ bf(W2)) * (1.0 - h1 ** 2)
    g = [(dz1.T @ x, dz1.sum(0)), (bf(dz2).T @ bf(h1), dz2.sum(0)), (bf(dz3).T @ bf(h2), dz3.sum(0)),
         (dy[None, :] @ h3, np.array([dy.sum()]))]
    A = np.abs
    # |dy| plus the size of y's own rounding terms (the residual y - t can be
    # far smaller than y, so an error in y is not bounded by |dy|)
    _, _, ya = forward_bf16(p, x)
    ady = A(dy) + ya / n
    az3 = ady[:, None] * A(W4[0])[None, :] * A(1.0 - h3 ** 2)
    az2 = (az3 @ A(W3)) * A(1.0 - h2 ** 2)
    az1 = (az2 @ A(W2)) * A(1.0 - h1 ** 2)
    a = [(az1.T @ A(x), az1.sum(0)), (az2.T @ A(h1), az2.sum(0)), (az3.T @ A(h2), az3.sum(0)),
         (ady[None, :] @ A(h3), np.array([ady.sum()]))]

    def flat(gs):
        return np.concatenate([np.concatenate([dW.ravel(), db.ravel()]) for dW, db in gs])

    return flat(g), flat(a)
