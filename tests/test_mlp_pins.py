"""Pins of the warm-start network's CPU reference (oracle/mlp.py) that do not
restate its own formulas: closed forms of Adam (Kingma & Ba, 2015) that follow
from the bias correction, the bfloat16 rounding against a library conversion,
and the BF16-operand network against the FP64 one within the BF16 error."""
import numpy as np
import pytest

from oracle import mlp as M


def _features(n, seed):
    rng = np.random.default_rng(seed)
    return np.stack([rng.integers(0, 2, n), 16.0 / rng.choice([8, 16, 32, 64], n), rng.choice([0.30103, 1.0], n),
                     rng.uniform(-2, 2, n), rng.uniform(0, 1, n)], axis=1)


def test_adam_first_step_is_the_normalised_gradient():
    """With zero moments the bias-corrected moments of step 1 are g and g^2,
    so the step is -lr g / (|g| + eps) whatever the gradient's scale; without
    the correction it would be 0.1 / sqrt(0.001) = 3.16 times larger, and with
    eps under the square root tiny gradients would barely move."""
    rng = np.random.default_rng(0)
    g = rng.normal(size=4000) * np.logspace(-12, 6, 4000)
    p = rng.normal(size=4000)
    lr = 1e-3
    p1, m1, v1 = M.adam_step(p, np.zeros_like(p), np.zeros_like(p), g, 1, lr)
    expect = -lr * g / (np.abs(g) + 1e-8)
    assert np.allclose(p1 - p, expect, rtol=1e-9, atol=1e-15)
    # a gradient ten times below eps moves by lr / 11
    q1, _, _ = M.adam_step(np.zeros(1), np.zeros(1), np.zeros(1), np.array([1e-9]), 1, lr)
    assert q1[0] == pytest.approx(-lr / 11.0, rel=1e-9)


def test_adam_constant_gradient_moves_lr_every_step():
    """A constant gradient g gives m_k = (1 - b1^k) g and v_k = (1 - b2^k) g^2,
    so every bias-corrected step is -lr sign(g) (up to eps) -- steps 2 and 3
    pin the correction's powers of the betas."""
    g = np.array([3.0, -0.25, 1e-4, -7e3])
    p, m, v = np.zeros(4), np.zeros(4), np.zeros(4)
    lr = 0.01
    for k in range(1, 6):
        p_new, m, v = M.adam_step(p, m, v, g, k, lr)
        assert np.allclose(p_new - p, -lr * g / (np.abs(g) + 1e-8), rtol=1e-9, atol=0)
        p = p_new


def test_adam_alternating_gradient_worked_example():
    """g, then -g: m_2 = 0.1 (0.9 g - g) = -0.01 g and 1 - 0.9^2 = 0.19, so the
    corrected first moment is -g / 19; v_2 = 0.001 (0.999 + 1) g^2 and
    1 - 0.999^2 = 0.001999, so the corrected second moment is g^2: the second
    step is +lr sign(g) / 19."""
    g = np.array([2.0, -0.5])
    lr = 0.1
    p1, m, v = M.adam_step(np.zeros(2), np.zeros(2), np.zeros(2), g, 1, lr)
    p2, _, _ = M.adam_step(p1, m, v, -g, 2, lr)
    assert np.allclose(p2 - p1, lr * np.sign(g) / 19.0, rtol=1e-7)


def test_adam_is_invariant_to_gradient_scale():
    rng = np.random.default_rng(3)
    gs = [rng.normal(size=50) for _ in range(4)]
    for c in (1e-2, 1e4):
        pa = pb = np.zeros(50)
        ma = va = mb = vb = np.zeros(50)
        for k, g in enumerate(gs, 1):
            pa, ma, va = M.adam_step(pa, ma, va, g, k, 0.01)
            pb, mb, vb = M.adam_step(pb, mb, vb, c * g, k, 0.01)
        assert np.allclose(pa, pb, rtol=2e-4, atol=1e-9)   # eps = 1e-8 against |c g| >= ~1e-5


def test_round_bf16_matches_library_conversion():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(5)
    x = rng.normal(size=200000) * np.logspace(-35, 35, 200000)
    ref = torch.tensor(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(M.round_bf16(x), ref)
    # ties go to the even significand: 1 + 2^-8 -> 1, 1 + 3 * 2^-8 -> 1 + 2^-6
    assert M.round_bf16(np.array([1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8])).tolist() == [1.0, 1 + 2.0 ** -6]


def test_bf16_network_within_bfloat16_error_of_fp64():
    """Every rounded operand carries a relative error of at most 2^-9; a few of
    them in sequence stay far inside 2^-6 of the sum of absolute terms."""
    p = M.init_params(3)
    x = _features(1024, 1)
    t = 0.3 * np.sin(2 * x[:, 3])
    y, _ = M.forward(p, x)
    yb, _, ya = M.forward_bf16(p, x)
    assert np.all(np.abs(yb - y) <= 2.0 ** -6 * ya)
    g = M.gradient(p, x, t)
    gb, a = M.gradient_bf16(p, x, t)
    assert np.all(np.abs(gb - g) <= 2.0 ** -6 * a)
    # and the rounding is not a no-op
    assert np.max(np.abs(gb - g)) > 0
