"""Pins for the FP64 oracle of the learned TDoA head (an extension, not in the
paper): the analytic gradient against central differences, closed forms of the
forward pass and of Adam's steps, and bfloat16 rounding."""
import math

import numpy as np
import pytest


@pytest.fixture(scope="module")
def O():
    from oracle import oracle
    oracle.build()
    return oracle


def _params(O, nin, H, seed, scale=0.3):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(O.mlp_nparams(nin, H)) * scale


def test_gradient_matches_central_differences(O):
    nin, H, n = 5, 7, 9
    rng = np.random.default_rng(1)
    p = _params(O, nin, H, 2)
    x = rng.standard_normal((n, nin))
    t = rng.uniform(-3, 3, n)
    tf = t + rng.normal(0, 0.5, n)
    loss, g = O.mlp_loss_grad(x, p, t, tf, nin, H, 0.3)
    h = 1e-6
    for k in rng.choice(len(p), 60, replace=False):
        e = np.zeros_like(p)
        e[k] = h
        lp, _ = O.mlp_loss_grad(x, p + e, t, tf, nin, H, 0.3)
        lm, _ = O.mlp_loss_grad(x, p - e, t, tf, nin, H, 0.3)
        num = (lp - lm) / (2 * h)
        assert abs(num - g[k]) <= 1e-6 * max(1.0, abs(num)), (k, num, g[k])


def test_forward_closed_forms(O):
    nin, H = 3, 4
    n_p = O.mlp_nparams(nin, H)
    assert n_p == H * nin + H + H * H + H + 2 * H + 2
    p = np.zeros(n_p)
    p[-2:] = [0.25, -1.5]  # b3
    y = O.mlp_forward(np.ones((2, nin)), p, nin, H)
    assert np.allclose(y, [[0.25, -1.5]] * 2)
    # one path through unit weights: y0 = gelu(gelu(1)), gelu(a) = a Phi(a)
    p = np.zeros(n_p)
    W1 = p[: H * nin].reshape(H, nin)
    W1[0, 0] = 1.0
    o = H * nin + H
    W2 = p[o: o + H * H].reshape(H, H)
    W2[0, 0] = 1.0
    o += H * H + H
    p[o] = 1.0  # W3[0, 0]
    y = O.mlp_forward(np.array([[1.0, 0.0, 0.0]]), p, nin, H)
    phi = lambda a: 0.5 * (1 + math.erf(a / math.sqrt(2)))
    g1 = 1.0 * 0.8413447460685429  # Phi(1) from the standard normal table
    assert abs(g1 - 1.0 * phi(1.0)) < 1e-15
    assert abs(y[0, 0] - g1 * phi(g1)) < 1e-14
    assert y[0, 1] == 0.0


def test_adam_first_step_is_signed_lr(O):
    p = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 1e-3])
    m, v = np.zeros(3), np.zeros(3)
    O.adam(p, g, m, v, 1, 0.01, eps=0.0)
    assert np.allclose(p, [1.0 - 0.01, -2.0 + 0.01, 0.5 - 0.01], atol=1e-15)


def test_round_bf16(O):
    vals = np.array([1.0, 1.00390625, 1.0078125, 3.14159265, -2.5e-3, 65504.0])
    r = O.round_bf16(vals)
    # bf16 keeps 8 significant bits: 1 + 2^-8 is a tie that rounds to the even 1.0
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0078125
    assert r[3] == 3.140625
    assert np.all(np.abs(r - vals) <= np.abs(vals) * 2.0 ** -8)


def test_adam_constant_gradient_moves_signed_lr_every_step(O):
    # With a constant gradient g the moments are m_t = (1 - b1^t) g and
    # v_t = (1 - b2^t) g^2, so the bias-corrected ratio is exactly g / |g| and
    # every step (eps = 0) moves each parameter by lr * sign(g).  An Adam that
    # forgets its moments between steps, or corrects the bias with the wrong
    # power of beta, moves by a different amount from step 2 on.
    g = np.array([0.3, -4.0, 1e-3, -7e-5])
    p0 = np.array([1.0, -2.0, 0.5, 3.0])
    p = p0.copy()
    m, v = np.zeros(4), np.zeros(4)
    lr = 0.01
    for step in range(1, 11):
        before = p.copy()
        O.adam(p, g, m, v, step, lr, eps=0.0)
        assert np.allclose(before - p, lr * np.sign(g), rtol=0, atol=1e-14), step
        assert np.allclose(m, (1 - 0.9 ** step) * g, rtol=1e-13, atol=0), step
        assert np.allclose(v, (1 - 0.999 ** step) * g * g, rtol=1e-13, atol=0), step
    assert np.allclose(p, p0 - 10 * lr * np.sign(g), rtol=0, atol=1e-13)
