"""Pins of the FP64 reference of the surrogate network (oracle/mlp_ref.py),
checked against things other than itself: BF16 rounding of known bit
patterns and torch's own BF16 conversion, a one-unit network worked out by
hand, and central finite differences of the loss."""
import math

import numpy as np
import pytest

from oracle import mlp_ref as R


def test_bf16_round_known_values_and_ties_to_even():
    # BF16 spacing just above 1 is 2^-7
    assert R.bf16_round(1.0) == 1.0
    assert R.bf16_round(1.0 + 2.0 ** -7) == 1.0 + 2.0 ** -7
    assert R.bf16_round(1.0 + 2.0 ** -8) == 1.0            # tie -> even
    assert R.bf16_round(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6  # tie -> even
    assert R.bf16_round(1.0 + 2.0 ** -8 + 2.0 ** -20) == 1.0 + 2.0 ** -7
    assert R.bf16_round(-2.5) == -2.5
    assert R.bf16_round(0.0) == 0.0


def test_bf16_round_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    a = np.concatenate([rng.standard_normal(5000) * 10.0 ** rng.integers(-6, 6, 5000),
                        rng.standard_normal(100)])
    t = torch.tensor(a.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(R.bf16_round(a), t)


def test_one_unit_network_by_hand():
    # y = v tanh(w x + b) + c;  loss = (y - t)^2 (one entry)
    w, b, v, c = 0.7, -0.2, 1.3, 0.1
    x, t = 0.5, 0.4
    ws = [np.array([[w]]), np.array([[v]])]
    bs = [np.array([b]), np.array([c])]
    acts, y = R.forward(ws, bs, np.array([[x]]))
    h = math.tanh(w * x + b)
    assert y[0, 0] == pytest.approx(v * h + c, abs=1e-15)
    loss, g = R.loss_grad(ws, bs, np.array([[x]]), np.array([[t]]))
    r = v * h + c - t
    assert loss == pytest.approx(r * r, abs=1e-15)
    dz = 2 * r * v * (1 - h * h)
    # packed order: W1, b1, W2, b2
    np.testing.assert_allclose(g, [dz * x, dz, 2 * r * h, 2 * r], atol=1e-15)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(1)
    shapes = [(5, 3), (5, 5), (4, 5)]
    ws = [rng.standard_normal(s) * 0.7 for s in shapes]
    bs = [rng.standard_normal(s[0]) * 0.3 for s in shapes]
    x = rng.standard_normal((7, 3))
    t = rng.standard_normal((7, 4))
    t[2, 1] = np.nan  # left out of the loss
    t[5, 3] = np.nan
    loss, g = R.loss_grad(ws, bs, x, t)
    theta = np.concatenate([p.ravel() for wb in zip(ws, bs) for p in wb])

    def loss_at(th):
        o, w2, b2 = 0, [], []
        for s in shapes:
            w2.append(th[o:o + s[0] * s[1]].reshape(s))
            o += s[0] * s[1]
            b2.append(th[o:o + s[0]])
            o += s[0]
        return R.loss_grad(w2, b2, x, t)[0]

    eps = 1e-6
    fd = np.empty_like(theta)
    for i in range(theta.size):
        e = np.zeros_like(theta)
        e[i] = eps
        fd[i] = (loss_at(theta + e) - loss_at(theta - e)) / (2 * eps)
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-9)
    assert loss == pytest.approx(loss_at(theta), abs=0)


def test_nan_targets_leave_the_gradient_unchanged():
    rng = np.random.default_rng(2)
    ws = [rng.standard_normal((6, 2)), rng.standard_normal((3, 6))]
    bs = [rng.standard_normal(6), rng.standard_normal(3)]
    x = rng.standard_normal((4, 2))
    t = rng.standard_normal((4, 3))
    t2 = t.copy()
    t2[1, :] = np.nan
    # dropping row 1's targets = same gradient as a target equal to y there
    _, y = R.forward(ws, bs, x)
    t3 = t.copy()
    t3[1, :] = y[1, :]
    np.testing.assert_allclose(R.loss_grad(ws, bs, x, t2)[1],
                               R.loss_grad(ws, bs, x, t3)[1], atol=1e-15)
