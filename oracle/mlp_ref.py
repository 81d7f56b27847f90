"""FP64 reference of the surrogate network (test infrastructure only).

Plain numpy in float64: the forward pass of the tanh perceptron that the
library's kernels run, the mean-squared-error loss with NaN targets left
out, and back-propagation written out layer by layer from the chain rule.
With ``bf16=True`` every operand of a matrix product is rounded to BF16
first -- weights, activations and back-propagated gradients, exactly where
the GPU path rounds them -- so that the two differ only by the order of
the FP32 accumulation.

Nothing here is used by the product path; the network is not part of the
paper (it learns the solver's trajectories).  Pinned by
tests/test_mlp_ref.py: finite differences of the loss, a network small
enough to evaluate by hand, and the BF16 rounding of known bit patterns.
"""
from __future__ import annotations

import numpy as np


def bf16_round(a) -> np.ndarray:
    """Rounds to the nearest BF16 value (ties to even), returned as float64.

    BF16 keeps the top 16 bits of an IEEE float32; rounding adds half of
    the dropped part's unit, plus one if the kept part is odd, before
    truncating (finite inputs)."""
    f = np.asarray(a, np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _op(a, bf16: bool):
    return bf16_round(a) if bf16 else np.asarray(a, np.float64)


def forward(ws, bs, x, bf16: bool = False):
    """Activations [x, h_1, .., h_L] and the output y (all float64)."""
    acts = [np.asarray(x, np.float64)]
    h = acts[0]
    L = len(ws) - 1
    for l, (w, b) in enumerate(zip(ws, bs)):
        z = _op(h, bf16) @ _op(w, bf16).T + np.asarray(b, np.float64)
        if l < L:
            h = np.tanh(z)
            acts.append(h)
        else:
            y = z
    return acts, y


def loss_and_dy(y, t):
    """Mean of (y - t)^2 over all entries, NaN targets contributing zero;
    and its gradient with respect to y."""
    t = np.asarray(t, np.float64)
    n = y.size
    d = np.where(np.isnan(t), 0.0, y - np.nan_to_num(t))
    return float((d * d).sum() / n), 2.0 * d / n


def backward(ws, acts, dy, bf16: bool = False):
    """Gradients (dW_l, db_l) per layer, from dL/dy."""
    L = len(ws) - 1
    gw, gb = [None] * (L + 1), [None] * (L + 1)
    dz = dy
    for l in range(L, -1, -1):
        gw[l] = _op(dz, bf16).T @ _op(acts[l], bf16)
        gb[l] = dz.sum(axis=0)
        if l > 0:
            dh = _op(dz, bf16) @ _op(ws[l], bf16)
            dz = dh * (1.0 - acts[l] ** 2)  # tanh' = 1 - tanh^2
    return gw, gb


def loss_grad(ws, bs, x, t, bf16: bool = False):
    """(loss, packed gradient) in the library's parameter order."""
    acts, y = forward(ws, bs, x, bf16)
    loss, dy = loss_and_dy(y, t)
    gw, gb = backward(ws, acts, dy, bf16)
    parts = []
    for w, b in zip(gw, gb):
        parts += [w.ravel(), b.ravel()]
    return loss, np.concatenate(parts)
