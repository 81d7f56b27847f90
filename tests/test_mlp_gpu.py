"""The surrogate network's kernels against the FP64 reference.

Forward outputs and gradients of lbm_mlp_* are compared with
oracle/mlp_ref.py evaluated with the same BF16 operand rounding (what is
left is the FP32 accumulation order, and the rare operand that FP32 and
FP64 round to neighbouring BF16 values) and, more loosely, with exact FP64
operands (the BF16 rounding itself).  Batches are ragged (not multiples of
the 64-row GEMM tile) and one shape has widths that are not multiples of
the tile either."""
import numpy as np
import pytest

from oracle import mlp_ref as R

pytestmark = pytest.mark.gpu


def _setup():
    import __graft_entry__
    __graft_entry__.build()
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1309_6726_gb300 import mlp
    return torch, mlp


def _init(rng, shapes):
    ws = [rng.uniform(-1, 1, s) * np.sqrt(6.0 / (s[0] + s[1])) for s in shapes]
    bs = [rng.uniform(-0.1, 0.1, s[0]) for s in shapes]
    # the GPU keeps FP32 master weights
    ws = [w.astype(np.float32).astype(np.float64) for w in ws]
    bs = [b.astype(np.float32).astype(np.float64) for b in bs]
    return ws, bs


@pytest.mark.parametrize("n_in,n_hidden,n_layers,n_out,batch",
                         [(4, 256, 3, 65, 1000), (3, 48, 2, 5, 77)])
def test_forward_and_gradient_match_the_fp64_reference(n_in, n_hidden,
                                                       n_layers, n_out,
                                                       batch):
    torch, mlp = _setup()
    rng = np.random.default_rng(7)
    shapes = mlp.layer_shapes(n_in, n_hidden, n_layers, n_out)
    ws, bs = _init(rng, shapes)
    x = rng.uniform(-1, 1, (batch, n_in)).astype(np.float32)
    t = rng.standard_normal((batch, n_out)).astype(np.float32)
    t[::7, 0] = np.nan
    net = mlp.Mlp(n_in, n_hidden, n_layers, n_out, max_batch=batch + 5)
    net.set_params(mlp.pack(ws, bs))
    np.testing.assert_array_equal(net.params(), mlp.pack(ws, bs))
    dev = torch.device("cuda", 0)
    xd = torch.from_numpy(x).to(dev)
    td = torch.from_numpy(t).to(dev)
    y = net.forward(xd).cpu().numpy().astype(np.float64)
    _, y_bf = R.forward(ws, bs, x, bf16=True)
    _, y_64 = R.forward(ws, bs, x, bf16=False)
    scale = np.abs(y_bf).max()
    # What is left is the FP32 accumulation order, except where an FP32
    # activation and its FP64 counterpart fall on two sides of a BF16
    # rounding boundary: one operand then differs by a BF16 unit (2^-8
    # relative).  That happens to a few percent of the rows (768 rounded
    # activations each) and moves all outputs of the row a little.
    dev_err = np.abs(y - y_bf)
    assert np.median(dev_err) < 1e-6 * scale
    assert np.mean(dev_err < 2e-5 * scale) > 0.9
    assert dev_err.max() < 2e-3 * scale
    # the median also on the first and on the last (ragged) tile of 64 rows
    # of the product kernel alone: a mistake confined to one tile moves
    # every output of its rows and cannot hide among the other rows there
    # (boundary flips touch a few rows, not the median)
    tail = batch % 64 or 64
    for part in (dev_err[:64], dev_err[-tail:]):
        assert np.median(part) < 1e-6 * scale
    # the BF16 operand rounding itself: about 1 percent of the output scale
    assert np.abs(y - y_64).max() < 5e-2 * scale

    g, loss = net.grad(xd, td)
    g = g.cpu().numpy().astype(np.float64)
    loss_bf, g_bf = R.loss_grad(ws, bs, x, t, bf16=True)
    loss_64, g_64 = R.loss_grad(ws, bs, x, t, bf16=False)
    assert loss == pytest.approx(loss_bf, rel=1e-5)
    gs = np.abs(g_bf).max()
    gerr = np.abs(g - g_bf)
    assert np.median(gerr) < 1e-5 * gs
    assert np.mean(gerr < 1e-4 * gs) > 0.9
    assert gerr.max() < 5e-3 * gs
    assert np.abs(g - g_64).max() < 5e-2 * gs
    # the weights did not move
    np.testing.assert_array_equal(net.params(), mlp.pack(ws, bs))
    net.close()


def test_adam_steps_match_a_reference_update_and_reduce_the_loss():
    torch, mlp = _setup()
    rng = np.random.default_rng(11)
    n_in, H, L, n_out, batch = 4, 64, 2, 8, 300
    shapes = mlp.layer_shapes(n_in, H, L, n_out)
    ws, bs = _init(rng, shapes)
    x = rng.uniform(-1, 1, (batch, n_in)).astype(np.float32)
    # a smooth target family: y_j = sin(j * (x . a) + x_0)
    a = rng.standard_normal(n_in)
    t = np.sin(np.outer(x @ a, np.arange(1, n_out + 1) * 0.5) +
               x[:, :1]).astype(np.float32)
    net = mlp.Mlp(n_in, H, L, n_out, max_batch=batch)
    theta0 = mlp.pack(ws, bs)
    net.set_params(theta0)
    dev = torch.device("cuda", 0)
    xd, td = torch.from_numpy(x).to(dev), torch.from_numpy(t).to(dev)
    # first step: Adam from zero moments moves each weight by lr * g/|g|
    g0, _ = net.grad(xd, td)
    g0 = g0.cpu().numpy().astype(np.float64)
    lr = 1e-3
    loss0 = net.train_step(xd, td, lr, want_loss=True)
    th1 = net.params().astype(np.float64)
    expect = theta0 - lr * g0 / (np.abs(g0) + 1e-8)
    np.testing.assert_allclose(th1, expect, atol=2e-6)
    for _ in range(400):
        net.train_step(xd, td, 3e-3)
    loss1 = net.train_step(xd, td, 3e-3, want_loss=True)
    assert loss1 < 0.1 * loss0
    net.close()
