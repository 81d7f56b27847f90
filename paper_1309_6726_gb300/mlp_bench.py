"""Timing of the surrogate network's kernels (forward, back-propagation,
Adam) at the surrogate's shape on random data, one JSON line:
``python -m paper_1309_6726_gb300.mlp_bench [--steps N] ...``."""
from __future__ import annotations

import numpy as np

from .mlp import Mlp, layer_shapes, pack


def main(argv=None):
    """Times the network's kernels at the surrogate's shape on random data:
    training steps (forward, back-propagation, Adam) at one batch size and
    inference at another; prints one JSON line."""
    import argparse
    import json
    import time
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--batch", type=int, default=1024)
    ap.add_argument("--infer-batch", type=int, default=8192)
    ap.add_argument("--steps", type=int, default=200)
    args = ap.parse_args(argv)
    import __graft_entry__
    __graft_entry__.build()
    n_in, H, L, n_out = 5, 256, 3, 65  # the surrogate's shape
    net = Mlp(n_in, H, L, n_out, max(args.batch, args.infer_batch))
    rng = np.random.default_rng(0)
    ws = [rng.uniform(-1, 1, s) * np.sqrt(3.0 / s[1])
          for s in layer_shapes(n_in, H, L, n_out)]
    net.set_params(pack(ws, [np.zeros(s[0]) for s in layer_shapes(n_in, H, L, n_out)]))
    dev = torch.device("cuda", 0)
    x = torch.rand((args.batch, n_in), device=dev) * 2 - 1
    t = torch.rand((args.batch, n_out), device=dev)
    xi = torch.rand((args.infer_batch, n_in), device=dev) * 2 - 1
    for _ in range(10):
        net.train_step(x, t, 1e-4)
        net.forward(xi)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        net.train_step(x, t, 1e-4)
    torch.cuda.synchronize()
    t_train = (time.perf_counter() - t0) / args.steps
    t0 = time.perf_counter()
    for _ in range(args.steps):
        net.forward(xi)
    torch.cuda.synchronize()
    t_inf = (time.perf_counter() - t0) / args.steps
    macs = n_in * H + (L - 1) * H * H + H * n_out  # per sample, forward
    print(json.dumps({
        "shape": [n_in, H, L, n_out], "train_batch": args.batch,
        "train_step_ms": 1e3 * t_train,
        "train_tflops": 3 * 2 * macs * args.batch / t_train / 1e12,
        "infer_batch": args.infer_batch, "infer_ms": 1e3 * t_inf,
        "infer_tflops": 2 * macs * args.infer_batch / t_inf / 1e12}))
    net.close()


if __name__ == "__main__":
    main()
