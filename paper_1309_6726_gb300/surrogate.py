"""A learned surrogate of the batched reactive solver (not part of the paper).

The network of lbm_mlp.h maps the parameters of one capillary run --
width W, reaction rate k_r, adhesion strength g_ads, viscosity ratio
tau_A / tau_B, and the capillary length L -- to its infiltration curve,
the front position z at 64 log-spaced times, and to its pore-closure time.
It is trained on trajectories that the batched lattice Boltzmann solver
generates (the members of a training set advance together in persistent
launches, one per step), and the solver stays the reference its error is
measured against on held-out parameters and the fallback for parameters
outside the training domain.

Parameters are drawn as in the batched sweep (W uniform over 16-128, L
uniform over 1024-4096, k_r log-uniform on [1e-5, 1e-2], contact angle
uniform on [20, 60] degrees mapped to g_ads by the calibrated table,
tau_A / tau_B uniform on [0.6, 1.5]) with the sweep's 64-column A
reservoir and 32-column outlet band.  The sweep draws L, so L is the fifth
input (Washburn's front speed scales as 1 / L, Eq. 1); a surrogate trained
on one length (a length range of one value) sees that input as constant.
The horizon is fixed for a surrogate.

    python -m paper_1309_6726_gb300.surrogate [--train 4096] [--held-out 256]
        [--length-min 1024] [--length-max 4096] [--steps 40000]
        [--ensemble 5] [--fit-steps 16000]

prints one JSON line with the dataset cost, the fit and the errors against
the solver.
"""
from __future__ import annotations

import argparse
import json
import math
import time
from dataclasses import dataclass

import numpy as np

from . import inputs as I

N_TIMES = 64
T_FIRST = 100
Z_SCALE = 10.0  # front targets are asinh(z / Z_SCALE)

W_RANGE = (16, 128)
K_RANGE = (1e-5, 1e-2)
THETA_RANGE = (20.0, 60.0)
RATIO_RANGE = (0.6, 1.5)
L_RANGE = (1024, 4096)
N_IN = 5  # W, log10 k_r, g_ads, tau ratio, L


def time_grid(t_max: int, n: int = N_TIMES, t_first: int = T_FIRST) -> np.ndarray:
    """n strictly increasing integer steps, log-spaced from t_first to t_max
    (both included).  Where rounding merges neighbours (a narrow range),
    they are pushed apart within [t_first, t_max]; ValueError when fewer
    than n integers lie in that range."""
    if n < 2 or t_first < 1 or t_max - t_first + 1 < n:
        raise ValueError("time_grid: need n >= 2 integers in [t_first, t_max]")
    t = np.round(np.geomspace(t_first, t_max, n)).astype(np.int64)
    t[0], t[-1] = t_first, t_max
    for i in range(1, n):  # strictly increasing from the bottom ...
        t[i] = max(t[i], t[i - 1] + 1)
    t[-1] = t_max
    for i in range(n - 2, -1, -1):  # ... and back under t_max from the top
        t[i] = min(t[i], t[i + 1] - 1)
    return t


def draw_members(count: int, seed: int, length=L_RANGE):
    """Run parameters drawn as in the batched sweep; `length` is a fixed
    capillary length or a (min, max) range drawn uniformly over integers."""
    lo, hi = (length, length) if isinstance(length, int) else length
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        w = int(rng.integers(W_RANGE[0], W_RANGE[1] + 1))
        k = float(10 ** rng.uniform(math.log10(K_RANGE[0]), math.log10(K_RANGE[1])))
        th = float(rng.uniform(*THETA_RANGE))
        tr = float(rng.uniform(*RATIO_RANGE))
        length_k = int(rng.integers(lo, hi + 1))
        out.append(I.SweepMember(w, length_k, k, th, tr))
    return out


def _g_range():
    # g_ads decreases as the contact angle grows
    a, b = I.g_ads_for_angle(THETA_RANGE[1]), I.g_ads_for_angle(THETA_RANGE[0])
    return min(a, b), max(a, b)


def _l_range(length):
    return (length, length) if isinstance(length, int) else tuple(length)


def features(members, length=L_RANGE) -> np.ndarray:
    """Network inputs in [-1, 1]: W, log10 k_r, g_ads, tau ratio and L over
    the length range (0 when the range is a single length)."""
    g0, g1 = _g_range()
    lk0, lk1 = math.log10(K_RANGE[0]), math.log10(K_RANGE[1])
    l0, l1 = _l_range(length)
    rows = []
    for m in members:
        g = I.g_ads_for_angle(m.theta_deg)
        rows.append([
            2 * (m.width - W_RANGE[0]) / (W_RANGE[1] - W_RANGE[0]) - 1,
            2 * (math.log10(m.k_r) - lk0) / (lk1 - lk0) - 1,
            2 * (g - g0) / (g1 - g0) - 1,
            2 * (m.tau_ratio - RATIO_RANGE[0]) / (RATIO_RANGE[1] - RATIO_RANGE[0]) - 1,
            0.0 if l1 == l0 else 2 * (m.length - l0) / (l1 - l0) - 1,
        ])
    return np.asarray(rows, np.float32)


def in_domain(members, length=L_RANGE) -> np.ndarray:
    """True where a run's parameters lie inside the training domain (the
    parameter box and the length range)."""
    l0, l1 = _l_range(length)
    f = features(members, length)
    ok = np.all(np.abs(f[:, :4]) <= 1.0 + 1e-6, axis=1)
    return ok & np.array([l0 <= m.length <= l1 for m in members])


def run_trajectories(members, t_grid, precision: str = "fp32",
                     chunk: int = 1024):
    """Advances the members on the GPU, `chunk` of them together in one
    batch, and records the front position at each time of t_grid and the
    closure step (-1: none)."""
    import torch
    from . import lbm
    z = np.full((len(members), len(t_grid)), np.nan)
    closure = np.full(len(members), -1, np.int64)
    bad = np.zeros(len(members), bool)
    nodes = 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for c0 in range(0, len(members), chunk):
        part = members[c0:c0 + chunk]
        pairs = [I.sweep_lattice(m) for m in part]
        s = lbm.Solver([g for g, _ in pairs], [p for _, p in pairs], precision)
        done = 0
        for j, t in enumerate(t_grid):
            s.step(int(t) - done)
            done = int(t)
            obs = s.observables(allow_nan=True)
            z[c0:c0 + len(part), j] = [o["front"] for o in obs]
        closure[c0:c0 + len(part)] = [o["closure_step"] for o in obs]
        bad[c0:c0 + len(part)] = [bool(o["nonfinite"]) for o in obs]
        nodes += sum(int((g.solid == 0).sum()) for g, _ in pairs)
        s.close()
    torch.cuda.synchronize()
    seconds = time.perf_counter() - t0
    z[bad] = np.nan
    return {"z": z, "closure": closure, "nonfinite": bad, "seconds": seconds,
            "fluid_nodes": nodes, "steps": int(t_grid[-1])}


def _log_tmax(t_max):
    return math.log10(t_max)


def targets(z, closure, t_max) -> np.ndarray:
    """Network targets: asinh(z / Z_SCALE) at each time (close to the
    relative error for fronts beyond Z_SCALE, the absolute one below it:
    the error measure of compare_to_solver), then the closure time as
    log10(t) / log10(t_max),
    or (log10(t_max) + 0.3) / log10(t_max) when the run did not close
    within t_max.  NaN marks what is unknown."""
    lt = _log_tmax(t_max)
    c = np.where(closure > 0, np.log10(np.maximum(closure, 1)) / lt,
                 (lt + 0.3) / lt)
    y = np.concatenate([np.arcsinh(z / Z_SCALE), c[:, None]],
                       axis=1).astype(np.float32)
    bad = np.all(np.isnan(z), axis=1)
    y[bad, -1] = np.nan
    return y


def decode(y, t_max):
    """(front [n, times] in lattice units, closure step or -1)."""
    lt = _log_tmax(t_max)
    z = np.sinh(y[:, :-1].astype(np.float64)) * Z_SCALE
    lc = y[:, -1].astype(np.float64) * lt
    closure = np.where(lc < lt + 0.15, np.round(10 ** np.minimum(lc, lt)), -1)
    return z, closure.astype(np.int64)


def spread_of(ys, t_max) -> np.ndarray:
    """Disagreement of an ensemble per run, in the units of the front error
    (compare_to_solver): the mean over the times of the members' standard
    deviation of the front, over the mean predicted front at the last time
    (at least 10 lattice units).  ys: (members, runs, outputs)."""
    zs = np.stack([decode(y, t_max)[0] for y in ys])
    scale = np.maximum(zs.mean(axis=0)[:, -1], 10.0)
    return zs.std(axis=0).mean(axis=1) / scale


def compare_to_solver(z_pred, c_pred, z_lb, c_lb, t_max):
    """Errors of the surrogate against the solver on the same runs.

    Front: per run, the mean over the times of |z_pred - z_lb| divided by
    the solver's last front position (at least 10 lattice units).
    Closure: the relative error of the closure time where both close, and
    the share of runs where they agree on closing within t_max at all."""
    ok = ~np.all(np.isnan(z_lb), axis=1)
    scale = np.maximum(np.nan_to_num(z_lb[:, -1]), 10.0)
    err = np.array([np.nanmean(np.abs(z_pred[i] - z_lb[i])) / scale[i]
                    for i in np.flatnonzero(ok)])
    both = (c_pred > 0) & (c_lb > 0) & ok
    cerr = np.abs(c_pred[both] / c_lb[both] - 1.0)
    agree = np.mean((c_pred[ok] > 0) == (c_lb[ok] > 0)) if ok.any() else float("nan")
    q = lambda a, p: float(np.percentile(a, p)) if a.size else None
    return {
        "runs": int(ok.sum()),
        "front_rel_err_mean": float(err.mean()) if err.size else None,
        "front_rel_err_median": q(err, 50),
        "front_rel_err_p90": q(err, 90),
        "front_within_2pct": float(np.mean(err <= 0.02)) if err.size else None,
        "closure_runs_both": int(both.sum()),
        "closure_rel_err_mean": float(cerr.mean()) if cerr.size else None,
        "closure_rel_err_median": q(cerr, 50),
        "closure_within_2pct": float(np.mean(cerr <= 0.02)) if cerr.size else None,
        "closure_agreement": float(agree),
    }


@dataclass
class FitLog:
    steps: int
    seconds: float
    first_loss: float
    last_loss: float


class Surrogate:
    """An ensemble of networks (5 inputs, 3 x 256 tanh, 65 outputs) on the
    GPU, each from its own initialisation and minibatch order; the
    prediction is their mean."""

    def __init__(self, hidden: int = 256, layers: int = 3, seed: int = 0,
                 max_batch: int = 8192, members: int = 1):
        from . import mlp
        self.nets = []
        for k in range(members):
            net = mlp.Mlp(N_IN, hidden, layers, N_TIMES + 1, max_batch)
            rng = np.random.default_rng([seed, k])
            ws, bs = [], []
            for r, c in mlp.layer_shapes(N_IN, hidden, layers, N_TIMES + 1):
                lim = math.sqrt(6.0 / (r + c))  # Glorot uniform
                ws.append(rng.uniform(-lim, lim, (r, c)))
                bs.append(np.zeros(r))
            net.set_params(mlp.pack(ws, bs))
            self.nets.append(net)

    @property
    def net(self):
        return self.nets[0]

    def fit(self, x, y, steps: int = 20000, batch: int = 512,
            lr: float = 2e-3, lr_end: float = 1e-5, seed: int = 0) -> FitLog:
        """Adam on minibatches with a cosine learning-rate decay, for each
        member of the ensemble; the log reports the mean losses."""
        import torch
        dev = torch.device("cuda", torch.cuda.current_device())
        xd = torch.from_numpy(np.ascontiguousarray(x, np.float32)).to(dev)
        yd = torch.from_numpy(np.ascontiguousarray(y, np.float32)).to(dev)
        n = xd.shape[0]
        batch = min(batch, n)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        firsts, lasts = [], []
        for m, net in enumerate(self.nets):
            g = torch.Generator(device="cpu").manual_seed(seed * 1000 + m)
            firsts.append(net.train_step(xd[:batch].contiguous(),
                                         yd[:batch].contiguous(), lr,
                                         want_loss=True))
            order = torch.randperm(n, generator=g).to(dev)
            pos = 0
            for k in range(1, steps):
                if pos + batch > n:
                    order = torch.randperm(n, generator=g).to(dev)
                    pos = 0
                idx = order[pos:pos + batch]
                pos += batch
                a = lr_end + 0.5 * (lr - lr_end) * (1 + math.cos(math.pi * k / steps))
                net.train_step(xd.index_select(0, idx), yd.index_select(0, idx), a)
            lasts.append(net.grad(xd, yd)[1] if n <= net.max_batch else float("nan"))
        torch.cuda.synchronize()
        return FitLog(steps * len(self.nets), time.perf_counter() - t0,
                      float(np.mean(firsts)), float(np.mean(lasts)))

    def predict(self, x) -> np.ndarray:
        import torch
        dev = torch.device("cuda", torch.cuda.current_device())
        xd = torch.from_numpy(np.ascontiguousarray(x, np.float32)).to(dev)
        out = self.nets[0].forward(xd)
        for net in self.nets[1:]:
            out += net.forward(xd)
        return (out / len(self.nets)).cpu().numpy()

    def predict_with_spread(self, x, t_max):
        """The mean prediction and, per run, the members' disagreement
        (spread_of)."""
        import torch
        dev = torch.device("cuda", torch.cuda.current_device())
        xd = torch.from_numpy(np.ascontiguousarray(x, np.float32)).to(dev)
        ys = np.stack([net.forward(xd).cpu().numpy() for net in self.nets])
        return self.predict(x), spread_of(ys, t_max)

    def params(self):
        return [net.params() for net in self.nets]

    def close(self):
        for net in self.nets:
            net.close()


def predict_or_solve(model: Surrogate, members, t_grid, length=L_RANGE,
                     max_spread=None):
    """Answers from the network inside the training domain (parameter box
    and length range) and, where max_spread is given, where the ensemble's
    members agree (spread_of at most max_spread); from the solver (the
    fallback) elsewhere.  Returns (front, closure, source)."""
    t_max = int(t_grid[-1])
    inside = in_domain(members, length)
    z = np.full((len(members), len(t_grid)), np.nan)
    c = np.full(len(members), -1, np.int64)
    if inside.any():
        yi, sp = model.predict_with_spread(features(
            [m for m, o in zip(members, inside) if o], length), t_max)
        zi, ci = decode(yi, t_max)
        idx = np.flatnonzero(inside)
        z[idx], c[idx] = zi, ci
        if max_spread is not None:
            inside[idx[sp > max_spread]] = False
    if (~inside).any():
        r = run_trajectories([m for m, o in zip(members, inside) if not o], t_grid)
        z[~inside], c[~inside] = r["z"], r["closure"]
    return z, c, np.where(inside, "network", "solver")


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=4096)
    ap.add_argument("--held-out", type=int, default=256)
    ap.add_argument("--length-min", type=int, default=L_RANGE[0])
    ap.add_argument("--length-max", type=int, default=L_RANGE[1])
    ap.add_argument("--steps", type=int, default=40000)
    ap.add_argument("--fit-steps", type=int, default=16000,
                    help="Adam steps per ensemble member")
    ap.add_argument("--batch", type=int, default=1024)
    ap.add_argument("--ensemble", type=int, default=5)
    ap.add_argument("--seed", type=int, default=1240)
    ap.add_argument("--save", default=None, help="write the weights (.npy)")
    ap.add_argument("--save-data", default=None,
                    help="write the trajectories (.npz)")
    ap.add_argument("--data", default=None,
                    help="read the trajectories (.npz from --save-data) "
                         "instead of running the solver")
    args = ap.parse_args(argv)
    import torch
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    grid = time_grid(args.steps)
    lr = (args.length_min, args.length_max)
    train_m = draw_members(args.train, args.seed, lr)
    test_m = draw_members(args.held_out, args.seed + 1, lr)
    if args.data:
        dd = np.load(args.data)
        tr = {"z": dd["z_train"], "closure": dd["c_train"],
              "nonfinite": np.all(np.isnan(dd["z_train"]), axis=1),
              "seconds": float("nan"), "fluid_nodes": 0, "steps": args.steps}
        te = {"z": dd["z_test"], "closure": dd["c_test"],
              "nonfinite": np.all(np.isnan(dd["z_test"]), axis=1),
              "seconds": float("nan"), "fluid_nodes": 0, "steps": args.steps}
        if not (np.array_equal(dd["x_train"], features(train_m, lr)) and
                np.array_equal(dd["times"], grid)):
            raise SystemExit("--data was written for other parameters")
    else:
        tr = run_trajectories(train_m, grid)
        te = run_trajectories(test_m, grid)
    x, y = features(train_m, lr), targets(tr["z"], tr["closure"], args.steps)
    if args.save_data:
        np.savez(args.save_data, x_train=x, z_train=tr["z"],
                 c_train=tr["closure"], x_test=features(test_m, lr),
                 z_test=te["z"], c_test=te["closure"], times=grid)
    model = Surrogate(seed=args.seed, members=args.ensemble)
    log = model.fit(x, y, steps=args.fit_steps, batch=args.batch)
    xt = features(test_m, lr)
    model.predict(xt)  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    yp = model.predict(xt)
    t_net = time.perf_counter() - t0
    zp, cp = decode(yp, args.steps)
    res = compare_to_solver(zp, cp, te["z"], te["closure"], args.steps)
    # with the solver as fallback where the members disagree (the threshold:
    # the 95th percentile of the spread over the training inputs, no
    # held-out information): the routed runs are solved again, timed
    _, sp_train = model.predict_with_spread(x, args.steps)
    thr = float(np.quantile(sp_train, 0.95))
    _, sp = model.predict_with_spread(xt, args.steps)
    routed = sp > thr
    zf, cf, t_fb = zp.copy(), cp.copy(), t_net
    if routed.any():
        r = run_trajectories([m for m, o in zip(test_m, routed) if o], grid)
        zf[routed], cf[routed] = r["z"], r["closure"]
        t_fb = t_net + r["seconds"]
    res_fb = compare_to_solver(zf, cf, te["z"], te["closure"], args.steps)
    res_fb.update({"max_spread": thr, "routed_runs": int(routed.sum()),
                   "routed_share": float(routed.mean()),
                   "seconds": t_fb,
                   "speedup_vs_solver": (te["seconds"] / t_fb
                                         if np.isfinite(te["seconds"]) else None)})
    if args.save:
        np.save(args.save, np.stack(model.params()))
    out = {
        "length_range": list(lr), "steps": args.steps, "times": len(grid),
        "train_runs": args.train, "held_out_runs": args.held_out,
        "train_nonfinite": int(tr["nonfinite"].sum()),
        "held_out_nonfinite": int(te["nonfinite"].sum()),
        "solver_seconds_train": tr["seconds"],
        "solver_seconds_held_out": te["seconds"],
        "solver_glups_held_out": (te["fluid_nodes"] * te["steps"] / te["seconds"] / 1e9
                                  if te["fluid_nodes"] else None),
        "fit": {"ensemble": args.ensemble, "steps": log.steps,
                "seconds": log.seconds,
                "first_loss": log.first_loss, "last_loss": log.last_loss},
        "network_seconds_held_out": t_net,
        "speedup_vs_solver": te["seconds"] / max(t_net, 1e-9),
        "vs_solver": res,
        "with_fallback": res_fb,
    }
    print(json.dumps(out))
    model.close()
    return out


if __name__ == "__main__":
    main()
