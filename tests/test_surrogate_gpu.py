"""The surrogate end to end at a small scale: trajectories from the batched
solver, training with the library's kernels, the solver as the reference on
held-out parameters, the solver as fallback outside the training domain,
and what the network gains over running the solver."""
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_surrogate_learns_solver_trajectories_and_saves_time():
    import __graft_entry__
    __graft_entry__.build()
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1309_6726_gb300 import surrogate as S

    length, steps = 96, 1500
    grid = S.time_grid(steps, n=S.N_TIMES, t_first=20)
    train_m = S.draw_members(320, seed=5, length=length)
    test_m = S.draw_members(48, seed=6, length=length)
    tr = S.run_trajectories(train_m, grid)
    te = S.run_trajectories(test_m, grid)
    assert tr["nonfinite"].sum() < 0.05 * len(train_m)
    # the fronts move (closure needs longer horizons than this one)
    assert np.nanmax(tr["z"][:, -1]) > 5.0

    model = S.Surrogate(hidden=128, layers=3, seed=1, max_batch=512)
    log = model.fit(S.features(train_m, length), S.targets(tr["z"], tr["closure"], steps),
                    steps=3000, batch=320, lr=3e-3)
    assert log.last_loss < 0.05 * log.first_loss

    xt = S.features(test_m, length)
    model.predict(xt)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    yp = model.predict(xt)
    t_net = time.perf_counter() - t0
    zp, cp = S.decode(yp, steps)
    res = S.compare_to_solver(zp, cp, te["z"], te["closure"], steps)
    print(res, "solver %.3f s, network %.5f s" % (te["seconds"], t_net))
    # a small training set at a short horizon: a looser bound than the
    # 2 percent of the full-size run, but well below an untrained guess
    assert res["front_rel_err_median"] < 0.10
    assert res["closure_agreement"] > 0.8
    # the gain: the answer for every held-out run, at that error, costs a
    # forward pass instead of a solver run
    assert te["seconds"] > 20 * t_net

    # outside the training domain (another capillary length) the solver
    # answers instead
    other = S.draw_members(3, seed=7, length=length + 8)
    z, c, src = S.predict_or_solve(model, other + test_m[:2], grid, length)
    assert list(src) == ["solver"] * 3 + ["network"] * 2
    ref = S.run_trajectories(other, grid)
    np.testing.assert_array_equal(z[:3], ref["z"])
    np.testing.assert_array_equal(c[:3], ref["closure"])
    zn, cn = S.decode(model.predict(S.features(test_m[:2], length)), steps)
    np.testing.assert_array_equal(z[3:], zn)
    # inside the domain, where the members disagree by more than
    # max_spread, the solver answers too: the runs with the largest spread
    # go to it, the others keep the network's answer
    _, sp = model.predict_with_spread(S.features(test_m[:6], length), steps)
    thr = float(np.sort(sp)[-3])  # the three largest spreads exceed it or equal it
    z2, c2, src2 = S.predict_or_solve(model, test_m[:6], grid, length,
                                      max_spread=thr - 1e-12)
    routed = sp > thr - 1e-12
    assert list(src2) == ["solver" if r else "network" for r in routed]
    assert routed.sum() >= 3
    ref2 = S.run_trajectories([m for m, r in zip(test_m[:6], routed) if r], grid)
    np.testing.assert_array_equal(z2[routed], ref2["z"])
    zn2, _ = S.decode(model.predict(S.features(test_m[:6], length)), steps)
    np.testing.assert_array_equal(z2[~routed], zn2[~routed])
    print("nonfinite runs: train %d/%d, held-out %d/%d, fallback %d/3" % (
        tr["nonfinite"].sum(), len(train_m), te["nonfinite"].sum(),
        len(test_m), ref["nonfinite"].sum()))
    model.close()


def test_surrogate_over_a_length_range_meets_its_held_out_bound():
    # Training runs drawn as in the sweep over a range of capillary lengths
    # (L is an input), the solver as the judge on held-out parameters.  A
    # small scale of the full run (L 128-384 instead of 1024-4096, 1024
    # training runs, 4000 steps): measured 1.4 % mean, 0.5 % median, 4.2 %
    # p90 front error.  Closure needs longer horizons than this one (no
    # training run closes); the runs agree on not closing.
    import __graft_entry__
    __graft_entry__.build()
    from paper_1309_6726_gb300 import surrogate as S

    lr, steps = (128, 384), 4000
    grid = S.time_grid(steps, n=S.N_TIMES, t_first=40)
    train_m = S.draw_members(1024, seed=11, length=lr)
    test_m = S.draw_members(128, seed=12, length=lr)
    tr = S.run_trajectories(train_m, grid)
    te = S.run_trajectories(test_m, grid)
    ok = ~np.all(np.isnan(tr["z"]), axis=1)
    model = S.Surrogate(hidden=256, layers=3, seed=2, max_batch=1024, members=2)
    model.fit(S.features(train_m, lr)[ok],
              S.targets(tr["z"], tr["closure"], steps)[ok],
              steps=6000, batch=512, lr=2e-3)
    zp, cp = S.decode(model.predict(S.features(test_m, lr)), steps)
    res = S.compare_to_solver(zp, cp, te["z"], te["closure"], steps)
    print("length range %s: %s" % (lr, res))
    assert res["runs"] >= 100
    assert res["front_rel_err_mean"] < 0.025
    assert res["front_rel_err_median"] < 0.01
    assert res["front_rel_err_p90"] < 0.08
    assert res["closure_agreement"] > 0.9
    # with the solver answering where the two members disagree most (the
    # 95th percentile of their spread over the training inputs): the
    # combined answer's error against the judge (measured 1.1 % mean,
    # 14 of 128 runs solved)
    _, sp_tr = model.predict_with_spread(S.features(train_m, lr)[ok], steps)
    thr = float(np.quantile(sp_tr, 0.95))
    z, c, src = S.predict_or_solve(model, test_m, grid, lr, max_spread=thr)
    fb = S.compare_to_solver(z, c, te["z"], te["closure"], steps)
    print("with fallback: %d of %d runs solved, %s"
          % ((src == "solver").sum(), len(test_m), fb))
    assert fb["front_rel_err_mean"] <= res["front_rel_err_mean"]
    assert fb["front_rel_err_mean"] < 0.02
    model.close()
