"""Host logic of the surrogate (no GPU): the time grid, the network's
inputs and targets and their decoding, the training-domain test and the
error measure against the solver."""
import numpy as np
import pytest

from paper_1309_6726_gb300 import inputs as I
from paper_1309_6726_gb300 import surrogate as S


@pytest.mark.parametrize("t_max,n,t_first", [
    (20000, 64, 100), (1500, 64, 20), (170, 64, 100), (163, 64, 100),
    (2, 2, 1)])
def test_time_grid_is_strictly_increasing_within_its_range(t_max, n, t_first):
    g = S.time_grid(t_max, n=n, t_first=t_first)
    assert g.size == n and g[0] == t_first and g[-1] == t_max
    assert np.all(np.diff(g) > 0)
    assert g.dtype.kind == "i"


def test_time_grid_is_log_spaced_where_it_can_be():
    g = S.time_grid(20000)
    r = g[1:] / g[:-1]
    # geometric ratio (200)^(1/63) up to integer rounding
    assert np.allclose(r, 200 ** (1 / 63), atol=0.01)


def test_time_grid_rejects_impossible_requests():
    with pytest.raises(ValueError):
        S.time_grid(120, n=64, t_first=100)
    with pytest.raises(ValueError):
        S.time_grid(100, n=1, t_first=1)


def test_targets_round_trip_and_missing_runs():
    z = np.array([[1.0, 2.0, 40.0], [3.0, np.nan, np.nan],
                  [np.nan, np.nan, np.nan]])
    c = np.array([1234, -1, -1])
    y = S.targets(z, c, 20000)
    assert y.shape == (3, 4) and y.dtype == np.float32
    assert np.isnan(y[2, -1])  # a run with no front at all: closure unknown
    zz, cc = S.decode(y, 20000)
    np.testing.assert_allclose(zz[0], z[0], rtol=1e-6)
    assert cc[0] == 1234 and cc[1] == -1
    # asinh(z / 10): close to the absolute front below 10 lu, relative above
    assert y[0, 0] == pytest.approx(np.arcsinh(0.1), rel=1e-6)


def test_features_span_the_training_domain():
    members = S.draw_members(400, seed=3)
    f = S.features(members)
    assert f.shape == (400, S.N_IN) and f.dtype == np.float32
    assert np.all(np.abs(f) <= 1.0 + 1e-6)
    # lengths drawn over the sweep's range, as the sweep draws them
    lengths = np.array([m.length for m in members])
    assert lengths.min() >= S.L_RANGE[0] and lengths.max() <= S.L_RANGE[1]
    assert lengths.max() - lengths.min() > 0.8 * (S.L_RANGE[1] - S.L_RANGE[0])
    # the corners of the ranges map to -1 and +1
    lo = I.SweepMember(S.W_RANGE[0], S.L_RANGE[0], S.K_RANGE[0],
                       S.THETA_RANGE[1], S.RATIO_RANGE[0])
    hi = I.SweepMember(S.W_RANGE[1], S.L_RANGE[1], S.K_RANGE[1],
                       S.THETA_RANGE[0], S.RATIO_RANGE[1])
    np.testing.assert_allclose(S.features([lo, hi]),
                               [[-1, -1, -1, -1, -1], [1, 1, 1, 1, 1]],
                               atol=1e-6)
    # a single training length: that input is constant (0)
    fixed = S.draw_members(10, seed=4, length=1024)
    assert {m.length for m in fixed} == {1024}
    assert np.all(S.features(fixed, 1024)[:, 4] == 0.0)


def test_in_domain_excludes_other_lengths_and_ranges():
    ok = I.SweepMember(64, 1024, 1e-3, 30.0, 1.0)
    wide = I.SweepMember(200, 1024, 1e-3, 30.0, 1.0)
    fast = I.SweepMember(64, 1024, 5e-2, 30.0, 1.0)
    longer = I.SweepMember(64, 2048, 1e-3, 30.0, 1.0)
    too_long = I.SweepMember(64, 5000, 1e-3, 30.0, 1.0)
    runs = [ok, wide, fast, longer, too_long]
    assert S.in_domain(runs, 1024).tolist() == [
        True, False, False, False, False]
    assert S.in_domain(runs, (1024, 4096)).tolist() == [
        True, False, False, True, False]


def test_compare_to_solver_by_hand():
    # run 0: fronts off by 1 lu at every time, final front 50 -> 2 %;
    # run 1: exact, final front 5 -> scale 10, error 0; run 2: no solver
    # front (left out).  Closure: run 0 closes in both (1100 vs 1000: 10 %).
    z_lb = np.array([[10.0, 30.0, 50.0], [1.0, 3.0, 5.0],
                     [np.nan, np.nan, np.nan]])
    z_pr = z_lb + np.array([[1.0, -1.0, 1.0], [0, 0, 0], [0, 0, 0]])
    c_lb = np.array([1000, -1, -1])
    c_pr = np.array([1100, -1, 500])
    r = S.compare_to_solver(z_pr, c_pr, z_lb, c_lb, 20000)
    assert r["runs"] == 2
    assert r["front_rel_err_mean"] == pytest.approx(0.01)
    assert r["front_within_2pct"] == 1.0
    assert r["closure_runs_both"] == 1
    assert r["closure_rel_err_mean"] == pytest.approx(0.1)
    assert r["closure_agreement"] == 1.0


def test_spread_is_the_members_front_std_over_the_error_scale():
    # two members whose fronts decode to 20 and 22 lu at every time: std 1,
    # mean last front 21 -> 1 / 21; fronts of 1 and 3 lu: std 1 over the
    # 10 lu floor -> 0.1; identical members -> 0
    t_max = 1000
    n_t = S.N_TIMES

    def member(z):
        y = np.zeros((1, n_t + 1), np.float32)
        y[0, :n_t] = np.arcsinh(z / S.Z_SCALE)
        return y

    ys = np.stack([member(20.0), member(22.0)])
    assert S.spread_of(ys, t_max)[0] == pytest.approx(1 / 21, rel=1e-5)
    ys = np.stack([member(1.0), member(3.0)])
    assert S.spread_of(ys, t_max)[0] == pytest.approx(0.1, rel=1e-5)
    ys = np.stack([member(15.0), member(15.0)])
    assert S.spread_of(ys, t_max)[0] == 0.0
