"""Pins of the oracle's observables and of the Eq. 1 helpers against
hand-computed values on small handmade masks and fields."""
import math

import numpy as np
import pytest

from oracle import analysis as A


def _straight(ny=10, nx=12, x0=2, x1=10):
    s = np.zeros((ny, nx), np.uint8)
    s[0, x0:x1] = 1
    s[ny - 1, x0:x1] = 1
    return s


def test_straight_channel_radii():
    # A straight capillary of height H: every radius is H/2, no growth.
    ny, nx, x0, x1 = 10, 12, 2, 10
    s = _straight(ny, nx, x0, x1)
    ra = np.where(s == 0, 1.0, 0.0)
    rb = np.where(s == 0, 0.01, 0.0)
    o = A.observables(ra, rb, ra * 0, ra * 0, s, s, x0, x1, np.zeros(4))
    H = ny - 2
    assert o["r_min"] == o["r_ave"] == o["r_h"] == H / 2
    assert o["delta_e"] == 0 and o["closed"] == 0
    assert o["wetted_lower"] == o["wetted_upper"] == x1 - x0


def test_grown_profile_by_hand():
    # Lower wall thickness b = [1,2,3,3,2,1] over six columns, upper wall
    # untouched, ny = 10 (centerline 4.5, walls' surface at b - 1/2):
    # A = sum(5 - b) = 18, P = 6 + 4 = 10 -> r_h = 1.8; h = 9 - b ->
    # r_min = 6/2 = 3, r_ave = mean(h)/2 = 3.5, Delta e = 2.
    ny, nx, x0, x1 = 10, 10, 2, 8
    s0 = _straight(ny, nx, x0, x1)
    s = s0.copy()
    for k, b in enumerate([1, 2, 3, 3, 2, 1]):
        s[:b, x0 + k] = 1
    ra = np.where(s == 0, 1.0, 0.0)
    o = A.observables(ra, ra * 0, ra * 0, ra * 0, s, s0, x0, x1,
                      np.zeros(4))
    assert o["r_h"] == pytest.approx(1.8)
    assert o["r_min"] == 3.0
    assert o["r_ave"] == 3.5
    assert o["delta_e"] == 2.0
    # close one column: Delta e becomes half the initial gap, H/2 = 4
    s[:, x0 + 3] = 1
    o = A.observables(ra * (s == 0), ra * 0, ra * 0, ra * 0, s, s0, x0, x1,
                      np.zeros(4))
    assert o["closed"] == 1.0 and o["delta_e"] == 4.0 and o["r_min"] == 0


def test_front_interpolation():
    # phi = rho_A - rho_B falls linearly from +1 at x = 6 to -1 at x = 7 on
    # the two centerline rows: the crossing is at 6.5, entrance plane at
    # x0 - 1/2 = 3.5, so z = 3.
    ny, nx, x0 = 6, 12, 4
    s = _straight(ny, nx, x0, 10)
    ra = np.zeros((ny, nx))
    rb = np.zeros((ny, nx))
    ra[:, :7] = 1.0
    rb[:, 7:] = 1.0
    assert A.front_position(ra, rb, s, x0) == pytest.approx(3.0)
    # asymmetric crossing: phi(6) = 0.5, phi(7) = -1.5 -> 6.25, z = 2.75
    ra[:, 6] = 0.75
    rb[:, 6] = 0.25
    ra[:, 7] = 0.0
    rb[:, 7] = 1.5
    assert A.front_position(ra, rb, s, x0) == pytest.approx(2.75)
    # no B anywhere on the centerline: no front
    assert math.isnan(A.front_position(ra * 0 + 1, rb * 0, s, x0))


def test_washburn_limits():
    # Eq. 1: z ~ v t^2 / (2 t_d) for t << t_d (inertial start) and
    # z ~ v (t - t_d) for t >> t_d, with v = gamma H cos / (6 mu L).
    gamma, mu, rho, H, L, c = 0.15, 0.17, 1.1, 30.0, 500.0, 0.866
    v = A.washburn_speed(gamma, mu, H, L, c)
    t_d = rho * H * H / (12 * mu)
    t = 1e-3 * t_d
    assert A.washburn_z(t, gamma, mu, rho, H, L, c) == pytest.approx(
        v * t * t / (2 * t_d), rel=1e-3)
    t = 60 * t_d
    assert A.washburn_z(t, gamma, mu, rho, H, L, c) == pytest.approx(
        v * (t - t_d), rel=1e-12)


def test_reff_recovers_height():
    # A front moving exactly at the Eq. 1 speed of height H gives r_eff = H/2.
    gamma, mu, L, c, H = 0.144, 0.17, 400.0, math.cos(math.radians(30)), 16
    v = A.washburn_speed(gamma, mu, H, L, c)
    t = np.arange(1000, 6000, 250.0)
    z = 2.0 + v * t
    assert A.fit_reff(t, z, gamma, mu, L, c) == pytest.approx(H / 2)
