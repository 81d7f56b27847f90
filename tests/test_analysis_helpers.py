"""Pin of the meniscus helper the contact-angle table and the 30-degree test
lean on, against hand-built fields whose answer is known: a phi field
whose zero contour is an exact circular arc of a chosen contact angle,
wetting (centre ahead of the interface) and non-wetting (centre behind
it).  A sign or centre mistake in the helper shifts the angle or flips the
sign and fails these.
"""
import math

import numpy as np
import pytest

from oracle import analysis as A


def _arc_field(ny: int, nx: int, theta_deg: float, x_mid: float):
    """rho_A, rho_B with phi = rho_A - rho_B = x_s(y) - x, the interface
    x_s(y) an arc of the circle of radius R = (H/2) / |cos theta| centred on
    the channel axis: ahead of the interface (x_c > x_s) when A wets
    (theta < 90 degrees), behind it otherwise."""
    H = ny - 2
    yc = (ny - 1) / 2.0
    c = math.cos(math.radians(theta_deg))
    R = (H / 2.0) / abs(c)
    y = np.arange(ny)[:, None] - yc
    half = np.sqrt(R * R - y * y)
    xc = x_mid + half[int(yc)] if c > 0 else x_mid - half[int(yc)]
    xs = xc - half if c > 0 else xc + half
    x = np.arange(nx)[None, :].astype(np.float64)
    phi = xs - x
    rho_a = 0.5 + 0.5 * phi
    rho_b = 0.5 - 0.5 * phi
    solid = np.zeros((ny, nx), np.uint8)
    solid[0, :] = solid[ny - 1, :] = 1
    return rho_a, rho_b, solid, R


@pytest.mark.parametrize("theta", [30.0, 60.0, 120.0, 150.0])
def test_meniscus_cos_theta_recovers_an_exact_arc(theta):
    ny, nx = 42, 160
    ra, rb, solid, R = _arc_field(ny, nx, theta, x_mid=70.0)
    cos_t, R_fit = A.meniscus_cos_theta(ra, rb, solid, x_from=10)
    assert R_fit == pytest.approx(R, rel=1e-9)
    assert math.degrees(math.acos(cos_t)) == pytest.approx(theta, abs=1e-6)


def test_meniscus_sign_follows_the_side_of_the_centre():
    ra, rb, solid, _ = _arc_field(30, 120, 45.0, x_mid=60.0)
    assert A.meniscus_cos_theta(ra, rb, solid, x_from=5)[0] > 0
    ra, rb, solid, _ = _arc_field(30, 120, 135.0, x_mid=60.0)
    assert A.meniscus_cos_theta(ra, rb, solid, x_from=5)[0] < 0
