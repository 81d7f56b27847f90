"""The oracle against the few numbers the paper prints (fixture
``tests/golden/paper_printed_values.txt``, each line with its citation):
Eq. 1's speed ratio between the two lengths of Fig. 3, Delta e = H / 2 for
a closed pore at each printed height, and the radii of Fig. 4 agreeing
(H / 2) for an ungrown capillary of the printed size."""
import math
import os

import numpy as np
import pytest

from oracle import analysis as A

GOLDEN = os.path.join(os.path.dirname(__file__), "golden",
                      "paper_printed_values.txt")


def _golden() -> dict:
    vals = {}
    with open(GOLDEN) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            key, val = (s.strip() for s in line.split("=", 1))
            nums = [float(v) for v in val.split()]
            vals[key] = nums if len(nums) > 1 else nums[0]
    return vals


G = _golden()
# lattice units of a BGK fluid at tau = 1 and an arbitrary surface tension:
# the checks below hold for any positive values
GAMMA, RHO = 0.11, 1.0
MU = A.lattice_viscosity(RHO, 1.0)


def test_fixture_holds_the_printed_values():
    assert G["contact_angle_deg"] == 30
    assert G["fig3_lengths_lu"] == [500, 1000]
    assert G["heights_lu"] == [25, 50, 100]


@pytest.mark.parametrize("H", G["heights_lu"])
def test_eq1_speed_ratio_between_the_fig3_lengths(H):
    # late-time slope of the full Eq. 1 (exponential transient included),
    # by finite differences far beyond t_d = rho H^2 / (12 mu)
    L1, L2 = G["fig3_lengths_lu"]
    c = math.cos(math.radians(G["contact_angle_deg"]))
    t_d = RHO * H * H / (12 * MU)
    t = np.array([40 * t_d, 60 * t_d])

    def slope(L):
        z = A.washburn_z(t, GAMMA, MU, RHO, H, L, c)
        return (z[1] - z[0]) / (t[1] - t[0])

    assert slope(L1) / slope(L2) == pytest.approx(
        G["eq1_speed_ratio_500_1000"], rel=1e-12)
    # and the early front is slower than the linear law (the transient)
    z_early = A.washburn_z(np.array([t_d]), GAMMA, MU, RHO, H, L1, c)[0]
    assert z_early < slope(L1) * t_d


def _channel(H: int, L: int, x_res: int = 8, x_out: int = 8):
    """Straight capillary of H fluid rows between 1-node walls."""
    ny, nx = H + 2, L + x_res + x_out
    solid = np.zeros((ny, nx), np.uint8)
    solid[0, x_res:nx - x_out] = 1
    solid[ny - 1, x_res:nx - x_out] = 1
    return solid, x_res, nx - x_out


def _obs(solid, initial, x0, x1):
    ny, nx = solid.shape
    ra = np.where(solid == 0, 1.0, 0.0)
    rb = np.where(solid == 0, 0.06, 0.0)
    z = np.zeros((ny, nx))
    return A.observables(ra, rb, z, z, solid, initial, x0, x1, [0, 0, 0, 0])


@pytest.mark.parametrize("H", G["heights_lu"])
def test_closed_pore_has_delta_e_half_height(H):
    solid0, x0, x1 = _channel(int(H), int(G["fig4_length_lu"]))
    grown = solid0.copy()
    grown[:, x0 + 100] = 1  # one section column entirely solid
    o = _obs(grown, solid0, x0, x1)
    assert o["closed"] == 1.0
    assert o["r_min"] == 0.0
    assert o["delta_e"] == G["closure_delta_e_over_h"] * H
    # one layer short of closure stays below H / 2
    partial = solid0.copy()
    partial[1:int(H) // 2, x0 + 100] = 1
    o = _obs(partial, solid0, x0, x1)
    assert o["closed"] == 0.0 and o["delta_e"] < H / 2


@pytest.mark.parametrize("H", G["heights_lu"])
def test_fig4_radii_agree_without_growth(H):
    # at the printed length, an ungrown capillary: r_min, r_ave, r_h and
    # r_eff (Eq. 1's late-time speed fed back through its inverse) all H / 2
    L = G["fig4_length_lu"]
    solid, x0, x1 = _channel(int(H), int(L))
    o = _obs(solid, solid, x0, x1)
    assert o["r_min"] == H / 2 and o["r_ave"] == H / 2
    assert o["r_h"] == pytest.approx(H / 2, rel=1e-12)
    c = math.cos(math.radians(G["contact_angle_deg"]))
    t = np.linspace(1e5, 5e5, 9)
    z = 3.0 + A.washburn_speed(GAMMA, MU, H, L, c) * t
    assert A.fit_reff(t, z, GAMMA, MU, L, c) == pytest.approx(H / 2,
                                                             rel=1e-9)
