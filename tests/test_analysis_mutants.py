"""The observables' pins catch plausible mistakes in ``oracle/analysis.py``.

Each case plants one mistake in a copy of the module (a temporary file),
imports the copy, and checks that a pin computed by hand holds for the real
module and fails for the copy."""
import importlib.util
import math

import numpy as np
import pytest

from oracle import analysis as REAL


def _straight(ny, nx, x0, x1):
    s = np.zeros((ny, nx), np.uint8)
    s[0, x0:x1] = 1
    s[ny - 1, x0:x1] = 1
    return s


def pin_front(A):
    # phi falls from +1 at x = 6 to -1 at x = 7 on the centerline rows:
    # crossing at 6.5, entrance plane at x0 - 1/2 = 3.5, z = 3
    ny, nx, x0 = 6, 12, 4
    s = _straight(ny, nx, x0, 10)
    ra = np.zeros((ny, nx))
    rb = np.zeros((ny, nx))
    ra[:, :7] = 1.0
    rb[:, 7:] = 1.0
    return abs(A.front_position(ra, rb, s, x0) - 3.0) < 1e-12


def _grown():
    # lower wall b = [1,2,3,3,2,1] over six columns, ny = 10: A = 18,
    # P = 6 + 4 = 10, r_h = 1.8; h = 9 - b: r_min = 3, r_ave = 3.5;
    # Delta e = 2
    ny, nx, x0, x1 = 10, 10, 2, 8
    s0 = _straight(ny, nx, x0, x1)
    s = s0.copy()
    for k, b in enumerate([1, 2, 3, 3, 2, 1]):
        s[:b, x0 + k] = 1
    return s0, s, x0, x1


def pin_radii(A):
    s0, s, x0, x1 = _grown()
    ra = np.where(s == 0, 1.0, 0.0)
    o = A.observables(ra, ra * 0, ra * 0, ra * 0, s, s0, x0, x1,
                      np.zeros(4))
    return (abs(o["r_h"] - 1.8) < 1e-12 and o["r_min"] == 3.0
            and o["r_ave"] == 3.5 and o["delta_e"] == 2.0)


def pin_closure(A):
    # one column of the grown profile closed: Delta e = H / 2 = 4
    s0, s, x0, x1 = _grown()
    s[:, x0 + 3] = 1
    ra = np.where(s == 0, 1.0, 0.0)
    o = A.observables(ra, ra * 0, ra * 0, ra * 0, s, s0, x0, x1,
                      np.zeros(4))
    return o["closed"] == 1.0 and o["delta_e"] == 4.0 and o["r_min"] == 0


def pin_wetted(A):
    # A fills the first 5 section columns, B the rest: 5 wetted nodes on
    # each wall of a straight channel
    ny, nx, x0, x1 = 8, 14, 2, 12
    s = _straight(ny, nx, x0, x1)
    ra = np.where(s == 0, 0.006, 0.0)
    rb = np.where(s == 0, 1.0, 0.0)
    ra[:, :x0 + 5] = np.where(s[:, :x0 + 5] == 0, 1.0, 0.0)
    rb[:, :x0 + 5] = np.where(s[:, :x0 + 5] == 0, 0.006, 0.0)
    o = A.observables(ra, rb, ra * 0, ra * 0, s, s, x0, x1, np.zeros(4))
    return o["wetted_lower"] == 5 and o["wetted_upper"] == 5


def pin_washburn(A):
    # Eq. 1 at t = t_d: z = v t_d / e, v = gamma H cos / (6 mu L)
    gamma, mu, rho, H, L, c = 0.15, 0.17, 1.1, 30.0, 500.0, 0.866
    t_d = rho * H * H / (12 * mu)
    v = gamma * H * c / (6 * mu * L)
    z = A.washburn_z(t_d, gamma, mu, rho, H, L, c)
    return abs(z - v * t_d / math.e) < 1e-12 * v * t_d


# (description, text in analysis.py, replacement, pin that must catch it)
MUTANTS = [
    ("front measured from x0 instead of the plane x0 - 1/2",
     "- (x0 - 0.5)", "- x0", pin_front),
    ("front crossing not interpolated",
     "found = x + phi[x] / (phi[x] - phi[x + 1]) - (x0 - 0.5)",
     "found = x + 1 - (x0 - 0.5)", pin_front),
    ("hydraulic perimeter without the vertical steps",
     "perim = len(b) + np.abs(np.diff(b)).sum()", "perim = len(b)",
     pin_radii),
    ("r_ave from the full aperture",
     "\"r_ave\": float(h.mean()) / 2.0,", "\"r_ave\": float(h.mean()),",
     pin_radii),
    ("closed column counts the whole gap",
     "half_gap = (ny - b0 - t0) / 2.0", "half_gap = (ny - b0 - t0) * 1.0",
     pin_closure),
    ("wetted length read on the wall row",
     "yl = b[k]\n", "yl = b[k] - 1\n", pin_wetted),
    ("Eq. 1 with t_d = rho H^2 / (6 mu)",
     "t_d = rho * H * H / (12.0 * mu)", "t_d = rho * H * H / (6.0 * mu)",
     pin_washburn),
]


@pytest.mark.parametrize("desc,old,new,pin", MUTANTS,
                         ids=[m[0] for m in MUTANTS])
def test_pin_catches_mutant(tmp_path, desc, old, new, pin):
    src = open(REAL.__file__).read()
    assert src.count(old) == 1, desc
    path = tmp_path / "analysis_mutant.py"
    path.write_text(src.replace(old, new))
    spec = importlib.util.spec_from_file_location("analysis_mutant", path)
    mutant = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mutant)
    assert pin(REAL), "pin fails on the real module: " + desc
    assert not pin(mutant), "pin misses the planted mistake: " + desc
