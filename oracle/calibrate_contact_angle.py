"""Calibrates the adhesion strength g against the static contact angle.

Runs the FP64 oracle on a closed straight channel (walls along its whole
length, periodic in x) holding a slug of A between two B regions, lets the
two menisci relax, and measures theta from a circle fitted to the meniscus
(``analysis.meniscus_cos_theta``).  The paper fixes the contact angle of
molten Si on carbon at 30 degrees (Sec. I) and adjusts the adhesive force to
reproduce it; this script produces the (theta, g) table that the input
generator interpolates.  It calls only the oracle.  Test infrastructure
like the rest of this package: the product path never runs it; only its
output table, committed beside the input generator, is used.

Usage: python -m oracle.calibrate_contact_angle
"""
from __future__ import annotations

import math
import sys

import numpy as np

from . import analysis
from .lattice import Lattice, Params

NX, NY, SLUG, STEPS = 120, 34, 60, 10_000
G_COH = 2.5
RHO_MAJOR, RHO_MINOR = 1.0, 0.006


def slug_fields():
    solid = np.zeros((NY, NX), np.uint8)
    solid[0, :] = 1
    solid[NY - 1, :] = 1
    x = np.arange(NX)[None, :].repeat(NY, 0)
    x0 = (NX - SLUG) // 2
    a_rich = (x >= x0) & (x < x0 + SLUG)
    rho_a = np.where(a_rich, RHO_MAJOR, RHO_MINOR).astype(np.float32)
    rho_b = np.where(a_rich, RHO_MINOR, RHO_MAJOR).astype(np.float32)
    rho_a[solid != 0] = 0
    rho_b[solid != 0] = 0
    return solid, rho_a, rho_b, np.zeros((NY, NX), np.float32)


def contact_angle(g_ads: float, steps: int = STEPS, tau: float = 1.0):
    """(theta in degrees, cos theta, R) of the slug's right meniscus."""
    solid, ra, rb, c = slug_fields()
    lat = Lattice(Params(tau_a=tau, tau_b=tau, g_coh=G_COH, g_ads=g_ads),
                  solid, ra, rb, c)
    lat.step(steps)
    rho_a, rho_b = lat.densities()
    cos, R = analysis.meniscus_cos_theta(rho_a, rho_b, solid, NX // 2)
    theta = math.degrees(math.acos(max(-1.0, min(1.0, cos))))
    return theta, cos, R


def main(argv=None):
    gs = [0.25, 0.30, 0.35, 0.40, 0.45, 0.50, 0.52, 0.54]
    rows = []
    for g in gs:
        th, cos, R = contact_angle(g)
        rows.append((th, g))
        print("g_ads %.3f  theta %.2f deg  cos %.4f  R %.2f" % (g, th, cos, R))
        sys.stdout.flush()
    print("CONTACT_ANGLE_TABLE = (")
    for th, g in rows:
        print("    (%.2f, %.3f)," % (th, g))
    print(")")


if __name__ == "__main__":
    main()
