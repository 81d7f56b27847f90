"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of the oracle source (on the CPU, in
a temporary directory), builds it, and checks that a pin which holds for the
real oracle fails for the copy.
"""
import os

import numpy as np
import pytest

from oracle import build as B
from oracle import lattice as OL
from oracle.lattice import Lattice, Params
from paper_1309_6726_gb300 import inputs as I

EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
EY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])


def pin_equilibrium(lib):
    f = OL.feq(0.8, 0.07, -0.03, lib)
    return (abs((f * EX * EX).sum() - (0.8 / 3 + 0.8 * 0.07 ** 2)) < 1e-14
            and abs((f * EX).sum() - 0.8 * 0.07) < 1e-15)


def pin_solute_equilibrium(lib):
    g = OL.geq(0.5, 0.05, 0.02, lib)
    return abs(g[0] - g[2] - 0.5 * 0.05) < 1e-15


def pin_poiseuille(lib):
    ny, gx, tau = 18, 1e-6, 0.8
    geom = I.channel(1, ny)
    lat = Lattice(Params(tau_a=tau, tau_b=tau, g_coh=0.0, body_force_x=gx),
                  geom.solid, geom.rho_a, geom.rho_b, geom.conc, lib=lib)
    lat.step(20000)
    f = lat.populations()[0][:, 1:ny - 1, 0]
    rho = f.sum(axis=0)
    u = ((f * EX[:, None]).sum(axis=0) + 0.5 * rho * gx) / rho
    y = np.arange(1, ny - 1)
    ua = gx / (2 * (tau - 0.5) / 3) * (y - 0.5) * (ny - 1.5 - y)
    return np.abs(u - ua).max() / ua.max() < 5e-3


def pin_cohesion(lib):
    nx, ny = 20, 6
    x = np.arange(nx)[None, :].repeat(ny, 0)
    ra = np.full((ny, nx), 0.9, np.float32)
    rb = (0.1 + 0.01 * x).astype(np.float32)
    lat = Lattice(Params(g_coh=2.5), np.zeros((ny, nx), np.uint8), ra, rb,
                  ra * 0, lib=lib)
    _, F = lat.moments_forces()
    return np.allclose(F[0, 0, 3, 5:15], -2.5 * 0.9 * 0.01 / 3, rtol=1e-6)


def pin_adhesion(lib):
    n = 8
    solid = np.zeros((n, n), np.uint8)
    solid[0, :] = 1
    ra = np.where(solid == 0, 0.8, 0).astype(np.float32)
    rb = np.where(solid == 0, 0.3, 0).astype(np.float32)
    lat = Lattice(Params(g_coh=0.0, g_ads=0.45), solid, ra, rb, ra * 0,
                  lib=lib)
    _, F = lat.moments_forces()
    return (abs(F[0, 1, 1, 3] + 0.45 * 0.8 / 6) < 1e-7
            and abs(F[1, 1, 1, 3] - 0.45 * 0.3 / 6) < 1e-7)


def pin_reaction(lib):
    n = 10
    solid = np.zeros((n, n), np.uint8)
    solid[4:6, 3:6] = 1
    solid[2, 8] = solid[3, 7] = solid[1, 7] = 1
    fl = solid == 0
    ra = np.where(fl, 1.0, 0).astype(np.float32)
    rb = np.where(fl, 0.006, 0).astype(np.float32)
    cc = np.where(fl, 0.75, 0).astype(np.float32)
    lat = Lattice(Params(g_coh=0.0, k_r=0.01, m_threshold=10.0), solid, ra,
                  rb, cc, lib=lib)
    lat.step(1)
    ns = np.zeros((n, n), int)
    for dx, dy in ((1, 0), (0, 1), (-1, 0), (0, -1)):
        ns += np.roll(solid, (-dy, -dx), axis=(0, 1))
    return np.allclose(lat.deposit(), 0.01 * ns * fl * np.float32(0.75),
                       rtol=1e-12, atol=1e-17)


def pin_mirror(lib):
    geom = I.capillary(48, 10, 12, 8)
    lat = Lattice(Params(g_ads=I.G_ADS_30, k_r=5e-3, inlet=1,
                         m_threshold=0.2, cap_x0=12, cap_x1=40), geom.solid,
                  geom.rho_a, geom.rho_b, geom.conc, lib=lib)
    lat.step(150)
    f = lat.populations()
    my = [0, 1, 4, 3, 2, 8, 7, 6, 5]
    return np.abs(f - f[:, my, ::-1, :]).max() < 1e-12


def pin_ledger(lib):
    geom = I.random_lattice(16, 12, seed=11, solid_fraction=0.15)
    lat = Lattice(Params(g_ads=0.4, k_r=2e-2, m_threshold=0.02), geom.solid,
                  geom.rho_a, geom.rho_b, geom.conc, lib=lib)
    f, g = I.random_populations(geom, seed=12)
    lat.set_populations(f)
    lat.set_solute(g)

    def tot():
        ra, rb = lat.densities()
        led = lat.ledger()
        return np.array([ra.sum() + led[0], rb.sum() + led[1],
                         lat.concentration().sum() + lat.deposit().sum()
                         + led[2] + led[3]])
    t0 = tot()
    lat.step(30)
    return lat.ledger()[0] > 0 and np.allclose(tot(), t0, rtol=1e-12)


def pin_threshold_inclusive(lib):
    # reading c10: a node turns solid once its deposit reaches the threshold
    # (m >= M_th).  At rest, k_r n_s C* = 0.25 * 1 * 0.5 = 0.125 exactly,
    # landing the four D2Q4 neighbours of one solid node on m = 1.0.
    n = 8
    solid = np.zeros((n, n), np.uint8)
    solid[4, 4] = 1
    fl = solid == 0
    ra = np.where(fl, 1.0, 0).astype(np.float32)
    rb = np.where(fl, 0.006, 0).astype(np.float32)
    cc = np.where(fl, 0.5, 0).astype(np.float32)
    lat = Lattice(Params(g_coh=0.0, g_ads=0.0, k_r=0.25, m_threshold=1.0),
                  solid, ra, rb, cc, lib=lib)
    lat.set_deposit(np.where(fl, 0.875, 0.0))
    lat.step(1)
    s = lat.solid()
    return (s.sum() == 5 and s[4, 3] == 1 and s[4, 5] == 1 and s[3, 4] == 1
            and s[5, 4] == 1)


def pin_solute_velocity(lib):
    # readings c4 and c7: the solute is advected by u = (sum j + F/2) /
    # sum rho.  From rest under a uniform acceleration gx, u = gx/2 in the
    # first collision, and the solute's x-moment after one step is
    # C u / tau_D.
    n, gx, tau_d, c = 4, 1e-4, 0.8, 0.6
    solid = np.zeros((n, n), np.uint8)
    ra = np.full((n, n), 0.7, np.float32)
    rb = np.full((n, n), 0.3, np.float32)
    cc = np.full((n, n), c, np.float32)
    lat = Lattice(Params(g_coh=0.0, g_ads=0.0, body_force_x=gx, tau_d=tau_d),
                  solid, ra, rb, cc, lib=lib)
    lat.step(1)
    g = lat.solute()
    mx = g[0] - g[2]
    # C as the oracle holds it: the float32 input widened to FP64
    return np.allclose(mx, float(np.float32(c)) * 0.5 * gx / tau_d,
                       rtol=1e-9, atol=0)


def pin_inlet(lib):
    # reading c12: the inlet column x = 0 leaves each collision at the
    # solute equilibrium of c_in (at rest: c_in / 4 per direction).  One
    # step from C = 0 therefore puts c_in / 4 into the east-moving solute at
    # x = 1, the west-moving one at x = nx - 1 (periodic), the two vertical
    # ones at x = 0, and nothing anywhere else.
    nx, ny, c_in = 8, 4, 0.8
    solid = np.zeros((ny, nx), np.uint8)
    ra = np.full((ny, nx), 1.0, np.float32)
    rb = np.full((ny, nx), 0.006, np.float32)
    lat = Lattice(Params(g_coh=0.0, g_ads=0.0, inlet=1, c_in=c_in), solid,
                  ra, rb, ra * 0, lib=lib)
    lat.step(1)
    g = lat.solute()
    expect = np.zeros((4, ny, nx))
    expect[0, :, 1] = c_in / 4       # (1, 0)
    expect[1, :, 0] = c_in / 4       # (0, 1)
    expect[2, :, nx - 1] = c_in / 4  # (-1, 0)
    expect[3, :, 0] = c_in / 4       # (0, -1)
    return np.abs(g - expect).max() < 1e-15


# (description, text in lbm_oracle.c, replacement, pin that must catch it)
MUTANTS = [
    ("equilibrium: second-order coefficient 9/2 -> 3",
     "4.5 * eu * eu", "3.0 * eu * eu", pin_equilibrium),
    ("solute equilibrium: advection factor 2 -> 3",
     "(1.0 + 2.0 * (SX[k] * ux", "(1.0 + 3.0 * (SX[k] * ux",
     pin_solute_equilibrium),
    ("bounce-back returns along the same direction",
     "L->f[(s * Q + OPP[i]) * N + n] += v;", "L->f[(s * Q + i) * N + n] += v;",
     pin_poiseuille),
    ("Shan-Chen shift without tau",
     "ux += tau[s] * L->F[(s * 2 + 0) * N + n] / r;",
     "ux += L->F[(s * 2 + 0) * N + n] / r;", pin_poiseuille),
    ("cohesion sign flipped",
     "Fx = -L->p.g_coh * r * cx", "Fx = +L->p.g_coh * r * cx", pin_cohesion),
    ("cohesion uses own density",
     "double rho_other = L->rho[(1 - s) * N + nb];",
     "double rho_other = L->rho[s * N + nb];", pin_cohesion),
    ("adhesion same sign for both components",
     "double Gads[2] = {-L->p.g_ads, +L->p.g_ads};",
     "double Gads[2] = {-L->p.g_ads, -L->p.g_ads};", pin_adhesion),
    ("reaction ignores the number of solid links",
     "double keep = 1.0 - L->p.k_r * ns;", "double keep = 1.0 - L->p.k_r;",
     pin_reaction),
    ("diagonal direction with a wrong y component",
     "static const int EY[Q] = {0, 0, 1, 0, -1, 1, 1, -1, -1};",
     "static const int EY[Q] = {0, 0, 1, 0, -1, 1, 1, -1, 1};", pin_mirror),
    ("growth forgets the deposit in the ledger",
     "L->ledger[3] += L->m[n];", "(void)0;", pin_ledger),
    ("threshold test strict (m > M_th)",
     "if (L->m[n] >= L->p.m_threshold) {", "if (L->m[n] > L->p.m_threshold) {",
     pin_threshold_inclusive),
    ("solute advected without the half-force term",
     "L->u[0 * N + n] = rt > 0 ? (jx + 0.5 * Fx) / rt : 0.0;",
     "L->u[0 * N + n] = rt > 0 ? jx / rt : 0.0;", pin_solute_velocity),
    ("inlet on the second column",
     "if (L->p.inlet && x == 0) {", "if (L->p.inlet && x == 1) {", pin_inlet),
    ("inlet relaxes towards c_in instead of imposing it",
     "for (int k = 0; k < QS; ++k) L->gc[k * N + n] = geq[k];",
     "for (int k = 0; k < QS; ++k) L->gc[k * N + n] = L->g[k * N + n]"
     " - (L->g[k * N + n] - geq[k]) / L->p.tau_d;", pin_inlet),
]


@pytest.fixture(scope="module")
def real_lib():
    return OL.load()


@pytest.mark.parametrize("desc,old,new,pin", MUTANTS,
                         ids=[m[0] for m in MUTANTS])
def test_pin_catches_mutant(tmp_path, real_lib, desc, old, new, pin):
    src = open(B.SRC).read()
    assert src.count(old) == 1, desc
    mutated = tmp_path / "lbm_oracle_mutant.c"
    mutated.write_text(src.replace(old, new))
    so = B.build(force=True, src=str(mutated),
                 out=str(tmp_path / "liblbm_oracle_mutant.so"))
    mlib = OL.load(so)
    assert pin(real_lib), "pin fails on the real oracle: " + desc
    assert not pin(mlib), "pin misses the planted mistake: " + desc
    assert os.path.exists(so)
