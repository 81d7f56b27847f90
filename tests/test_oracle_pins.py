"""Pins of the FP64 oracle against what the mathematics fixes exactly.

Each test checks the oracle against a closed form, an exact invariant or a
special case with a known answer, never against a retyped copy of its own
formulas.  The slower physical checks (Laplace law, contact angle, Washburn
law, Poiseuille flow) are in ``test_oracle_physics.py``.
"""
import numpy as np
import pytest

from oracle import lattice as OL
from oracle.lattice import Lattice, Params
from paper_1309_6726_gb300 import inputs as I

EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
EY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
SX = np.array([1, 0, -1, 0])
SY = np.array([0, 1, 0, -1])


def _lat(geom, **kw):
    p = Params(cap_x0=geom.cap_x0, cap_x1=geom.cap_x1, **kw)
    return Lattice(p, geom.solid, geom.rho_a, geom.rho_b, geom.conc)


def _momentum(lat):
    f = lat.populations()
    return np.array([(f * EX[None, :, None, None]).sum(),
                     (f * EY[None, :, None, None]).sum()])


@pytest.mark.parametrize("rho,ux,uy", [(1.0, 0.0, 0.0), (0.7, 0.05, -0.02),
                                       (0.006, -0.1, 0.08)])
def test_equilibrium_moments(oracle_lib, rho, ux, uy):
    # Hydrodynamic moments of the D2Q9 equilibrium: density, momentum and
    # momentum flux rho/3 I + rho u u (the BGK equilibrium's defining
    # properties, paper Sec. II).
    f = OL.feq(rho, ux, uy, oracle_lib)
    assert f.sum() == pytest.approx(rho, rel=1e-14)
    assert (f * EX).sum() == pytest.approx(rho * ux, abs=1e-15)
    assert (f * EY).sum() == pytest.approx(rho * uy, abs=1e-15)
    assert (f * EX * EX).sum() == pytest.approx(rho / 3 + rho * ux * ux,
                                                rel=1e-14)
    assert (f * EY * EY).sum() == pytest.approx(rho / 3 + rho * uy * uy,
                                                rel=1e-14)
    assert (f * EX * EY).sum() == pytest.approx(rho * ux * uy, abs=1e-15)
    # D2Q4 solute equilibrium: zeroth moment C, first moment C u, second
    # moment C/2 (sound speed squared 1/2 gives D = (tau_D - 1/2)/2).
    c = 0.37
    g = OL.geq(c, ux, uy, oracle_lib)
    assert g.sum() == pytest.approx(c, rel=1e-14)
    assert (g * SX).sum() == pytest.approx(c * ux, abs=1e-15)
    assert (g * SY).sum() == pytest.approx(c * uy, abs=1e-15)
    assert (g * SX * SX).sum() == pytest.approx(c / 2, rel=1e-14)


def test_rest_state_is_fixed_point(oracle_lib):
    # A uniform single-phase fluid at rest with no solid is a fixed point of
    # collide + stream (no forces: uniform densities give zero cohesion).
    n = 12
    z = np.zeros((n, n), np.float32)
    ra = np.full((n, n), 1.0, np.float32)
    rb = np.full((n, n), 0.006, np.float32)
    c = np.full((n, n), 0.5, np.float32)
    lat = Lattice(Params(k_r=0.0), z.astype(np.uint8), ra, rb, c)
    f0, g0 = lat.populations(), lat.solute()
    lat.step(25)
    assert np.abs(lat.populations() - f0).max() < 1e-15
    assert np.abs(lat.solute() - g0).max() < 1e-15


def test_translation_invariance_exact(oracle_lib):
    # The update is the same rule at every node of a periodic lattice, so
    # shifting the initial state shifts the result bit for bit.
    geom = I.random_lattice(23, 17, seed=5, solid_fraction=0.12)
    kw = dict(g_ads=0.4, k_r=5e-3, m_threshold=0.01)
    a = _lat(geom, **kw)
    dx, dy = 7, 4
    rolled = I.Geometry(*(np.roll(x, (dy, dx), axis=(0, 1)) for x in
                          (geom.solid, geom.rho_a, geom.rho_b, geom.conc)),
                        0, 23)
    b = _lat(rolled, **kw)
    a.step(30)
    b.step(30)
    assert np.array_equal(np.roll(a.populations(), (dy, dx), axis=(2, 3)),
                          b.populations())
    assert np.array_equal(np.roll(a.solid(), (dy, dx), axis=(0, 1)),
                          b.solid())
    assert np.array_equal(np.roll(a.deposit(), (dy, dx), axis=(0, 1)),
                          b.deposit())


def _mirror_y(f9):
    # populations mirrored about the channel axis: y -> ny-1-y and the
    # direction index maps to the one with e_y negated.
    my = [0, 1, 4, 3, 2, 8, 7, 6, 5]
    return f9[..., my, ::-1, :]


def test_mirror_symmetry_of_capillary(oracle_lib):
    # The capillary is symmetric about its axis; the update must keep an
    # axis-symmetric state symmetric (a wrong direction index or a one-sided
    # stencil breaks it).
    geom = I.capillary(96, 14, 24, 16)
    lat = _lat(geom, g_ads=I.G_ADS_30, k_r=5e-3, inlet=1, m_threshold=0.2)
    lat.step(400)
    f = lat.populations()
    assert lat.ledger()[0] > 0  # growth happened
    assert np.abs(f - _mirror_y(f)).max() < 1e-12
    g = lat.solute()
    assert np.abs(g - g[[0, 3, 2, 1], ::-1, :]).max() < 1e-12
    s = lat.solid()
    assert np.array_equal(s, s[::-1, :])


def test_momentum_conserved_with_cohesion(oracle_lib):
    # With no solid and no body force, cohesion is a pair interaction:
    # the forces sum to zero over a periodic lattice, and with the Shan-Chen
    # shift the total momentum after collision equals the total before plus
    # the total force, so momentum is conserved.
    geom = I.random_lattice(20, 16, seed=3, solid_fraction=0.0)
    lat = _lat(geom, g_coh=2.5)
    f, g = I.random_populations(geom, seed=4)
    lat.set_populations(f)
    lat.set_solute(g)
    rho, F = lat.moments_forces()
    assert np.abs(F).max() > 1e-3
    assert abs(F[:, 0].sum()) < 1e-14 and abs(F[:, 1].sum()) < 1e-14
    p0 = _momentum(lat)
    lat.step(1)
    assert np.abs(_momentum(lat) - p0).max() < 1e-13


def test_adhesion_force_closed_form(oracle_lib):
    # A fluid node right above a flat wall sees solid at e = (0,-1), (1,-1),
    # (-1,-1): sum_i w_i s e_i = (0, -(1/9 + 2/36)) = (0, -1/6), so
    # F_A = -G_ads,A rho_A (0, -1/6) = (0, -g rho_A / 6) (towards the wall)
    # and F_B = (0, +g rho_B / 6).
    n = 8
    solid = np.zeros((n, n), np.uint8)
    solid[0, :] = 1
    ra = np.where(solid == 0, 0.8, 0).astype(np.float32)
    rb = np.where(solid == 0, 0.3, 0).astype(np.float32)
    g = 0.45
    lat = Lattice(Params(g_coh=0.0, g_ads=g), solid, ra, rb, ra * 0)
    _, F = lat.moments_forces()
    assert F[0, 1, 1, 3] == pytest.approx(-g * 0.8 / 6, rel=1e-6)
    assert F[1, 1, 1, 3] == pytest.approx(+g * 0.3 / 6, rel=1e-6)
    assert F[0, 0, 1, 3] == pytest.approx(0.0, abs=1e-15)
    # a node two rows up sees no solid
    assert F[0, 1, 2, 3] == pytest.approx(0.0, abs=1e-15)


def test_cohesion_force_closed_form(oracle_lib):
    # Linear rho_B(x) = a + b x (periodic jumps kept away): the stencil gives
    # sum_i w_i rho_B(x + e_i) e_x = b sum_i w_i e_x^2 = b/3, so
    # F_A,x = -G_c rho_A b / 3 exactly.
    nx, ny = 20, 6
    x = np.arange(nx)[None, :].repeat(ny, 0)
    ra = np.full((ny, nx), 0.9, np.float32)
    rb = (0.1 + 0.01 * x).astype(np.float32)
    lat = Lattice(Params(g_coh=2.5), np.zeros((ny, nx), np.uint8), ra, rb,
                  ra * 0)
    _, F = lat.moments_forces()
    b = 0.01
    got = F[0, 0, 3, 5:15]
    assert np.allclose(got, -2.5 * 0.9 * b / 3, rtol=1e-6)
    assert np.allclose(F[0, 1, 3, 5:15], 0, atol=1e-15)


def test_mass_ledgers_close_with_growth(oracle_lib):
    # Collision conserves each component, streaming only moves mass, and
    # growth moves a node's content to the ledger: sum(rho_s) + ledger_s is
    # constant; for the closed solute, sum C + sum m + ledger_C + ledger_m
    # is constant (no inlet).
    geom = I.random_lattice(24, 18, seed=11, solid_fraction=0.15)
    lat = _lat(geom, g_ads=0.4, k_r=2e-2, m_threshold=0.02)
    f, g = I.random_populations(geom, seed=12)
    lat.set_populations(f)
    lat.set_solute(g)

    def totals():
        ra, rb = lat.densities()
        led = lat.ledger()
        return np.array([ra.sum() + led[0], rb.sum() + led[1],
                         lat.concentration().sum() + lat.deposit().sum()
                         + led[2] + led[3]])

    t0 = totals()
    s0 = lat.solid().copy()
    lat.step(60)
    t1 = totals()
    assert lat.ledger()[0] > 0 and lat.ledger()[3] > 0  # nodes turned solid
    assert np.all(lat.solid() >= s0)                     # solid only grows
    assert np.allclose(t1, t0, rtol=1e-12, atol=0)


def test_d2q4_diffusion_variance_exact():
    # Pure diffusion on a fluid at rest: for BGK D2Q4 the variance of a
    # point release grows by exactly 2 D per step with D = (tau_D - 1/2)/2
    # (sound speed squared 1/2), once the first moment's transient is gone.
    nx = 400
    solid = np.zeros((1, nx), np.uint8)
    ra = np.ones((1, nx), np.float32)
    rb = np.zeros((1, nx), np.float32)
    c = np.zeros((1, nx), np.float32)
    c[0, nx // 2] = 1.0
    tau_d = 0.8
    lat = Lattice(Params(tau_d=tau_d, g_coh=0.0), solid, ra, rb, c)
    x = np.arange(nx)
    var = []
    for _ in range(4):
        lat.step(400)
        C = lat.concentration()[0]
        mean = (C * x).sum() / C.sum()
        var.append((C * (x - mean) ** 2).sum() / C.sum())
        assert C.sum() == pytest.approx(1.0, rel=1e-13)
    slopes = np.diff(var) / 400
    assert np.allclose(slopes, 2 * (tau_d - 0.5) / 2, rtol=1e-9)


def test_reaction_one_step_closed_form(oracle_lib):
    # Uniform A-rich fluid at rest around a 3x2 solid block, uniform C0.
    # After one step each fluid node with n_s solid D2Q4 neighbours holds
    # m = k_r n_s C0 exactly (collision keeps C; the reaction takes
    # k_r n_s C*), and the solute lost equals the mass deposited.
    n = 10
    solid = np.zeros((n, n), np.uint8)
    solid[4:6, 3:6] = 1
    solid[2, 8] = solid[3, 7] = solid[1, 7] = 1  # a notch: n_s = 2 and 3
    ra = np.where(solid == 0, 1.0, 0).astype(np.float32)
    rb = np.where(solid == 0, 0.006, 0).astype(np.float32)
    c0 = 0.75
    cc = np.where(solid == 0, c0, 0).astype(np.float32)
    k = 0.01
    lat = Lattice(Params(g_coh=0.0, k_r=k, m_threshold=10.0), solid, ra, rb,
                  cc)
    C0 = lat.concentration().sum()
    lat.step(1)
    m = lat.deposit()
    ns = np.zeros((n, n), int)
    for dx, dy in ((1, 0), (0, 1), (-1, 0), (0, -1)):
        ns += np.roll(solid, (-dy, -dx), axis=(0, 1))
    ns = ns * (solid == 0)
    assert set(np.unique(ns)) >= {0, 1, 2, 3}
    np.testing.assert_allclose(m, k * ns * np.float32(c0), rtol=1e-12,
                               atol=1e-17)
    assert lat.concentration().sum() + m.sum() == pytest.approx(C0,
                                                                rel=1e-14)


def test_reaction_gated_by_wetting_phase(oracle_lib):
    # Reading of where the reactant deposits: only where the melt (A) is the
    # majority.  B-rich nodes next to the solid get nothing.
    n = 10
    solid = np.zeros((n, n), np.uint8)
    solid[0, :] = 1
    x = np.arange(n)[None, :].repeat(n, 0)
    a_rich = x < 5
    ra = np.where(a_rich, 1.0, 0.006).astype(np.float32) * (solid == 0)
    rb = np.where(a_rich, 0.006, 1.0).astype(np.float32) * (solid == 0)
    cc = np.where(solid == 0, 1.0, 0).astype(np.float32)
    lat = Lattice(Params(g_coh=0.0, k_r=0.01, m_threshold=10.0), solid, ra,
                  rb, cc)
    lat.step(1)
    m = lat.deposit()
    # rows 1 and n-1 (periodic in y) touch the wall row 0
    for row in (1, n - 1):
        assert np.all(m[row, :5] > 0)
        assert np.all(m[row, 5:] == 0)
    assert np.all(m[2:n - 1, :] == 0)


def test_growth_moves_post_stream_content_to_ledger(oracle_lib):
    # Nodes turn solid after streaming.  Everything up to the end of the
    # streaming is the same with and without the flip, so the ledger of a
    # run whose threshold is crossed in step 1 equals the post-stream
    # content of the same nodes in a run with an unreachable threshold.
    geom = I.random_lattice(16, 12, seed=21, solid_fraction=0.2)
    f, g = I.random_populations(geom, seed=22)
    m0 = np.where(geom.solid == 0, 0.999, 0.0)

    def run(th):
        lat = _lat(geom, g_ads=0.3, k_r=0.05, m_threshold=th)
        lat.set_populations(f)
        lat.set_solute(g)
        lat.set_deposit(m0)
        lat.step(1)
        return lat

    a = run(1.0)
    b = run(1e9)
    flipped = (a.solid() == 1) & (geom.solid == 0)
    assert flipped.sum() > 5
    fb = b.populations()
    led = a.ledger()
    assert led[0] == pytest.approx(fb[0][:, flipped].sum(), rel=1e-13)
    assert led[1] == pytest.approx(fb[1][:, flipped].sum(), rel=1e-13)
    assert led[2] == pytest.approx(b.solute()[:, flipped].sum(), rel=1e-13)
    assert led[3] == pytest.approx(b.deposit()[flipped].sum(), rel=1e-13)
    # exactly the nodes whose deposit reached the threshold flipped
    assert np.array_equal(flipped, (b.deposit() >= 1.0) & (geom.solid == 0))
    # and they hold nothing afterwards
    assert np.all(a.populations()[:, :, flipped] == 0)


def test_closure_step_brute_force(oracle_lib):
    # The pore-closure step is the first step count after which some column
    # of the capillary section is entirely solid: check it by stepping one
    # at a time and inspecting the mask.  A narrow walled channel full of A
    # with solute only in a few columns closes there first.
    nx, ny = 30, 7
    solid = np.zeros((ny, nx), np.uint8)
    solid[0, :] = solid[ny - 1, :] = 1
    fl = solid == 0
    ra = np.where(fl, 1.0, 0).astype(np.float32)
    rb = np.where(fl, 0.006, 0).astype(np.float32)
    cc = np.zeros((ny, nx), np.float32)
    cc[:, 12:16] = 1.0
    cc[~fl] = 0
    lat = Lattice(Params(g_ads=I.G_ADS_30, k_r=2e-2, m_threshold=0.1,
                         cap_x0=2, cap_x1=28), solid, ra, rb, cc)
    seen = -1
    for t in range(1, 3000):
        lat.step(1)
        s = lat.solid()[:, 2:28]
        if s.all(axis=0).any():
            seen = t
            break
    assert seen > 0
    assert lat.closure_step == seen
