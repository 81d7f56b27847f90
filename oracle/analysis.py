"""Observables and theory of the capillary problem, in plain numpy.

Test infrastructure only (the tests, the smoke check and the benchmark's
CPU-baseline leg).  Everything here reads the oracle's post-stream state
(densities, solute, deposit, solid mask) and follows the definitions below;
none of it is shared with the CUDA library.

Definitions (paper Sec. III and Figs. 2-4; the paper names the quantities
but not their lattice formulas, so the formulas are readings):

* capillary section: columns x in [x0, x1); walls were one node thick at
  y = 0 and y = ny - 1 at the start; centerline y_c = (ny - 1) / 2.
* front z (Fig. 2, Eq. 1): on each centerline row (rows floor(y_c) and
  ceil(y_c)), the first x >= x0 - 1 where phi = rho_A - rho_B goes from
  > 0 at x to <= 0 at x + 1 with both nodes fluid, placed by linear
  interpolation, minus the entrance plane x0 - 1/2; the mean over the
  centerline rows.  NaN where no such crossing exists.
* lower-wall thickness b(x): number of solid nodes stacked from y = 0 up
  to the first fluid node; upper t(x) likewise from y = ny - 1 down.
* Delta e (Fig. 3): the largest grown thickness b(x) - b0(x) or
  t(x) - t0(x) over the section (b0, t0 from the initial mask); a fully
  solid column counts half of its initial gap, i.e. H/2.
* aperture h(x): fluid nodes in column x; r_min = min h / 2,
  r_ave = mean h / 2 (Fig. 4).
* r_h = A / P (Fig. 4): A = fluid area between the lower-wall profile
  (surface at y = b(x) - 1/2) and the centerline, P = length of that
  profile, one per column plus |b(x+1) - b(x)| between columns.
* r_eff (Fig. 4): Eq. 1 solved for H with the least-squares front speed,
  cos(theta) of the non-reactive run and the fluid's gamma and mu; half
  of that H.
* wetted length, per wall: fluid nodes next to that wall's profile, in
  the section, where rho_A > rho_B.
"""
from __future__ import annotations

import math

import numpy as np

OBS_KEYS = ("front", "wetted_lower", "wetted_upper", "r_min", "r_h",
            "r_ave", "delta_e", "precip_mass", "mass_a", "mass_b",
            "mass_c", "ledger_a", "ledger_b", "ledger_c", "ledger_m",
            "closed")


def wall_profiles(solid: np.ndarray, x0: int, x1: int):
    """b(x), t(x) and h(x) over columns [x0, x1) (see module text)."""
    ny = solid.shape[0]
    cols = solid[:, x0:x1].astype(bool)
    fluid = ~cols
    h = fluid.sum(axis=0)
    b = np.where(fluid.any(axis=0), np.argmax(fluid, axis=0), ny)
    t = np.where(fluid.any(axis=0), np.argmax(fluid[::-1], axis=0), ny)
    return b, t, h


def centerline_rows(ny: int) -> list[int]:
    yc = (ny - 1) / 2.0
    return sorted({int(math.floor(yc)), int(math.ceil(yc))})


def front_position(rho_a, rho_b, solid, x0: int) -> float:
    """Centerline front z (see module text)."""
    ny, nx = solid.shape
    zs = []
    for y in centerline_rows(ny):
        phi = rho_a[y] - rho_b[y]
        found = math.nan
        for x in range(max(x0 - 1, 0), nx - 1):
            if solid[y, x] or solid[y, x + 1]:
                continue
            if phi[x] > 0 and phi[x + 1] <= 0:
                found = x + phi[x] / (phi[x] - phi[x + 1]) - (x0 - 0.5)
                break
        zs.append(found)
    return float(np.mean(zs))


def observables(rho_a, rho_b, conc, deposit, solid, initial_solid,
                x0: int, x1: int, ledger) -> dict:
    """All observables of one lattice state (see module text)."""
    ny, nx = solid.shape
    fl = solid == 0
    b, t, h = wall_profiles(solid, x0, x1)
    b0, t0, _ = wall_profiles(initial_solid, x0, x1)
    closed_cols = h == 0
    grown = np.maximum(b - b0, t - t0).astype(np.float64)
    half_gap = (ny - b0 - t0) / 2.0
    grown = np.where(closed_cols, half_gap, grown)
    yc = (ny - 1) / 2.0
    area = np.maximum(0.0, yc - (b - 0.5))
    perim = len(b) + np.abs(np.diff(b)).sum()
    wet_lo = 0
    wet_up = 0
    for k, x in enumerate(range(x0, x1)):
        if closed_cols[k]:
            continue
        yl = b[k]
        yu = ny - 1 - t[k]
        if rho_a[yl, x] > rho_b[yl, x]:
            wet_lo += 1
        if rho_a[yu, x] > rho_b[yu, x]:
            wet_up += 1
    led = np.asarray(ledger, dtype=np.float64)
    return {
        "front": front_position(rho_a, rho_b, solid, x0),
        "wetted_lower": float(wet_lo),
        "wetted_upper": float(wet_up),
        "r_min": float(h.min()) / 2.0,
        "r_h": float(area.sum() / perim) if perim > 0 else 0.0,
        "r_ave": float(h.mean()) / 2.0,
        "delta_e": float(grown.max()),
        "precip_mass": float(deposit[fl].sum() + led[3]),
        "mass_a": float(rho_a[fl].sum()),
        "mass_b": float(rho_b[fl].sum()),
        "mass_c": float(conc[fl].sum()),
        "ledger_a": float(led[0]),
        "ledger_b": float(led[1]),
        "ledger_c": float(led[2]),
        "ledger_m": float(led[3]),
        "closed": float(closed_cols.any()),
    }


def lattice_observables(lat) -> dict:
    """Observables of an :class:`oracle.lattice.Lattice`."""
    ra, rb = lat.densities()
    return observables(ra, rb, lat.concentration(), lat.deposit(),
                       lat.solid(), lat.initial_solid, lat.params.cap_x0,
                       lat.params.cap_x1, lat.ledger())


# ---- theory ---------------------------------------------------------------

def washburn_z(t, gamma: float, mu: float, rho: float, H: float, L: float,
               cos_theta: float):
    """Eq. 1: z(t) = (V_cap H cos(theta) / 6L) t_d [exp(-t/t_d) + t/t_d - 1]
    with V_cap = gamma / mu and t_d = rho H^2 / (12 mu)."""
    t = np.asarray(t, dtype=np.float64)
    v_cap = gamma / mu
    t_d = rho * H * H / (12.0 * mu)
    return v_cap * H * cos_theta / (6.0 * L) * t_d * (
        np.exp(-t / t_d) + t / t_d - 1.0)


def washburn_speed(gamma: float, mu: float, H: float, L: float,
                   cos_theta: float) -> float:
    """Late-time slope of Eq. 1, dz/dt = gamma H cos(theta) / (6 mu L)."""
    return gamma * H * cos_theta / (6.0 * mu * L)


def lattice_viscosity(rho: float, tau: float) -> float:
    """Dynamic viscosity of a BGK D2Q9 fluid, mu = rho (tau - 1/2) / 3."""
    return rho * (tau - 0.5) / 3.0


def fit_reff(t, z, gamma: float, mu: float, L: float,
             cos_theta0: float) -> float:
    """Effective radius: least-squares front speed v put into the late-time
    form of Eq. 1 solved for H, r_eff = H / 2 = 3 mu L v / (gamma cos)."""
    t = np.asarray(t, dtype=np.float64)
    z = np.asarray(z, dtype=np.float64)
    v = np.polyfit(t, z, 1)[0]
    return 3.0 * mu * L * v / (gamma * cos_theta0)


def mixture_pressure(rho_a, rho_b, g_coh: float):
    """Bulk pressure of the two-component fluid with the cohesion force
    above: p = (rho_A + rho_B) / 3 + G_c rho_A rho_B / 3 (second moment of
    the force stencil: sum_i w_i e_i e_i = I / 3)."""
    return (rho_a + rho_b) / 3.0 + g_coh * rho_a * rho_b / 3.0


def meniscus_cos_theta(rho_a, rho_b, solid, x_from: int, wall_skip: int = 3):
    """cos(theta) of a meniscus in a straight channel with walls at y = 0 and
    ny - 1: interface points phi = 0 on each fluid row (first + to - crossing
    at x >= x_from), a circle with centre on the channel axis fitted to the
    rows at least ``wall_skip`` rows from the walls, cos = (H/2) / R, positive
    when the centre lies ahead of the interface (A wets).  Returns (cos, R)."""
    ny, nx = solid.shape
    H = ny - 2
    yc = (ny - 1) / 2.0
    xs, ys = [], []
    for y in range(1, ny - 1):
        phi = rho_a[y] - rho_b[y]
        for x in range(x_from, nx - 1):
            if phi[x] > 0 and phi[x + 1] <= 0:
                xs.append(x + phi[x] / (phi[x] - phi[x + 1]))
                ys.append(y - yc)
                break
    xs = np.array(xs)
    ys = np.array(ys)
    sel = np.abs(ys) <= H / 2.0 - wall_skip
    X, Y = xs[sel], ys[sel]
    A = np.c_[2.0 * X, np.ones_like(X)]
    (a, c), *_ = np.linalg.lstsq(A, X ** 2 + Y ** 2, rcond=None)
    R = math.sqrt(c + a * a)
    sign = 1.0 if a > X.mean() else -1.0
    return sign * (H / 2.0) / R, R
