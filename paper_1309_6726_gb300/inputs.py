"""Seeded synthetic inputs: geometries, initial fields and model constants.

This module holds no arithmetic of the method.  It only lays out solid
masks, initial densities and concentrations, and picks constants, so both
the CUDA path and the FP64 oracle can be fed the same inputs.  Random
draws use ``numpy.random.default_rng(seed)``.

Geometry conventions (lattice nx by ny, periodic in x and y, row-major):

* capillary: solid walls one node thick at y = 0 and y = ny - 1 over the
  capillary section x in [x_res, nx - x_out); the wall-free band
  x < x_res is a reservoir of the wetting melt A (and of solute at c_in);
  the rest is filled with the displaced component B.  The periodic wrap
  joins the B outlet band to the A reservoir through a flat interface, so
  only the meniscus inside the capillary drives the flow (the paper's
  single capillary in the linear Washburn regime, Sec. III).
* the capillary height H is the number of fluid rows, ny - 2, and its
  length L is nx - x_res - x_out.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, asdict

import numpy as np

#: densities of the majority and minority component in each bulk phase
RHO_MAJOR = 1.0
RHO_MINOR = 0.006

#: Adhesion strength g (G_ads,A = -g, G_ads,B = +g) giving the contact
#: angle theta with G_c = 2.5, rho 1.0 / 0.006, tau_A = tau_B = 1.0, from the
#: static-meniscus calibration in ``oracle/calibrate_contact_angle.py``.
#: Pairs (theta in degrees, g).
CONTACT_ANGLE_TABLE: tuple[tuple[float, float], ...] = (
    (66.43, 0.250),
    (61.54, 0.300),
    (55.31, 0.350),
    (48.06, 0.400),
    (40.26, 0.450),
    (30.48, 0.500),
    (25.14, 0.520),
    (18.24, 0.540),
)

#: g for the paper's 30 degree contact angle (paper Sec. I), interpolated
#: in the table above.
G_ADS_30 = 0.502


def g_ads_for_angle(theta_deg: float) -> float:
    """Adhesion g for a contact angle, by linear interpolation in the table."""
    if not CONTACT_ANGLE_TABLE:
        raise RuntimeError("contact-angle table not calibrated")
    th = np.array([t for t, _ in CONTACT_ANGLE_TABLE])
    gs = np.array([g for _, g in CONTACT_ANGLE_TABLE])
    order = np.argsort(th)
    return float(np.interp(theta_deg, th[order], gs[order]))


@dataclass
class ModelParams:
    """Constants of one lattice; field names match the C-ABI struct."""
    tau_a: float = 1.0
    tau_b: float = 1.0
    tau_d: float = 0.8
    g_coh: float = 2.5
    g_ads: float = 0.0
    k_r: float = 0.0
    m_threshold: float = 1.0
    c_in: float = 1.0
    body_force_x: float = 0.0
    inlet: int = 0

    def as_dict(self) -> dict:
        return asdict(self)


@dataclass
class Geometry:
    """Solid mask and initial fields of one lattice, all shaped (ny, nx)."""
    solid: np.ndarray
    rho_a: np.ndarray
    rho_b: np.ndarray
    conc: np.ndarray
    cap_x0: int = 0
    cap_x1: int = 0
    extra: dict = field(default_factory=dict)

    @property
    def nx(self) -> int:
        return int(self.solid.shape[1])

    @property
    def ny(self) -> int:
        return int(self.solid.shape[0])


def _phase_fields(a_rich: np.ndarray, solid: np.ndarray):
    rho_a = np.where(a_rich, RHO_MAJOR, RHO_MINOR).astype(np.float32)
    rho_b = np.where(a_rich, RHO_MINOR, RHO_MAJOR).astype(np.float32)
    rho_a[solid != 0] = 0
    rho_b[solid != 0] = 0
    return rho_a, rho_b


def capillary(nx: int, ny: int, x_res: int, x_out: int,
              c_in: float = 1.0) -> Geometry:
    """Single straight capillary between an A reservoir and a B outlet band."""
    if not (0 < x_res and 0 < x_out and x_res + x_out < nx and ny >= 3):
        raise ValueError("bad capillary dimensions")
    solid = np.zeros((ny, nx), np.uint8)
    solid[0, x_res:nx - x_out] = 1
    solid[ny - 1, x_res:nx - x_out] = 1
    xs = np.arange(nx)[None, :].repeat(ny, 0)
    a_rich = xs < x_res
    rho_a, rho_b = _phase_fields(a_rich, solid)
    conc = np.where(a_rich, c_in, 0.0).astype(np.float32)
    conc[solid != 0] = 0
    return Geometry(solid, rho_a, rho_b, conc, x_res, nx - x_out,
                    {"kind": "capillary", "x_res": x_res, "x_out": x_out})


def channel(nx: int, ny: int, rho: float = 1.0) -> Geometry:
    """Straight channel with walls along its whole length, filled with A only
    (single-component limit, for the Poiseuille check)."""
    solid = np.zeros((ny, nx), np.uint8)
    solid[0, :] = 1
    solid[ny - 1, :] = 1
    rho_a = np.where(solid == 0, rho, 0.0).astype(np.float32)
    z = np.zeros((ny, nx), np.float32)
    return Geometry(solid, rho_a, z.copy(), z.copy(), 0, nx,
                    {"kind": "channel"})


def drop(n: int, radius: float) -> Geometry:
    """Disc of A of the given radius centred in an n by n periodic box of B."""
    solid = np.zeros((n, n), np.uint8)
    y, x = np.mgrid[0:n, 0:n]
    c = (n - 1) / 2.0
    inside = (x - c) ** 2 + (y - c) ** 2 <= radius ** 2
    rho_a, rho_b = _phase_fields(inside, solid)
    return Geometry(solid, rho_a, rho_b, np.zeros((n, n), np.float32), 0, n,
                    {"kind": "drop", "radius": radius})


def flat_interface(nx: int, ny: int) -> Geometry:
    """A in the left half, B in the right half of a periodic box."""
    solid = np.zeros((ny, nx), np.uint8)
    x = np.arange(nx)[None, :].repeat(ny, 0)
    rho_a, rho_b = _phase_fields(x < nx // 2, solid)
    return Geometry(solid, rho_a, rho_b, np.zeros((ny, nx), np.float32), 0,
                    nx, {"kind": "flat"})


def slug(nx: int, ny: int, length: int) -> Geometry:
    """Closed channel (walls along the whole length, periodic in x) holding a
    slug of A of the given length in the middle, B on both sides: two static
    menisci (contact-angle calibration)."""
    solid = np.zeros((ny, nx), np.uint8)
    solid[0, :] = 1
    solid[ny - 1, :] = 1
    x = np.arange(nx)[None, :].repeat(ny, 0)
    x0 = (nx - length) // 2
    a_rich = (x >= x0) & (x < x0 + length)
    rho_a, rho_b = _phase_fields(a_rich, solid)
    return Geometry(solid, rho_a, rho_b, np.zeros((ny, nx), np.float32), 0,
                    nx, {"kind": "slug", "x0": x0, "length": length})


def random_lattice(nx: int, ny: int, seed: int,
                   solid_fraction: float = 0.15,
                   conc: bool = True) -> Geometry:
    """Random solid nodes and random two-phase blobs (parity inputs)."""
    rng = np.random.default_rng(seed)
    solid = (rng.random((ny, nx)) < solid_fraction).astype(np.uint8)
    a_rich = rng.random((ny, nx)) < 0.5
    rho_a, rho_b = _phase_fields(a_rich, solid)
    c = (rng.random((ny, nx)) if conc else np.zeros((ny, nx))).astype(
        np.float32)
    c[solid != 0] = 0
    return Geometry(solid, rho_a, rho_b, c, 0, nx,
                    {"kind": "random", "seed": seed})


def random_populations(geom: Geometry, seed: int,
                       spread: float = 0.3) -> tuple[np.ndarray, np.ndarray]:
    """Random positive, non-equilibrium populations for a geometry: fluid
    (2, 9, ny, nx) and solute (4, ny, nx), zero at solid nodes.  Each value
    is a lattice weight times the node's initial density (or a quarter of its
    concentration) times a factor drawn uniformly from [1 - spread,
    1 + spread]."""
    rng = np.random.default_rng(seed)
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4, np.float64)
    ny, nx = geom.solid.shape
    fl = (geom.solid == 0)
    f = np.zeros((2, 9, ny, nx), np.float64)
    for s, rho in enumerate((geom.rho_a, geom.rho_b)):
        fac = 1.0 + spread * (2 * rng.random((9, ny, nx)) - 1)
        f[s] = w[:, None, None] * rho[None].astype(np.float64) * fac
    g = 0.25 * geom.conc[None].astype(np.float64) * (
        1.0 + spread * (2 * rng.random((4, ny, nx)) - 1))
    f = (f * fl[None, None]).astype(np.float32)
    g = (g * fl[None]).astype(np.float32)
    return f, g


# --------------------------------------------------------------------------
# The five workloads the project is measured on, with fixed seeds.
# --------------------------------------------------------------------------

def config_small() -> tuple[Geometry, ModelParams, int]:
    """256 x 32 capillary, reservoir 64 columns, outlet band 32 columns,
    tau = 1.0 both, D2Q4 tau_D = 0.8, c_in = 1.0, k_r = 1e-3, threshold 1.0,
    2000 steps."""
    geom = capillary(256, 32, 64, 32)
    p = ModelParams(g_ads=G_ADS_30, k_r=1e-3, inlet=1)
    return geom, p, 2000


def config_paper_scale(k_r: float = 1e-3) -> tuple[Geometry, ModelParams,
                                                    int]:
    """4096 x 128 capillary (H = 126, L = 3712), k_r in {0, 1e-4, 1e-3}."""
    geom = capillary(4096, 128, 256, 128)
    p = ModelParams(g_ads=G_ADS_30, k_r=k_r, inlet=1)
    return geom, p, 200_000


@dataclass
class SweepMember:
    width: int        # H, fluid rows of the capillary
    length: int       # L, capillary length
    k_r: float
    theta_deg: float
    tau_ratio: float  # tau_A / tau_B with tau_B = 1.0


def sweep_members(count: int = 512, seed: int = 1236) -> list[SweepMember]:
    """Parameters of the batched sweep: widths uniform over integers 16-128,
    lengths uniform over integers 1024-4096, k_r log-uniform on
    [1e-5, 1e-2], contact angle uniform on [20, 60] degrees, viscosity
    ratio tau_A / tau_B uniform on [0.6, 1.5]."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        w = int(rng.integers(16, 129))
        ln = int(rng.integers(1024, 4097))
        k = float(10 ** rng.uniform(-5, -2))
        th = float(rng.uniform(20, 60))
        tr = float(rng.uniform(0.6, 1.5))
        out.append(SweepMember(w, ln, k, th, tr))
    return out


def sweep_lattice(member: SweepMember, x_res: int = 64,
                  x_out: int = 32) -> tuple[Geometry, ModelParams]:
    geom = capillary(member.length + x_res + x_out, member.width + 2, x_res,
                     x_out)
    p = ModelParams(tau_a=member.tau_ratio * 1.0, tau_b=1.0,
                    g_ads=g_ads_for_angle(member.theta_deg), k_r=member.k_r,
                    inlet=1)
    return geom, p


def preform(n: int = 2048, seed: int = 1237, x_res: int = 128,
            x_out: int = 128, median_radius: float = 12.0,
            sigma: float = 0.4, solid_fraction: float = 0.5,
            max_tries: int = 2_000_000) -> Geometry:
    """Synthetic carbon preform: non-overlapping solid discs with lognormal
    radii (median 12, sigma 0.4), placed by random sequential addition with
    at least one fluid node between discs, in x in [x_res, n - x_out), until
    the solid fraction there reaches ``solid_fraction``.  A reservoir of A
    (with solute) fills x < x_res, B fills the rest; y is periodic."""
    rng = np.random.default_rng(seed)
    solid = np.zeros((n, n), np.uint8)
    x_lo, x_hi = x_res, n - x_out
    area = (x_hi - x_lo) * n
    filled = 0
    tries = 0
    while filled < solid_fraction * area and tries < max_tries:
        tries += 1
        r = float(median_radius * math.exp(sigma * rng.standard_normal()))
        r = max(1.5, min(r, 0.25 * (x_hi - x_lo)))
        cx = rng.uniform(x_lo + r, x_hi - r)
        cy = rng.uniform(0, n)
        ri = int(math.ceil(r)) + 1
        xs = np.arange(int(cx) - ri, int(cx) + ri + 2)
        ys = np.arange(int(cy) - ri, int(cy) + ri + 2)
        xs = xs[(xs >= x_lo) & (xs < x_hi)]
        X, Y = np.meshgrid(xs, ys)
        d2 = (X - cx) ** 2 + (Y - cy) ** 2
        disc = d2 <= r * r
        halo = d2 <= (r + 1.5) ** 2
        if solid[Y[halo] % n, X[halo]].any():
            continue
        ty = (Y[disc] % n)
        tx = X[disc]
        newly = solid[ty, tx] == 0
        solid[ty, tx] = 1
        filled += int(newly.sum())
    xs = np.arange(n)[None, :].repeat(n, 0)
    a_rich = xs < x_res
    rho_a, rho_b = _phase_fields(a_rich, solid)
    conc = np.where(a_rich & (solid == 0), 1.0, 0.0).astype(np.float32)
    return Geometry(solid, rho_a, rho_b, conc, x_lo, x_hi,
                    {"kind": "preform", "seed": seed,
                     "solid_fraction": filled / area})


def config_preform() -> tuple[Geometry, ModelParams, int]:
    """2048 x 2048 disc preform, k_r = 1e-3, 100k steps."""
    geom = preform()
    p = ModelParams(g_ads=G_ADS_30, k_r=1e-3, inlet=1)
    return geom, p, 100_000
