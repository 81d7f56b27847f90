"""Shared helpers of the GPU parity tests: run the same seeded input through
the CUDA library (via its C ABI) and through the FP64 oracle, and compare."""
import numpy as np

from oracle.lattice import Lattice, Params

W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
W22 = np.concatenate([W9, W9, [0.25] * 4])

#: planes of each component in the 22-plane population stack
COMPONENTS = (("A", 0, 9), ("B", 9, 18), ("C", 18, 22))

#: density floor of the relative error: a node enters a component's
#: relative error when the oracle's density of that component there is at
#: least this (six times below the minority density 0.006, so the minority
#: phase is included; nodes a component has practically left are not)
REL_FLOOR = 1e-3


def oracle_for(geom, mp):
    p = Params(**mp.as_dict(), cap_x0=geom.cap_x0, cap_x1=geom.cap_x1)
    return Lattice(p, geom.solid, geom.rho_a, geom.rho_b, geom.conc)


def oracle_pops(lat):
    ny, nx = lat.ny, lat.nx
    return np.concatenate([lat.populations().reshape(18, ny, nx),
                           lat.solute()])


def pop_error(f_gpu, f_ora, scale_rho=1.0):
    """Largest |f_gpu - f_oracle| over all populations, each divided by its
    lattice weight times a reference density (so 1e-5 means 1e-5 of a
    population of a fluid at density ``scale_rho``)."""
    d = np.abs(f_gpu.astype(np.float64) - f_ora) / (W22[:, None, None] *
                                                   scale_rho)
    return float(d.max())


def pop_rel_error(f_gpu, f_ora, floor=REL_FLOOR):
    """Per-component relative error: the largest
    |f_gpu - f_oracle| / (w_i rho_sigma(x)) over the populations of each
    component (A, B, and the solute with C(x) and w = 1/4), where
    rho_sigma(x) is the oracle's density of that component at the node
    (C for the solute), over the nodes where it is at least ``floor``.
    Returns a dict {"A": ..., "B": ..., "C": ...} (0 where no node
    qualifies)."""
    d = np.abs(f_gpu.astype(np.float64) - f_ora)
    out = {}
    for name, lo, hi in COMPONENTS:
        rho = f_ora[lo:hi].sum(axis=0)
        sel = rho >= floor
        if not sel.any():
            out[name] = 0.0
            continue
        e = d[lo:hi][:, sel] / (W22[lo:hi, None] * rho[sel])
        out[name] = float(e.max())
    return out


def assert_rel(f_gpu, f_ora, tol, floor=REL_FLOOR):
    """Asserts the per-component relative error (pop_rel_error) of every
    component below ``tol`` (a number, or a dict per component); returns the
    errors."""
    err = pop_rel_error(f_gpu, f_ora, floor)
    for name, v in err.items():
        t = tol[name] if isinstance(tol, dict) else tol
        assert v < t, "component %s: relative error %.3g >= %.3g" % (name, v, t)
    return err
