"""Shared helpers of the GPU parity tests: run the same seeded input through
the CUDA library (via its C ABI) and through the FP64 oracle, and compare."""
import numpy as np

from oracle.lattice import Lattice, Params

W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
W22 = np.concatenate([W9, W9, [0.25] * 4])


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
