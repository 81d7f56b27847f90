"""ctypes wrapper of the FP64 oracle library (``lbm_oracle.c``).

Test infrastructure only: the tests, the smoke check and the benchmark's
CPU-baseline leg use it; the CUDA library never does.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np

from . import build as _build

Q, QS = 9, 4


class _Params(C.Structure):
    _fields_ = [
        ("tau_a", C.c_double), ("tau_b", C.c_double), ("tau_d", C.c_double),
        ("g_coh", C.c_double), ("g_ads", C.c_double), ("k_r", C.c_double),
        ("m_threshold", C.c_double), ("c_in", C.c_double),
        ("body_force_x", C.c_double), ("inlet", C.c_int32),
        ("cap_x0", C.c_int32), ("cap_x1", C.c_int32),
    ]


_lib = None


def load(path: str | None = None):
    """Loads (building first if needed) the oracle library."""
    global _lib
    if path is not None:
        return _bind(C.CDLL(path))
    if _lib is None:
        _lib = _bind(C.CDLL(_build.build()))
    return _lib


def _bind(lib):
    dp = C.POINTER(C.c_double)
    u8p = C.POINTER(C.c_uint8)
    lib.orc_create.restype = C.c_void_p
    lib.orc_create.argtypes = [C.POINTER(_Params), C.c_int, C.c_int, u8p, dp,
                               dp, dp]
    lib.orc_destroy.argtypes = [C.c_void_p]
    lib.orc_step.argtypes = [C.c_void_p, C.c_int64]
    lib.orc_step_count.restype = C.c_int64
    lib.orc_step_count.argtypes = [C.c_void_p]
    lib.orc_closure_step.restype = C.c_int64
    lib.orc_closure_step.argtypes = [C.c_void_p]
    lib.orc_ledger.argtypes = [C.c_void_p, dp]
    lib.orc_get.restype = C.c_int
    lib.orc_get.argtypes = [C.c_void_p, C.c_int, dp]
    lib.orc_set.restype = C.c_int
    lib.orc_set.argtypes = [C.c_void_p, C.c_int, dp]
    lib.orc_get_solid.argtypes = [C.c_void_p, u8p]
    lib.orc_moments_forces.argtypes = [C.c_void_p, dp, dp]
    lib.orc_feq.argtypes = [C.c_double, C.c_double, C.c_double, dp]
    lib.orc_geq.argtypes = [C.c_double, C.c_double, C.c_double, dp]
    return lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def feq(rho: float, ux: float, uy: float, lib=None) -> np.ndarray:
    """D2Q9 BGK equilibrium (9 values) as the oracle evaluates it."""
    lib = lib or load()
    out = np.zeros(Q)
    lib.orc_feq(rho, ux, uy, _dptr(out))
    return out


def geq(c: float, ux: float, uy: float, lib=None) -> np.ndarray:
    """D2Q4 solute equilibrium (4 values) as the oracle evaluates it."""
    lib = lib or load()
    out = np.zeros(QS)
    lib.orc_geq(c, ux, uy, _dptr(out))
    return out


@dataclass
class Params:
    """Model constants of one lattice (same meaning as the C struct)."""
    tau_a: float = 1.0
    tau_b: float = 1.0
    tau_d: float = 0.8
    g_coh: float = 3.0
    g_ads: float = 0.0
    k_r: float = 0.0
    m_threshold: float = 1.0
    c_in: float = 1.0
    body_force_x: float = 0.0
    inlet: int = 0
    cap_x0: int = 0
    cap_x1: int = 0

    def to_c(self) -> _Params:
        return _Params(self.tau_a, self.tau_b, self.tau_d, self.g_coh,
                       self.g_ads, self.k_r, self.m_threshold, self.c_in,
                       self.body_force_x, int(self.inlet), int(self.cap_x0),
                       int(self.cap_x1))


class Lattice:
    """One FP64 oracle lattice, nx by ny, periodic in x and y.

    ``solid``, ``rho_a``, ``rho_b`` and ``conc`` are (ny, nx) arrays; every
    fluid node starts at rest equilibrium for its densities and
    concentration.
    """

    def __init__(self, params: Params, solid, rho_a, rho_b, conc, lib=None):
        self._lib = lib or load()
        solid = np.ascontiguousarray(solid, dtype=np.uint8)
        self.ny, self.nx = solid.shape
        ra = np.ascontiguousarray(rho_a, dtype=np.float64)
        rb = np.ascontiguousarray(rho_b, dtype=np.float64)
        cc = np.ascontiguousarray(conc, dtype=np.float64)
        for a in (ra, rb, cc):
            if a.shape != solid.shape:
                raise ValueError("field shape %s != solid shape %s"
                                 % (a.shape, solid.shape))
        self.params = params
        self._cp = params.to_c()
        self.initial_solid = solid.copy()
        self._h = self._lib.orc_create(
            C.byref(self._cp), self.nx, self.ny,
            solid.ctypes.data_as(C.POINTER(C.c_uint8)), _dptr(ra), _dptr(rb),
            _dptr(cc))
        if not self._h:
            raise MemoryError("orc_create failed")

    def close(self):
        if getattr(self, "_h", None):
            self._lib.orc_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    @property
    def N(self) -> int:
        return self.nx * self.ny

    def step(self, n: int = 1) -> None:
        self._lib.orc_step(self._h, int(n))

    @property
    def step_count(self) -> int:
        return int(self._lib.orc_step_count(self._h))

    @property
    def closure_step(self) -> int:
        return int(self._lib.orc_closure_step(self._h))

    def ledger(self) -> np.ndarray:
        """Mass moved out of the fluid by growth: [A, B, solute, deposit]."""
        out = np.zeros(4)
        self._lib.orc_ledger(self._h, _dptr(out))
        return out

    def populations(self) -> np.ndarray:
        """Post-stream populations, shape (2, 9, ny, nx): A then B."""
        out = np.zeros(2 * Q * self.N)
        self._lib.orc_get(self._h, 0, _dptr(out))
        return out.reshape(2, Q, self.ny, self.nx)

    def solute(self) -> np.ndarray:
        """Post-stream solute populations, shape (4, ny, nx)."""
        out = np.zeros(QS * self.N)
        self._lib.orc_get(self._h, 1, _dptr(out))
        return out.reshape(QS, self.ny, self.nx)

    def deposit(self) -> np.ndarray:
        """Precipitated mass per node, shape (ny, nx)."""
        out = np.zeros(self.N)
        self._lib.orc_get(self._h, 2, _dptr(out))
        return out.reshape(self.ny, self.nx)

    def solid(self) -> np.ndarray:
        out = np.zeros(self.N, dtype=np.uint8)
        self._lib.orc_get_solid(self._h, out.ctypes.data_as(
            C.POINTER(C.c_uint8)))
        return out.reshape(self.ny, self.nx)

    def set_populations(self, f: np.ndarray) -> None:
        a = np.ascontiguousarray(f, dtype=np.float64).reshape(-1)
        assert a.size == 2 * Q * self.N
        self._lib.orc_set(self._h, 0, _dptr(a))

    def set_solute(self, g: np.ndarray) -> None:
        a = np.ascontiguousarray(g, dtype=np.float64).reshape(-1)
        assert a.size == QS * self.N
        self._lib.orc_set(self._h, 1, _dptr(a))

    def set_deposit(self, m: np.ndarray) -> None:
        a = np.ascontiguousarray(m, dtype=np.float64).reshape(-1)
        assert a.size == self.N
        self._lib.orc_set(self._h, 2, _dptr(a))

    def densities(self) -> tuple[np.ndarray, np.ndarray]:
        f = self.populations()
        return f[0].sum(axis=0), f[1].sum(axis=0)

    def concentration(self) -> np.ndarray:
        return self.solute().sum(axis=0)

    def moments_forces(self) -> tuple[np.ndarray, np.ndarray]:
        """(rho[2, ny, nx], F[2 comps, 2 axes, ny, nx]) of the current state."""
        rho = np.zeros(2 * self.N)
        F = np.zeros(4 * self.N)
        self._lib.orc_moments_forces(self._h, _dptr(rho), _dptr(F))
        return (rho.reshape(2, self.ny, self.nx),
                F.reshape(2, 2, self.ny, self.nx))
