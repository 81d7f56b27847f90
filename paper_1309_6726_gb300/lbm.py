"""Python binding of the CUDA library (``liblbm.so``, C ABI in
``include/lbm.h``).  Argument marshalling only: every step of the method
runs in the library's kernels.  There is no fallback: if the library or a
CUDA device is missing, constructing a :class:`Solver` raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "liblbm.so")

LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_ETIMEOUT, LBM_ENAN, LBM_EIO = \
    range(7)
LBM_FP32, LBM_FP16, LBM_BF16 = 0, 1, 2
FIELD_POPS, FIELD_DEPOSIT, FIELD_DENSITY = 0, 1, 2
NPOP = 22

#: exported symbols (every entry point the header declares)
SYMBOLS = ("lbm_create", "lbm_create_batch", "lbm_set_stream", "lbm_step",
           "lbm_step_count", "lbm_count", "lbm_observables",
           "lbm_get_solid_mask", "lbm_get_solid_masks", "lbm_get_fields",
           "lbm_set_fields",
           "lbm_save", "lbm_load", "lbm_destroy", "lbm_last_error",
           "lbm_fit_reff", "lbm_observables_static", "lbm_autotune",
           "lbm_get_tuning", "lbm_plan_tiles")


class LbmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("lbm status %d: %s" % (status, msg))
        self.status = status


class Geometry(C.Structure):
    # the arrays as plain addresses (lbm_geometry's typed pointers have the
    # same representation); integers are quicker to marshal than casts
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32),
                ("solid", C.c_void_p), ("rho_a", C.c_void_p),
                ("rho_b", C.c_void_p), ("conc", C.c_void_p),
                ("cap_x0", C.c_int32), ("cap_x1", C.c_int32)]


class Params(C.Structure):
    _fields_ = [("tau_a", C.c_double), ("tau_b", C.c_double),
                ("tau_d", C.c_double), ("g_coh", C.c_double),
                ("g_ads", C.c_double), ("k_r", C.c_double),
                ("m_threshold", C.c_double), ("c_in", C.c_double),
                ("body_force_x", C.c_double), ("inlet", C.c_int32),
                ("precision", C.c_int32)]


class Tuning(C.Structure):
    _fields_ = [("kernel", C.c_int32), ("tx", C.c_int32), ("ty", C.c_int32),
                ("ms_per_step", C.c_double)]

    def as_dict(self) -> dict:
        return {"kernel": "tma" if self.kernel else "direct",
                "tile": "%dx%d" % (self.tx, self.ty),
                "ms_per_step": self.ms_per_step}


class Obs(C.Structure):
    _fields_ = [("step", C.c_int64), ("front", C.c_double),
                ("wetted_lower", C.c_double), ("wetted_upper", C.c_double),
                ("r_min", C.c_double), ("r_h", C.c_double),
                ("r_ave", C.c_double), ("delta_e", C.c_double),
                ("precip_mass", C.c_double), ("mass_a", C.c_double),
                ("mass_b", C.c_double), ("mass_c", C.c_double),
                ("ledger_a", C.c_double), ("ledger_b", C.c_double),
                ("ledger_c", C.c_double), ("ledger_m", C.c_double),
                ("closed", C.c_int32), ("nonfinite", C.c_int32),
                ("closure_step", C.c_int64)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


#: lbm_obs as a numpy record (the same bytes as Obs)
OBS_DTYPE = np.dtype([(n, {C.c_int64: np.int64, C.c_int32: np.int32,
                           C.c_double: np.float64}[t]) for n, t in Obs._fields_],
                     align=True)
assert OBS_DTYPE.itemsize == C.sizeof(Obs)


_lib = None


def load_library(path: str = LIB_PATH):
    """Loads the compiled library (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(
            "liblbm.so not built (run __graft_entry__.build()): %s" % path)
    lib = C.CDLL(path)
    vp = C.c_void_p
    lib.lbm_create.argtypes = [C.POINTER(Geometry), C.POINTER(Params),
                               C.POINTER(vp)]
    lib.lbm_create_batch.argtypes = [C.POINTER(Geometry), C.POINTER(Params),
                                     C.c_int32, C.POINTER(vp)]
    lib.lbm_set_stream.argtypes = [vp, vp]
    lib.lbm_step.argtypes = [vp, C.c_int64]
    lib.lbm_step_count.argtypes = [vp]
    lib.lbm_step_count.restype = C.c_int64
    lib.lbm_count.argtypes = [vp]
    lib.lbm_count.restype = C.c_int32
    lib.lbm_observables.argtypes = [vp, C.POINTER(Obs)]
    lib.lbm_get_solid_mask.argtypes = [vp, C.c_int32, C.POINTER(C.c_uint8),
                                       C.c_size_t]
    lib.lbm_get_solid_masks.argtypes = [vp, C.POINTER(C.c_uint8), C.c_size_t]
    lib.lbm_get_fields.argtypes = [vp, C.c_int32, C.c_int32, vp, C.c_size_t]
    lib.lbm_set_fields.argtypes = [vp, C.c_int32, C.c_int32, vp, C.c_size_t]
    lib.lbm_save.argtypes = [vp, C.c_char_p]
    lib.lbm_load.argtypes = [vp, C.c_char_p]
    lib.lbm_destroy.argtypes = [vp]
    lib.lbm_destroy.restype = None
    lib.lbm_last_error.argtypes = [vp]
    lib.lbm_last_error.restype = C.c_char_p
    dp = C.POINTER(C.c_double)
    lib.lbm_fit_reff.argtypes = [dp, dp, C.c_int32, C.c_double, C.c_double,
                                 C.c_double, C.c_double, dp]
    ip = C.POINTER(C.c_int32)
    lib.lbm_plan_tiles.argtypes = [ip, ip, C.c_int32, C.c_int32, C.c_int32,
                                   C.c_int32, ip, C.c_int64, ip]
    lib.lbm_autotune.argtypes = [vp, C.c_int32, C.POINTER(Tuning)]
    lib.lbm_get_tuning.argtypes = [vp, C.POINTER(Tuning)]
    lib.lbm_observables_static.argtypes = [vp, vp, vp, vp, C.c_int32,
                                           C.c_int32, C.c_int32, C.c_int32,
                                           dp, C.c_int64, C.c_int64, vp, vp]
    _lib = lib
    return lib


_PARAM_KEYS = ("tau_a", "tau_b", "tau_d", "g_coh", "g_ads", "k_r",
               "m_threshold", "c_in", "body_force_x")


def _param_values(p) -> tuple:
    """The model constants of one lattice and its inlet flag, in Params
    order (p: a dict or an object with those attributes)."""
    if isinstance(p, dict):
        return tuple(float(p[k]) for k in _PARAM_KEYS) + (int(p["inlet"]),)
    return tuple(float(getattr(p, k)) for k in _PARAM_KEYS) + (int(p.inlet),)


def _params(p, precision: int) -> Params:
    return Params(*_param_values(p), int(precision))


#: Geometry and Params as numpy records (the same bytes)
GEOM_DTYPE = np.dtype([("nx", np.int32), ("ny", np.int32), ("solid", np.uintp),
                       ("rho_a", np.uintp), ("rho_b", np.uintp),
                       ("conc", np.uintp), ("cap_x0", np.int32),
                       ("cap_x1", np.int32)], align=True)
PARAMS_DTYPE = np.dtype([(k, np.float64) for k in _PARAM_KEYS]
                        + [("inlet", np.int32), ("precision", np.int32)],
                        align=True)
assert GEOM_DTYPE.itemsize == C.sizeof(Geometry)
assert PARAMS_DTYPE.itemsize == C.sizeof(Params)


class Solver:
    """A batch of lattices on the GPU (one lattice is a batch of one).

    ``geoms`` are :class:`paper_1309_6726_gb300.inputs.Geometry` objects (or
    anything with ``solid``, ``rho_a``, ``rho_b``, ``conc``, ``cap_x0``,
    ``cap_x1``) and ``params`` matching :class:`inputs.ModelParams` (or
    dicts).  ``precision`` is ``"fp32"``, ``"fp16"`` or ``"bf16"`` (the
    16-bit formats share one layout).
    """

    def __init__(self, geoms, params, precision: str = "fp32"):
        if not isinstance(geoms, (list, tuple)):
            geoms, params = [geoms], [params]
        if len(geoms) != len(params) or not geoms:
            raise ValueError("need as many params as geometries (>= 1)")
        self._lib = load_library()
        prec = {"fp32": LBM_FP32, "fp16": LBM_FP16, "bf16": LBM_BF16}[precision]
        self.precision = precision
        self._keep = []
        self.shapes = []
        grows, prows = [], []
        for k, (g, p) in enumerate(zip(geoms, params)):
            solid = np.ascontiguousarray(g.solid, dtype=np.uint8)
            if solid.ndim != 2:
                raise ValueError("lattice %d: solid must be (ny, nx)" % k)
            ny, nx = solid.shape
            ra = np.ascontiguousarray(g.rho_a, dtype=np.float32)
            rb = np.ascontiguousarray(g.rho_b, dtype=np.float32)
            cc = np.ascontiguousarray(g.conc, dtype=np.float32)
            # the library reads ny * nx values from each array
            for name, a in (("rho_a", ra), ("rho_b", rb), ("conc", cc)):
                if a.shape != solid.shape:
                    raise ValueError("lattice %d: %s has shape %s, solid %s"
                                     % (k, name, a.shape, solid.shape))
            self._keep += [solid, ra, rb, cc]
            grows.append((nx, ny, solid.ctypes.data, ra.ctypes.data,
                          rb.ctypes.data, cc.ctypes.data, int(g.cap_x0),
                          int(g.cap_x1)))
            prows.append(_param_values(p) + (int(prec),))
            self.shapes.append((ny, nx))
        # both struct arrays built in one call each (the same bytes as
        # arrays of Geometry / Params)
        G = np.array(grows, GEOM_DTYPE)
        P = np.array(prows, PARAMS_DTYPE)
        h = C.c_void_p()
        st = self._lib.lbm_create_batch(G.ctypes.data_as(C.POINTER(Geometry)),
                                        P.ctypes.data_as(C.POINTER(Params)),
                                        len(geoms), C.byref(h))
        self._keep = []
        if st != LBM_OK:
            raise LbmError(st, self._lib.lbm_last_error(None).decode())
        self._h = h
        self.count = len(geoms)

    # -- life cycle ----------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            self._lib.lbm_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _check(self, st: int):
        if st != LBM_OK:
            raise LbmError(st, self._lib.lbm_last_error(self._h).decode())

    # -- stepping ------------------------------------------------------------
    def set_stream(self, stream) -> None:
        """Binds a CUDA stream (an int handle, e.g. a torch stream's
        ``cuda_stream``) or None for the solver's own.  The legacy default
        stream (handle 0) cannot be bound: it would mean the solver's own."""
        if stream == 0:
            raise ValueError("bind a created stream, not the legacy default "
                             "stream (0)")
        self._check(self._lib.lbm_set_stream(self._h, stream))

    def step(self, n: int = 1) -> None:
        self._check(self._lib.lbm_step(self._h, int(n)))

    @property
    def step_count(self) -> int:
        return int(self._lib.lbm_step_count(self._h))

    # -- outputs -------------------------------------------------------------
    def observables_array(self, allow_nan: bool = False) -> np.ndarray:
        """Observables of every lattice as one record array (OBS_DTYPE,
        the fields of observables())."""
        out = np.empty(self.count, OBS_DTYPE)
        st = self._lib.lbm_observables(
            self._h, out.ctypes.data_as(C.POINTER(Obs)))
        if not (st == LBM_ENAN and allow_nan):
            self._check(st)
        return out

    def observables(self, allow_nan: bool = False) -> list[dict]:
        """Observables of every lattice, one dict each."""
        a = self.observables_array(allow_nan)
        names = a.dtype.names
        return [dict(zip(names, r)) for r in a.tolist()]

    def solid_mask(self, k: int = 0) -> np.ndarray:
        ny, nx = self.shapes[k]
        out = np.zeros((ny, nx), np.uint8)
        self._check(self._lib.lbm_get_solid_mask(
            self._h, k, out.ctypes.data_as(C.POINTER(C.c_uint8)), out.size))
        return out

    def solid_masks(self, out: np.ndarray | None = None) -> list[np.ndarray]:
        """Solid masks of every lattice, read back in one call: views of
        one buffer of all lattices' nodes, ``out`` if given (a contiguous
        uint8 array of that size, e.g. in pinned memory, where the copy
        runs at the link's full rate)."""
        sizes = [ny * nx for ny, nx in self.shapes]
        if out is None:
            buf = np.empty(sum(sizes), np.uint8)
        else:
            buf = out.reshape(-1)
            if (buf.dtype != np.uint8 or buf.size != sum(sizes)
                    or not buf.flags.c_contiguous):
                raise ValueError("out: need %d contiguous uint8 values"
                                 % sum(sizes))
        self._check(self._lib.lbm_get_solid_masks(
            self._h, buf.ctypes.data_as(C.POINTER(C.c_uint8)), buf.size))
        out, o = [], 0
        for (ny, nx), n in zip(self.shapes, sizes):
            out.append(buf[o:o + n].reshape(ny, nx))
            o += n
        return out

    def populations(self, k: int = 0) -> np.ndarray:
        """Post-streaming populations (22, ny, nx): A 0-8, B 9-17, solute
        18-21."""
        ny, nx = self.shapes[k]
        out = np.zeros((NPOP, ny, nx), np.float32)
        self._check(self._lib.lbm_get_fields(self._h, k, FIELD_POPS,
                                             out.ctypes.data, out.nbytes))
        return out

    def densities(self, k: int = 0) -> np.ndarray:
        """(3, ny, nx): rho_A, rho_B, C of the post-streaming state."""
        ny, nx = self.shapes[k]
        out = np.zeros((3, ny, nx), np.float32)
        self._check(self._lib.lbm_get_fields(self._h, k, FIELD_DENSITY,
                                             out.ctypes.data, out.nbytes))
        return out

    def deposit(self, k: int = 0) -> np.ndarray:
        ny, nx = self.shapes[k]
        out = np.zeros((ny, nx), np.float64)
        self._check(self._lib.lbm_get_fields(self._h, k, FIELD_DEPOSIT,
                                             out.ctypes.data, out.nbytes))
        return out

    def set_populations(self, f, k: int = 0) -> None:
        a = np.ascontiguousarray(f, dtype=np.float32)
        ny, nx = self.shapes[k]
        if a.size != NPOP * ny * nx:
            raise ValueError("populations: need %d values, got %d"
                             % (NPOP * ny * nx, a.size))
        self._check(self._lib.lbm_set_fields(self._h, k, FIELD_POPS,
                                             a.ctypes.data, a.nbytes))

    def set_deposit(self, m, k: int = 0) -> None:
        a = np.ascontiguousarray(m, dtype=np.float64)
        self._check(self._lib.lbm_set_fields(self._h, k, FIELD_DEPOSIT,
                                             a.ctypes.data, a.nbytes))

    def autotune(self, steps: int = 32) -> dict:
        """Times every step-kernel variant on this state (restored after
        each trial) and keeps the fastest; returns the choice."""
        t = Tuning()
        self._check(self._lib.lbm_autotune(self._h, int(steps), C.byref(t)))
        return t.as_dict()

    def tuning(self) -> dict:
        t = Tuning()
        self._check(self._lib.lbm_get_tuning(self._h, C.byref(t)))
        return t.as_dict()

    def save(self, path: str) -> None:
        self._check(self._lib.lbm_save(self._h, path.encode()))

    def load(self, path: str) -> None:
        self._check(self._lib.lbm_load(self._h, path.encode()))


def fit_reff(t, z, gamma: float, mu: float, length: float,
             cos_theta0: float) -> float:
    """Effective radius from a front history (``lbm_fit_reff``)."""
    lib = load_library()
    t = np.ascontiguousarray(t, dtype=np.float64)
    z = np.ascontiguousarray(z, dtype=np.float64)
    out = C.c_double()
    dp = C.POINTER(C.c_double)
    st = lib.lbm_fit_reff(t.ctypes.data_as(dp), z.ctypes.data_as(dp), len(t),
                          gamma, mu, length, cos_theta0, C.byref(out))
    if st != LBM_OK:
        raise LbmError(st, "lbm_fit_reff: bad arguments")
    return out.value


def plan_tiles(sizes, tx: int, ty: int, grid: int) -> np.ndarray:
    """Tile schedule of the TMA step kernel (``lbm_plan_tiles``) for
    lattices of (nx, ny) ``sizes``: int32 [slots, grid, 3] of (lattice,
    first column, first row), lattice -1 after a block's last tile."""
    lib = load_library()
    nx = np.ascontiguousarray([s[0] for s in sizes], dtype=np.int32)
    ny = np.ascontiguousarray([s[1] for s in sizes], dtype=np.int32)
    ip = C.POINTER(C.c_int32)
    slots = C.c_int32()
    args = (nx.ctypes.data_as(ip), ny.ctypes.data_as(ip), len(nx), tx, ty,
            grid)
    st = lib.lbm_plan_tiles(*args, None, 0, C.byref(slots))
    if st != LBM_OK:
        raise LbmError(st, lib.lbm_last_error(None).decode())
    out = np.empty((slots.value, grid, 3), dtype=np.int32)
    st = lib.lbm_plan_tiles(*args, out.ctypes.data_as(ip), out.size,
                            C.byref(slots))
    if st != LBM_OK:
        raise LbmError(st, lib.lbm_last_error(None).decode())
    return out


#: most columns lbm_observables_static accepts (its fixed scratch size)
STATIC_MAX_COLUMNS = 16384


def observables_static(pops_ptr: int, solid_ptr: int, solid0_ptr: int,
                       deposit_ptr: int, nx: int, ny: int, cap_x0: int,
                       cap_x1: int, ledger, step: int, closure_step: int,
                       out_ptr: int, stream: int = 0) -> None:
    """``lbm_observables_static``: observables of one lattice held in
    caller-owned device buffers (raw device addresses), written to the
    device address ``out_ptr`` (one lbm_obs, 144 bytes); allocates nothing.
    """
    lib = load_library()
    led = (C.c_double * 4)(*[float(v) for v in ledger])
    st = lib.lbm_observables_static(pops_ptr, solid_ptr, solid0_ptr,
                                    deposit_ptr, nx, ny, cap_x0, cap_x1, led,
                                    int(step), int(closure_step), out_ptr,
                                    stream or None)
    if st != LBM_OK:
        raise LbmError(st, "lbm_observables_static failed")
