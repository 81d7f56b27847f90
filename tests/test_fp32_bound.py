"""Where the FP32 parity bound comes from.

The kernels compute in FP32.  To separate "FP32 arithmetic" from "kernel
error", the oracle's own source is compiled with every double turned into a
float (a copy built in a temporary directory, on the CPU) and run on the
small capillary next to the FP64 oracle.  Its deviation after 2000 steps,
about 6e-5 of a population's weight, is what a plain FP32 evaluation of
the textbook formulas carries as the meniscus moves.  The kernels evaluate
the equilibrium pairwise and close the rest population on the density,
which keeps them near 6e-6, so the GPU parity test can hold them to 1e-5.
"""
import ctypes as C
import subprocess

import numpy as np

from oracle import build as B
from paper_1309_6726_gb300 import inputs as I
from tests.gpu_helpers import W22, oracle_for, oracle_pops


class _P32(C.Structure):
    _fields_ = [(n, C.c_float) for n in (
        "tau_a", "tau_b", "tau_d", "g_coh", "g_ads", "k_r", "m_threshold",
        "c_in", "body_force_x")] + [("inlet", C.c_int32),
                                    ("cap_x0", C.c_int32),
                                    ("cap_x1", C.c_int32)]


def _fp32_oracle(tmp_path):
    src = open(B.SRC).read().replace("double", "float")
    p = tmp_path / "orc32.c"
    p.write_text(src)
    so = str(tmp_path / "orc32.so")
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared",
                    "-ffp-contract=off", str(p), "-o", so, "-lm"], check=True)
    lib = C.CDLL(so)
    fp = C.POINTER(C.c_float)
    lib.orc_create.restype = C.c_void_p
    lib.orc_create.argtypes = [C.POINTER(_P32), C.c_int, C.c_int,
                               C.POINTER(C.c_uint8), fp, fp, fp]
    lib.orc_step.argtypes = [C.c_void_p, C.c_int64]
    lib.orc_get.argtypes = [C.c_void_p, C.c_int, fp]
    lib.orc_destroy.argtypes = [C.c_void_p]
    return lib


def test_fp32_arithmetic_deviation_sets_the_bound(tmp_path):
    lib = _fp32_oracle(tmp_path)
    geom, mp, steps = I.config_small()
    d = mp.as_dict()
    p = _P32(d["tau_a"], d["tau_b"], d["tau_d"], d["g_coh"], d["g_ads"],
             d["k_r"], d["m_threshold"], d["c_in"], d["body_force_x"],
             d["inlet"], geom.cap_x0, geom.cap_x1)
    f32 = lambda a: np.ascontiguousarray(a, np.float32)
    ra, rb, cc = f32(geom.rho_a), f32(geom.rho_b), f32(geom.conc)
    sol = np.ascontiguousarray(geom.solid, np.uint8)
    fp = C.POINTER(C.c_float)
    h = lib.orc_create(C.byref(p), geom.nx, geom.ny,
                       sol.ctypes.data_as(C.POINTER(C.c_uint8)),
                       ra.ctypes.data_as(fp), rb.ctypes.data_as(fp),
                       cc.ctypes.data_as(fp))
    o = oracle_for(geom, mp)
    N = geom.nx * geom.ny
    errs = {}
    for t in (500, 2000):
        lib.orc_step(h, t - o.step_count)
        o.step(t - o.step_count)
        f = np.zeros(18 * N, np.float32)
        g = np.zeros(4 * N, np.float32)
        lib.orc_get(h, 0, f.ctypes.data_as(fp))
        lib.orc_get(h, 1, g.ctypes.data_as(fp))
        ff = np.concatenate([f.reshape(18, geom.ny, geom.nx),
                             g.reshape(4, geom.ny, geom.nx)])
        errs[t] = float((np.abs(ff - oracle_pops(o)) / W22[:, None, None]).max())
    lib.orc_destroy(h)
    print("FP32-arithmetic oracle vs FP64 oracle:", errs)
    # plain FP32 evaluation drifts as the meniscus moves: well above the
    # 1e-5 the kernels are held to
    assert 2e-5 < errs[2000] < 1e-4
    assert errs[500] < 1e-4
