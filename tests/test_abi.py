"""The C-ABI library builds, loads and exports every entry point that
include/*.h declares (no compute calls: this runs without a GPU)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        for m in re.finditer(r"\b(lbm_\w+)\s*\(", text):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1309_6726_gb300 import build
    return ctypes.CDLL(build.build())


def test_header_declares_entry_points():
    names = _declared()
    assert {"lbm_create", "lbm_step", "lbm_observables", "lbm_destroy",
            "lbm_get_solid_mask", "lbm_get_fields"} <= names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_every_declared_symbol():
    from paper_1309_6726_gb300 import lbm, mlp
    assert set(lbm.SYMBOLS) | set(mlp.SYMBOLS) == _declared()


def test_create_rejects_bad_arguments_without_touching_the_gpu(lib):
    # Argument checks happen before any CUDA call.
    from paper_1309_6726_gb300 import lbm
    L = lbm.load_library()
    h = ctypes.c_void_p()
    assert L.lbm_create_batch(None, None, 1, ctypes.byref(h)) == lbm.LBM_EINVAL
    assert b"NULL" in L.lbm_last_error(None)
    assert L.lbm_step(None, 1) == lbm.LBM_EINVAL
    lbm_obs_size = ctypes.sizeof(lbm.Obs)
    assert lbm_obs_size == 144


def test_binding_rejects_mismatched_arrays_without_touching_the_gpu(lib):
    # the library reads ny * nx values from each field: the binding checks
    # the shapes before it calls create
    from paper_1309_6726_gb300 import inputs as I, lbm
    geom, mp, _ = I.config_small()
    bad = I.Geometry(geom.solid, geom.rho_a[:, :-1], geom.rho_b, geom.conc,
                     geom.cap_x0, geom.cap_x1)
    with pytest.raises(ValueError, match="rho_a"):
        lbm.Solver(bad, mp)
    flat = I.Geometry(geom.solid.ravel(), geom.rho_a, geom.rho_b, geom.conc,
                      geom.cap_x0, geom.cap_x1)
    with pytest.raises(ValueError, match="solid"):
        lbm.Solver(flat, mp)
    with pytest.raises(ValueError):
        lbm.Solver([geom, geom], [mp])


def test_fit_reff_host_helper(lib):
    # Host-only arithmetic: a front at exactly the Eq. 1 speed for height H
    # gives r_eff = H / 2.
    import math
    import numpy as np
    from paper_1309_6726_gb300 import lbm
    gamma, mu, L, c, H = 0.144, 0.17, 400.0, math.cos(math.radians(30)), 16
    v = gamma * H * c / (6 * mu * L)
    t = np.arange(1000, 6000, 250.0)
    assert lbm.fit_reff(t, 3.0 + v * t, gamma, mu, L, c) == pytest.approx(
        H / 2, rel=1e-12)


def test_mlp_create_rejects_bad_shapes_without_touching_the_gpu(lib):
    from paper_1309_6726_gb300 import lbm, mlp
    L = mlp.load_library()
    h = ctypes.c_void_p()
    bad = mlp.Shape(4, 250, 3, 65, 64)  # hidden width not a multiple of 16
    assert L.lbm_mlp_create(ctypes.byref(bad), ctypes.byref(h)) == lbm.LBM_EINVAL
    assert b"shape" in L.lbm_mlp_last_error(None)
    assert L.lbm_mlp_create(None, ctypes.byref(h)) == lbm.LBM_EINVAL
    assert L.lbm_mlp_param_count(None) == -1
    assert mlp.layer_shapes(4, 256, 3, 65) == [(256, 4), (256, 256),
                                               (256, 256), (65, 256)]


def test_create_rejects_degenerate_parameters_without_touching_the_gpu(lib):
    # every check runs before any CUDA call
    import numpy as np
    from paper_1309_6726_gb300 import inputs as I, lbm
    L = lbm.load_library()
    geom = I.capillary(40, 8, 8, 8)
    keep = []

    def arr(a, t):
        a = np.ascontiguousarray(a, t)
        keep.append(a)
        return a.ctypes.data

    def geo(nx=geom.nx, ny=geom.ny, x0=geom.cap_x0, x1=geom.cap_x1):
        return lbm.Geometry(nx, ny, arr(geom.solid, np.uint8),
                            arr(geom.rho_a, np.float32),
                            arr(geom.rho_b, np.float32),
                            arr(geom.conc, np.float32), x0, x1)

    def params(**kw):
        d = I.ModelParams().as_dict()
        d.update(kw)
        return lbm._params(d, kw.pop("precision", 0))

    h = ctypes.c_void_p()
    cases = [
        (geo(), params(m_threshold=0.0), b"m_threshold"),
        (geo(), params(tau_a=0.5), b"relaxation"),
        (geo(), params(k_r=-1e-3), b"k_r"),
        (geo(), params(g_coh=float("nan")), b"non-finite"),
        (geo(ny=2), params(), b"ny >= 3"),
        (geo(nx=0), params(), b"nx >= 1"),
        (geo(x0=5, x1=5), params(), b"section"),
        (geo(nx=20000, ny=20000), params(), b"too large"),
        (geo(), params(precision=3), b"unknown precision"),
    ]
    for g, p, msg in cases:
        assert L.lbm_create(ctypes.byref(g), ctypes.byref(p),
                            ctypes.byref(h)) == lbm.LBM_EINVAL, msg
        assert msg in L.lbm_last_error(None), (msg, L.lbm_last_error(None))
    # a batch may not mix storage precisions; an empty batch is refused
    G2 = (lbm.Geometry * 2)(geo(), geo())
    P2 = (lbm.Params * 2)(params(), lbm._params(I.ModelParams().as_dict(), 1))
    assert L.lbm_create_batch(G2, P2, 2, ctypes.byref(h)) == lbm.LBM_EINVAL
    assert b"mixed precision" in L.lbm_last_error(None)
    assert L.lbm_create_batch(G2, P2, 0, ctypes.byref(h)) == lbm.LBM_EINVAL
    # FP16 and BF16 share a layout but not a codec: not mixed either
    P3 = (lbm.Params * 2)(lbm._params(I.ModelParams().as_dict(), lbm.LBM_FP16),
                          lbm._params(I.ModelParams().as_dict(), lbm.LBM_BF16))
    assert L.lbm_create_batch(G2, P3, 2, ctypes.byref(h)) == lbm.LBM_EINVAL
    assert b"mixed precision" in L.lbm_last_error(None)
