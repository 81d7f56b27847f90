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
