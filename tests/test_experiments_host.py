"""Host logic of the paper-scale analysis and of the binding's batch
marshalling, on the CPU.

* The Eq. 1 fit window (paper Sec. III, Eq. 1: the front advances
  linearly in the Washburn regime): from t_lo, finite samples only, before
  the front passes the reservoir bound, and no further than the front's
  farthest advance when it stalls and recedes first.
* The record arrays the binding hands to lbm_create_batch hold the same
  bytes as arrays of the ctypes structures the header mirrors.
"""
import ctypes as C

import numpy as np

from paper_1309_6726_gb300 import experiments as E
from paper_1309_6726_gb300 import inputs as I
from paper_1309_6726_gb300 import lbm


def test_fit_window_stops_before_the_reservoir_bound():
    t = np.arange(0, 100_000, 500)
    z = 3e-3 * t
    idx = E._fit_window(t, z, 16_000, 230.0)
    assert t[idx[0]] == 16_000
    assert z[idx[-1]] < 230.0 <= z[idx[-1] + 1]
    assert np.all(np.diff(idx) == 1)


def test_fit_window_stops_at_the_farthest_advance():
    # linear advance to step 60 000, then the front recedes, then the run
    # breaks down (non-finite samples)
    t = np.arange(0, 100_000, 500).astype(float)
    z = np.where(t <= 60_000, 2.5e-3 * t, 150.0 - 1e-4 * (t - 60_000))
    z[t >= 95_000] = np.nan
    idx = E._fit_window(t, z, 16_000, 230.0)
    assert t[idx[0]] == 16_000 and t[idx[-1]] == 60_000
    v = np.polyfit(t[idx], z[idx], 1)[0]
    assert abs(v - 2.5e-3) < 1e-12


def test_fit_window_skips_non_finite_and_early_samples():
    t = np.arange(0, 40_000, 1000).astype(float)
    z = 1e-3 * t
    z[20] = np.nan
    idx = E._fit_window(t, z, 10_000, 1e9)
    assert t[idx[0]] == 10_000 and 20 not in idx
    assert np.all(np.isfinite(z[idx]))


def test_batch_records_match_the_ctypes_structures():
    geom, mp, _ = I.config_small()
    ny, nx = geom.solid.shape
    ptrs = [a.ctypes.data for a in (geom.solid, geom.rho_a, geom.rho_b, geom.conc)]
    g = lbm.Geometry(nx, ny, *ptrs, int(geom.cap_x0), int(geom.cap_x1))
    rec = np.array([(nx, ny, *ptrs, int(geom.cap_x0), int(geom.cap_x1))],
                   lbm.GEOM_DTYPE)
    assert rec.tobytes() == bytes(g)
    for src in (mp, mp.as_dict()):
        p = lbm._params(src, lbm.LBM_FP16)
        prec = np.array([lbm._param_values(src) + (lbm.LBM_FP16,)],
                        lbm.PARAMS_DTYPE)
        assert prec.tobytes() == bytes(p)
    assert lbm.GEOM_DTYPE.itemsize == C.sizeof(lbm.Geometry)
    assert lbm.PARAMS_DTYPE.itemsize == C.sizeof(lbm.Params)
