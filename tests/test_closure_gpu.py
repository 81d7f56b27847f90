"""Pore closure on the GPU path against the FP64 oracle.

Closure is the paper's result (Sec. III, Figs. 2 and 3): the solid grown
from both walls of a narrow capillary meets across the section, the front
stops, and Delta e reaches H/2.  The closure step is the first step count
after which some column of the capillary section is entirely solid.  On
the GPU it is recorded by the node flips of one step: each flip decrements
its section column's fluid counter, and the flip that empties a column
takes the step count by an atomic minimum per lattice.

These cases close within a few hundred steps (oracle: steps 607, 391 and
353).  Every check asserts first that the oracle closed, so no comparison
is -1 against -1.  FP32 and FP16 storage: the closure step and the solid
mask must be equal at every check, including each single step around the
closure; populations within the stated FP32 / FP16 bounds.
"""
import numpy as np
import pytest

from oracle import analysis as A
from paper_1309_6726_gb300 import inputs as I
from paper_1309_6726_gb300 import lbm
from tests.gpu_helpers import assert_rel, oracle_for, oracle_pops, pop_error

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5
FP32_REL = 1e-4
FP16_TOL = 1e-3
FP16_REL_LONG = 1.5e-2


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _closing(nx, ny, x_res, x_out, k_r, m_th, theta=30.0):
    geom = I.capillary(nx, ny, x_res, x_out)
    mp = I.ModelParams(g_ads=I.g_ads_for_angle(theta), k_r=k_r,
                       m_threshold=m_th, inlet=1)
    return geom, mp


# H = 10 fluid rows, L = 136: the oracle closes it at step 607
CASE = (200, 12, 40, 24, 4e-3, 0.25)


@pytest.mark.parametrize("precision,tol,rtol", [
    ("fp32", FP32_TOL, FP32_REL), ("fp16", FP16_TOL, FP16_REL_LONG)])
def test_narrow_capillary_closes_at_the_oracle_step(precision, tol, rtol):
    geom, mp = _closing(*CASE)
    s, o = lbm.Solver(geom, mp, precision), oracle_for(geom, mp)
    # up to shortly before the closure in chunks, then one step at a time
    while o.step_count < 590:
        n = min(50, 590 - o.step_count)
        s.step(n)
        o.step(n)
        np.testing.assert_array_equal(s.solid_mask(), o.solid())
        assert s.observables()[0]["closure_step"] == o.closure_step == -1
    closed_at = None
    while o.step_count < 625:
        s.step(1)
        o.step(1)
        np.testing.assert_array_equal(s.solid_mask(), o.solid())
        go = s.observables()[0]
        assert go["closure_step"] == o.closure_step, o.step_count
        if o.closure_step > 0 and closed_at is None:
            closed_at = o.step_count
            assert o.closure_step == o.step_count
    assert closed_at is not None and closed_at > 0
    print("%s: closure at step %d on both sides" % (precision, closed_at))
    go = s.observables()[0]
    oo = A.lattice_observables(o)
    assert go["closed"] == 1 and oo["closed"] == 1.0
    # a closed column counts H / 2 (reading c15)
    assert go["delta_e"] == oo["delta_e"] == (geom.ny - 2) / 2
    assert go["r_min"] == oo["r_min"] == 0.0
    fg, fo = s.populations(), oracle_pops(o)
    assert pop_error(fg, fo) < tol
    print("%s closure case: %s" % (precision, assert_rel(fg, fo, rtol)))
    s.close()


@pytest.mark.parametrize("precision", ["fp32", "fp16", "bf16"])
def test_batch_closes_each_lattice_at_its_own_step(precision):
    # Four capillaries in one handle: three close at different steps, one
    # (wide, slow reaction) stays open.  The per-lattice closure minimum and
    # the per-column counters must not leak between lattices.
    cases = [_closing(*CASE),
             _closing(150, 10, 30, 20, 4e-3, 0.2, theta=40.0),
             _closing(180, 30, 40, 24, 1e-3, 1.0),
             _closing(130, 11, 30, 20, 5e-3, 0.2, theta=25.0)]
    geoms = [g for g, _ in cases]
    mps = [p for _, p in cases]
    s = lbm.Solver(geoms, mps, precision)
    ors = [oracle_for(g, p) for g, p in zip(geoms, mps)]
    for chunk in (300, 40, 40, 40, 40, 40, 40, 40, 60):
        s.step(chunk)
        for o in ors:
            o.step(chunk)
        obs = s.observables()
        masks = s.solid_masks()  # all lattices in one call
        for k, o in enumerate(ors):
            np.testing.assert_array_equal(s.solid_mask(k), o.solid())
            np.testing.assert_array_equal(masks[k], o.solid())
            assert obs[k]["closure_step"] == o.closure_step, (k, o.step_count)
    steps = [o.closure_step for o in ors]
    print("%s closure steps: %s" % (precision, steps))
    assert steps[2] == -1
    assert all(t > 0 for i, t in enumerate(steps) if i != 2)
    assert len({steps[0], steps[1], steps[3]}) == 3
