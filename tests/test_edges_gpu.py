"""Edge cases and the benchmark's own configuration on the GPU path,
against the FP64 oracle.

* The batched sweep at full size (512 capillaries, about 1e8 nodes) in the
  launch configuration bench.py times (default tile, persistent TMA
  kernel, FP16 headline and FP32 comparison): three capillaries sampled
  from it (smallest, median and largest) are advanced by the oracle alone
  and compared element by element.
* The 2048 x 2048 disc preform at its full size, both storages.
* Degenerate rates: k_r = 0 (no deposit, the mask never changes) and a
  vanishing threshold (every reacting node turns solid at once, growth
  cascades one layer per step) -- masks exact against the oracle.
* A section that is solid from the start (closed at step 0) and the
  smallest lattices (one column, three rows)."""
import numpy as np
import pytest

from oracle import analysis as A
from paper_1309_6726_gb300 import inputs as I
from paper_1309_6726_gb300 import lbm
from tests.gpu_helpers import assert_rel, oracle_for, oracle_pops, pop_error

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5
FP16_TOL_SHORT = 5e-3
# per-component relative bound (gpu_helpers.pop_rel_error; the reason is
# given in test_parity_gpu.py)
FP32_REL = 1e-4
FP16_REL = 1.5e-2


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


@pytest.mark.parametrize("precision,tol", [("fp16", FP16_TOL_SHORT),
                                           ("fp32", FP32_TOL)])
def test_full_sweep_sampled_capillaries(precision, tol):
    members = I.sweep_members(512)
    pairs = [I.sweep_lattice(m) for m in members]
    sizes = np.array([g.solid.size for g, _ in pairs])
    order = np.argsort(sizes)
    picks = [int(order[0]), int(order[len(order) // 2]), int(order[-1])]
    s = lbm.Solver([g for g, _ in pairs], [p for _, p in pairs], precision)
    steps = 10
    s.step(steps)
    for k in picks:
        g, p = pairs[k]
        o = oracle_for(g, p)
        o.step(steps)
        np.testing.assert_array_equal(s.solid_mask(k), o.solid())
        assert pop_error(s.populations(k), oracle_pops(o)) < tol, k
        rel = assert_rel(s.populations(k), oracle_pops(o),
                         FP32_REL if precision == "fp32" else FP16_REL)
        print("sweep sample %s lattice %d: %s" % (precision, k, rel))
    s.close()


def test_full_size_preform_both_storages():
    # One 2048 x 2048 lattice (4.2e6 nodes, its tall tile columns cut into
    # strips over every block, walls around thousands of discs) for three
    # steps, element by element against the oracle in both storages.  No
    # node reacts this early (no disc touches the reservoir); growth on a
    # preform is compared on the 192 x 192 one.
    geom, mp, _ = I.config_preform()
    o = oracle_for(geom, mp)
    o.step(3)
    fo = oracle_pops(o)
    for precision, tol in (("fp32", FP32_TOL), ("fp16", FP16_TOL_SHORT)):
        with lbm.Solver(geom, mp, precision) as s:
            s.step(3)
            np.testing.assert_array_equal(s.solid_mask(), o.solid())
            assert pop_error(s.populations(), fo) < tol, precision
            rel = assert_rel(s.populations(), fo,
                             FP32_REL if precision == "fp32" else FP16_REL)
            print("full preform %s: %s" % (precision, rel))


def _capillary(k_r, m_threshold, nx=96, ny=14):
    geom = I.capillary(nx, ny, 24, 16)
    mp = I.ModelParams(g_ads=I.G_ADS_30, k_r=k_r, m_threshold=m_threshold,
                       inlet=1)
    return geom, mp


def test_zero_rate_never_grows():
    geom, mp = _capillary(0.0, 1.0)
    s, o = lbm.Solver(geom, mp), oracle_for(geom, mp)
    s.step(300)
    o.step(300)
    np.testing.assert_array_equal(s.solid_mask(), geom.solid)
    np.testing.assert_array_equal(o.solid(), geom.solid)
    assert np.all(s.deposit() == 0.0)
    assert pop_error(s.populations(), oracle_pops(o)) < FP32_TOL
    assert_rel(s.populations(), oracle_pops(o), FP32_REL)
    assert s.observables()[0]["ledger_m"] == 0.0


def test_tiny_threshold_cascades_exactly():
    # every reacting node turns solid in the step it first reacts: growth
    # cascades one layer per step
    geom, mp = _capillary(1e-3, 1e-9)
    s, o = lbm.Solver(geom, mp), oracle_for(geom, mp)
    grown = []
    for _ in range(6):
        s.step(3)
        o.step(3)
        np.testing.assert_array_equal(s.solid_mask(), o.solid())
        grown.append(int((o.solid() != geom.solid).sum()))
        assert pop_error(s.populations(), oracle_pops(o)) < FP32_TOL
        assert_rel(s.populations(), oracle_pops(o), FP32_REL)
    assert grown[-1] > grown[0] > 0


def test_section_closed_from_the_start():
    geom, mp = _capillary(1e-3, 1.0)
    solid = geom.solid.copy()
    solid[:, 50] = 1  # one section column fully solid
    geom2 = I.Geometry(solid, np.where(solid, 0, geom.rho_a).astype(np.float32),
                       np.where(solid, 0, geom.rho_b).astype(np.float32),
                       np.where(solid, 0, geom.conc).astype(np.float32),
                       geom.cap_x0, geom.cap_x1, geom.extra)
    s, o = lbm.Solver(geom2, mp), oracle_for(geom2, mp)
    s.step(20)
    o.step(20)
    go = s.observables()[0]
    oo = A.lattice_observables(o)
    assert go["closed"] == 1 and oo["closed"]
    assert go["r_min"] == 0.0 == oo["r_min"]
    # closed from the start: the first step with a solid column is step 0
    assert go["closure_step"] == o.closure_step == 0
    np.testing.assert_array_equal(s.solid_mask(), o.solid())
    assert pop_error(s.populations(), oracle_pops(o)) < FP32_TOL
    assert_rel(s.populations(), oracle_pops(o), FP32_REL)


@pytest.mark.parametrize("nx,ny", [(1, 3), (2, 3), (3, 5)])
def test_smallest_lattices(nx, ny):
    geom = I.random_lattice(nx, ny, seed=nx * 10 + ny, solid_fraction=0.2)
    mp = I.ModelParams(g_ads=0.3, k_r=0.05, m_threshold=1.0)
    s, o = lbm.Solver(geom, mp), oracle_for(geom, mp)
    f, g = I.random_populations(geom, seed=3)
    pops = np.concatenate([f.reshape(18, ny, nx), g])
    s.set_populations(pops)
    o.set_populations(f.astype(np.float64))
    o.set_solute(g.astype(np.float64))
    for _ in range(3):
        s.step(2)
        o.step(2)
        np.testing.assert_array_equal(s.solid_mask(), o.solid())
        assert pop_error(s.populations(), oracle_pops(o)) < FP32_TOL
        assert_rel(s.populations(), oracle_pops(o), FP32_REL)
