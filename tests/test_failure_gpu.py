"""Failure detection without a GPU fault: every wait of the step kernel on
an mbarrier is bounded (about two seconds), and on time-out the kernel
records an error, lets its copies in flight land and returns, so the host
reads a status and the context stays usable.

The test makes one wait run out: the library's test hook (environment
variable LBM_TEST_STALL, read when a handle is created) has block 0 expect
16 bytes more for its first tile than any copy delivers -- a completion
that nothing triggers.  The step returns, the next observables call
reports LBM_ETIMEOUT, and a fresh handle on the same context steps
normally."""
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_with_a_status(monkeypatch):
    import __graft_entry__
    __graft_entry__.build()
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1309_6726_gb300 import inputs as I, lbm
    from tests.gpu_helpers import oracle_for, oracle_pops, pop_error

    geom = I.capillary(96, 14, 24, 16)
    mp = I.ModelParams(g_ads=I.G_ADS_30, k_r=1e-3, inlet=1)
    monkeypatch.setenv("LBM_TEST_STALL", "16")
    s = lbm.Solver(geom, mp)
    monkeypatch.delenv("LBM_TEST_STALL")
    t0 = time.perf_counter()
    s.step(1)
    with pytest.raises(lbm.LbmError) as err:
        s.observables()
    waited = time.perf_counter() - t0
    assert err.value.status == lbm.LBM_ETIMEOUT
    assert waited < 30.0
    s.close()

    # the context is intact: a new handle steps and matches the oracle
    s2, o = lbm.Solver(geom, mp), oracle_for(geom, mp)
    s2.step(40)
    o.step(40)
    np.testing.assert_array_equal(s2.solid_mask(), o.solid())
    assert pop_error(s2.populations(), oracle_pops(o)) < 1e-5
    s2.close()


@pytest.mark.parametrize("precision", ["fp32", "fp16", "bf16"])
def test_non_finite_lattice_is_flagged_alone(precision):
    # A batch of two capillaries; one gets a NaN population (a blown-up
    # state).  Observables report LBM_ENAN, flag that lattice only, and the
    # other lattice goes on exactly as it would alone.
    import __graft_entry__
    __graft_entry__.build()
    from paper_1309_6726_gb300 import inputs as I, lbm

    geom = I.capillary(96, 14, 24, 16)
    mp = I.ModelParams(g_ads=I.G_ADS_30, k_r=1e-3, inlet=1)
    s = lbm.Solver([geom, geom], [mp, mp], precision)
    alone = lbm.Solver(geom, mp, precision)
    bad = s.populations(1)
    bad[3, 7, 50] = np.nan
    s.set_populations(bad, 1)
    s.step(20)
    alone.step(20)
    with pytest.raises(lbm.LbmError) as err:
        s.observables()
    assert err.value.status == lbm.LBM_ENAN
    obs = s.observables(allow_nan=True)
    assert obs[0]["nonfinite"] == 0 and obs[1]["nonfinite"] == 1
    np.testing.assert_array_equal(s.populations(0), alone.populations())
    s.close()
    alone.close()
