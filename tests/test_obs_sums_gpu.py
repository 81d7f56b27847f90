"""The lattice totals the step kernel adds up against the observables pass
that reads the whole stored state.

The last launch of every step call also sums, per lattice, the fluid
content of the nodes it updates: rho_A and rho_B as the collision
conserves them and C after the update and the reaction.  The observables
call then reads the mask, the deposit, the nodes that turned solid in
that step and the phase rows, not the populations of every node.
Loading a checkpoint (or setting a field) drops those totals, and the next
observables call sums the stored state itself.  A node's stored values
sum to its conserved densities up to FP32 rounding, so a checkpoint saved
and loaded into the same handle gives the same observables by the other
route: every field equal, the fluid content within 1e-7 relative (the
rounding of a node's sums, of random sign, over at least a thousand
nodes).  The cases react, grow solid and close, so the nodes turned solid
in the last step (subtracted from the fluid content) are part of what is
compared."""
import numpy as np
import pytest

from paper_1309_6726_gb300 import inputs as I
from paper_1309_6726_gb300 import lbm

pytestmark = pytest.mark.gpu

FLUID_KEYS = ("mass_a", "mass_b", "mass_c")
LEDGER_KEYS = ("precip_mass", "ledger_a", "ledger_b", "ledger_c", "ledger_m")


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _closing_batch():
    def cap(nx, ny, x_res, x_out, k_r, m_th, theta):
        geom = I.capillary(nx, ny, x_res, x_out)
        mp = I.ModelParams(g_ads=I.g_ads_for_angle(theta), k_r=k_r,
                           m_threshold=m_th, inlet=1)
        return geom, mp
    cases = [cap(200, 12, 40, 24, 4e-3, 0.25, 30.0),
             cap(150, 10, 30, 20, 4e-3, 0.2, 40.0),
             cap(180, 30, 40, 24, 1e-3, 1.0, 30.0)]
    return [g for g, _ in cases], [p for _, p in cases]


def _compare(fused, full, where):
    assert len(fused) == len(full)
    for k, (a, b) in enumerate(zip(fused, full)):
        for key, va in a.items():
            vb = b[key]
            if key in FLUID_KEYS:
                assert va == pytest.approx(vb, rel=1e-7), (where, k, key)
            elif key in LEDGER_KEYS:
                assert va == pytest.approx(vb, rel=1e-12, abs=1e-12), (where, k, key)
            elif isinstance(va, float) and np.isnan(va):
                assert np.isnan(vb), (where, k, key)
            else:
                assert va == vb, (where, k, key)


@pytest.mark.parametrize("kernel", ["tma", "direct"])
@pytest.mark.parametrize("precision", ["fp32", "fp16", "bf16"])
def test_step_totals_match_the_full_observables_pass(tmp_path, monkeypatch,
                                                     precision, kernel):
    monkeypatch.delenv("LBM_KERNEL", raising=False)
    if kernel == "direct":
        monkeypatch.setenv("LBM_KERNEL", "direct")
    geoms, mps = _closing_batch()
    s = lbm.Solver(geoms, mps, precision)
    ck = str(tmp_path / "state.ckpt")
    flips = 0
    # plain launches, graph replays (16 steps from buffer 0), a graph
    # followed by plain launches, and single steps across the growth and
    # the first lattice's closure (step 607)
    chunks = [7, 16, 33, 200, 1, 1, 50, 1, 16, 40, 1, 1, 1, 60, 1, 1, 30,
              120] + [1] * 35
    for n in chunks:
        s.step(n)
        fused = s.observables(allow_nan=True)
        s.save(ck)
        s.load(ck)
        full = s.observables(allow_nan=True)
        _compare(fused, full, s.step_count)
        # the record array carries the same values (NaN where no front)
        arr = s.observables_array(allow_nan=True)
        for k, o in enumerate(full):
            for key, v in o.items():
                np.testing.assert_equal(arr[key][k], v, err_msg=key)
        flips += sum(o["ledger_m"] > 0 for o in fused)
    closed = [o["closure_step"] for o in s.observables()]
    print("%s %s: closure steps %s after %d steps" % (precision, kernel, closed,
                                                     s.step_count))
    assert flips > 0, "no node turned solid: the deposit path went unchecked"
    assert closed[0] > 0
    s.close()


def test_setting_populations_drops_the_step_totals():
    # populations set by the caller after a step: the observables must
    # report the new content, not the totals of the step before
    geoms, mps = _closing_batch()
    s = lbm.Solver(geoms[:1], mps[:1], "fp32")
    s.step(21)
    before = s.observables()[0]
    f = s.populations(0)
    s.set_populations(f * np.float32(1.25), 0)
    after = s.observables()[0]
    solid = s.solid_mask(0).astype(bool)
    fluid_a = float(f[0:9][:, ~solid].astype(np.float64).sum()) * 1.25
    assert after["mass_a"] == pytest.approx(fluid_a, rel=1e-6)
    assert after["mass_a"] == pytest.approx(1.25 * before["mass_a"], rel=1e-5)
    s.close()


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_summing_launches_leave_the_state_unchanged(precision):
    # every launch summing (one step per call) against one summing launch
    # in 60 steps: the same populations and masks, bit for bit
    geoms, mps = _closing_batch()
    a = lbm.Solver(geoms, mps, precision)
    b = lbm.Solver(geoms, mps, precision)
    for _ in range(60):
        a.step(1)
    b.step(60)
    for k in range(len(geoms)):
        np.testing.assert_array_equal(a.populations(k), b.populations(k))
        np.testing.assert_array_equal(a.solid_mask(k), b.solid_mask(k))
    for oa, ob in zip(a.observables(), b.observables()):
        for key in FLUID_KEYS:
            assert oa[key] == pytest.approx(ob[key], rel=1e-12)
    a.close()
    b.close()
