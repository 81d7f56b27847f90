"""Batch creation reads the caller's input arrays in place when the device
can address them (pinned host memory, device memory: one gather kernel
for the whole batch) and copies them otherwise (pageable host memory).
Both routes must give the same stored state, bit for bit, and the same
trajectory; a batch that mixes pinned and pageable arrays takes both
routes at once."""
import dataclasses

import numpy as np
import pytest

from paper_1309_6726_gb300 import inputs as I
from paper_1309_6726_gb300 import lbm

pytestmark = pytest.mark.gpu

ARRAYS = (("solid", np.uint8), ("rho_a", np.float32), ("rho_b", np.float32),
          ("conc", np.float32))


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _pinned(g, which=None):
    """The geometry with (some of) its input arrays in pinned host memory."""
    import torch
    rep = {}
    for k, t in ARRAYS:
        if which is None or k in which:
            rep[k] = torch.from_numpy(np.ascontiguousarray(getattr(g, k), t)) \
                .pin_memory().numpy()
    return dataclasses.replace(g, **rep)


def _batch():
    members = [I.SweepMember(14, 90, 2e-2, 30.0, 1.0),
               I.SweepMember(9, 61, 5e-3, 50.0, 1.3),
               I.SweepMember(21, 120, 1e-2, 20.0, 0.8),
               I.SweepMember(17, 75, 1e-3, 40.0, 0.7)]
    geoms, mps = zip(*[I.sweep_lattice(m, x_res=16, x_out=8) for m in members])
    return list(geoms), list(mps)


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_pinned_and_pageable_inputs_give_the_same_state(precision):
    geoms, mps = _batch()
    ref = lbm.Solver(geoms, mps, precision)
    # all pinned; and a mix: lattice 0 pinned, lattice 1 half pinned,
    # lattices 2 and 3 pageable
    mixed = [_pinned(geoms[0]), _pinned(geoms[1], {"rho_a", "solid"}),
             geoms[2], geoms[3]]
    runs = {"pinned": lbm.Solver([_pinned(g) for g in geoms], mps, precision),
            "mixed": lbm.Solver(mixed, mps, precision)}
    for name, s in runs.items():
        for k in range(len(geoms)):
            np.testing.assert_array_equal(s.populations(k), ref.populations(k),
                                          err_msg=name)
            np.testing.assert_array_equal(s.solid_mask(k), ref.solid_mask(k),
                                          err_msg=name)
    ref.step(120)
    for name, s in runs.items():
        s.step(120)
        for k in range(len(geoms)):
            np.testing.assert_array_equal(s.populations(k), ref.populations(k),
                                          err_msg=name)
        s.close()
    ref.close()


def test_device_resident_inputs_give_the_same_state():
    # Inputs already on this device, given to the C ABI as device pointers:
    # the gather kernel reads them in place.
    import ctypes as C
    import torch
    geoms, mps = _batch()
    ref = lbm.Solver(geoms, mps, "fp16")
    lib = lbm.load_library()
    dev = torch.device("cuda", 0)
    keep = []
    G = (lbm.Geometry * len(geoms))()
    P = (lbm.Params * len(geoms))()
    for k, (g, p) in enumerate(zip(geoms, mps)):
        arrs = [torch.from_numpy(np.ascontiguousarray(getattr(g, name), t)).to(dev)
                for name, t in ARRAYS]
        keep += arrs
        ny, nx = g.solid.shape
        G[k] = lbm.Geometry(nx, ny, arrs[0].data_ptr(), arrs[1].data_ptr(),
                            arrs[2].data_ptr(), arrs[3].data_ptr(),
                            int(g.cap_x0), int(g.cap_x1))
        P[k] = lbm._params(p, lbm.LBM_FP16)
    h = C.c_void_p()
    assert lib.lbm_create_batch(G, P, len(geoms), C.byref(h)) == lbm.LBM_OK
    s = lbm.Solver.__new__(lbm.Solver)
    s._lib, s._h, s._keep = lib, h, []
    s.precision, s.count = "fp16", len(geoms)
    s.shapes = [g.solid.shape for g in geoms]
    for k in range(len(geoms)):
        np.testing.assert_array_equal(s.populations(k), ref.populations(k))
        np.testing.assert_array_equal(s.solid_mask(k), ref.solid_mask(k))
    s.step(60)
    ref.step(60)
    for k in range(len(geoms)):
        np.testing.assert_array_equal(s.populations(k), ref.populations(k))
    s.close()
    ref.close()


def test_masks_into_pinned_and_pageable_buffers_agree():
    # The batch's solid masks read back into a new pageable buffer, into a
    # caller's pinned buffer and lattice by lattice, after growth has
    # changed them.
    import torch
    geoms, mps = _batch()
    s = lbm.Solver(geoms, mps, "fp16")
    s.step(400)
    pageable = s.solid_masks()
    n = sum(g.solid.size for g in geoms)
    out = torch.empty(n, dtype=torch.uint8, pin_memory=True).numpy()
    out[:] = 7  # every byte must be written
    pinned = s.solid_masks(out=out)
    for k in range(len(geoms)):
        single = s.solid_mask(k)
        np.testing.assert_array_equal(pageable[k], single)
        np.testing.assert_array_equal(pinned[k], single)
        assert np.shares_memory(pinned[k], out)
    assert set(np.unique(out)) <= {0, 1}
    grown = sum(int(m.sum()) for m in pinned) - sum(int(g.solid.sum()) for g in geoms)
    print("nodes grown: %d" % grown)
    with pytest.raises(ValueError):
        s.solid_masks(out=np.empty(n - 1, np.uint8))
    s.close()
