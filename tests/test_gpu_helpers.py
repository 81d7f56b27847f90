"""The comparison helpers of the GPU parity tests, checked on the CPU on
hand-built population stacks: the per-component relative error sees a
mistake confined to the minority phase or to dilute solute, which the
error normalised by the weight alone lets through."""
import numpy as np

from tests.gpu_helpers import W22, pop_error, pop_rel_error


def _stack(rho_a, rho_b, conc):
    """Rest-state populations w_i rho of a (1, n) lattice."""
    f = np.zeros((22, 1, len(rho_a)))
    f[0:9] = W22[0:9, None, None] * np.asarray(rho_a)[None, None, :]
    f[9:18] = W22[9:18, None, None] * np.asarray(rho_b)[None, None, :]
    f[18:22] = W22[18:22, None, None] * np.asarray(conc)[None, None, :]
    return f


def test_minority_mistake_is_relative_to_its_own_density():
    fo = _stack([1.0, 0.006], [0.006, 1.0], [1.0, 1e-3])
    fg = fo.copy()
    fg[5, 0, 1] *= 1 + 1e-3       # A population at the A-minority node
    assert pop_error(fg, fo) < 1e-5   # 6e-6 of the weight: unseen there
    rel = pop_rel_error(fg, fo)
    assert abs(rel["A"] - 1e-3) < 1e-12
    assert rel["B"] == 0.0 and rel["C"] == 0.0


def test_solute_is_relative_to_c_and_the_floor_excludes_empty_nodes():
    fo = _stack([1.0, 1.0, 1.0], [0.006] * 3, [0.5, 2e-3, 1e-5])
    fg = fo.copy()
    fg[19, 0, 1] += 0.25 * 2e-3 * 4e-4   # 4e-4 of the solute at C = 2e-3
    fg[20, 0, 2] += 0.25 * 1e-5 * 0.5    # at C = 1e-5: below the floor
    rel = pop_rel_error(fg, fo)
    assert abs(rel["C"] - 4e-4) < 1e-12
    assert pop_rel_error(fg, fo, floor=1e-6)["C"] > 0.49


def test_components_do_not_mix():
    fo = _stack([0.5], [0.5], [0.0])
    fg = fo.copy()
    fg[12] *= 1 + 2e-6
    rel = pop_rel_error(fg, fo)
    assert rel["A"] == 0.0 and abs(rel["B"] - 2e-6) < 1e-12
    assert rel["C"] == 0.0  # no node with C above the floor
