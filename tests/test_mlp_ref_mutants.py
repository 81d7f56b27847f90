"""The surrogate network's FP64 reference (``oracle/mlp_ref.py``) against
planted mistakes: each case changes one line in a copy of the module and
checks that a pin computed by hand holds for the real module and fails for
the copy (an exception in the copy counts as caught)."""
import importlib.util
import math

import numpy as np
import pytest

from oracle import mlp_ref as REAL


def pin_loss(R):
    # mean over every entry, a NaN target contributing zero but still
    # counted: (1 + 4 + 9 + 0) / 4
    y = np.array([[1.0, 2.0], [3.0, 5.0]])
    t = np.array([[0.0, 0.0], [0.0, np.nan]])
    loss, dy = R.loss_and_dy(y, t)
    return (loss == 3.5
            and np.array_equal(dy, np.array([[0.5, 1.0], [1.5, 0.0]])))


def pin_gradient(R):
    # y = v tanh(w x + b) + c, one sample: the gradient by hand
    w, b, v, c, x, t = 0.7, -0.2, 1.3, 0.1, 0.5, 0.4
    ws = [np.array([[w]]), np.array([[v]])]
    bs = [np.array([b]), np.array([c])]
    _, g = R.loss_grad(ws, bs, np.array([[x]]), np.array([[t]]))
    h = math.tanh(w * x + b)
    r = v * h + c - t
    dz = 2 * r * v * (1 - h * h)
    return np.allclose(g, [dz * x, dz, 2 * r * h, 2 * r], atol=1e-15)


def pin_bias_batch(R):
    # two samples: bias gradients add over the batch
    ws = [np.array([[0.3, -0.4]]), np.array([[0.9]])]
    bs = [np.array([0.1]), np.array([-0.2])]
    x = np.array([[0.5, 0.25], [-1.0, 2.0]])
    t = np.array([[0.3], [-0.1]])
    acts, y = R.forward(ws, bs, x)
    _, dy = R.loss_and_dy(y, t)
    gw, gb = R.backward(ws, acts, dy)
    return gb[1].shape == (1,) and abs(gb[1][0] - dy.sum()) < 1e-15


def pin_bf16(R):
    # 1 + 2^-8 lies halfway between BF16 neighbours 1 and 1 + 2^-7: ties go
    # to the even one (1); 1 + 3 * 2^-8 goes up to 1 + 2^-6
    a = np.array([1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8, -(1 + 2.0 ** -8)])
    return np.array_equal(R.bf16_round(a),
                          [1.0, 1 + 2.0 ** -6, -1.0])


MUTANTS = [
    ("loss averaged over rows instead of entries",
     "    n = y.size\n", "    n = y.shape[0]\n", pin_loss),
    ("NaN targets still pull the output",
     "d = np.where(np.isnan(t), 0.0, y - np.nan_to_num(t))",
     "d = y - np.nan_to_num(t)", pin_loss),
    ("tanh derivative 1 - tanh",
     "dz = dh * (1.0 - acts[l] ** 2)", "dz = dh * (1.0 - acts[l])",
     pin_gradient),
    ("bias gradient averaged over the batch",
     "gb[l] = dz.sum(axis=0)", "gb[l] = dz.mean(axis=0)", pin_bias_batch),
    ("BF16 rounding without ties to even",
     "u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000",
     "u = (u + 0x8000) & 0xFFFF0000", pin_bf16),
]


def _caught(pin, module):
    try:
        return not pin(module)
    except Exception:
        return True


@pytest.mark.parametrize("desc,old,new,pin", MUTANTS,
                         ids=[m[0] for m in MUTANTS])
def test_pin_catches_mutant(tmp_path, desc, old, new, pin):
    src = open(REAL.__file__).read()
    assert src.count(old) == 1, desc
    path = tmp_path / "mlp_ref_mutant.py"
    path.write_text(src.replace(old, new))
    spec = importlib.util.spec_from_file_location("mlp_ref_mutant", path)
    mutant = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mutant)
    assert pin(REAL), "pin fails on the real module: " + desc
    assert _caught(pin, mutant), "pin misses the planted mistake: " + desc
