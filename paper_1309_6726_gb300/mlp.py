"""Thin ctypes binding of the surrogate network's C ABI (include/lbm_mlp.h).

Argument marshalling only: the forward pass, back-propagation and the Adam
update run in the library's kernels.  Activations, targets and gradients
are CUDA tensors passed by device pointer; parameters cross as host
float32 arrays.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import lbm

SYMBOLS = ("lbm_mlp_create", "lbm_mlp_param_count", "lbm_mlp_set_params",
           "lbm_mlp_get_params", "lbm_mlp_set_stream", "lbm_mlp_forward",
           "lbm_mlp_grad", "lbm_mlp_train_step", "lbm_mlp_destroy",
           "lbm_mlp_last_error")


class Shape(C.Structure):
    _fields_ = [("n_in", C.c_int32), ("n_hidden", C.c_int32),
                ("n_layers", C.c_int32), ("n_out", C.c_int32),
                ("max_batch", C.c_int32)]


_ready = False


def load_library():
    """The shared library with the network's argument types declared."""
    global _ready
    lib = lbm.load_library()
    if _ready:
        return lib
    vp, fp, dp = C.c_void_p, C.POINTER(C.c_float), C.POINTER(C.c_double)
    lib.lbm_mlp_create.argtypes = [C.POINTER(Shape), C.POINTER(vp)]
    lib.lbm_mlp_param_count.argtypes = [vp]
    lib.lbm_mlp_param_count.restype = C.c_int64
    lib.lbm_mlp_set_params.argtypes = [vp, fp, C.c_int64]
    lib.lbm_mlp_get_params.argtypes = [vp, fp, C.c_int64]
    lib.lbm_mlp_set_stream.argtypes = [vp, vp]
    lib.lbm_mlp_forward.argtypes = [vp, vp, C.c_int32, vp]
    lib.lbm_mlp_grad.argtypes = [vp, vp, vp, C.c_int32, vp, dp]
    lib.lbm_mlp_train_step.argtypes = [vp, vp, vp, C.c_int32, C.c_float, dp]
    lib.lbm_mlp_destroy.argtypes = [vp]
    lib.lbm_mlp_destroy.restype = None
    lib.lbm_mlp_last_error.argtypes = [vp]
    lib.lbm_mlp_last_error.restype = C.c_char_p
    _ready = True
    return lib


def layer_shapes(n_in: int, n_hidden: int, n_layers: int, n_out: int):
    """(rows, cols) of each weight matrix, in the packed order."""
    dims = [n_in] + [n_hidden] * n_layers + [n_out]
    return [(dims[i + 1], dims[i]) for i in range(len(dims) - 1)]


def pack(weights, biases) -> np.ndarray:
    """Packs per-layer W (rows x cols) and b into the library's layout."""
    parts = []
    for w, b in zip(weights, biases):
        parts += [np.asarray(w, np.float32).ravel(),
                  np.asarray(b, np.float32).ravel()]
    return np.concatenate(parts)


def unpack(theta, n_in, n_hidden, n_layers, n_out):
    """Inverse of :func:`pack`: lists of W and b (float64 views)."""
    theta = np.asarray(theta, np.float64)
    ws, bs, o = [], [], 0
    for r, c in layer_shapes(n_in, n_hidden, n_layers, n_out):
        ws.append(theta[o:o + r * c].reshape(r, c))
        o += r * c
        bs.append(theta[o:o + r])
        o += r
    return ws, bs


class Mlp:
    """One network on the GPU (tanh hidden layers, linear output)."""

    def __init__(self, n_in: int, n_hidden: int, n_layers: int, n_out: int,
                 max_batch: int):
        self._lib = load_library()
        self.n_in, self.n_hidden, self.n_layers, self.n_out = (
            n_in, n_hidden, n_layers, n_out)
        self.max_batch = max_batch
        h = C.c_void_p()
        st = self._lib.lbm_mlp_create(
            C.byref(Shape(n_in, n_hidden, n_layers, n_out, max_batch)),
            C.byref(h))
        if st != lbm.LBM_OK:
            raise lbm.LbmError(st, self._lib.lbm_mlp_last_error(None).decode())
        self._h = h
        self.param_count = int(self._lib.lbm_mlp_param_count(h))

    def _check(self, st):
        if st != lbm.LBM_OK:
            raise lbm.LbmError(st, self._lib.lbm_mlp_last_error(self._h).decode())

    def set_params(self, theta: np.ndarray):
        theta = np.ascontiguousarray(theta, np.float32)
        self._check(self._lib.lbm_mlp_set_params(
            self._h, theta.ctypes.data_as(C.POINTER(C.c_float)), theta.size))

    def params(self) -> np.ndarray:
        out = np.empty(self.param_count, np.float32)
        self._check(self._lib.lbm_mlp_get_params(
            self._h, out.ctypes.data_as(C.POINTER(C.c_float)), out.size))
        return out

    def set_stream(self, stream_handle):
        self._check(self._lib.lbm_mlp_set_stream(self._h, stream_handle))

    def _bind(self):
        # run on torch's current stream, so that inputs written by torch
        # are ready and torch's reads of the outputs wait for the kernels;
        # torch's default stream is CUDA's legacy stream (cudaStreamLegacy)
        import torch
        s = torch.cuda.current_stream().cuda_stream
        self.set_stream(s if s else 1)

    @staticmethod
    def _dev(t, cols):
        import torch
        if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()
                and t.dim() == 2 and t.shape[1] == cols):
            raise ValueError("expected a contiguous float32 CUDA tensor "
                             "with %d columns" % cols)
        return t.data_ptr()

    def forward(self, x, out=None):
        """y = network(x) for a float32 CUDA tensor x [batch, n_in]."""
        import torch
        if out is None:
            out = torch.empty((x.shape[0], self.n_out), device=x.device,
                              dtype=torch.float32)
        self._bind()
        self._check(self._lib.lbm_mlp_forward(
            self._h, self._dev(x, self.n_in), x.shape[0],
            self._dev(out, self.n_out)))
        return out

    def grad(self, x, target):
        """(gradient as a float32 CUDA tensor, loss) at the current weights."""
        import torch
        g = torch.empty(self.param_count, device=x.device, dtype=torch.float32)
        loss = C.c_double()
        self._bind()
        self._check(self._lib.lbm_mlp_grad(
            self._h, self._dev(x, self.n_in), self._dev(target, self.n_out),
            x.shape[0], g.data_ptr(), C.byref(loss)))
        return g, loss.value

    def train_step(self, x, target, lr: float, want_loss: bool = False):
        loss = C.c_double()
        self._bind()
        self._check(self._lib.lbm_mlp_train_step(
            self._h, self._dev(x, self.n_in), self._dev(target, self.n_out),
            x.shape[0], float(lr), C.byref(loss) if want_loss else None))
        return loss.value if want_loss else None

    def close(self):
        if getattr(self, "_h", None):
            self._lib.lbm_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
