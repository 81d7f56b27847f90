"""The reciprocal the step kernels use for the Shan-Chen shift and the
barycentric velocity (rcp_nr in lbm_device.cuh: the hardware approximation
refined by one Newton-Raphson step) against the correctly rounded quotient
1/x that CUDA's IEEE division gives, on the GPU, over a sweep of inputs
that includes the kernels' guards (the callers only pass x > 1e-30 for the
mixture density and x > 1e-12 for a component's density).

Bound: at most one unit in the last place, and correctly rounded for at
least 99 % of the inputs.  A small test library is compiled from the
library's own header with nvcc for this check."""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = r'''
#include "lbm_device.cuh"
__global__ void k(const float *x, float *r, float *q, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) { r[i] = lbmk::rcp_nr(x[i]); q[i] = __fdiv_rn(1.0f, x[i]); }
}
extern "C" int run(const float *x, float *r, float *q, int n) {
    k<<<(n + 255) / 256, 256>>>(x, r, q, n);
    return (int)cudaDeviceSynchronize();
}
'''


@pytest.fixture(scope="module")
def rcp_lib(tmp_path_factory):
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    d = tmp_path_factory.mktemp("rcp")
    src = d / "rcp.cu"
    src.write_text(SRC)
    so = str(d / "librcp.so")
    nvcc = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a",
                    "-O3", "-std=c++17", "--expt-relaxed-constexpr",
                    "-Xcompiler", "-fPIC", "-shared",
                    "-I", os.path.join(ROOT, "paper_1309_6726_gb300", "csrc"),
                    str(src), "-o", so], check=True)
    lib = C.CDLL(so)
    lib.run.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]
    return lib


def _ulps(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    ia = a.view(np.int32).astype(np.int64)
    ib = b.view(np.int32).astype(np.int64)
    return np.abs(ia - ib)


def test_rcp_nr_within_one_ulp_of_the_quotient(rcp_lib):
    import torch
    rng = np.random.default_rng(5)
    xs = [10.0 ** rng.uniform(-30, 30, 200_000),            # the whole range
          rng.uniform(0.5, 2.0, 200_000),                    # densities ~1
          rng.uniform(1e-3, 1e-2, 100_000),                  # minority phase
          1e-30 * (1 + rng.uniform(0, 1e-3, 1000)),          # guard of rho_A+rho_B
          1e-12 * (1 + rng.uniform(0, 1e-3, 1000)),          # guard of rho_s
          np.array([1.0, 2.0, 3.0, 1.0 / 3.0, 0.006, 1.006])]
    x = np.concatenate(xs).astype(np.float32)
    dx = torch.from_numpy(x).cuda()
    r = torch.empty_like(dx)
    q = torch.empty_like(dx)
    assert rcp_lib.run(dx.data_ptr(), r.data_ptr(), q.data_ptr(), x.size) == 0
    r, q = r.cpu().numpy(), q.cpu().numpy()
    assert np.isfinite(r).all()
    u = _ulps(r, q)
    print("rcp_nr against 1/x: max %d ulp, %.4f %% not correctly rounded"
          % (u.max(), 100.0 * (u > 0).mean()))
    assert u.max() <= 1
    assert (u > 0).mean() < 0.01
