"""The FP16 storage codec alone (enc_node16 / dec_pair / dec_sol16 in
lbm_device.cuh), on the GPU, against what it must guarantee, on scaled
equilibria f^_i = rho (1 + 3 e.u + 9/2 (e.u)^2 - 3/2 u.u) of two
components and random solute values:

* mass: the nine read-back values of each component, weighted, sum to
  the written content within a few FP32 roundings at rho's magnitude
  (the quantisation error is taken up by the rest reference);
* every value read back within one unit of the 16-bit format (FP16 or
  BF16) of its deviation from the reference (plus FP32 rounding): the deviation is 2^10 (f^_i - r_i),
  r_i = rho~ + e_i . v;
* v is the odd part of the axis populations for the component with the
  larger rest population where |v_x| + |v_y| <= f^_0, for the other one
  only at a node next to a wall and where |v_x| + |v_y| <= 4 f^_0, and 0
  otherwise; with it, the deviations of a slow flow are second order in
  u, so the read-back error of such a node is far below the rest-only
  reference's.  Both kinds of node are encoded.

A small test library is compiled from the library's own header with nvcc."""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = r'''
#include "lbm_device.cuh"
using namespace lbmk;
// f: n x 9 {A, B} pairs (scaled), g: n x 4 scaled solute; out: n x 9 pairs
// read back, gout: n x 4, words: n x NW16
template <class F>
__global__ void k(const float2 *f, const float *g, float2 *out, float *gout,
                  uint32_t *words, int n, bool wall) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    float2 fv[Q];
    float gv[QS];
    for (int i = 0; i < Q; ++i) fv[i] = f[j * Q + i];
    for (int k = 0; k < QS; ++k) gv[k] = g[j * QS + k];
    uint32_t w[NW16];
    enc_node16<F>(fv, gv, w, wall);
    for (int q = 0; q < NW16; ++q) words[j * NW16 + q] = w[q];
    const float2 ref = make_float2(__uint_as_float(w[W16_REF]),
                                   __uint_as_float(w[W16_REF + 1]));
    out[j * Q] = ref;
    for (int i = 1; i < Q; ++i)
        out[j * Q + i] = dec_pair<F>(i, false, w[i - 1], ref, w[W16_VEL], w[W16_VEL + 1]);
    const float rc = __uint_as_float(w[W16_REF + 2]);
    for (int k = 0; k < QS; ++k)
        gout[j * QS + k] = dec_sol16<F>(w[W16_SOL + (k >> 1)], k, rc);
}
extern "C" int run(int bf16, int wall, const float *f, const float *g,
                   float *out, float *gout, unsigned *words, int n) {
    if (bf16)
        k<BF16><<<(n + 127) / 128, 128>>>((const float2 *)f, g, (float2 *)out, gout,
                                          (uint32_t *)words, n, wall != 0);
    else
        k<F16><<<(n + 127) / 128, 128>>>((const float2 *)f, g, (float2 *)out, gout,
                                         (uint32_t *)words, n, wall != 0);
    return (int)cudaDeviceSynchronize();
}
'''
EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
EY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
NW16, W16_SOL, W16_VEL, W16_REF = 15, 8, 10, 12


@pytest.fixture(scope="module")
def codec(tmp_path_factory):
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    d = tmp_path_factory.mktemp("codec")
    (d / "codec.cu").write_text(SRC)
    so = str(d / "libcodec.so")
    nvcc = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a",
                    "-O3", "-std=c++17", "--expt-relaxed-constexpr",
                    "-Xcompiler", "-fPIC", "-shared",
                    "-I", os.path.join(ROOT, "paper_1309_6726_gb300", "csrc"),
                    str(d / "codec.cu"), "-o", so], check=True)
    lib = C.CDLL(so)
    lib.run.argtypes = [C.c_int, C.c_int] + [C.c_void_p] * 5 + [C.c_int]

    def call(f, g, fmt, wall):
        n = f.shape[0]
        dev = torch.device("cuda", 0)
        fd = torch.from_numpy(np.ascontiguousarray(f, np.float32)).to(dev)
        gd = torch.from_numpy(np.ascontiguousarray(g, np.float32)).to(dev)
        out = torch.empty_like(fd)
        gout = torch.empty_like(gd)
        words = torch.empty((n, NW16), dtype=torch.int32, device=dev)
        assert lib.run(1 if fmt == "bf16" else 0, int(wall), fd.data_ptr(),
                       gd.data_ptr(), out.data_ptr(), gout.data_ptr(),
                       words.data_ptr(), n) == 0
        return (out.cpu().numpy().astype(np.float64),
                gout.cpu().numpy().astype(np.float64),
                words.cpu().numpy().view(np.uint32))
    return call


def _equilibria(rng, n, u_max):
    """n nodes x 9 x {A, B}: scaled equilibria, A the majority in half of
    the nodes, B in the other half."""
    rho = np.empty((n, 2))
    maj = rng.uniform(0.5, 1.5, n)
    mino = rng.uniform(0.004, 0.02, n)
    a_major = rng.random(n) < 0.5
    rho[:, 0] = np.where(a_major, maj, mino)
    rho[:, 1] = np.where(a_major, mino, maj)
    ang = rng.uniform(0, 2 * np.pi, (n, 2))
    mag = rng.uniform(0, u_max, (n, 2))
    ux, uy = mag * np.cos(ang), mag * np.sin(ang)
    eu = EX[None, :, None] * ux[:, None, :] + EY[None, :, None] * uy[:, None, :]
    f = rho[:, None, :] * (1 + 3 * eu + 4.5 * eu ** 2
                           - 1.5 * (ux ** 2 + uy ** 2)[:, None, :])
    return f.astype(np.float32), rho, a_major


def _half(bits, fmt):
    b = np.asarray(bits, np.uint32)
    if fmt == "bf16":  # BF16: the upper half of an FP32
        return (b << 16).astype(np.uint32).view(np.float32).astype(np.float64)
    return b.astype(np.uint16).view(np.float16).astype(np.float64)


# significand bits below the leading one, smallest normal exponent
FORMATS = {"fp16": (10, -14), "bf16": (7, -126)}


def _ulp(x, fmt):
    m, emin = FORMATS[fmt]
    return 2.0 ** (np.floor(np.log2(np.maximum(np.abs(x), 2.0 ** emin))) - m)


@pytest.mark.parametrize("wall", [False, True])
@pytest.mark.parametrize("fmt", ["fp16", "bf16"])
@pytest.mark.parametrize("u_max", [1e-3, 0.1, 0.6])
def test_codec_round_trip(codec, u_max, fmt, wall):
    rng = np.random.default_rng(int(u_max * 1e4) + 3)
    n = 20000
    f, rho, a_major = _equilibria(rng, n, u_max)
    g = rng.uniform(0.0, 1.2, (n, 4)).astype(np.float32)
    out, gout, words = codec(f, g, fmt, wall)
    f64 = f.astype(np.float64)
    # mass of each component: weighted sum of the read-back values against
    # the written one (FP32 inputs summed in FP64)
    m_in = np.einsum("i,nic->nc", W9, f64)
    m_out = np.einsum("i,nic->nc", W9, out)
    size = np.einsum("i,nic->nc", W9, np.abs(f64))  # the values' magnitude
    assert np.all(np.abs(m_out - m_in) <= 8 * 2.0 ** -24 * size)
    # v: the odd axis part where |v_x| + |v_y| <= f^_0 (majority) or
    # 4 f^_0 (minority at a wall node), else 0
    vx = np.stack([_half(words[:, W16_VEL] & 0xFFFF, fmt),
                   _half(words[:, W16_VEL] >> 16, fmt)], 1)
    vy = np.stack([_half(words[:, W16_VEL + 1] & 0xFFFF, fmt),
                   _half(words[:, W16_VEL + 1] >> 16, fmt)], 1)
    ox = 0.5 * (f64[:, 1] - f64[:, 3])
    oy = 0.5 * (f64[:, 2] - f64[:, 4])
    major = np.stack([a_major, ~a_major], 1)
    lim = np.where(major, 1.0, 4.0 if wall else 0.0) * f64[:, 0]
    odd = np.abs(ox) + np.abs(oy)
    use = odd <= lim * (1 - 1e-6)
    outside = odd > lim * (1 + 1e-6)
    assert np.all(vx[outside] == 0) and np.all(vy[outside] == 0)
    if wall:
        assert use[~major].mean() > 0.5  # the minority takes v here
    rt = 2.0 ** -FORMATS[fmt][0]
    np.testing.assert_allclose(vx[use], ox[use], rtol=rt, atol=2.0 ** -24)
    np.testing.assert_allclose(vy[use], oy[use], rtol=rt, atol=2.0 ** -24)
    # every moving value: within one unit of the format of its deviation (in
    # the 2^10-scaled units it is stored in) plus FP32 rounding
    # (the writer's deviation is taken from the rest population f^_0 before
    # the reference takes up the quantisation error; the read-back adds
    # that error, |rho~ - f^_0|, to every value)
    ref = out[:, 0, :]
    lin = EX[None, 1:, None] * vx[:, None, :] + EY[None, 1:, None] * vy[:, None, :]
    r = ref[:, None, :] + lin
    dev = 1024.0 * (f64[:, 1:, :] - (f64[:, :1, :] + lin))
    ulp16 = _ulp(dev, fmt)
    err = np.abs(out[:, 1:, :] - f64[:, 1:, :])
    # (FP32 rounding at the larger of the value and its reference r_i, which
    # the read-back forms first)
    bound = ulp16 / 1024.0 \
        + 4 * 2.0 ** -24 * np.maximum(np.abs(f64[:, 1:, :]), np.abs(r)) \
        + np.abs(ref - f64[:, 0, :])[:, None, :]
    bad = err > bound * (1 + 1e-9)
    if bad.any():
        j, i, c = np.unravel_index(np.argmax(err / bound), err.shape)
        raise AssertionError(
            "%d values above the bound; worst node %d dir %d comp %d: f %.9g "
            "read %.9g err %.3g bound %.3g dev %.6g ref %.9g f0 %.9g v %.6g %.6g"
            % (bad.sum(), j, i + 1, c, f64[j, i + 1, c], out[j, i + 1, c],
               err[j, i, c], bound[j, i, c], dev[j, i, c], ref[j, c],
               f64[j, 0, c], vx[j, c], vy[j, c]))
    # the solute: within its FP16 rounding (its own and its share of the
    # error taken up by C~) of its deviation from C~; its total exact to
    # FP32 rounding
    c = 0.25 * g.astype(np.float64).sum(1)
    gd = 1024.0 * (g.astype(np.float64) - c[:, None])
    ulp16 = _ulp(np.abs(gd).max(1), fmt)
    assert np.all(np.abs(gout - g) <= 2 * ulp16[:, None] / 1024.0 + 4 * 2.0 ** -24 * (1 + np.abs(g)))
    assert np.abs(gout.sum(1) - g.astype(np.float64).sum(1)).max() < 1e-6
    if u_max <= 1e-3:
        # a slow flow: the majority's read-back is as accurate as FP32
        # (second-order deviations: measured bit-exact, the FP16 rounding
        # being far below half an FP32 unit of the value); the rest-only
        # reference would round 3 rho e.u to 11 bits: a mean error of
        # 2.0e-7 rho here, max 2e-6
        emaj = np.where(a_major[:, None], err[:, :, 0], err[:, :, 1]) \
            / np.where(a_major, rho[:, 0], rho[:, 1])[:, None]
        print("slow flow: majority read-back error / rho: mean %.3g, max %.3g"
              % (emaj.mean(), emaj.max()))
        assert emaj.mean() < 6e-8
        assert emaj.max() < 6e-7
