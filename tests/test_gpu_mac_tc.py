"""Tensor-core MAC (byte planes on the tcgen05 tensor cores) against the
oracle's MAC and against the CUDA-core MAC: bit-exact on every residue, for
dense and conv layers whose groups have at least 32 outputs and at most 512
taps (the layers it runs), including fan-in that is not a multiple of the MMA's
K step, several output tiles, zero taps, extreme weights and residues near q,
and the feature add."""
import numpy as np
import pytest
import torch

import workloads
from oracle import oracle as O
from paper_2402_01296_gb300 import bcn

pytestmark = pytest.mark.gpu

_ctx = {}


def pair(p):
    if p not in _ctx:
        _ctx[p] = (bcn.Context(*p, device=0), O.Params(*p))
    return _ctx[p]


def host(t):
    torch.cuda.synchronize()
    return bcn.to_host_u32(t)


def run_model(ctx, layer, w, x, pt, impl):
    m = bcn.Model(ctx, [layer], [w], [1.0])
    m.set_mac_impl(impl)
    out = torch.full(m.out_shape(), -1, dtype=torch.int32, device="cuda")
    xd = bcn.to_device(x)
    pts = [bcn.to_device(pt)] if layer["add"] else []
    key = torch.zeros(ctx.evk_words(), dtype=torch.int32, device="cuda")  # no square: the key is not read
    m.eval(key, xd, pts, out, m.alloc_workspace())
    r = host(out)
    assert ctx.device_status() == 0
    m.close()
    return r


@pytest.mark.parametrize("n_in,n_out,extreme", [(180, 100, False), (512, 64, True), (37, 33, False),
                                                (100, 130, False), (16, 32, True), (100, 10, True),
                                                (64, 12, False)])
def test_dense_matches_oracle(n_in, n_out, extreme):
    c, P = pair((13, 3, 1, 1))
    rng = np.random.default_rng(n_in * 7 + n_out)
    level = P.L
    if extreme:  # residues at q - 1 - small, weights +-127: the largest exact sums
        x = np.empty((n_in, 2, level, P.N), dtype=np.uint32)
        for i, q in enumerate(P.q[:level]):
            x[:, :, i, :] = q - 1 - rng.integers(0, 3, size=(n_in, 2, P.N))
        w = np.where(rng.random((n_out, n_in)) < 0.5, -127, 127).astype(np.int8)
        w[0] = 127
        w[1] = -127
    else:
        x = workloads.random_residues(P.q[:level], (n_in, 2), P.N, 5)
        w = rng.integers(-127, 128, size=(n_out, n_in)).astype(np.int8)
    pt = workloads.random_residues(P.q[:level], (n_out,), P.N, 6)
    layer = dict(type="dense", n_in=n_in, n_out=n_out, add=True, square=False)
    got = run_model(c, layer, w, x, pt, 0)
    idx = np.tile(np.arange(n_in, dtype=np.int32), (n_out, 1))
    assert np.array_equal(got, P.mac(level, idx, w, x, pt))
    assert np.array_equal(got, run_model(c, layer, w, x, pt, 1))


def test_conv_with_padding_matches_cuda_cores():
    """16 -> 32 channels, 3x3, stride 2, padding 1 (the CIFAR-shaped second
    conv) on a 9 x 7 map: border positions have zero taps."""
    c, P = pair((12, 4, 1, 1))
    layer = dict(type="conv", cin=16, h=9, w=7, cout=32, k=3, stride=2, pad=1, add=True, square=False)
    ho, wo = workloads.conv_out_hw(9, 7, 3, 2, 1)
    rng = np.random.default_rng(9)
    w = rng.integers(-127, 128, size=(32, 16, 3, 3)).astype(np.int8)
    x = workloads.random_residues(P.q, (16 * 9 * 7, 2), P.N, 10)
    pt = workloads.random_residues(P.q, (32 * ho * wo,), P.N, 11)
    got = run_model(c, layer, w, x, pt, 0)
    assert np.array_equal(got, run_model(c, layer, w, x, pt, 1))
    # and against the oracle's MAC with the conv's taps written out
    idx = np.full((32 * ho * wo, 16 * 9), -1, dtype=np.int32)
    wt = np.zeros((32 * ho * wo, 16 * 9), dtype=np.int8)
    for co in range(32):
        for oy in range(ho):
            for ox in range(wo):
                o = (co * ho + oy) * wo + ox
                for ci in range(16):
                    for ky in range(3):
                        for kx in range(3):
                            iy, ix = oy * 2 - 1 + ky, ox * 2 - 1 + kx
                            if 0 <= iy < 9 and 0 <= ix < 7:
                                t = (ci * 3 + ky) * 3 + kx
                                idx[o, t] = (ci * 9 + iy) * 7 + ix
                                wt[o, t] = w[co, ci, ky, kx]
    assert np.array_equal(got, P.mac(P.L, idx, wt, x, pt))


def test_cifar_conv2_shape_at_full_ring():
    """The CIFAR-shaped second convolution's groups (16 -> 32 channels, 3x3,
    stride 2, padding 1: 144 taps x 32 outputs, on the tensor cores) at
    N = 16384 with its 10 live limbs of the 11 + 2 prime chain and the feature
    add, on a 4 x 4 map (border positions with zero taps, inner ones with all
    144): bit-exact against the oracle and the CUDA-core MAC."""
    c, P = pair((14, 11, 2, 2))
    level = 10
    layer = dict(type="conv", cin=16, h=4, w=4, cout=32, k=3, stride=2, pad=1, add=True, square=False)
    rng = np.random.default_rng(23)
    w = rng.integers(-127, 128, size=(32, 16, 3, 3)).astype(np.int8)
    w[0] = 127
    w[1] = -127
    n_in, n_out = workloads.cipher_layer_io(layer)
    x = workloads.random_residues(P.q[:level], (n_in, 2), P.N, 24)
    x[:3] = np.array(P.q[:level], dtype=np.uint32)[None, None, :, None] - 1  # residues at q - 1
    pt = workloads.random_residues(P.q[:level], (n_out,), P.N, 25)
    # the model runs at the chain's top level: evaluate at level 10 through the op entry point
    idx, wt = O.layer_table(layer, w)  # [n_out][144] input index (-1: padding) and weight
    want = P.mac(level, idx, wt, x, pt)
    got = torch.full((n_out, 2, level, P.N), -1, dtype=torch.int32, device="cuda")
    c.op_mac(level, n_in, torch.from_numpy(idx).cuda(), torch.from_numpy(wt).cuda(), bcn.to_device(x),
             bcn.to_device(pt), got)
    assert np.array_equal(host(got), want)
    # the model path (tensor cores, groups of 32 outputs) on the same layer at the top level
    xl = workloads.random_residues(P.q, (n_in, 2), P.N, 26)
    ptl = workloads.random_residues(P.q, (n_out,), P.N, 27)
    tc = run_model(c, layer, w, xl, ptl, 0)
    assert np.array_equal(tc, P.mac(P.L, idx, wt, xl, ptl))
    assert np.array_equal(tc, run_model(c, layer, w, xl, ptl, 1))


def test_cifar_dense_2048_to_10_at_full_ring():
    """The CIFAR-shaped output layer: 2048 -> 10 at N = 16384, 9 limbs of the
    11 + 2 chain (more taps than the tensor cores' exact 512, so the CUDA-core
    MAC), extreme weights and residues near q, against the oracle."""
    c, P = pair((14, 11, 2, 2))
    level, n_in, n_out = 9, 2048, 10
    rng = np.random.default_rng(31)
    x = workloads.random_residues(P.q[:level], (n_in, 2), P.N, 32)
    x[: n_in // 4] = np.array(P.q[:level], dtype=np.uint32)[None, None, :, None] - 1
    w = rng.integers(-127, 128, size=(n_out, n_in)).astype(np.int8)
    w[0] = 127
    w[1] = -127
    idx = np.tile(np.arange(n_in, dtype=np.int32), (n_out, 1))
    got = torch.full((n_out, 2, level, P.N), -1, dtype=torch.int32, device="cuda")
    c.op_mac(level, n_in, torch.from_numpy(idx).cuda(), torch.from_numpy(w).cuda(), bcn.to_device(x), None, got)
    assert np.array_equal(host(got), P.mac(level, idx, w, x, None))
    assert c.device_status() == 0


@pytest.mark.parametrize("n_in,n_out", [(27, 16), (2048, 10), (37, 33)])
def test_dp4a_mac_matches_oracle(n_in, n_out):
    """The byte-plane dp4a MAC (mac impl 2): fan-in not a multiple of 4, extreme
    weights, residues near q, the feature add; against the oracle."""
    c, P = pair((13, 3, 1, 1))
    rng = np.random.default_rng(n_in + 3 * n_out)
    level = P.L
    x = workloads.random_residues(P.q[:level], (n_in, 2), P.N, 41)
    x[: n_in // 3] = np.array(P.q[:level], dtype=np.uint32)[None, None, :, None] - 1
    w = rng.integers(-127, 128, size=(n_out, n_in)).astype(np.int8)
    w[0] = -127
    pt = workloads.random_residues(P.q[:level], (n_out,), P.N, 42)
    layer = dict(type="dense", n_in=n_in, n_out=n_out, add=True, square=False)
    got = run_model(c, layer, w, x, pt, 2)
    idx = np.tile(np.arange(n_in, dtype=np.int32), (n_out, 1))
    assert np.array_equal(got, P.mac(level, idx, w, x, pt))
