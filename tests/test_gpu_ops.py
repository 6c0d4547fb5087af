"""Op-level parity of the CUDA kernels (through the C ABI) with the oracle.

Bit-exact on every residue: the operations are exact modular integer maps.
Sizes span several thread blocks and ragged tails (counts that are not
multiples of the chunk or block sizes), the smallest ring, digit sets whose
last digit is truncated, and K = 2 special primes.
"""
import numpy as np
import pytest
import torch

import workloads
from oracle import oracle as O
from paper_2402_01296_gb300 import bcn

pytestmark = pytest.mark.gpu

PARAMS = [(4, 3, 1, 1), (12, 3, 1, 1), (13, 7, 1, 1), (14, 11, 2, 2), (13, 5, 2, 2), (12, 4, 2, 1)]
_cache = {}


def pair(p):
    if p not in _cache:
        _cache[p] = (bcn.Context(*p, device=0), O.Params(*p))
    return _cache[p]


def dev(a):
    return bcn.to_device(a)


def host(t):
    torch.cuda.synchronize()
    return bcn.to_host_u32(t)


@pytest.mark.parametrize("p", PARAMS)
def test_ntt_roundtrip(p):
    c, P = pair(p)
    x = workloads.random_residues(P.q, (3,), P.N, 1)
    t = dev(x)
    c.op_ntt(t, 3, P.L, inverse=False)
    y = host(t)
    assert not np.array_equal(x, y)
    c.op_ntt(t, 3, P.L, inverse=True)
    assert np.array_equal(host(t), x)


@pytest.mark.parametrize("p", PARAMS)
def test_tensor_square(p):
    """The device NTT is a negacyclic convolution: the tensor square through it
    equals the oracle's (textbook NTT) product, residue by residue."""
    c, P = pair(p)
    n_ct = 5
    for level in (P.L, 1):
        x = workloads.random_residues(P.q[:level], (n_ct, 2), P.N, 2 + level)
        out = torch.empty((n_ct, 3, level, P.N), dtype=torch.int32, device="cuda")
        c.op_tensor_square(level, dev(x), n_ct, out)
        assert np.array_equal(host(out), P.square(level, x))


@pytest.mark.parametrize("p", PARAMS[:4])
def test_mac_with_feature_add(p):
    c, P = pair(p)
    rng = np.random.default_rng(3)
    level, n_in, n_out, K = P.L, 11, 7, 9
    x = workloads.random_residues(P.q, (n_in, 2), P.N, 4)
    idx = rng.integers(-1, n_in, size=(n_out, K)).astype(np.int32)
    w = rng.integers(-127, 128, size=(n_out, K)).astype(np.int8)
    w[0, :] = 127
    w[1, :] = -127  # extreme weights
    pt = workloads.random_residues(P.q, (n_out,), P.N, 5)
    out = torch.empty((n_out, 2, level, P.N), dtype=torch.int32, device="cuda")
    c.op_mac(level, n_in, torch.from_numpy(idx).cuda(), torch.from_numpy(w).cuda(), dev(x), dev(pt), out)
    assert np.array_equal(host(out), P.mac(level, idx, w, x, pt))
    c.op_mac(level, n_in, torch.from_numpy(idx).cuda(), torch.from_numpy(w).cuda(), dev(x), None, out)
    assert np.array_equal(host(out), P.mac(level, idx, w, x, None))


def test_mac_large_fan_in():
    """Fan-in 2048 (the CIFAR-shaped dense layer) with all weights -127 and
    residues near q: the signed 64-bit accumulation and its reduction."""
    c, P = pair((12, 3, 1, 1))
    n_in, K = 2048, 2048
    x = np.empty((n_in, 2, 2, P.N), dtype=np.uint32)
    for i, q in enumerate(P.q[:2]):
        x[:, :, i, :] = q - 1 - np.random.default_rng(i).integers(0, 3, size=(n_in, 2, P.N))
    idx = np.tile(np.arange(K, dtype=np.int32), (3, 1))
    w = np.full((3, K), -127, dtype=np.int8)
    w[1] = 127
    w[2, ::2] = 127
    out = torch.empty((3, 2, 2, P.N), dtype=torch.int32, device="cuda")
    c.op_mac(2, n_in, torch.from_numpy(idx).cuda(), torch.from_numpy(w).cuda(), dev(x), None, out)
    assert np.array_equal(host(out), P.mac(2, idx, w, x, None))


def test_mac_fan_in_spanning_tap_chunks():
    """Fan-in 5000 (above the 2048 taps a block stages at a time: two full
    chunks and a ragged third) with zero taps and repeated inputs, as in a dense
    layer over a large segment."""
    c, P = pair((12, 3, 1, 1))
    rng = np.random.default_rng(17)
    n_in, n_out, K = 700, 5, 5000
    x = workloads.random_residues(P.q[:2], (n_in, 2), P.N, 18)
    idx = rng.integers(-1, n_in, size=(n_out, K)).astype(np.int32)
    w = rng.integers(-127, 128, size=(n_out, K)).astype(np.int8)
    w[0] = -127
    out = torch.empty((n_out, 2, 2, P.N), dtype=torch.int32, device="cuda")
    c.op_mac(2, n_in, torch.from_numpy(idx).cuda(), torch.from_numpy(w).cuda(), dev(x), None, out)
    assert np.array_equal(host(out), P.mac(2, idx, w, x, None))


@pytest.mark.parametrize("p", PARAMS)
def test_rescale(p):
    c, P = pair(p)
    if P.L < 2:
        pytest.skip("needs two primes")
    for level in (P.L, 2):
        x = workloads.random_residues(P.q[:level], (4, 2), P.N, 6 + level)
        out = torch.empty((4, 2, level - 1, P.N), dtype=torch.int32, device="cuda")
        c.op_rescale(level, dev(x), 4, out)
        assert np.array_equal(host(out), P.rescale(level, x))


@pytest.mark.parametrize("p", PARAMS)
def test_square_relin_rescale(p):
    """Tensor square, hybrid key switching (ModUp, inner product with the
    device evaluation key, ModDown) and rescale, bit-exact; at the top level
    and one below (a truncated last digit when alpha > 1)."""
    c, P = pair(p)
    sk, evk = P.keygen(3)
    evk_eval = c.evk_prepare(dev(evk))
    n_ct = 3 if P.N >= 8192 else 6
    for level in (P.L, P.L - 1):
        if level < 2:
            continue
        x = workloads.random_residues(P.q[:level], (n_ct, 2), P.N, 10 + level)
        out = torch.empty((n_ct, 2, level - 1, P.N), dtype=torch.int32, device="cuda")
        c.op_square_relin_rescale(level, evk_eval, dev(x), n_ct, out)
        assert np.array_equal(host(out), P.square_relin_rescale(level, evk, x))


def test_square_relin_rescale_many_chunks():
    """More ciphertexts than one key-switching chunk holds (ragged last chunk)."""
    c, P = pair((12, 3, 1, 1))
    sk, evk = P.keygen(3)
    evk_eval = c.evk_prepare(dev(evk))
    ws_one = c.op_workspace_bytes(3, 1)
    per_chunk = c.op_workspace_bytes(3, 10**6) // ws_one
    n_ct = int(per_chunk) + 3
    x = workloads.random_residues(P.q, (n_ct, 2), P.N, 21)
    out = torch.empty((n_ct, 2, 2, P.N), dtype=torch.int32, device="cuda")
    c.op_square_relin_rescale(3, evk_eval, dev(x), n_ct, out)
    assert np.array_equal(host(out), P.square_relin_rescale(3, evk, x))


def test_errors_are_statuses():
    c, P = pair((12, 3, 1, 1))
    x = torch.zeros((1, 2, 1, P.N), dtype=torch.int32, device="cuda")
    with pytest.raises(bcn.BcnError):
        c.op_rescale(1, x, 1, x)  # nothing left to drop
    y = torch.zeros((9, P.N), dtype=torch.int32, device="cuda")
    with pytest.raises(bcn.BcnError):
        c.op_ntt(y, 1, 9, inverse=False)  # level beyond the chain
