"""Edge inputs through the NTT-based kernels, bit-exact against the oracle.

The random-residue tests never feed the lazy butterflies ([0, 4q) forward on
the data primes) or the strict ones (the special primes) their extreme values.
Here every limb is one of: all zero, all q - 1, all (q - 1)/2 and all
(q + 1)/2 (the two sides of the centred lift's boundary, which ModUp, ModDown
and the rescale branch on), alternating 0 / q - 1, and single spikes (one
coefficient q - 1 or 1, the rest zero).  Through the device NTT (round trip,
and the forward output against the oracle's evaluations in bit-reversed
order), the tensor square, and the square activation (tensor square, key
switching through the special primes, ModDown, rescale) at every ring degree,
on the top level and one below.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2402_01296_gb300 import bcn

pytestmark = pytest.mark.gpu

PARAMS = [(4, 3, 1, 1), (12, 3, 1, 1), (13, 7, 1, 1), (14, 11, 2, 2), (13, 5, 2, 2)]
_cache = {}


def pair(p):
    if p not in _cache:
        _cache[p] = (bcn.Context(*p, device=0), O.Params(*p))
    return _cache[p]


def host(t):
    torch.cuda.synchronize()
    return bcn.to_host_u32(t)


def patterns(primes, N):
    """[n_pattern][len(primes)][N] uint32 limbs, one edge pattern per row (the
    same pattern on every limb, with that limb's prime)."""
    rows = []
    for kind in ("zero", "qm1", "half", "half1", "alt", "spike_hi", "spike_one", "spike_last"):
        limbs = []
        for q in primes:
            a = np.zeros(N, dtype=np.uint64)
            if kind == "qm1":
                a[:] = q - 1
            elif kind == "half":
                a[:] = (q - 1) // 2
            elif kind == "half1":
                a[:] = (q + 1) // 2
            elif kind == "alt":
                a[1::2] = q - 1
            elif kind == "spike_hi":
                a[N // 3] = q - 1
            elif kind == "spike_one":
                a[0] = 1
            elif kind == "spike_last":
                a[N - 1] = q - 1
            limbs.append(a)
        rows.append(np.stack(limbs))
    return np.stack(rows).astype(np.uint32)


def bitrev(n_bits):
    r = np.zeros(1 << n_bits, dtype=np.int64)
    for i in range(1 << n_bits):
        r[i] = int(format(i, f"0{n_bits}b")[::-1], 2) if n_bits else 0
    return r


@pytest.mark.parametrize("p", PARAMS)
def test_ntt_edge_inputs(p):
    c, P = pair(p)
    x = patterns(P.q, P.N)
    t = bcn.to_device(x)
    c.op_ntt(t, x.shape[0], P.L, inverse=False)
    y = host(t)
    perm = bitrev(P.log_n)
    for r in range(x.shape[0]):
        for i in range(P.L):
            # canonical, and element e is the evaluation at psi^(2 brv(e) + 1)
            want = P.ntt_fwd(i, x[r, i])
            assert np.array_equal(y[r, i], want[perm]), (r, i)
    c.op_ntt(t, x.shape[0], P.L, inverse=True)
    assert np.array_equal(host(t), x)
    assert c.device_status() == 0


def edge_cts(P, level):
    """Ciphertexts (c0, c1) from pairs of edge patterns, [n][2][level][N]."""
    pat = patterns(P.q[:level], P.N)
    n = pat.shape[0]
    pairs = [(a, (a * 3 + 1) % n) for a in range(n)] + [(1, 1), (4, 4), (5, 5)]
    return np.stack([np.stack([pat[a], pat[b]]) for a, b in pairs])


@pytest.mark.parametrize("p", PARAMS)
def test_tensor_square_edge_inputs(p):
    c, P = pair(p)
    for level in (P.L, 1):
        x = edge_cts(P, level)
        out = torch.empty((x.shape[0], 3, level, P.N), dtype=torch.int32, device="cuda")
        c.op_tensor_square(level, bcn.to_device(x), x.shape[0], out)
        assert np.array_equal(host(out), P.square(level, x))
    assert c.device_status() == 0


@pytest.mark.parametrize("p", PARAMS)
def test_square_relin_rescale_edge_inputs(p):
    c, P = pair(p)
    _, evk = P.keygen(3)
    evk_eval = c.evk_prepare(bcn.to_device(evk))
    for level in (P.L, P.L - 1):
        if level < 2:
            continue
        x = edge_cts(P, level)
        out = torch.empty((x.shape[0], 2, level - 1, P.N), dtype=torch.int32, device="cuda")
        c.op_square_relin_rescale(level, evk_eval, bcn.to_device(x), x.shape[0], out)
        got = host(out)
        want = P.square_relin_rescale(level, evk, x)
        assert np.array_equal(got, want), f"level {level}: rows {np.unique(np.nonzero(got != want)[0])}"
    assert c.device_status() == 0
