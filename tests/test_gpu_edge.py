"""Edge inputs through the NTT-based kernels, bit-exact against the oracle.

The random-residue tests never feed the lazy butterflies ([0, 4q) forward on
the data primes) or the strict ones (the special primes) their extreme values.
Here every limb is one of: all zero, all q - 1, all (q - 1)/2 and all
(q + 1)/2 (the two sides of the centred lift's boundary, which ModUp, ModDown
and the rescale branch on), alternating 0 / q - 1, and single spikes (one
coefficient q - 1 or 1, the rest zero).  Through the device NTT (round trip,
and the forward output against the oracle's evaluations at the same points),
the tensor square, and the square activation (tensor square, key
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


@pytest.mark.parametrize("p", PARAMS)
def test_ntt_edge_inputs(p):
    """The device's forward NTT evaluates at the same 2N-th roots as the
    oracle's (any primitive root of the library's choosing: the order of the
    evaluation points is internal).  The transform of X gives each element's
    point, hence the permutation between the two; every edge pattern's
    transform must then equal the oracle's, permuted, residue for residue."""
    c, P = pair(p)
    x = patterns(P.q, P.N)
    mono = np.zeros((1, P.L, P.N), dtype=np.uint32)
    mono[0, :, 1] = 1  # the polynomial X on every limb
    t = bcn.to_device(np.concatenate([x, mono]))
    c.op_ntt(t, x.shape[0] + 1, P.L, inverse=False)
    y = host(t)
    for i in range(P.L):
        pts_dev = y[-1, i]  # element e: the evaluation point itself
        pts_ora = P.ntt_fwd(i, mono[0, i])  # oracle index k: psi^(2k+1)
        assert len(set(pts_dev.tolist())) == P.N and sorted(pts_dev.tolist()) == sorted(pts_ora.tolist())
        where = {int(v): k for k, v in enumerate(pts_ora)}
        perm = np.array([where[int(v)] for v in pts_dev])
        for r in range(x.shape[0]):
            want = P.ntt_fwd(i, x[r, i])
            assert np.array_equal(y[r, i], want[perm]), (r, i)
    c.op_ntt(t, x.shape[0] + 1, P.L, inverse=True)
    assert np.array_equal(host(t)[:-1], x)
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
