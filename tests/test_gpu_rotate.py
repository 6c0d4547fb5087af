"""Slot rotation on the GPU (automorphism, key switching with the Galois key,
ModDown; App. A Rot) against the oracle: bit-exact on every residue for data
and special primes, one- and two-prime digits, full and lower levels, and
rotations by 1, by a few slots, by N/2 - 1 and to the right; the decrypted
result is the rotated slot vector."""
import numpy as np
import pytest
import torch

import workloads
from oracle import oracle as O
from paper_2402_01296_gb300 import bcn

pytestmark = pytest.mark.gpu

PARAMS = [(12, 3, 1, 1), (13, 7, 1, 1), (14, 11, 2, 2), (12, 4, 2, 1)]
_cache = {}


def pair(p):
    if p not in _cache:
        _cache[p] = (bcn.Context(*p, device=0), O.Params(*p))
    return _cache[p]


@pytest.mark.parametrize("p", PARAMS)
def test_rotate_bit_exact(p):
    c, P = pair(p)
    sk, _ = P.keygen(3)
    for steps in (1, 5, -3, P.N // 2 - 1):
        gk = P.galois_keygen(sk, steps, 21)
        gk_eval = c.evk_prepare(bcn.to_device(gk))
        for level in (P.L, max(1, P.L - 2)):
            x = workloads.random_residues(P.q[:level], (3, 2), P.N, 30 + level + steps)
            out = torch.empty((3, 2, level, P.N), dtype=torch.int32, device="cuda")
            c.op_rotate(level, gk_eval, steps, bcn.to_device(x), 3, out)
            torch.cuda.synchronize()
            assert np.array_equal(bcn.to_host_u32(out), P.rotate(level, gk, steps, x)), (steps, level)


def test_rotate_decrypts_to_rotated_slots():
    c, P = pair((13, 7, 1, 1))
    sk, _ = P.keygen(3)
    z = np.random.default_rng(5).uniform(-1, 1, (2, P.N // 2))
    S = 2.0**30
    ct = P.encrypt(sk, O.encode(z, P.N, S, P.q), P.L, 4)
    steps = 7
    gk_eval = c.evk_prepare(bcn.to_device(c.galois_keygen(sk, steps, 9)))
    out = torch.empty(ct.shape, dtype=torch.int32, device="cuda")
    c.op_rotate(P.L, gk_eval, steps, bcn.to_device(ct), 2, out)
    dec = c.decrypt_decode(sk, bcn.to_host_u32(out), P.L, S, P.N // 2)
    # key-switching noise of one-prime digits over one special prime: well below 2^20
    assert np.abs(dec - np.roll(z, -steps, axis=1)).max() < 2.0**20 / S


def test_rotate_rejects_overlap_and_bad_level():
    c, P = pair((12, 3, 1, 1))
    x = torch.zeros((2, 2, 3, P.N), dtype=torch.int32, device="cuda")
    gk = torch.zeros(c.evk_words(), dtype=torch.int32, device="cuda")
    with pytest.raises(bcn.BcnError):
        c.op_rotate(3, gk, 1, x, 2, x)  # in place
    big = torch.zeros((2, 2, 4, P.N), dtype=torch.int32, device="cuda")
    with pytest.raises(bcn.BcnError):
        c.op_rotate(4, gk, 1, big, 2, torch.zeros_like(big))  # level beyond the chain
