"""Hoisted rotations (bcn_op_rotate_many: one ModUp per ciphertext, shared by
all its rotations) against the oracle's one-at-a-time rotation (App. A Rot),
bit-exact on every residue: identity, positive, negative and large steps, more
ciphertexts than one chunk holds and more rotations than one batch, one and two
special primes, alpha 1 and 2, at the top level and below it."""
import numpy as np
import pytest
import torch

import workloads
from oracle import oracle as O
from paper_2402_01296_gb300 import bcn

pytestmark = pytest.mark.gpu


def host(t):
    torch.cuda.synchronize()
    return bcn.to_host_u32(t)


@pytest.mark.parametrize("params,steps,n_ct", [
    ((12, 3, 1, 1), [1, 0, -1, 5, 2047, -300, 64, 3], 10),
    ((12, 4, 2, 2), list(range(-17, 18)) + [1000], 2),          # 36 rotations: two batches
    ((13, 5, 2, 1), [1, 16, -16, 4095], 3),
    ((14, 11, 2, 2), [1, -1, 17, 8191], 2),
])
def test_rotate_many_matches_oracle(params, steps, n_ct):
    P = O.Params(*params)
    ctx = bcn.Context(*params, device=0)
    sk, _ = P.keygen(3)
    half = P.N // 2
    keys = {}
    for r in steps:
        if r % half and r % half not in keys:
            keys[r % half] = P.galois_keygen(sk, r % half, 50 + (r % half))
    gks = {r: ctx.evk_prepare(bcn.to_device(k)) for r, k in keys.items()}
    for level in (P.L, max(1, P.L - 2)):
        x = workloads.random_residues(P.q[:level], (n_ct, 2), P.N, 60 + level)
        out = torch.full((n_ct, len(steps), 2, level, P.N), -1, dtype=torch.int32, device="cuda")
        ctx.op_rotate_many(level, gks, steps, bcn.to_device(x), n_ct, out)
        got = host(out)
        for k, r in enumerate(steps):
            want = x if r % half == 0 else P.rotate(level, keys[r % half], r % half, x)
            assert np.array_equal(got[:, k], want), f"level {level}, step {r}"
    assert ctx.device_status() == 0


def test_rotate_many_equals_rotate_one_at_a_time():
    """The hoisted path and bcn_op_rotate give the same residues (GPU vs GPU,
    beside the oracle check above), on the CryptoNets-scale ring."""
    P = O.Params(13, 7, 1, 1)
    ctx = bcn.Context(13, 7, 1, 1, device=0)
    sk, _ = P.keygen(3)
    steps = [1, 2, 3, 16, 17]
    gks = {r: ctx.evk_prepare(bcn.to_device(P.galois_keygen(sk, r, 70 + r))) for r in steps}
    x = bcn.to_device(workloads.random_residues(P.q, (4, 2), P.N, 71))
    out = torch.empty((4, len(steps), 2, P.L, P.N), dtype=torch.int32, device="cuda")
    ctx.op_rotate_many(P.L, gks, steps, x, 4, out)
    for k, r in enumerate(steps):
        one = torch.empty((4, 2, P.L, P.N), dtype=torch.int32, device="cuda")
        ctx.op_rotate(P.L, gks[r], r, x, 4, one)
        assert np.array_equal(host(out[:, k].contiguous()), host(one))
