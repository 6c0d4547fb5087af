"""The CIFAR-shaped network at full size through bcn_eval, bit-exact against
the oracle on every output limb.

Full size: 768 input ciphertexts (a 16x16x3 segment), conv 3x3 with 16 maps
(4096 ciphertexts squared at 11 limbs), conv 3x3 stride 2 with 32 maps (2048
squared at 10 limbs: the tensor-core MAC's 144-tap x 32-output groups), dense
2048 -> 10 at 9 limbs; N = 16384, 11 + 2 primes, alpha 2.  The homomorphic work
does not depend on the slot batch, so the batch is kept small (the oracle's
encoder and plaintext branch then finish quickly); everything the ciphertext
branch computes is at the benchmark's size.  Decrypted logits also against the
fp64 network (1e-3, same argmax).  The oracle's evaluation takes minutes on the
host cores.
"""
import numpy as np
import pytest
import torch

import workloads
from oracle import oracle as O
from paper_2402_01296_gb300 import bcn

pytestmark = pytest.mark.gpu


def test_full_size_cifar_bit_exact():
    cfg = workloads.with_batch(workloads.get_config("cifar_cnn"), 256)
    assert workloads.n_input_cts(cfg) == 768
    prob = O.Problem(cfg)
    ctx = bcn.Context.from_config(cfg)
    model = bcn.Model(ctx, cfg["cipher"], prob.w_int, prob.s_w)
    assert [model.n_outs[i] for i in range(3)] == [4096, 2048, 10]
    assert model.levels == prob.levels == [11, 10, 9]
    evk_eval = ctx.evk_prepare(bcn.to_device(prob.evk))
    out = torch.empty(model.out_shape(), dtype=torch.int32, device="cuda")
    ws = model.alloc_workspace()
    model.eval(evk_eval, bcn.to_device(prob.cts), [bcn.to_device(p) for p in prob.pts], out, ws)
    torch.cuda.synchronize()
    got = bcn.to_host_u32(out)
    assert ctx.device_status() == 0
    del ws
    torch.cuda.empty_cache()
    ref = prob.evaluate()
    assert got.shape == ref.shape == (10, 2, 9, 16384)
    assert np.array_equal(got, ref), f"{np.mean(got != ref):.3%} of residues differ"
    dec = prob.decode_output(got)
    fp = prob.fp64_logits()
    assert np.abs(dec - fp).max() < 1e-3
    top2 = np.sort(fp, axis=0)[-2:]
    clear = (top2[1] - top2[0]) > 2e-3
    assert np.all(np.argmax(dec, 0)[clear] == np.argmax(fp, 0)[clear])
