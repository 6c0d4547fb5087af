"""Stacked evaluation (bcn_model_create_stacked / bcn_eval_stacked): several
requests of one model, each from its own client with its own evaluation key,
in one launch sequence.  Every request's output must equal its separate
evaluation bit for bit: the small MNIST-shaped network (N = 4096) and the
CryptoNets-scale one (N = 8192, tensor-core dense layer, square layers split
in halves), with the evaluator's stream overlap on and off, and a chunk that
cuts through a request."""
import numpy as np
import pytest
import torch

import workloads
from paper_2402_01296_gb300 import bcn

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,stack,chunk", [("cnn3_small", 3, 0), ("cryptonets", 2, 0), ("cnn3_small", 4, 50)])
def test_stacked_equals_separate(name, stack, chunk):
    cfg = workloads.get_config(name)
    ctx = bcn.Context.from_config(cfg)
    wq = [bcn.quantize(w) for w in workloads.cipher_weights(cfg)]
    single = bcn.Model(ctx, cfg["cipher"], [a for a, _ in wq], [s for _, s in wq])
    stacked = single.stacked(stack)
    assert stacked.stack == stack and stacked.n_in == stack * single.n_in and stacked.n_out == stack * single.n_out
    if chunk:
        stacked.set_chunk(chunk)  # chunks of 50 ciphertexts cut through the requests' blocks of 80
    keys = [ctx.evk_prepare(bcn.to_device(ctx.keygen(500 + r)[1])) for r in range(stack)]
    cts = [workloads.random_residues(ctx.q, (single.n_in, 2), ctx.N, 600 + r) for r in range(stack)]
    pts = [[workloads.random_residues(ctx.q[:s[1]], (s[0],), ctx.N, 700 + 5 * r + k)
            for k, s in enumerate(single.pt_shapes())] for r in range(stack)]
    refs = []
    ws1 = single.alloc_workspace()
    for r in range(stack):
        o = torch.empty(single.out_shape(), dtype=torch.int32, device="cuda")
        single.eval(keys[r], bcn.to_device(cts[r]), [bcn.to_device(p) for p in pts[r]], o, ws1)
        refs.append(bcn.to_host_u32(o))
    cts_s = bcn.to_device(np.concatenate(cts))
    pts_s = [bcn.to_device(np.concatenate([pts[r][k] for r in range(stack)])) for k in range(len(single.pt_shapes()))]
    ws = stacked.alloc_workspace()
    for overlap in (True, False):
        stacked.set_overlap(overlap)
        out = torch.full(stacked.out_shape(), -1, dtype=torch.int32, device="cuda")
        stacked.eval_stacked(keys, cts_s, pts_s, out, ws)
        got = bcn.to_host_u32(out)
        n1 = single.n_out
        for r in range(stack):
            assert np.array_equal(got[r * n1:(r + 1) * n1], refs[r]), (overlap, r)
    assert ctx.device_status() == 0
    with pytest.raises(bcn.BcnError):
        stacked.eval_stacked(keys[:-1], cts_s, pts_s, out, ws)  # one key per request
