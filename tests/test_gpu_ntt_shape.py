"""The alternative block shape of the NTT-based kernels (bcn_ctx_set_ntt_shape)
computes the same residues as the default one: an evaluation at each of
N = 4096, 8192 and 16384 (two square layers, digits of one and of two primes)
is bit-identical under both shapes, and so are a rotation and a forward and
inverse transform; the selection is reported and validated."""
import numpy as np
import pytest
import torch

import workloads
from paper_2402_01296_gb300 import bcn

pytestmark = pytest.mark.gpu

CASES = [("cnn3_small", None), ("cryptonets", None), ("cifar", workloads.reduced_cifar(cout1=4, cout2=8, seg=8))]


@pytest.mark.parametrize("name,cfg", CASES)
def test_shapes_agree(name, cfg):
    cfg = cfg or workloads.with_batch(workloads.get_config(name), 64)
    ctx = bcn.Context.from_config(cfg)
    wq = [bcn.quantize(w) for w in workloads.cipher_weights(cfg)]
    model = bcn.Model(ctx, cfg["cipher"], [a for a, _ in wq], [s for _, s in wq])
    sk, evk = ctx.keygen(7)
    cts = bcn.to_device(workloads.random_residues(ctx.q, (model.n_in, 2), ctx.N, 3))
    pts = [bcn.to_device(workloads.random_residues(ctx.q[:s[1]], (s[0],), ctx.N, 4 + k))
           for k, s in enumerate(model.pt_shapes())]
    ws = model.alloc_workspace()
    gk = ctx.galois_keygen(sk, 3, 5)
    outs = []
    for shape in (0, 1):
        ctx.set_ntt_shape(shape)
        assert ctx.ntt_shape()[0] == shape
        ev = ctx.evk_prepare(bcn.to_device(evk))  # the prepared key does not depend on the shape
        out = torch.zeros(model.out_shape(), dtype=torch.int32, device="cuda")
        model.eval(ev, cts, pts, out, ws)
        rot = torch.zeros((3, 2, ctx.L, ctx.N), dtype=torch.int32, device="cuda")
        ctx.op_rotate(ctx.L, ctx.evk_prepare(bcn.to_device(gk)), 3, cts[:3].contiguous(), 3, rot)
        t = cts[:2].clone()
        ctx.op_ntt(t, 4, ctx.L, inverse=False)
        fwd = bcn.to_host_u32(t)
        ctx.op_ntt(t, 4, ctx.L, inverse=True)
        assert np.array_equal(bcn.to_host_u32(t), bcn.to_host_u32(cts[:2]))
        outs.append((bcn.to_host_u32(out), bcn.to_host_u32(rot), bcn.to_host_u32(ev), fwd))
    ctx.set_ntt_shape(0)
    for a, b in zip(*outs):
        assert np.array_equal(a, b)
    assert ctx.ntt_shape()[1] == {4096: 16, 8192: 16, 16384: 32}[ctx.N]
    assert ctx.device_status() == 0
    with pytest.raises(bcn.BcnError):
        ctx.set_ntt_shape(2)
