"""Seeded ciphertexts on the GPU: the device draws c1 from the seed exactly as
the client's encryption does -- checked against the oracle's encryption (its
own implementation of the same SplitMix64 streams), at the smallest and the
largest ring, with enough draws that rejected ones occur -- and an evaluation
from c0 and the seed equals the evaluation from the full ciphertexts."""
import numpy as np
import pytest
import torch

import workloads
from oracle import oracle as O
from paper_2402_01296_gb300 import bcn

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("params,n_ct", [((4, 3, 1, 1), 5), ((13, 7, 1, 1), 6), ((14, 11, 2, 2), 9)])
def test_expand_equals_oracle_encryption(params, n_ct):
    c, P = bcn.Context(*params, device=0), O.Params(*params)
    sk, _ = P.keygen(3)
    pts = workloads.random_residues(P.q, (n_ct,), P.N, 21)
    want = P.encrypt(sk, pts, P.L, 77)
    c0 = c.encrypt_seeded(sk, pts, P.L, 77)
    assert np.array_equal(c0, want[:, 0])
    out = torch.zeros((n_ct, 2, P.L, P.N), dtype=torch.int32, device="cuda")
    c.expand_seeded(bcn.to_device(c0), n_ct, P.L, 77, out)
    assert np.array_equal(bcn.to_host_u32(out), want)
    assert c.device_status() == 0
    # a later range of the same call: the stream index continues from ct_base
    part = torch.zeros((2, 2, P.L, P.N), dtype=torch.int32, device="cuda")
    c.expand_seeded(bcn.to_device(np.ascontiguousarray(c0[3:5])), 2, P.L, 77, part, ct_base=3)
    assert np.array_equal(bcn.to_host_u32(part), want[3:5])


def test_eval_from_seeded_equals_full():
    cfg = workloads.with_batch(workloads.get_config("cnn3_small"), 64)
    ctx = bcn.Context.from_config(cfg)
    wq = [bcn.quantize(w) for w in workloads.cipher_weights(cfg)]
    model = bcn.Model(ctx, cfg["cipher"], [a for a, _ in wq], [s for _, s in wq])
    sk, evk = ctx.keygen(5)
    evk_eval = ctx.evk_prepare(bcn.to_device(evk))
    imgs = workloads.images(cfg)
    full = ctx.encrypt_segment(sk, imgs, cfg["segment"], 2.0**25, 9)
    c0 = ctx.encrypt_segment_seeded(sk, imgs, cfg["segment"], 2.0**25, 9)
    assert np.array_equal(full[:, 0], c0)
    pts = [workloads.random_residues(ctx.q[:s[1]], (s[0],), ctx.N, 30 + k) for k, s in enumerate(model.pt_shapes())]
    ws = model.alloc_workspace(host=True)
    a = np.zeros(model.out_shape(), dtype=np.uint32)
    b = np.zeros(model.out_shape(), dtype=np.uint32)
    model.eval_host_async(evk_eval, full, pts, a, ws)
    torch.cuda.synchronize()
    for _ in range(2):  # twice in a row on the same workspace
        b[:] = 0
        model.eval_host_seeded_async(evk_eval, c0, 9, pts, b, ws)
        torch.cuda.synchronize()
        assert np.array_equal(a, b)
    assert ctx.device_status() == 0


def test_eval_from_integer_features_equals_residues():
    """The compact upload (c0, the seed, the features' integer coefficients)
    gives the same outputs as the full upload of the same encodings, twice in a
    row on one workspace; bcn_expand_i64 alone equals the host encoder."""
    cfg = workloads.with_batch(workloads.get_config("cryptonets"), 64)
    ctx = bcn.Context.from_config(cfg)
    wq = [bcn.quantize(w) for w in workloads.cipher_weights(cfg)]
    model = bcn.Model(ctx, cfg["cipher"], [a for a, _ in wq], [s for _, s in wq])
    sk, evk = ctx.keygen(5)
    evk_eval = ctx.evk_prepare(bcn.to_device(evk))
    imgs = workloads.images(cfg)
    scale = 2.0 ** cfg["log_scale"]
    full = ctx.encrypt_segment(sk, imgs, cfg["segment"], scale, 9)
    c0 = np.ascontiguousarray(full[:, 0])
    adds, _ = model.scales(scale)
    rng = np.random.default_rng(3)
    vals = [rng.uniform(-1, 1, (s[0], 64)) for s in model.pt_shapes()]
    pts = [ctx.encode(v, s[1], sc) for v, s, sc in zip(vals, model.pt_shapes(), adds)]
    feats = [ctx.encode_i64(v, sc) for v, sc in zip(vals, adds)]
    dev = torch.from_numpy(feats[0]).cuda()
    got = torch.zeros((feats[0].shape[0], pts[0].shape[1], ctx.N), dtype=torch.int32, device="cuda")
    ctx.expand_i64(dev, feats[0].shape[0], pts[0].shape[1], got)
    assert np.array_equal(bcn.to_host_u32(got), pts[0])
    ws = model.alloc_workspace(host=True)
    a = np.zeros(model.out_shape(), dtype=np.uint32)
    b = np.zeros(model.out_shape(), dtype=np.uint32)
    model.eval_host_async(evk_eval, full, pts, a, ws)
    torch.cuda.synchronize()
    for _ in range(2):
        b[:] = 0
        model.eval_host_compact_async(evk_eval, c0, 9, feats, b, ws)
        torch.cuda.synchronize()
        assert np.array_equal(a, b)
    assert ctx.device_status() == 0
