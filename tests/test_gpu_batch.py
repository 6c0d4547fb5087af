"""Batched evaluation (bcn_batch): evaluations of different ring degrees and
segment sizes captured as one CUDA graph over several lanes.  Every item's
output must equal bcn_eval of the same inputs (itself bit-exact to the
oracle), on the first launch and on a replay."""
import numpy as np
import pytest
import torch

import workloads
from paper_2402_01296_gb300 import bcn

pytestmark = pytest.mark.gpu


def small_uneven():
    # (base config, segment h, w): three ring degrees, uneven segment sizes
    specs = [("cnn3_small", 9, 11), ("cnn3_small", 14, 13), ("cryptonets", 12, 10), ("cryptonets", 17, 16),
             ("cifar_cnn", 4, 5), ("cifar_cnn", 5, 4), ("cnn3_small", 6, 7)]
    return [workloads.segment_network(workloads.get_config(b), h, w) for b, h, w in specs]


@pytest.fixture(scope="module")
def setup():
    cfgs = small_uneven()
    ctxs, evks = {}, {}
    items, refs = [], []
    for i, cfg in enumerate(cfgs):
        key = cfg["log_n"]
        if key not in ctxs:
            ctxs[key] = bcn.Context.from_config(cfg)
            _, evk = ctxs[key].keygen(workloads.SEED_KEYS)
            evks[key] = ctxs[key].evk_prepare(bcn.to_device(evk))
        ctx = ctxs[key]
        wq = [bcn.quantize(w) for w in workloads.cipher_weights(cfg)]
        model = bcn.Model(ctx, cfg["cipher"], [a for a, _ in wq], [s for _, s in wq])
        cts = bcn.to_device(workloads.random_residues(ctx.q, (model.n_in, 2), ctx.N, 50 + i))
        pts = [bcn.to_device(workloads.random_residues(ctx.q[:s[1]], (s[0],), ctx.N, 80 + i * 3 + k))
               for k, s in enumerate(model.pt_shapes())]
        out = torch.full(model.out_shape(), -1, dtype=torch.int32, device="cuda")
        ref = torch.empty_like(out)
        model.eval(evks[key], cts, pts, ref, model.alloc_workspace())
        items.append((model, evks[key], cts, pts, out))
        refs.append(ref)
    torch.cuda.synchronize()
    return items, refs


@pytest.mark.parametrize("lanes", [1, 3, 8])
def test_batch_matches_single_evaluations(setup, lanes):
    items, refs = setup
    b = bcn.Batch(items, lanes)
    assert sorted(set(b.lane_of_item)) == list(range(min(lanes, len(items))))
    for rep in range(2):  # the captured graph replays
        for it in items:
            it[4].fill_(-1)
        b.launch()
        torch.cuda.synchronize()
        for it, ref in zip(items, refs):
            assert torch.equal(it[4], ref)
    b.close()


def test_lane_assignment_balances_cost(setup):
    items, _ = setup
    costs = [bcn.model_cost(it[0]) for it in items]
    b = bcn.Batch(items, 2)
    loads = [sum(c for c, l in zip(costs, b.lane_of_item) if l == k) for k in range(2)]
    # longest-processing-time: no lane exceeds the other by more than the largest item
    assert abs(loads[0] - loads[1]) <= max(costs)
    b.close()
