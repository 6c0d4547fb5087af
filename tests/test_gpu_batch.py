"""Batched evaluation (bcn_batch): evaluations of different ring degrees and
segment sizes captured as one CUDA graph over several lanes.  Every item's
output must equal bcn_eval of the same inputs, on the first launch and on a
replay; one item of each ring degree (segments other than the configurations'
own) equals the oracle's evaluation residue for residue; the plain
one-stream path (no overlap inside an evaluation) gives the same residues."""
import numpy as np
import pytest
import torch

import workloads
from oracle import oracle as O
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
    ctxs, evks, host_evks = {}, {}, {}
    items, refs, host = [], [], []
    for i, cfg in enumerate(cfgs):
        key = cfg["log_n"]
        if key not in ctxs:
            ctxs[key] = bcn.Context.from_config(cfg)
            _, evk = ctxs[key].keygen(workloads.SEED_KEYS)
            host_evks[key] = evk
            evks[key] = ctxs[key].evk_prepare(bcn.to_device(evk))
        ctx = ctxs[key]
        wq = [bcn.quantize(w) for w in workloads.cipher_weights(cfg)]
        model = bcn.Model(ctx, cfg["cipher"], [a for a, _ in wq], [s for _, s in wq])
        cts_h = workloads.random_residues(ctx.q, (model.n_in, 2), ctx.N, 50 + i)
        pts_h = [workloads.random_residues(ctx.q[:s[1]], (s[0],), ctx.N, 80 + i * 3 + k)
                 for k, s in enumerate(model.pt_shapes())]
        cts, pts = bcn.to_device(cts_h), [bcn.to_device(p) for p in pts_h]
        out = torch.full(model.out_shape(), -1, dtype=torch.int32, device="cuda")
        ref = torch.empty_like(out)
        model.eval(evks[key], cts, pts, ref, model.alloc_workspace())
        items.append((model, evks[key], cts, pts, out))
        refs.append(ref)
        host.append((cfg, [a for a, _ in wq], host_evks[key], cts_h, pts_h))
    torch.cuda.synchronize()
    return items, refs, host


@pytest.mark.parametrize("lanes", [1, 3, 8])
def test_batch_matches_single_evaluations(setup, lanes):
    items, refs, _ = setup
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
    items, _, _ = setup
    costs = [bcn.model_cost(it[0]) for it in items]
    b = bcn.Batch(items, 2)
    loads = [sum(c for c, l in zip(costs, b.lane_of_item) if l == k) for k in range(2)]
    # longest-processing-time: no lane exceeds the other by more than the largest item
    assert abs(loads[0] - loads[1]) <= max(costs)
    b.close()


def test_batch_items_match_oracle(setup):
    """One uneven item per ring degree (N = 4096, 8192, 16384 with their own
    segment shapes), run through a 3-lane batch graph, against the oracle."""
    items, refs, host = setup
    b = bcn.Batch(items, 3)
    for it in items:
        it[4].fill_(-1)
    b.launch()
    torch.cuda.synchronize()
    seen = set()
    for it, (cfg, w_int, evk, cts_h, pts_h) in zip(items, host):
        if cfg["log_n"] in seen:
            continue
        seen.add(cfg["log_n"])
        P = O.Params.from_config(cfg)
        tables = [O.layer_table(l, w) for l, w in zip(cfg["cipher"], w_int)]
        want = O.evaluate(P, cfg, tables, evk, cts_h, pts_h)
        assert np.array_equal(bcn.to_host_u32(it[4]), want), cfg["name"] if "name" in cfg else cfg["log_n"]
    assert seen == {12, 13, 14}
    b.close()


def test_plain_one_stream_path_matches(setup):
    items, refs, _ = setup
    for (m, evk, cts, pts, out), ref in zip(items, refs):
        m.set_overlap(False)
        out.fill_(-1)
        m.eval(evk, cts, pts, out, m.alloc_workspace())
        m.set_overlap(True)
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
