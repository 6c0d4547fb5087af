"""Continuous-batching server: requests of two models from several clients,
arriving while others run, admitted under a device-memory budget.  Every
result must equal the stand-alone evaluation of the same request (bit-exact),
in the mix and on the per-request path."""
import numpy as np
import pytest
import torch

import workloads
from paper_2402_01296_gb300 import bcn, serve

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def world():
    models, images = {}, {}
    for name in ("cnn3_small", "cryptonets"):
        cfg = workloads.get_config(name)
        ctx = bcn.Context.from_config(cfg)
        wq = [bcn.quantize(w) for w in workloads.cipher_weights(cfg)]
        model = bcn.Model(ctx, cfg["cipher"], [a for a, _ in wq], [s for _, s in wq])
        evks = [ctx.evk_prepare(bcn.to_device(ctx.keygen(100 + c)[1])) for c in range(3)]
        models[name] = (model, evks)
        images[name] = cfg["batch"]
    rng = np.random.default_rng(7)
    reqs = []
    for i in range(12):
        name = ["cnn3_small", "cryptonets"][int(rng.random() < 0.3)]
        model = models[name][0]
        ctx = model.ctx
        cts = workloads.random_residues(ctx.q, (model.n_in, 2), ctx.N, 200 + i)
        pts = [workloads.random_residues(ctx.q[:s[1]], (s[0],), ctx.N, 300 + 5 * i + k)
               for k, s in enumerate(model.pt_shapes())]
        reqs.append(serve.Request(rid=i, client=int(rng.integers(0, 3)), model=name, arrival=0.002 * i,
                                  cts=cts, pts=pts))
    refs = []
    for r in reqs:
        model, evks = models[r.model]
        out = torch.empty(model.out_shape(), dtype=torch.int32, device="cuda")
        model.eval(evks[r.client], bcn.to_device(r.cts), [bcn.to_device(p) for p in r.pts], out,
                   model.alloc_workspace())
        refs.append(bcn.to_host_u32(out))
    return models, images, reqs, refs


def _fresh(reqs):
    return [serve.Request(rid=r.rid, client=r.client, model=r.model, arrival=r.arrival, cts=r.cts, pts=r.pts)
            for r in reqs]


def test_budget_limits_lanes_and_results_equal_standalone(world):
    models, images, reqs, refs = world
    keys = sum(e.numel() * 4 for _, evks in models.values() for e in evks)
    lane = max(m.workspace_bytes() for m, _ in models.values()) + sum(
        serve.request_bytes(m) for m, _ in models.values())
    # asked for 3 lanes, the budget holds 2: requests queue for a free lane
    srv = serve.Server(models, lanes=3, budget_bytes=keys + 2 * lane + lane // 2)
    assert len(srv.lanes) == 2 and srv.budget.used == keys + 2 * lane
    done = srv.run(_fresh(reqs), keep_outputs=True)
    for r in done:
        assert r.done >= r.arrival
        assert np.array_equal(r.out, refs[r.rid])
    stats = serve.latency_stats(done, images)
    assert stats["requests"] == 12 and stats["p99_ms"] >= stats["p50_ms"] > 0
    with pytest.raises(MemoryError):
        serve.Server(models, lanes=1, budget_bytes=keys + lane // 2)


def test_mixed_in_flight_equals_alone(world):
    """Many requests in flight on several lanes: the same residues as alone."""
    models, images, reqs, refs = world
    srv = serve.Server(models, lanes=4, budget_bytes=1 << 40)
    burst = _fresh(reqs)
    for r in burst:
        r.arrival = 0.0  # all at once
    done = srv.run(burst, keep_outputs=True)
    for r in done:
        assert np.array_equal(r.out, refs[r.rid])


def test_plain_path_equals_standalone(world):
    models, images, reqs, refs = world
    done = serve.run_plain(models, _fresh(reqs), keep_outputs=True)
    for r in done:
        assert np.array_equal(r.out, refs[r.rid])
