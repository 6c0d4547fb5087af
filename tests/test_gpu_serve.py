"""Continuous-batching server on the GPU: requests of two models from several
clients, arriving while others run, admitted by their own working sets under a
device-memory budget.  Every result must equal the stand-alone evaluation of
the same request (bit-exact), in the mix, under a budget that holds only a few
working sets, with malformed and cancelled requests among them, and on the
per-request path."""
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


def _keys(models):
    return sum(e.numel() * 4 for _, evks in models.values() for e in evks)


def test_tight_budget_admits_by_working_set_and_results_equal_standalone(world):
    models, images, reqs, refs = world
    specs = {n: serve.model_spec(m, len(e)) for n, (m, e) in models.items()}
    big, small = specs["cryptonets"].working_set(), specs["cnn3_small"].working_set()
    arena = big + 2 * small  # one CryptoNets-scale request and two small ones at a time
    srv = serve.Server(models, lanes=8, budget_bytes=_keys(models) + arena)
    done = srv.run(_fresh(reqs), keep_outputs=True)
    for r in done:
        assert r.status == "ok" and r.done >= r.arrival
        assert np.array_equal(r.out, refs[r.rid])
    assert srv.scheduler.peak_used <= arena
    srv.scheduler.close()
    assert srv.scheduler.arena.used == 0
    stats = serve.latency_stats(done, images)
    assert stats["requests"] == 12 and stats["p99_ms"] >= stats["p50_ms"] > 0
    with pytest.raises(MemoryError):
        serve.Server(models, lanes=1, budget_bytes=_keys(models) + small // 2)


def test_mixed_in_flight_equals_alone(world):
    """Many requests in flight on several streams: the same residues as alone."""
    models, images, reqs, refs = world
    srv = serve.Server(models, lanes=6, budget_bytes=_keys(models) + (4 << 30))
    burst = _fresh(reqs)
    for r in burst:
        r.arrival = 0.0  # all at once
    done = srv.run(burst, keep_outputs=True)
    for r in done:
        assert r.status == "ok" and np.array_equal(r.out, refs[r.rid])


def test_failures_in_the_mix_leave_the_others_exact(world):
    """A malformed request (a limb short), one for a client without a key, one
    cancelled before it starts and one whose producer stalls: each ends with
    its status, and every other request still equals its stand-alone result."""
    models, images, reqs, refs = world
    srv = serve.Server(models, lanes=4, budget_bytes=_keys(models) + (4 << 30), payload_timeout=0.05)
    mix = _fresh(reqs)
    short = mix[0]
    short.cts = np.ascontiguousarray(short.cts[:, :, :-1])
    mix[1].client = 7
    mix[2].cancel()
    mix[3].ready = lambda: False
    done = srv.run(mix, keep_outputs=True)
    want = {0: "rejected", 1: "rejected", 2: "cancelled", 3: "timeout"}
    for r in done:
        assert r.status == want.get(r.rid, "ok"), (r.rid, r.status, r.detail)
        if r.status == "ok":
            assert np.array_equal(r.out, refs[r.rid])
    srv.scheduler.close()
    assert srv.scheduler.arena.used == 0


def test_plain_path_equals_standalone(world):
    models, images, reqs, refs = world
    done = serve.run_plain(models, _fresh(reqs), keep_outputs=True)
    for r in done:
        assert np.array_equal(r.out, refs[r.rid])


def test_small_requests_share_launches_and_equal_standalone(world):
    """With stacks of the small model, requests that wait together run as one
    stacked evaluation (each with its client's key); every result still equals
    its stand-alone evaluation."""
    models, images, reqs, refs = world
    srv = serve.Server(models, lanes=4, budget_bytes=_keys(models) + (4 << 30),
                       stacks={"cnn3_small": [2, 4], "cryptonets": [2]})
    burst = _fresh(reqs)
    for r in burst:
        r.arrival = 0.0
    done = srv.run(burst, keep_outputs=True)
    for r in done:
        assert r.status == "ok" and np.array_equal(r.out, refs[r.rid]), r.rid
    assert srv.scheduler.stats["batches"] < len(reqs)  # some launches were shared
