"""Host logic of the server that needs no GPU: the arena allocator, admission
by each request's working set, and the statuses of injected failures (a
malformed request, one too large for the arena, a cancelled request before and
during its run, a producer that stalls and one that is late but finishes),
over a fake executor that completes a request after a set number of polls."""
import numpy as np
import pytest

from paper_2402_01296_gb300 import serve


def test_memory_budget_admission():
    b = serve.MemoryBudget(100)
    assert b.reserve(60) and not b.reserve(41) and b.reserve(40)
    b.release(60)
    assert b.used == 40 and b.reserve(60) and not b.reserve(1)
    with pytest.raises(AssertionError):
        b.release(101)


def test_poisson_arrivals_rate():
    t = serve.poisson_arrivals(500.0, 20.0, seed=3)
    assert np.all(np.diff(t) > 0) and t[-1] <= 20.0
    assert abs(len(t) / 20.0 - 500.0) < 5 * np.sqrt(500.0 / 20.0)  # within 5 sigma of the rate


def test_arena_first_fit_alignment_and_coalescing():
    a = serve.Arena(4096, align=256)
    x = a.alloc(1)
    y = a.alloc(300)        # rounds up to 512
    z = a.alloc(256)
    assert (x, y, z) == (0, 256, 768) and a.used == 1024
    assert a.alloc(4096) is None
    a.free(y)
    assert a.alloc(256) == 256   # first fit reuses the hole
    a.free(256)
    a.free(x)
    a.free(z)
    assert a.free_list == [(0, 4096)] and a.used == 0  # everything coalesced back
    rng = np.random.default_rng(0)
    live = []
    for _ in range(2000):  # random traffic never overlaps and never leaks
        if live and rng.random() < 0.5:
            a.free(live.pop(rng.integers(len(live))))
        else:
            off = a.alloc(int(rng.integers(1, 900)))
            if off is not None:
                live.append(off)
        spans = sorted((o, a.live[o]) for o in a.live)
        assert all(o1 + s1 <= o2 for (o1, s1), (o2, _) in zip(spans, spans[1:]))
        assert all(o % 256 == 0 for o in a.live)
        assert a.used + sum(s for _, s in a.free_list) == 4096
    for off in live:
        a.free(off)
    assert a.free_list == [(0, 4096)]


class FakeExecutor:
    """Completes a request after `polls[model]` polls; records starts."""

    def __init__(self, polls):
        self.polls, self.started, self.live = polls, [], 0
        self.max_live = 0
        self.slots_used, self.dropped, self.batches = [], [], []

    def start(self, reqs, slot):
        assert len(reqs) == slot.stack and all(r.model == slot.model for r in reqs)
        self.started.extend(r.rid for r in reqs)
        self.batches.append([r.rid for r in reqs])
        self.slots_used.append(slot.sid)
        self.live += 1
        self.max_live = max(self.max_live, self.live)
        return [reqs, self.polls[slot.model], slot]

    def drop(self, slot):
        self.dropped.append(slot.sid)

    def poll(self, h):
        h[1] -= 1
        if h[1] <= 0:
            if h[1] == 0:
                self.live -= 1
            return True
        return False

    def finish(self, h, reqs):
        for r in reqs:
            r.out = np.full(1, r.rid, dtype=np.uint32)


def specs():
    small = serve.ModelSpec(cts_shape=(4, 2, 3, 16), pt_shapes=[(2, 3, 16)], out_shape=(2, 2, 2, 16),
                            workspace=3000, n_clients=4)
    big = serve.ModelSpec(cts_shape=(16, 2, 5, 32), pt_shapes=[(8, 5, 32), (4, 4, 32)], out_shape=(2, 2, 3, 32),
                          workspace=30000, n_clients=4)
    return {"small": small, "big": big}


def make(rid, model, client=0, arrival=0.0, **kw):
    s = specs()[model]
    return serve.Request(rid=rid, client=client, model=model, arrival=arrival,
                         cts=np.zeros(s.cts_shape, np.uint32), pts=[np.zeros(p, np.uint32) for p in s.pt_shapes], **kw)


def test_admission_by_working_set_lets_small_requests_pass():
    sp = specs()
    cap = sp["big"].working_set() + sp["small"].working_set()  # one big and one small fit together
    ex = FakeExecutor({"small": 3, "big": 50})
    sch = serve.Scheduler(sp, cap, slots=8, executor=ex)
    reqs = [make(0, "big"), make(1, "big"), make(2, "small"), make(3, "small"), make(4, "small")]
    done = sch.run(reqs, t0=None, keep_outputs=True, sleep=False)
    assert [r.status for r in done] == ["ok"] * 5
    assert all(int(r.out[0]) == r.rid for r in done)
    # the second big request waits for the first; the small ones overtake it
    assert ex.started.index(1) > ex.started.index(2) and ex.started.index(1) > ex.started.index(4)
    assert sch.peak_used <= cap
    sch.close()
    assert sch.arena.used == 0 and sch.arena.free_list == [(0, cap)]


def test_idle_slots_are_reused_and_reclaimed_for_other_models():
    sp = specs()
    cap = sp["big"].working_set() + sp["small"].working_set()
    ex = FakeExecutor({"small": 2, "big": 2})
    sch = serve.Scheduler(sp, cap, slots=1, executor=ex)
    done = sch.run([make(i, "small", arrival=0.0) for i in range(4)], sleep=False)
    assert all(r.status == "ok" for r in done)
    assert len(set(ex.slots_used)) == 1  # one request at a time: the same slot every time
    # a big request needs the memory the idle small slot holds... it fits beside it here
    done = sch.run([make(10, "big")], sleep=False)
    assert done[0].status == "ok" and ex.dropped == []
    # two big ones in flight need the small slot's memory: it goes back to the arena
    sch2 = serve.Scheduler(sp, 2 * sp["big"].working_set(), slots=2, executor=ex)
    sch2.run([make(20, "small")], sleep=False)
    assert len(sch2.idle) == 1
    done = sch2.run([make(21, "big"), make(22, "big")], sleep=False)
    assert [r.status for r in done] == ["ok", "ok"] and sch2.evictions == 1
    assert sch2.peak_used <= 2 * sp["big"].working_set()


def test_without_slot_cache_memory_returns_at_completion():
    sp = specs()
    sch = serve.Scheduler(sp, 1 << 20, slots=4, executor=FakeExecutor({"small": 2, "big": 2}), cache_slots=False)
    sch.run([make(i, "small") for i in range(5)], sleep=False)
    assert sch.arena.used == 0 and not sch.idle


def test_slots_bound_requests_in_flight():
    sp = specs()
    ex = FakeExecutor({"small": 4, "big": 4})
    sch = serve.Scheduler(sp, 1 << 30, slots=2, executor=ex)
    done = sch.run([make(i, "small") for i in range(9)], t0=None, sleep=False)
    assert all(r.status == "ok" for r in done) and ex.max_live == 2


def test_injected_failures_surface_as_statuses():
    sp = specs()
    ex = FakeExecutor({"small": 3, "big": 5})
    sch = serve.Scheduler(sp, sp["big"].working_set() * 2, slots=4, executor=ex, payload_timeout=0.05)
    bad_level = make(0, "small")
    bad_level.cts = np.zeros((4, 2, 2, 16), np.uint32)            # one limb short
    bad_pts = make(1, "big")
    bad_pts.pts = bad_pts.pts[:1]                                  # a feature plaintext missing
    bad_client = make(2, "small", client=9)                        # no key for this client
    cancelled = make(3, "small")
    cancelled.cancel()
    stalled = make(4, "small", ready=lambda: False)                # the producer never finishes
    flag = {"n": 0}

    def late():  # the producer finishes after a few polls, well within the timeout
        flag["n"] += 1
        return flag["n"] > 5

    late_ok = make(5, "small", ready=late)
    good = make(6, "big")
    unknown = make(7, "small")
    unknown.model = "nope"
    done = sch.run([bad_level, bad_pts, bad_client, cancelled, stalled, late_ok, good, unknown], t0=None,
                   keep_outputs=True, sleep=False)
    st = {r.rid: r.status for r in done}
    assert st == {0: "rejected", 1: "rejected", 2: "rejected", 3: "cancelled", 4: "timeout", 5: "ok", 6: "ok",
                  7: "rejected"}
    assert "limb" in done[0].detail or "expected" in done[0].detail
    assert 3 not in ex.started and 4 not in ex.started  # never reserved, never started
    sch.close()
    assert sch.arena.used == 0


def test_cancel_in_flight_discards_the_result_and_frees_its_memory():
    sp = specs()

    class CancelOnStart(FakeExecutor):
        def start(self, reqs, slot):
            h = super().start(reqs, slot)
            for r in reqs:
                if r.rid == 1:
                    r.cancel()  # the client gives up while its request runs
            return h

    ex = CancelOnStart({"small": 3, "big": 3})
    sch = serve.Scheduler(sp, 1 << 20, slots=4, executor=ex)
    done = sch.run([make(0, "small"), make(1, "small"), make(2, "small")], t0=None, keep_outputs=True, sleep=False)
    assert [r.status for r in done] == ["ok", "cancelled", "ok"]
    sch.close()
    assert done[1].out is None and sch.arena.used == 0


def test_too_large_for_the_arena():
    sp = specs()
    sch = serve.Scheduler(sp, sp["small"].working_set(), slots=4, executor=FakeExecutor({"small": 1, "big": 1}))
    done = sch.run([make(0, "big"), make(1, "small")], t0=None, sleep=False)
    assert [r.status for r in done] == ["too_large", "ok"]


def stacked_specs(sizes=(2, 4)):
    sp = specs()
    small = sp["small"]
    by = {k: serve.ModelSpec(cts_shape=(k * small.cts_shape[0],) + small.cts_shape[1:],
                             pt_shapes=[(k * p[0],) + tuple(p[1:]) for p in small.pt_shapes],
                             out_shape=(k * small.out_shape[0],) + small.out_shape[1:],
                             workspace=small.workspace * k, n_clients=4) for k in sizes}
    return sp, {"small": by}


def test_small_requests_share_launches():
    """Seven small requests waiting together run as stacks of 4 and 2 and a
    single one (the largest stack the waiting requests fill, first); the big
    request among them runs alone; a stack is one batch of the executor."""
    sp, st = stacked_specs()
    ex = FakeExecutor({"small": 3, "big": 3})
    sch = serve.Scheduler(sp, 1 << 24, slots=8, executor=ex, stacks=st)
    reqs = [make(i, "small") for i in range(5)] + [make(5, "big")] + [make(6 + i, "small", client=i % 4)
                                                                      for i in range(2)]
    done = sch.run(reqs, keep_outputs=True, sleep=False)
    assert all(r.status == "ok" and int(r.out[0]) == r.rid for r in done)
    assert ex.batches[0] == [0, 1, 2, 3] and [5] in ex.batches
    # the other three small ones: a stack of 2 (the largest they fill), then one alone; the big one alone
    assert sorted(len(b) for b in ex.batches) == [1, 1, 2, 4]
    assert sch.stats["requests"] == 8 and sch.stats["batches"] == len(ex.batches)


def test_cancel_inside_a_stack_discards_only_that_result():
    sp, st = stacked_specs((2,))

    class CancelOnStart(FakeExecutor):
        def start(self, reqs, slot):
            h = super().start(reqs, slot)
            reqs[1].cancel()
            return h

    ex = CancelOnStart({"small": 2, "big": 2})
    sch = serve.Scheduler(sp, 1 << 24, slots=4, executor=ex, stacks=st)
    done = sch.run([make(0, "small"), make(1, "small")], keep_outputs=True, sleep=False)
    assert [r.status for r in done] == ["ok", "cancelled"] and done[1].out is None and int(done[0].out[0]) == 0


def test_stack_that_does_not_fit_falls_back_to_smaller():
    """An arena that holds a stack of 2 but not of 4: four waiting requests run as
    two stacks of 2."""
    sp, st = stacked_specs((2, 4))
    cap = st["small"][2].working_set()
    ex = FakeExecutor({"small": 2, "big": 2})
    sch = serve.Scheduler(sp, cap, slots=4, executor=ex, stacks=st)
    done = sch.run([make(i, "small") for i in range(4)], sleep=False)
    assert all(r.status == "ok" for r in done) and [len(b) for b in ex.batches] == [2, 2]
    assert sch.peak_used <= cap
