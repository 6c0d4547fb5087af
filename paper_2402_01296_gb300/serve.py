"""Continuous-batching server for encrypted inference requests.

A request is one slot batch of one client: the encrypted sensitive segment and
the encoded plaintext-branch features of one model (Sec. 2 threat model: the
client sends ciphertexts, the server evaluates without the secret key).  Every
client's evaluation key stays resident on the device; the rest of the
device-memory budget is an arena from which each request's own working set --
its input ciphertexts, its feature plaintexts, its output ciphertexts and its
model's evaluation workspace -- is reserved when it is admitted and returned
when it completes.  A request is admitted as soon as a stream is free and its
working set fits in what the requests in flight leave of the arena, so small
requests pass large ones that do not fit yet (first fit over the arrival-order
queue, with a bounded number of requests allowed to overtake a waiting one);
requests that arrive while others are on the GPU start at once on their own
streams, and their copies and kernels overlap on the device.  A completed
request's working set stays reserved as an idle slot of its model (its device
buffers keep their addresses, so the executor can replay the evaluation it
captured for them); idle slots are handed to the next requests of that model
and are returned to the arena, least recently used first, as soon as a
request of another model needs the memory (with cache_slots=False a working
set goes back to the arena at completion).

Every request ends with a status: "ok"; "rejected" (malformed: an unknown
model or client, or ciphertexts / plaintexts whose level, limb count or shape
does not match the model); "too_large" (its working set exceeds the whole
arena); "cancelled" (Request.cancel() before it started; once started its work
completes but the result is discarded); "timeout" (its producer did not
finish the payload -- Request.ready() stayed false -- within `payload_timeout`
seconds of its arrival).  Nothing of a request that does not end "ok" is kept.

Requests of one model that wait together share their launches: the first
ready request in the queue is started together with the next ready requests of
its model, up to the largest stack size configured for that model, as one
stacked evaluation (bcn_model_create_stacked: every kernel launch serves all of
them, each ciphertext's key switch with its own client's key) in a slot sized
for the stack.

The scheduling (admission, arena, slots, batches, statuses) is host logic over
an executor that starts a batch's copies and evaluation and reports
completion; the GPU executor copies the payloads into the slot's device
buffers and replays a CUDA graph of bcn_eval captured once per (slot, client
key) for a single request, or runs bcn_eval_stacked with the batch's keys, one
stream per batch in flight.  The per-request baseline ("plain") serves the same
arrivals one at a time on one stream.
"""
from __future__ import annotations

import dataclasses
import time
from typing import Callable

import numpy as np


@dataclasses.dataclass
class Request:
    rid: int
    client: int
    model: str                 # model name (a key of Server.models)
    arrival: float             # seconds, relative to the start of the run
    cts: np.ndarray            # host uint32 (page-locked for full-rate copies), [n_in][2][L][N]
    pts: list                  # host uint32 arrays, one per add layer
    ready: Callable[[], bool] | None = None  # producer done with the payload (None: ready on arrival)
    done: float = -1.0         # completion time (seconds since start)
    status: str = "pending"
    detail: str = ""
    out: np.ndarray | None = None
    cancelled: bool = False

    def cancel(self):
        self.cancelled = True


class MemoryBudget:
    """Device-memory budget: reservations succeed while they fit."""

    def __init__(self, budget_bytes: int):
        self.budget = int(budget_bytes)
        self.used = 0

    def reserve(self, nbytes: int) -> bool:
        if self.used + nbytes > self.budget:
            return False
        self.used += int(nbytes)
        return True

    def release(self, nbytes: int) -> None:
        self.used -= int(nbytes)
        assert self.used >= 0


class Arena:
    """First-fit allocator over [0, capacity) bytes with coalescing of freed
    neighbours; every block starts on an `align`-byte boundary."""

    def __init__(self, capacity: int, align: int = 256):
        self.capacity, self.align = int(capacity), int(align)
        self.free_list = [(0, self.capacity)] if capacity > 0 else []  # sorted (offset, size)
        self.live = {}  # offset -> size

    def alloc(self, nbytes: int):
        n = max(self.align, (int(nbytes) + self.align - 1) // self.align * self.align)
        for i, (off, size) in enumerate(self.free_list):
            if size >= n:
                if size == n:
                    self.free_list.pop(i)
                else:
                    self.free_list[i] = (off + n, size - n)
                self.live[off] = n
                return off
        return None

    def free(self, off: int) -> None:
        n = self.live.pop(off)
        fl = self.free_list
        i = 0
        while i < len(fl) and fl[i][0] < off:
            i += 1
        fl.insert(i, (off, n))
        # coalesce with the right, then the left neighbour
        if i + 1 < len(fl) and fl[i][0] + fl[i][1] == fl[i + 1][0]:
            fl[i] = (fl[i][0], fl[i][1] + fl[i + 1][1])
            fl.pop(i + 1)
        if i > 0 and fl[i - 1][0] + fl[i - 1][1] == fl[i][0]:
            fl[i - 1] = (fl[i - 1][0], fl[i - 1][1] + fl[i][1])
            fl.pop(i)

    @property
    def used(self) -> int:
        return sum(self.live.values())


@dataclasses.dataclass
class ModelSpec:
    """What the scheduler needs of a model: input / plaintext / output shapes
    (uint32 words), workspace bytes, and the clients it has keys for."""
    cts_shape: tuple
    pt_shapes: list
    out_shape: tuple
    workspace: int
    n_clients: int

    def parts(self, align: int = 256):
        """Byte sizes of the working set's parts: cts, each pt, out, workspace."""
        a = lambda b: (int(b) + align - 1) // align * align  # noqa: E731
        return ([a(np.prod(self.cts_shape) * 4)] + [a(np.prod(s) * 4) for s in self.pt_shapes]
                + [a(np.prod(self.out_shape) * 4), a(self.workspace)])

    def working_set(self, align: int = 256) -> int:
        return sum(self.parts(align))


def request_bytes(model) -> int:
    """Input, plaintext and output bytes of one request of a bcn.Model."""
    N, L = model.ctx.N, model.ctx.L
    b = model.n_in * 2 * L * N * 4 + int(np.prod(model.out_shape())) * 4
    for s in model.pt_shapes():
        b += int(np.prod(s)) * 4
    return b


def validate(req: Request, spec: ModelSpec) -> str:
    """'' if the request matches its model, else why not."""
    if not (0 <= req.client < spec.n_clients):
        return f"no key for client {req.client}"
    c = np.asarray(req.cts)
    if c.dtype != np.uint32 or tuple(c.shape) != tuple(spec.cts_shape):
        return f"ciphertexts {tuple(c.shape)} {c.dtype}, expected {tuple(spec.cts_shape)} uint32"
    if len(req.pts) != len(spec.pt_shapes):
        return f"{len(req.pts)} feature plaintexts, expected {len(spec.pt_shapes)}"
    for p, s in zip(req.pts, spec.pt_shapes):
        p = np.asarray(p)
        if p.dtype != np.uint32 or tuple(p.shape) != tuple(s):
            return f"feature plaintexts {tuple(p.shape)} {p.dtype}, expected {tuple(s)} uint32"
    return ""


@dataclasses.dataclass
class Slot:
    """One batch's working set in the arena: offsets of its parts."""
    sid: int
    model: str
    stack: int
    offs: list


class Scheduler:
    """Admission and completion over an executor (host logic only).

    executor: start(reqs, slot) -> handle (copies + evaluation of the batch
    queued), poll(handle) -> bool, finish(handle, reqs) (fetch the results into
    each req.out), drop(slot) (the slot's memory goes back to the arena).
    specs: {model name: ModelSpec} (one request); stacks: {model name: {size:
    ModelSpec of that many requests side by side}} (size 1 may be left out);
    capacity: arena bytes (the budget left after the keys); slots: batches in
    flight at most; overtake: how many later requests may start ahead of a
    waiting one before admission stops at it; cache_slots: keep a completed
    batch's working set as an idle slot of its model and stack size."""

    def __init__(self, specs: dict, capacity: int, slots: int, executor, payload_timeout: float = 1.0,
                 overtake: int = 64, cache_slots: bool = True, stacks: dict | None = None):
        self.specs, self.executor = specs, executor
        self.stacks = {m: {1: sp} for m, sp in specs.items()}
        for m, by_size in (stacks or {}).items():
            self.stacks[m].update(by_size)
        self.arena = Arena(capacity)
        self.slots, self.payload_timeout, self.overtake = int(slots), float(payload_timeout), int(overtake)
        self.cache_slots = cache_slots
        self.stats = {"loops": 0, "start_s": 0.0, "poll_s": 0.0, "max_in_flight": 0, "batches": 0, "requests": 0}
        self.idle = []  # idle slots, least recently used first
        self.n_slots = 0
        self.peak_used = 0
        self.evictions = 0

    def _carve(self, spec):
        offs = []
        for nbytes in spec.parts(self.arena.align):
            off = self.arena.alloc(nbytes)
            if off is None:
                for o in offs:
                    self.arena.free(o)
                return None
            offs.append(off)
        return offs

    def _drop(self, slot: Slot):
        for o in slot.offs:
            self.arena.free(o)
        self.executor.drop(slot)

    def _acquire(self, model: str, stack: int = 1):
        """An idle slot of (model, stack), else a new one carved from the arena,
        after returning other idle slots (least recently used first) while it
        does not fit."""
        for i, sl in enumerate(self.idle):
            if sl.model == model and sl.stack == stack:
                return self.idle.pop(i)
        spec = self.stacks[model][stack]
        offs = self._carve(spec)
        while offs is None:
            victim = next((i for i, sl in enumerate(self.idle) if (sl.model, sl.stack) != (model, stack)), None)
            if victim is None:
                return None
            self._drop(self.idle.pop(victim))
            self.evictions += 1
            offs = self._carve(spec)
        self.n_slots += 1
        self.peak_used = max(self.peak_used, self.arena.used)
        return Slot(self.n_slots - 1, model, stack, offs)

    def _release(self, slot: Slot):
        if self.cache_slots:
            self.idle.append(slot)
        else:
            self._drop(slot)

    def close(self):
        """Return every idle slot to the arena."""
        while self.idle:
            self._drop(self.idle.pop())

    def run(self, requests: list, t0: float | None = None, keep_outputs: bool = False, sleep: bool = True):
        """Serve `requests`; returns them (arrival order) with status and completion times."""
        pending = sorted(requests, key=lambda r: r.arrival)
        queue, in_flight = [], []
        t0 = time.perf_counter() if t0 is None else t0
        nxt, finished = 0, 0
        st = self.stats = {"loops": 0, "start_s": 0.0, "poll_s": 0.0, "max_in_flight": 0, "batches": 0,
                           "requests": 0}
        clock = time.perf_counter

        def end(r, status, detail="", now=None):
            nonlocal finished
            r.status, r.detail = status, detail
            r.done = (time.perf_counter() - t0) if now is None else now
            finished += 1

        def ready(r):
            return r.ready is None or r.ready()

        while finished < len(pending):
            now = time.perf_counter() - t0
            while nxt < len(pending) and pending[nxt].arrival <= now:
                r = pending[nxt]
                nxt += 1
                spec = self.specs.get(r.model)
                why = "unknown model" if spec is None else validate(r, spec)
                if why:
                    end(r, "rejected", why)
                elif spec.working_set(self.arena.align) > self.arena.capacity:
                    end(r, "too_large", f"working set {spec.working_set()} > arena {self.arena.capacity}")
                else:
                    queue.append(r)
            progressed = False
            st["loops"] += 1
            tp = clock()
            for item in list(in_flight):  # completions
                batch, slot, h = item
                if self.executor.poll(h):
                    live = [r for r in batch if not r.cancelled]
                    if keep_outputs and live:
                        self.executor.finish(h, batch)
                    for r in batch:
                        if r.cancelled:
                            r.out = None
                            end(r, "cancelled", "cancelled while in flight; result discarded")
                        else:
                            end(r, "ok")
                    self._release(slot)
                    in_flight.remove(item)
                    progressed = True
            st["poll_s"] += clock() - tp
            # admission: first fit over the queue, in arrival order; a request
            # starts together with the next ready requests of its model
            skipped = 0
            for r in list(queue):
                if r not in queue:  # started in an earlier batch of this pass
                    continue
                if r.cancelled:
                    queue.remove(r)
                    end(r, "cancelled", "cancelled before it started")
                    continue
                if not ready(r):
                    if now - r.arrival > self.payload_timeout:
                        queue.remove(r)
                        end(r, "timeout", f"payload not ready {now - r.arrival:.3f} s after arrival")
                    continue
                if len(in_flight) >= self.slots:
                    break
                sizes = sorted(self.stacks[r.model], reverse=True)
                mates = [r]
                for x in queue:
                    if len(mates) >= sizes[0]:
                        break
                    if x is not r and x.model == r.model and not x.cancelled and ready(x):
                        mates.append(x)
                slot = None
                for size in sizes:  # the largest stack the waiting requests fill, else smaller ones
                    if size <= len(mates):
                        slot = self._acquire(r.model, size)
                        if slot is not None:
                            mates = mates[:size]
                            break
                if slot is not None:
                    for x in mates:
                        queue.remove(x)
                    ts = clock()
                    in_flight.append((mates, slot, self.executor.start(mates, slot)))
                    st["start_s"] += clock() - ts
                    st["batches"] += 1
                    st["requests"] += len(mates)
                    st["max_in_flight"] = max(st["max_in_flight"], len(in_flight))
                    progressed = True
                else:
                    skipped += 1
                    if skipped > self.overtake:
                        break
            if not progressed and sleep and not queue and not in_flight and nxt < len(pending):
                wait = pending[nxt].arrival - (time.perf_counter() - t0)
                if wait > 2e-4:
                    time.sleep(wait - 1e-4)
        return pending


class GpuExecutor:
    """Runs a batch on the device on a stream of its own: copies the payloads
    into the slot's device buffers (request i in the i-th block of each), then
    for a single request replays the evaluation captured for that slot and the
    request's client key (bcn_batch of one item, captured on first use), for a
    stack runs bcn_eval_stacked with the requests' keys; copies the outputs back
    to a page-locked host buffer."""

    def __init__(self, models: dict, arena_bytes: int, streams: int, device: int = 0, stacked: dict | None = None):
        import torch

        from . import bcn

        self.torch, self.bcn = torch, bcn
        self.models = models
        self.stacked = stacked or {}  # {name: {size: bcn.Model}}
        self.dev = f"cuda:{device}"
        self.buf = torch.empty(max(1, arena_bytes // 4), dtype=torch.int32, device=self.dev)
        self.streams = [torch.cuda.Stream(device=device) for _ in range(max(1, streams))]
        self.free_streams = list(range(len(self.streams)))
        self.views, self.graphs, self.out_host = {}, {}, {}

    def _model(self, slot):
        return self.models[slot.model][0] if slot.stack == 1 else self.stacked[slot.model][slot.stack]

    def _view(self, off, shape):
        n = int(np.prod(shape))
        return self.buf[off // 4: off // 4 + n].view(*shape)

    def _slot_views(self, slot):
        v = self.views.get(slot.sid)
        if v is None:
            model = self._model(slot)
            N, L = model.ctx.N, model.ctx.L
            offs = slot.offs
            cts = self._view(offs[0], (model.n_in, 2, L, N))
            pts = [self._view(o, tuple(sh)) for o, sh in zip(offs[1:-2], model.pt_shapes())]
            out = self._view(offs[-2], tuple(model.out_shape()))
            ws = self.buf[offs[-1] // 4: offs[-1] // 4 + (model.workspace_bytes() + 3) // 4]
            v = (cts, pts, out, ws)
            self.views[slot.sid] = v
            self.out_host[slot.sid] = self.torch.empty(model.out_shape(), dtype=self.torch.int32).pin_memory()
        return v

    def graph(self, slot, client: int):
        key = (slot.sid, client)
        g = self.graphs.get(key)
        if g is None:
            model, evks = self.models[slot.model]
            cts, pts, out, ws = self._slot_views(slot)
            g = self.bcn.Batch([(model, evks[client], cts, pts, out)], 1, workspace=ws)
            self.graphs[key] = g
        return g

    def start(self, reqs: list, slot: Slot):
        torch = self.torch
        cts, pts, out, ws = self._slot_views(slot)
        _, evks = self.models[slot.model]
        si = self.free_streams.pop()
        st = self.streams[si]
        oh = self.out_host[slot.sid]
        with torch.cuda.stream(st):
            n_in = cts.shape[0] // slot.stack
            for i, r in enumerate(reqs):
                cts[i * n_in:(i + 1) * n_in].copy_(torch.from_numpy(np.asarray(r.cts).view(np.int32)),
                                                   non_blocking=True)
                for d, h in zip(pts, r.pts):
                    n_pt = d.shape[0] // slot.stack
                    d[i * n_pt:(i + 1) * n_pt].copy_(torch.from_numpy(np.asarray(h).view(np.int32)),
                                                     non_blocking=True)
            if slot.stack == 1:
                self.graph(slot, reqs[0].client).launch(st)
            else:
                self._model(slot).eval_stacked([evks[r.client] for r in reqs], cts, pts, out, ws, stream=st)
            oh.copy_(out, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(st)
        return [si, ev, oh, False]

    def poll(self, h) -> bool:
        if h[3]:
            return True
        if h[1].query():
            h[3] = True
            self.free_streams.append(h[0])
            return True
        return False

    def finish(self, h, reqs: list):
        full = h[2].numpy().view(np.uint32)
        n_out = full.shape[0] // len(reqs)
        for i, r in enumerate(reqs):
            r.out = full[i * n_out:(i + 1) * n_out].copy()

    def drop(self, slot):
        for key in [k for k in self.graphs if k[0] == slot.sid]:
            self.graphs.pop(key).close()
        self.views.pop(slot.sid, None)
        self.out_host.pop(slot.sid, None)


def model_spec(model, n_clients: int) -> ModelSpec:
    N, L = model.ctx.N, model.ctx.L
    return ModelSpec(cts_shape=(model.n_in, 2, L, N), pt_shapes=[tuple(s) for s in model.pt_shapes()],
                     out_shape=tuple(model.out_shape()), workspace=model.workspace_bytes(), n_clients=n_clients)


class Server:
    """models: {name: (bcn.Model, [evk_eval per client])}.  The keys are
    reserved from the budget first; the rest (at most the device's free memory
    less 1 GiB) is the requests' arena.  `lanes`: batches in flight at most
    (one stream each).  stacks: {name: [sizes > 1]}: requests of that model
    that wait together run as one stacked evaluation of up to the largest size."""

    def __init__(self, models: dict, lanes: int, budget_bytes: int, device: int = 0, payload_timeout: float = 1.0,
                 stacks: dict | None = None):
        self.models = models
        self.device = device
        self.budget = MemoryBudget(budget_bytes)
        keys = sum(e.numel() * e.element_size() for _, evks in models.values() for e in evks)
        if not self.budget.reserve(keys):
            raise MemoryError("evaluation keys alone exceed the device-memory budget")
        import torch

        # the arena: what the budget leaves after the keys, at most what the
        # device has free (less 1 GiB for the library's own tables and streams)
        torch.cuda.empty_cache()  # what torch's allocator holds but does not use counts as free
        free = torch.cuda.mem_get_info(device)[0]
        arena = min(self.budget.budget - self.budget.used, max(0, free - (1 << 30)))
        self.specs = {name: model_spec(m, len(evks)) for name, (m, evks) in models.items()}
        if min(s.working_set() for s in self.specs.values()) > arena:
            raise MemoryError("no request fits the device-memory budget left after the keys")
        self.budget.reserve(arena)
        stacked = {name: {int(k): models[name][0].stacked(int(k)) for k in sizes if int(k) > 1}
                   for name, sizes in (stacks or {}).items()}
        stack_specs = {name: {k: model_spec(m, len(models[name][1])) for k, m in by.items()}
                       for name, by in stacked.items()}
        self.executor = GpuExecutor(models, arena, lanes, device, stacked=stacked)
        self.scheduler = Scheduler(self.specs, arena, lanes, self.executor, payload_timeout=payload_timeout,
                                   stacks=stack_specs)
        self.lanes = list(range(lanes))

    def warm(self, slots_per_model: int):
        """Carve up to `slots_per_model` idle slots per model (as the budget
        allows) and capture their evaluations for every client key, so that the
        first requests replay instead of capturing."""
        sch = self.scheduler
        for name, (model, evks) in self.models.items():
            got = []
            for _ in range(slots_per_model):
                sl = sch._acquire(name)
                if sl is None:
                    break
                got.append(sl)
                for c in range(len(evks)):
                    self.executor.graph(sl, c)
            for size in sch.stacks[name]:  # and a few slots of every stack size
                for _ in range(min(4, slots_per_model)):
                    if size == 1:
                        break
                    sl = sch._acquire(name, size)
                    if sl is None:
                        break
                    self.executor._slot_views(sl)
                    got.append(sl)
            sch.idle.extend(got)

    def run(self, requests: list, t0: float | None = None, keep_outputs: bool = False, sleep: bool = True):
        return self.scheduler.run(requests, t0=t0, keep_outputs=keep_outputs, sleep=sleep)


def run_plain(models: dict, requests: list, device: int = 0, keep_outputs: bool = False):
    """The per-request path: one request at a time on one stream with bcn_eval,
    in arrival order (a request starts at max(arrival, previous completion))."""
    import torch

    dev = f"cuda:{device}"
    bufs = {}
    big = max((m for m, _ in models.values()), key=lambda m: m.workspace_bytes())
    ws = big.alloc_workspace()
    for name, (model, _) in models.items():
        cts = torch.empty((model.n_in, 2, model.ctx.L, model.ctx.N), dtype=torch.int32, device=dev)
        pts = [torch.empty(s, dtype=torch.int32, device=dev) for s in model.pt_shapes()]
        out = torch.empty(model.out_shape(), dtype=torch.int32, device=dev)
        bufs[name] = (cts, pts, out, torch.empty(model.out_shape(), dtype=torch.int32).pin_memory())
    pending = sorted(requests, key=lambda r: r.arrival)
    t0 = time.perf_counter()
    for r in pending:
        now = time.perf_counter() - t0
        if r.arrival > now:
            time.sleep(r.arrival - now)
        model, evks = models[r.model]
        cts, pts, out, oh = bufs[r.model]
        cts.copy_(torch.from_numpy(r.cts.view(np.int32)), non_blocking=True)
        for d, h in zip(pts, r.pts):
            d.copy_(torch.from_numpy(h.view(np.int32)), non_blocking=True)
        model.eval(evks[r.client], cts, pts, out, ws)
        oh.copy_(out)
        r.done = time.perf_counter() - t0
        r.status = "ok"
        if keep_outputs:
            r.out = oh.numpy().view(np.uint32).copy()
    return pending


def latency_stats(requests: list, images: dict) -> dict:
    ok = [r for r in requests if r.status == "ok"]
    lat = np.array([r.done - r.arrival for r in ok]) * 1e3
    span = max(r.done for r in ok) - min(r.arrival for r in ok)
    imgs = sum(images[r.model] for r in ok)
    return {"requests": len(ok), "not_ok": len(requests) - len(ok), "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
            "throughput_inferences_per_s": imgs / span, "throughput_requests_per_s": len(ok) / span}


def poisson_arrivals(rate: float, duration: float, seed: int) -> np.ndarray:
    g = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += g.exponential(1.0 / rate)
        if t > duration:
            return np.array(out)
        out.append(t)
