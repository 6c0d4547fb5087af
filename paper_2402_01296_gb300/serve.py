"""Continuous-batching server for encrypted inference requests.

A request is one slot batch of one client: the encrypted sensitive segment and
the encoded plaintext-branch features of one model (Sec. 2 threat model: the
client sends ciphertexts, the server evaluates without the secret key).  Every
client's evaluation key stays resident on the device.  The device-memory
budget is spent on the keys first, then on lanes: a lane owns a workspace and
device buffers for one request of every model, and as many lanes are built as
the budget holds (at most the number asked for).  Requests wait in arrival
order; a lane that finishes takes the next arrived request at once, so
requests that arrive while others are on the GPU start as soon as a lane is
free and their work overlaps on the device.  Each lane replays a captured
graph of the evaluation for the request's model and client key (bcn_batch with
one item), fed through the lane's buffers.

The per-request baseline ("plain") serves the same arrivals one at a time on one
stream with bcn_eval.
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np
import torch

from . import bcn


@dataclasses.dataclass
class Request:
    rid: int
    client: int
    model: str                 # model name (a key of Server.models)
    arrival: float             # seconds, relative to the start of the run
    cts: np.ndarray            # host (page-locked torch uint32 view), [n_in][2][L][N]
    pts: list                  # host arrays, one per add layer
    done: float = -1.0         # completion time (seconds since start)
    out: np.ndarray | None = None


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


def request_bytes(model: bcn.Model) -> int:
    N, L = model.ctx.N, model.ctx.L
    b = model.n_in * 2 * L * N * 4 + int(np.prod(model.out_shape())) * 4
    for s in model.pt_shapes():
        b += int(np.prod(s)) * 4
    return b


class _Lane:
    def __init__(self, server: "Server", idx: int):
        self.idx = idx
        self.stream = torch.cuda.Stream(device=server.device)
        self.event = torch.cuda.Event()
        self.req: Request | None = None
        dev = f"cuda:{server.device}"
        # one set of input/output buffers and one captured evaluation per model
        # and client key; all graphs of a lane share the lane's workspace (a lane
        # runs one request at a time)
        self.buf, self.graph, self.out_host = {}, {}, {}
        self.ws_bytes = max(m.workspace_bytes() for m, _ in server.models.values())
        self.ws = torch.empty(max(1, (self.ws_bytes + 3) // 4), dtype=torch.int32, device=dev)
        for name, (model, evks) in server.models.items():
            cts = torch.empty((model.n_in, 2, model.ctx.L, model.ctx.N), dtype=torch.int32, device=dev)
            pts = [torch.empty(s, dtype=torch.int32, device=dev) for s in model.pt_shapes()]
            out = torch.empty(model.out_shape(), dtype=torch.int32, device=dev)
            self.buf[name] = (cts, pts, out)
            self.out_host[name] = torch.empty(model.out_shape(), dtype=torch.int32).pin_memory()
            self.graph[name] = [bcn.Batch([(model, evk, cts, pts, out)], 1, workspace=self.ws) for evk in evks]


class Server:
    """models: {name: (bcn.Model, [evk_eval per client])}."""

    def __init__(self, models: dict, lanes: int, budget_bytes: int, device: int = 0):
        self.models = models
        self.device = device
        self.budget = MemoryBudget(budget_bytes)
        keys = sum(e.numel() * e.element_size() for _, evks in models.values() for e in evks)
        if not self.budget.reserve(keys):
            raise MemoryError("evaluation keys alone exceed the device-memory budget")
        self.lanes = []
        for i in range(lanes):
            lane_bytes = max(m.workspace_bytes() for m, _ in models.values()) + sum(
                request_bytes(m) for m, _ in models.values())
            if not self.budget.reserve(lane_bytes):
                break  # no room for another lane
            self.lanes.append(_Lane(self, i))
        if not self.lanes:
            raise MemoryError("no lane fits the device-memory budget")

    def _start(self, lane: _Lane, req: Request, now: float):
        cts, pts, out = lane.buf[req.model]
        with torch.cuda.stream(lane.stream):
            cts.copy_(torch.from_numpy(req.cts.view(np.int32)), non_blocking=True)
            for d, h in zip(pts, req.pts):
                d.copy_(torch.from_numpy(h.view(np.int32)), non_blocking=True)
            lane.graph[req.model][req.client].launch(lane.stream)
            lane.out_host[req.model].copy_(out, non_blocking=True)
            lane.event.record(lane.stream)
        lane.req = req

    def run(self, requests: list, t0: float | None = None, keep_outputs: bool = False, sleep: bool = True):
        """Serve `requests` (sorted by arrival); returns them with completion times."""
        pending = list(requests)
        pending.sort(key=lambda r: r.arrival)
        queue: list = []  # arrived, waiting for a lane and memory (FIFO)
        t0 = time.perf_counter() if t0 is None else t0
        nxt, finished = 0, 0
        while finished < len(pending):
            now = time.perf_counter() - t0
            while nxt < len(pending) and pending[nxt].arrival <= now:
                queue.append(pending[nxt])
                nxt += 1
            progressed = False
            for lane in self.lanes:
                if lane.req is not None and lane.event.query():
                    r = lane.req
                    r.done = time.perf_counter() - t0
                    if keep_outputs:
                        r.out = lane.out_host[r.model].numpy().view(np.uint32).copy()
                    lane.req = None
                    finished += 1
                    progressed = True
                if lane.req is None and queue:
                    self._start(lane, queue.pop(0), now)
                    progressed = True
            if not progressed and sleep and not queue and nxt < len(pending):
                # idle until the next arrival -- unless a lane is busy, whose
                # completion must be seen (and its lane reused) when it happens
                if not any(lane.req is not None for lane in self.lanes):
                    wait = pending[nxt].arrival - (time.perf_counter() - t0)
                    if wait > 2e-4:
                        time.sleep(wait - 1e-4)
        return pending


def run_plain(models: dict, requests: list, device: int = 0, keep_outputs: bool = False):
    """The per-request path: one request at a time on one stream with bcn_eval,
    in arrival order (a request starts at max(arrival, previous completion))."""
    dev = f"cuda:{device}"
    bufs, ws = {}, None
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
        if keep_outputs:
            r.out = oh.numpy().view(np.uint32).copy()
    return pending


def latency_stats(requests: list, images: dict) -> dict:
    lat = np.array([r.done - r.arrival for r in requests]) * 1e3
    span = max(r.done for r in requests) - min(r.arrival for r in requests)
    imgs = sum(images[r.model] for r in requests)
    return {"requests": len(requests), "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
            "throughput_inferences_per_s": imgs / span, "throughput_requests_per_s": len(requests) / span}


def poisson_arrivals(rate: float, duration: float, seed: int) -> np.ndarray:
    g = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += g.exponential(1.0 / rate)
        if t > duration:
            return np.array(out)
        out.append(t)
