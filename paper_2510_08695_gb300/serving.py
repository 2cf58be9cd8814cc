"""Continuous-batching decode server.

Requests are syndrome batches of any registered graph.  The server owns
``slots`` CUDA streams, each with preallocated device buffers (syndromes in,
corrections / status / logical flips / iterations out) sized for
``max_shots`` shots; nothing is allocated per request.  Whenever a slot is
free, every pending request that fits is copied host->device into it and the
whole group is decoded by one multi-batch persistent launch
(``bpdc_decode_multi``), then copied back; requests that arrive while other
slots are busy are admitted as soon as a slot frees up, so their work overlaps
on the device with the work already running.  A request's result depends only
on its syndromes and global shot offsets, so it is the same alone and in any
mix.

The plain baseline (``PlainDecoder``) decodes one request at a time with the
per-batch kernel on one stream.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Request:
    graph_id: int
    syndromes: "object"          # pinned host int32 tensor [B, ceil(M/32)]
    shot_offset: int = 0
    arrival: float = 0.0         # host clock (s) when the request arrived
    rid: int = 0
    done: float | None = None    # host clock when its results were on the host
    result: dict | None = None


@dataclass
class _Slot:
    stream: "object"
    bufs: dict                   # graph_id -> device buffers sized for max_shots
    host_out: dict               # graph_id -> pinned host output buffers
    event: "object" = None
    busy: list = field(default_factory=list)   # [(request, graph_id, row0, n)]


class Server:
    """Continuous-batching server over a fixed set of graphs."""

    def __init__(self, graphs, slots: int = 4, max_shots: int = 4096):
        import torch
        from . import _bpdc
        self.torch = torch
        self._bpdc = _bpdc
        self.graphs = list(graphs)
        self.max_shots = max_shots
        self.pending = collections.deque()
        self.slots = []
        for _ in range(slots):
            st = torch.cuda.Stream(device=self.graphs[0].device)
            bufs, host = {}, {}
            for gid, g in enumerate(self.graphs):
                bufs[gid] = dict(syn=torch.empty((max_shots, g.MW), dtype=torch.int32, device="cuda"),
                                 out=g.alloc_outputs(max_shots))
                host[gid] = {k: torch.empty(v.shape, dtype=v.dtype, pin_memory=True)
                             for k, v in bufs[gid]["out"].items()}
            self.slots.append(_Slot(st, bufs, host))
        self.completed = []
        self.launches = 0
        self.requests_per_launch = []
        self.max_busy = 0

    def submit(self, req: Request):
        if req.syndromes.shape[0] > self.max_shots:
            raise ValueError("request larger than the slot capacity")
        self.pending.append(req)

    def _launch(self, slot: _Slot):
        torch = self.torch
        used = {gid: 0 for gid in range(len(self.graphs))}
        group = []
        while self.pending:
            req = self.pending[0]
            n = req.syndromes.shape[0]
            if used[req.graph_id] + n > self.max_shots:
                break
            self.pending.popleft()
            group.append((req, req.graph_id, used[req.graph_id], n))
            used[req.graph_id] += n
        if not group:
            return False
        with torch.cuda.stream(slot.stream):
            items = []
            for req, gid, r0, n in group:
                b = slot.bufs[gid]
                b["syn"][r0:r0 + n].copy_(req.syndromes, non_blocking=True)
                out = {k: v[r0:r0 + n] for k, v in b["out"].items()}
                items.append(dict(graph=self.graphs[gid], syndromes=b["syn"][r0:r0 + n],
                                  shot_offset=req.shot_offset, out=out))
            self._bpdc.decode_multi(items, slot.stream)
            for req, gid, r0, n in group:
                for k, v in slot.bufs[gid]["out"].items():
                    slot.host_out[gid][k][r0:r0 + n].copy_(v[r0:r0 + n], non_blocking=True)
            slot.event = torch.cuda.Event()
            slot.event.record(slot.stream)
        slot.busy = group
        self.launches += 1
        self.requests_per_launch.append(len(group))
        return True

    def _harvest(self, slot: _Slot, now: float):
        for req, gid, r0, n in slot.busy:
            req.result = {k: v[r0:r0 + n].clone() for k, v in slot.host_out[gid].items()}
            req.done = now
            self.completed.append(req)
        slot.busy = []
        slot.event = None

    def step(self) -> int:
        """Harvests finished slots and admits pending requests into free ones.
        Returns the number of busy slots."""
        now = time.perf_counter()
        busy = 0
        for slot in self.slots:
            if slot.busy and slot.event.query():
                self._harvest(slot, time.perf_counter())
            if not slot.busy and self.pending:
                self._launch(slot)
            busy += bool(slot.busy)
        self.max_busy = max(self.max_busy, busy)
        return busy


class PlainDecoder:
    """Baseline: one request at a time, plain per-batch kernel, one stream."""

    def __init__(self, graphs, max_shots: int = 4096):
        import torch
        self.torch = torch
        self.graphs = list(graphs)
        self.stream = torch.cuda.Stream(device=self.graphs[0].device)
        self.bufs = {gid: dict(syn=torch.empty((max_shots, g.MW), dtype=torch.int32, device="cuda"),
                               out=g.alloc_outputs(max_shots)) for gid, g in enumerate(self.graphs)}
        self.host = {gid: {k: torch.empty(v.shape, dtype=v.dtype, pin_memory=True)
                           for k, v in self.bufs[gid]["out"].items()} for gid in range(len(self.graphs))}
        self.pending = collections.deque()
        self.current = None
        self.event = None
        self.completed = []

    def submit(self, req: Request):
        self.pending.append(req)

    def step(self) -> int:
        torch = self.torch
        if self.current is not None and self.event.query():
            req = self.current
            gid, n = req.graph_id, req.syndromes.shape[0]
            req.result = {k: v[:n].clone() for k, v in self.host[gid].items()}
            req.done = time.perf_counter()
            self.completed.append(req)
            self.current = None
        if self.current is None and self.pending:
            req = self.pending.popleft()
            gid, n = req.graph_id, req.syndromes.shape[0]
            b = self.bufs[gid]
            with torch.cuda.stream(self.stream):
                b["syn"][:n].copy_(req.syndromes, non_blocking=True)
                out = {k: v[:n] for k, v in b["out"].items()}
                self.graphs[gid].decode(b["syn"][:n], req.shot_offset, out=out, persistent=False,
                                        stream=self.stream)
                for k, v in out.items():
                    self.host[gid][k][:n].copy_(v, non_blocking=True)
                self.event = torch.cuda.Event()
                self.event.record(self.stream)
            self.current = req
        return int(self.current is not None)


def poisson_trace(n_requests: int, rate_per_s: float, n_graphs: int, seed: int = 7,
                  min_shots: int = 1, max_shots: int = 1024):
    """Seeded arrival trace: (arrival time s, graph id, shots) with Poisson arrivals
    and request sizes uniform in [min_shots, max_shots]."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_per_s, size=n_requests))
    g = rng.integers(0, n_graphs, size=n_requests)
    n = rng.integers(min_shots, max_shots + 1, size=n_requests)
    return [(float(t[i]), int(g[i]), int(n[i])) for i in range(n_requests)]


def replay(engine, trace, syndromes_by_graph, shot_cursor=None):
    """Feeds a trace to an engine (Server or PlainDecoder) in real time.

    syndromes_by_graph[gid] is a pinned host tensor of shots; request i takes the
    next rows of its graph.  Returns the completed requests (with latency =
    done - arrival in seconds)."""
    cursor = dict(shot_cursor or {})
    reqs = []
    for i, (t, gid, n) in enumerate(trace):
        c = cursor.get(gid, 0)
        pool = syndromes_by_graph[gid]
        if c + n > pool.shape[0]:
            c = 0
        reqs.append(Request(gid, pool[c:c + n], c, t, i))
        cursor[gid] = c + n
    t0 = time.perf_counter()
    k = 0
    while k < len(reqs) or len(engine.completed) < len(reqs):
        now = time.perf_counter() - t0
        while k < len(reqs) and reqs[k].arrival <= now:
            reqs[k].arrival = t0 + reqs[k].arrival
            engine.submit(reqs[k])
            k += 1
        engine.step()
    return reqs
