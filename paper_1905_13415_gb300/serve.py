"""Continuous-batching parse server.

Requests (an input already resident on the device, a parser) arrive over
time.  The server admits every waiting request whose outputs fit the
remaining output-memory budget, parses all admitted requests of one round in
a single batched launch (parparaw_parse_batch: one persistent launch over all
their tiles, each request keeping its own look-back chains), and issues
rounds on several streams so that requests arriving while earlier rounds run
are admitted and overlap with them on the device.  Memory of a request is
released, and its latency (completion seen by the host minus arrival) taken,
when its round's completion event fires.  Parser tables stay resident (they
travel as kernel parameters / a device table per launch).
"""
from __future__ import annotations

import collections
import dataclasses
import time

import numpy as np
import torch

from . import _abi
from .parser import Output, Parser, parse_batch


@dataclasses.dataclass
class Request:
    rid: int
    parser: Parser
    data: torch.Tensor        # uint8 on the device
    rows_cap: int
    values_caps: list
    arrival: float = 0.0      # host time (perf_counter seconds)
    done: float = 0.0
    out: Output | None = None

    def out_bytes(self) -> int:
        rows = self.rows_cap
        n = 2 * ((rows + 7) // 8) + 1024
        for t, cap in zip(self.parser.types, self.values_caps):
            if t == _abi.SKIP:  # a column that is not selected holds nothing
                continue
            n += (cap + 8 * (rows + 1)) if t == _abi.STRING else 8 * rows
            n += (rows + 7) // 8
        return n


class Server:
    def __init__(self, arena_bytes: int, streams: int = 4, max_batch: int = 1024, device="cuda",
                 keep_outputs: bool = False):
        self.keep_outputs = keep_outputs
        self.arena_bytes = int(arena_bytes)
        self.in_use = 0
        self.streams = [torch.cuda.Stream(device=device) for _ in range(streams)]
        self.next_stream = 0
        self.max_batch = max_batch
        self.device = device
        self.waiting: collections.deque[Request] = collections.deque()
        self.inflight: list[tuple[torch.cuda.Event, list[Request], int]] = []
        self.completed: list[Request] = []
        self.rounds = 0

    def submit(self, req: Request) -> None:
        self.waiting.append(req)

    def _admit(self) -> list[Request]:
        """Takes waiting requests while their outputs fit.  Called with the
        round's stream current, so the outputs (and the zero fill of their
        result buffers) are allocated on that stream, ordered before its
        parse."""
        batch = []
        while self.waiting and len(batch) < self.max_batch:
            need = self.waiting[0].out_bytes()
            if self.in_use + need > self.arena_bytes and (batch or self.inflight):
                break  # wait for memory; a request larger than the arena runs alone
            req = self.waiting.popleft()
            req.out = req.parser.allocate(req.rows_cap, req.values_caps, device=self.device)
            self.in_use += need
            batch.append(req)
        return batch

    def poll(self) -> None:
        """Retires finished rounds (releases their memory, stamps latency)."""
        still = []
        now = time.perf_counter()
        for ev, reqs, nbytes in self.inflight:
            if ev.query():
                for r in reqs:
                    r.done = now
                    if not self.keep_outputs:
                        r.out = None  # back to the caching allocator
                    self.completed.append(r)
                self.in_use -= nbytes
            else:
                still.append((ev, reqs, nbytes))
        self.inflight = still

    def step(self) -> int:
        """Admits and launches one round; returns the number of requests launched."""
        self.poll()
        stream = self.streams[self.next_stream]
        with torch.cuda.stream(stream):
            batch = self._admit()
        if not batch:
            return 0
        self.next_stream = (self.next_stream + 1) % len(self.streams)
        with torch.cuda.stream(stream):
            parse_batch([(r.parser, r.data, r.out) for r in batch], stream=stream)
            ev = torch.cuda.Event()
            ev.record(stream)
        self.inflight.append((ev, batch, sum(r.out_bytes() for r in batch)))
        self.rounds += 1
        return len(batch)

    def drain(self) -> None:
        while self.waiting or self.inflight:
            if not self.step():
                time.sleep(20e-6)


def run_trace(server: Server, requests: list[Request], offsets_s: np.ndarray) -> dict:
    """Feeds requests at their arrival offsets (seconds from start) in real
    time and runs the server until all complete.  Returns latency stats."""
    t0 = time.perf_counter()
    i = 0
    n = len(requests)
    while i < n or server.waiting or server.inflight:
        now = time.perf_counter() - t0
        while i < n and offsets_s[i] <= now:
            requests[i].arrival = t0 + offsets_s[i]
            server.submit(requests[i])
            i += 1
        if not server.step():
            time.sleep(20e-6)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    lat = np.array([(r.done - r.arrival) * 1e3 for r in requests])
    nbytes = sum(r.data.numel() for r in requests)
    return {"requests": n, "wall_s": round(wall, 3), "bytes": int(nbytes),
            "gbs": round(nbytes / wall / 1e9, 4), "p50_ms": round(float(np.percentile(lat, 50)), 4),
            "p99_ms": round(float(np.percentile(lat, 99)), 4), "rounds": server.rounds}


def run_trace_plain(requests: list[Request], offsets_s: np.ndarray, device="cuda") -> dict:
    """The same trace with one parparaw_parse per request on one stream, in
    arrival order (the plain per-request parse)."""
    stream = torch.cuda.Stream(device=device)
    pending = collections.deque()
    t0 = time.perf_counter()
    i = 0
    n = len(requests)
    done = 0
    while done < n:
        now = time.perf_counter() - t0
        while i < n and offsets_s[i] <= now:
            r = requests[i]
            r.arrival = t0 + offsets_s[i]
            with torch.cuda.stream(stream):  # the outputs' zero fill is ordered before the parse
                r.out = r.parser.allocate(r.rows_cap, r.values_caps, device=device)
                r.parser.parse_into(r.data, r.out, stream=stream)
                ev = torch.cuda.Event()
                ev.record(stream)
            pending.append((ev, r))
            i += 1
        progressed = False
        while pending and pending[0][0].query():
            _, r = pending.popleft()
            r.done = time.perf_counter()
            r.out = None
            done += 1
            progressed = True
        if not progressed:
            time.sleep(20e-6)
    wall = time.perf_counter() - t0
    lat = np.array([(r.done - r.arrival) * 1e3 for r in requests])
    nbytes = sum(r.data.numel() for r in requests)
    return {"requests": n, "wall_s": round(wall, 3), "bytes": int(nbytes),
            "gbs": round(nbytes / wall / 1e9, 4), "p50_ms": round(float(np.percentile(lat, 50)), 4),
            "p99_ms": round(float(np.percentile(lat, 99)), 4)}
