"""Continuous-batching parse server.

Requests (an input already resident on the device, a parser) arrive over
time.  The server admits every waiting request whose outputs fit the
remaining output-memory budget, parses all admitted requests of one round in
a single batched launch (parparaw_parse_batch: one persistent launch over all
their tiles, each request keeping its own look-back chains), and issues
rounds on several streams so that requests arriving while earlier rounds run
are admitted and overlap with them on the device.

A request does not need to know its row count: its outputs are sized from
its length (one record per 16 bytes, string columns as long as the input),
and a request whose parse reports PP_E_CAPACITY is admitted again with the
exact sizes the device reported.  The results of a round come back to the
host in one copy.  Memory of a request is released, and its latency taken,
when its round's completion event fires; the event's device timestamp gives
the completion time on the GPU as well, so that the host's share of the
latency (dispatch, polling) can be told apart.
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
    rows_cap: int | None = None     # None: sized from the input's length
    values_caps: list | None = None
    arrival: float = 0.0      # host time (perf_counter seconds)
    done: float = 0.0         # host time the completion was seen
    done_dev_ms: float = 0.0  # device time of the completion, ms after the trace's reference event
    retries: int = 0          # admissions again after PP_E_CAPACITY
    status: int = 0
    rows: int = 0
    keep: bool = False        # keep the outputs after completion (for checks)
    out: Output | None = None

    def sizes(self) -> tuple[int, list]:
        n = self.data.numel()
        rows = self.rows_cap if self.rows_cap is not None else max(64, n // 16)
        caps = self.values_caps if self.values_caps is not None else [max(n, 1)] * len(self.parser.types)
        return rows, caps

    def out_bytes(self) -> int:
        rows, caps = self.sizes()
        n = 2 * ((rows + 7) // 8) + 1024
        for t, cap in zip(self.parser.types, caps):
            if t == _abi.SKIP:  # a column that is not selected holds nothing
                continue
            n += (cap + 8 * (rows + 1)) if t == _abi.STRING else 8 * rows
            n += (rows + 7) // 8
        return n


class Server:
    def __init__(self, arena_bytes: int, streams: int = 4, max_batch: int = 1024, device="cuda",
                 keep_outputs: bool = False, host_buffers: int = 32):
        self.keep_outputs = keep_outputs
        self.arena_bytes = int(arena_bytes)
        self.in_use = 0
        self.device = torch.device(device)
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(streams)]
        self.next_stream = 0
        self.max_batch = max_batch
        self.waiting: collections.deque[Request] = collections.deque()
        self.inflight: list = []
        self.completed: list[Request] = []
        self.rounds = 0
        self.retries = 0
        # pinned blocks the rounds' results come back into (one per round in flight)
        self.free_host = [torch.empty(max_batch * _abi.RESULT_BYTES, dtype=torch.uint8, pin_memory=True)
                          for _ in range(host_buffers)]
        self.ref_event = None

    def start_clock(self) -> None:
        """Records the reference event that device completion times count from."""
        self.ref_event = torch.cuda.Event(enable_timing=True)
        self.ref_event.record(self.streams[0])

    def submit(self, req: Request) -> None:
        self.waiting.append(req)

    def _admit(self, res_block: torch.Tensor) -> list[Request]:
        """Takes waiting requests while their outputs fit.  Called with the
        round's stream current, so the outputs are allocated on that stream,
        ordered before its parse; results go to slices of res_block."""
        batch = []
        while self.waiting and len(batch) < self.max_batch:
            need = self.waiting[0].out_bytes()
            if self.in_use + need > self.arena_bytes and (batch or self.inflight):
                break  # wait for memory; a request larger than the arena runs alone
            req = self.waiting.popleft()
            rows, caps = req.sizes()
            k = len(batch)
            req.out = req.parser.allocate(rows, caps, device=self.device,
                                          result_buf=res_block[k * _abi.RESULT_BYTES:(k + 1) * _abi.RESULT_BYTES])
            self.in_use += need
            batch.append(req)
        return batch

    def poll(self) -> None:
        """Retires finished rounds: reads their results, admits again the
        requests that reported PP_E_CAPACITY (with the exact sizes), releases
        the others' memory and stamps their latency."""
        still = []
        now = time.perf_counter()
        for ev, reqs, nbytes, host in self.inflight:
            if not ev.query():
                still.append((ev, reqs, nbytes, host))
                continue
            dev_ms = self.ref_event.elapsed_time(ev) if self.ref_event is not None else 0.0
            raw = host[: len(reqs) * _abi.RESULT_BYTES].numpy()
            again = []
            for k, r in enumerate(reqs):
                res = _abi.pp_parse_result.from_buffer_copy(raw[k * _abi.RESULT_BYTES:(k + 1) * _abi.RESULT_BYTES])
                if res.status == _abi.E_CAPACITY:
                    r.rows_cap = max(int(res.rows), 1)
                    r.values_caps = [max(int(b), 1) for b in res.values_bytes_needed[: len(r.parser.types)]]
                    r.retries += 1
                    r.out = None
                    again.append(r)
                    continue
                r.status, r.rows = res.status, int(res.rows)
                r.done, r.done_dev_ms = now, dev_ms
                if not (self.keep_outputs or r.keep):
                    r.out = None  # back to the caching allocator
                self.completed.append(r)
            self.retries += len(again)
            self.waiting.extendleft(reversed(again))  # first in line, in their order
            self.in_use -= nbytes
            self.free_host.append(host)
        self.inflight = still

    def step(self) -> int:
        """Admits and launches one round; returns the number of requests launched."""
        self.poll()
        if not self.waiting or not self.free_host:
            return 0
        stream = self.streams[self.next_stream]
        with torch.cuda.stream(stream):
            res_block = torch.empty(self.max_batch * _abi.RESULT_BYTES, dtype=torch.uint8, device=self.device)
            batch = self._admit(res_block)
            if not batch:
                return 0
            self.next_stream = (self.next_stream + 1) % len(self.streams)
            parse_batch([(r.parser, r.data, r.out) for r in batch], stream=stream)
            host = self.free_host.pop()
            host[: len(batch) * _abi.RESULT_BYTES].copy_(res_block[: len(batch) * _abi.RESULT_BYTES], non_blocking=True)
            ev = torch.cuda.Event(enable_timing=True)
            ev.record(stream)
        self.inflight.append((ev, batch, sum(r.out_bytes() for r in batch), host))
        self.rounds += 1
        return len(batch)

    def drain(self) -> None:
        while self.waiting or self.inflight:
            if not self.step():
                time.sleep(0)


def _stats(requests, wall: float, t0: float) -> dict:
    lat = np.array([(r.done - r.arrival) * 1e3 for r in requests])
    dev = np.array([r.done_dev_ms - (r.arrival - t0) * 1e3 for r in requests])
    nbytes = sum(r.data.numel() for r in requests)
    return {"requests": len(requests), "wall_s": round(wall, 3), "bytes": int(nbytes),
            "gbs": round(nbytes / wall / 1e9, 4), "p50_ms": round(float(np.percentile(lat, 50)), 4),
            "p99_ms": round(float(np.percentile(lat, 99)), 4),
            "p50_device_ms": round(float(np.percentile(dev, 50)), 4),
            "p99_device_ms": round(float(np.percentile(dev, 99)), 4),
            "failed": int(sum(1 for r in requests if r.status != _abi.OK))}


def run_trace(server: Server, requests: list[Request], offsets_s: np.ndarray) -> dict:
    """Feeds requests at their arrival offsets (seconds from start) in real
    time and runs the server until all complete.  Latency = arrival to the
    host seeing the completion; the device latency counts to the completion
    event's device timestamp instead."""
    torch.cuda.synchronize()
    server.start_clock()
    torch.cuda.synchronize()
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
            time.sleep(0)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    out = _stats(requests, wall, t0)
    out.update(rounds=server.rounds, capacity_retries=server.retries)
    return out


def run_trace_plain(requests: list[Request], offsets_s: np.ndarray, device="cuda") -> dict:
    """The same trace with one parparaw_parse per request on one stream, in
    arrival order (the plain per-request parse), outputs sized the same way
    (exact sizes from the first parse when it reports PP_E_CAPACITY)."""
    device = torch.device(device)
    stream = torch.cuda.Stream(device=device)
    pending = collections.deque()
    torch.cuda.synchronize()
    ref = torch.cuda.Event(enable_timing=True)
    ref.record(stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    i = 0
    n = len(requests)
    done = 0
    retries = 0
    while done < n:
        now = time.perf_counter() - t0
        while i < n and offsets_s[i] <= now:
            r = requests[i]
            r.arrival = t0 + offsets_s[i]
            rows, caps = r.sizes()
            with torch.cuda.stream(stream):  # the outputs' zero fill is ordered before the parse
                r.out = r.parser.allocate(rows, caps, device=device)
                r.parser.parse_into(r.data, r.out, stream=stream)
                ev = torch.cuda.Event(enable_timing=True)
                ev.record(stream)
            pending.append((ev, r))
            i += 1
        progressed = False
        while pending and pending[0][0].query():
            ev, r = pending.popleft()
            res = r.out.result()  # read on the current stream: this request's parse has completed
            if res.status == _abi.E_CAPACITY:  # once more with the exact sizes, synchronously
                retries += 1
                with torch.cuda.stream(stream):
                    r.out = r.parser.allocate(max(res.rows, 1), [max(int(b), 1) for b in res.values_bytes_needed],
                                              device=device)
                    r.parser.parse_into(r.data, r.out, stream=stream)
                    ev = torch.cuda.Event(enable_timing=True)
                    ev.record(stream)
                ev.synchronize()
                res = r.out.result()
            r.status, r.rows = res.status, int(res.rows)
            r.done = time.perf_counter()
            r.done_dev_ms = ref.elapsed_time(ev)
            r.out = None
            done += 1
            progressed = True
        if not progressed:
            time.sleep(0)
    wall = time.perf_counter() - t0
    out = _stats(requests, wall, t0)
    out.update(capacity_retries=retries)
    return out
