"""End-to-end streaming parse of host-resident input (Sec. 4.4).

The input is split into partitions.  Two device input buffers alternate:
while partition k is parsed from one, partition k+1 is copied into the other
and the columns of partition k-1 are copied back to the host, on three
streams.  Each buffer keeps a carry-over region in front of its partition:
the incomplete last record of partition k (the bytes after its last record
delimiter, reported by the device as `consumed`) is copied there so that it
is parsed at the start of partition k+1.  Partitions are parsed with
PP_OPT_PARTIAL_INPUT; the last one as a whole input.  The output is one
Arrow-like record batch per partition, in host memory.

The carry-over restarts each partition in the DFA's start state, which holds
for formats whose record delimiters lead back to the start state (both
formats shipped here).
"""
from __future__ import annotations

import dataclasses

import torch

from . import _abi
from .parser import Output, Parser, ParparawError


@dataclasses.dataclass
class Partition:
    rows: int
    nbytes: int                      # input bytes parsed (carry-over included)
    columns: list                    # per column: dict of host tensors
    row_valid: torch.Tensor


class HostArena:
    """One pinned host buffer that the columns of a stream's partitions are
    carved from, so that a parse allocates no pinned memory per partition.
    Reusable across parses: the partitions of a parse stay valid until the
    arena's next parse (reset)."""

    def __init__(self, nbytes: int):
        self.buf = torch.empty(int(nbytes), dtype=torch.uint8, pin_memory=True)
        self.used = 0

    def reset(self) -> None:
        self.used = 0

    def take(self, n: int, dtype) -> torch.Tensor | None:
        size = torch.empty(0, dtype=dtype).element_size()
        start = (self.used + 63) & ~63
        end = start + max(n, 1) * size
        if end > self.buf.numel():
            return None
        self.used = end
        return self.buf[start:end].view(dtype)


class StreamParser:
    def __init__(self, parser: Parser, partition_bytes: int = 256 << 20, carry_bytes: int | None = None,
                 rows_per_byte: float = 1 / 16, device="cuda"):
        self.parser = parser
        self.part = int(partition_bytes)
        self.carry = int(carry_bytes or partition_bytes)
        self.device = torch.device(device)
        self.rows_per_byte = rows_per_byte
        self.bufs = [torch.empty(self.carry + self.part, dtype=torch.uint8, device=self.device) for _ in range(2)]
        self.s_h2d = torch.cuda.Stream(device=self.device)
        self.s_parse = torch.cuda.Stream(device=self.device)
        self.s_d2h = torch.cuda.Stream(device=self.device)
        self.outs = [None, None]
        self.arena = None

    def _out(self, b: int) -> Output:
        if self.outs[b] is None:
            nbytes = self.carry + self.part
            rows = max(1024, int(nbytes * self.rows_per_byte))
            with torch.cuda.stream(self.s_parse):  # zero fill ordered before the parses on s_parse
                self.outs[b] = self.parser.allocate(rows, [nbytes] * len(self.parser.types), device=self.device)
        return self.outs[b]

    def _host_like(self, t: torch.Tensor, n: int) -> torch.Tensor:
        if self.arena is not None:
            x = self.arena.take(n, t.dtype)
            if x is not None:
                return x
        return torch.empty(max(n, 1), dtype=t.dtype, pin_memory=True)

    def _copy_back(self, out: Output, res, nbytes_in: int, done: torch.cuda.Event) -> Partition:
        _host_like = self._host_like
        rows = res.rows
        nb = (rows + 7) // 8
        cols = []
        with torch.cuda.stream(self.s_d2h):
            for c, t in enumerate(out.types):
                col = {}
                if t == _abi.SKIP:  # not selected: nothing to copy
                    cols.append({"values": None, "offsets": None, "validity": None})
                    continue
                if t == _abi.STRING:
                    nbytes = int(res.values_bytes_needed[c])
                    col["values"] = _host_like(out.values[c], nbytes)
                    col["values"][:nbytes].copy_(out.values[c][:nbytes], non_blocking=True)
                    col["offsets"] = _host_like(out.offsets[c], rows + 1)
                    col["offsets"][:rows + 1].copy_(out.offsets[c][:rows + 1], non_blocking=True)
                else:
                    col["values"] = _host_like(out.values[c], rows)
                    col["values"][:rows].copy_(out.values[c][:rows], non_blocking=True)
                col["validity"] = _host_like(out.validity[c], nb)
                col["validity"][:nb].copy_(out.validity[c][:nb], non_blocking=True)
                cols.append(col)
            rv = _host_like(out.row_valid, nb)
            rv[:nb].copy_(out.row_valid[:nb], non_blocking=True)
            done.record(self.s_d2h)
        return Partition(rows, nbytes_in, cols, rv)

    def parse(self, host: torch.Tensor, arena: HostArena | None = None) -> list[Partition]:
        """Parses the pinned uint8 host tensor; returns the partitions' columns,
        in pinned host memory (carved from `arena` when given: then they stay
        valid until the arena's next use)."""
        self.arena = arena
        if arena is not None:
            arena.reset()
        n = host.numel()
        nparts = max(1, (n + self.part - 1) // self.part)
        ev = lambda: torch.cuda.Event()  # noqa: E731
        h2d_done = [ev(), ev()]
        parse_done = [ev(), ev()]
        d2h_done = [ev(), ev()]
        carry_done = ev()
        for e in (*parse_done, *d2h_done, carry_done):
            e.record(self.s_parse)

        def h2d(k):
            b = k % 2
            lo = k * self.part
            ln = min(self.part, n - lo)
            self.s_h2d.wait_event(carry_done)  # the carry-over out of this buffer is taken
            with torch.cuda.stream(self.s_h2d):
                self.bufs[b][self.carry:self.carry + ln].copy_(host[lo:lo + ln], non_blocking=True)
                h2d_done[b].record(self.s_h2d)
            return ln

        skip = self.parser.skip_records  # Sec. 4.3: they are all in the first partition
        try:
            results: list[Partition] = []
            lens = [0] * nparts
            lens[0] = h2d(0)
            prev = None  # (buffer, start, length, Output) of partition k-1
            for k in range(nparts):
                b = k % 2
                last = k + 1 == nparts
                carry_len = 0
                if prev is not None:
                    pb, pstart, plen, pout = prev
                    parse_done[pb].synchronize()
                    res = self._checked(pout, pb, pstart, plen, partial=True)
                    results.append(self._copy_back(self.outs[pb], res, plen, d2h_done[pb]))
                    if k == 1 and skip and res.rows == 0:
                        raise ParparawError(_abi.E_UNSUPPORTED, "the skipped records reach past the first partition")
                    carry_len = plen - res.consumed
                    if carry_len > self.carry:
                        raise ParparawError(_abi.E_UNSUPPORTED, "a record is longer than the carry-over region")
                    self.s_parse.wait_event(h2d_done[b])
                    if carry_len:
                        with torch.cuda.stream(self.s_parse):
                            self.bufs[b][self.carry - carry_len:self.carry].copy_(
                                self.bufs[pb][pstart + res.consumed:pstart + plen], non_blocking=True)
                    carry_done.record(self.s_parse)
                start = self.carry - carry_len
                length = carry_len + lens[k]
                self.s_parse.wait_event(h2d_done[b])
                self.s_parse.wait_event(d2h_done[b])  # this buffer's previous copy-back
                out = self._out(b)
                self.parser.set_option(_abi.OPT_PARTIAL_INPUT, 0 if last else 1)
                self.parser.set_option(_abi.OPT_SKIP_RECORDS, skip if k == 0 else 0)
                self.parser.parse_into(self.bufs[b][start:start + length], out, stream=self.s_parse)
                parse_done[b].record(self.s_parse)
                if not last:
                    lens[k + 1] = h2d(k + 1)  # overlaps with this partition's parse
                prev = (b, start, length, out)
            pb, pstart, plen, pout = prev
            parse_done[pb].synchronize()
            res = self._checked(pout, pb, pstart, plen, partial=False)
            results.append(self._copy_back(self.outs[pb], res, plen, d2h_done[pb]))
            torch.cuda.synchronize()
            return results
        finally:
            self.parser.set_option(_abi.OPT_PARTIAL_INPUT, 0)
            self.parser.set_option(_abi.OPT_SKIP_RECORDS, skip)

    def _checked(self, out: Output, b: int, start: int, length: int, partial: bool):
        res = out.result()
        if res.status == _abi.E_CAPACITY:  # grow this buffer's outputs and parse the partition again
            with torch.cuda.stream(self.s_parse):
                self.outs[b] = self.parser.allocate(max(res.rows, 1),
                                                    [max(int(x), 1) for x in res.values_bytes_needed],
                                                    device=self.device)
            self.parser.set_option(_abi.OPT_PARTIAL_INPUT, 1 if partial else 0)
            self.parser.parse_into(self.bufs[b][start:start + length], self.outs[b], stream=self.s_parse)
            torch.cuda.current_stream().wait_stream(self.s_parse)
            self.s_parse.synchronize()
            res = self.outs[b].result()
        if res.status != _abi.OK:
            raise ParparawError(res.status, "partition")
        return res
