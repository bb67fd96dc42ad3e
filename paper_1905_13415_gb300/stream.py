"""End-to-end streaming parse of host-resident input (Sec. 4.4): binding of
parparaw_stream_create / _parse / _destroy.

The library owns the pipeline: two device input buffers with a carry-over
region each, two sets of device output columns and three CUDA streams
(copy in, parse, copy out).  While partition k is parsed, partition k+1 is
copied in and the columns of partition k-1 are copied out to a host arena;
the incomplete record at the end of a partition is carried over on the device
to the front of the next one.  This module only marshals arguments and wraps
the partitions' host columns as tensors.
"""
from __future__ import annotations

import ctypes
import dataclasses
import time

import torch

from . import _abi
from .parser import Parser, ParparawError

_TORCH_OF = {_abi.INT32: torch.int32, _abi.DATE_D: torch.int32, _abi.INT64: torch.int64,
             _abi.TIMESTAMP_S: torch.int64, _abi.TIMESTAMP_CLF: torch.int64, _abi.FLOAT64: torch.float64}


@dataclasses.dataclass
class Partition:
    rows: int
    row0: int                        # first row of the whole parse in this partition
    input_offset: int                # first input byte parsed for it (carry-over included)
    nbytes: int                      # input bytes parsed (carry-over included)
    columns: list                    # per column: dict of host tensors (views of the arena)
    row_valid: torch.Tensor
    h2d_ms: float = 0.0              # device time of the partition's copy in, parse and copy out
    parse_ms: float = 0.0
    d2h_ms: float = 0.0


class HostArena:
    """A pinned host buffer that the partitions' columns are carved from (by
    the library).  The partitions of a parse stay valid until the arena's
    next parse."""

    def __init__(self, nbytes: int):
        self.buf = torch.empty(max(int(nbytes), 64), dtype=torch.uint8, pin_memory=True)

    def view(self, ptr: int, n: int, dtype) -> torch.Tensor:
        size = torch.empty(0, dtype=dtype).element_size()
        off = ptr - self.buf.data_ptr()
        assert 0 <= off and off + n * size <= self.buf.numel()
        return self.buf[off: off + n * size].view(dtype)


class StreamParser:
    """Streams pinned host input through the parser in partitions of
    `partition_bytes`; a record may be at most `carry_bytes` long."""

    def __init__(self, parser: Parser, partition_bytes: int = 256 << 20, carry_bytes: int | None = None,
                 device="cuda", **_unused):
        self.parser = parser
        self.part = int(partition_bytes)
        self._lib = _abi.load()
        self.handle = ctypes.c_void_p()
        with torch.cuda.device(torch.device(device)):
            rc = self._lib.parparaw_stream_create(parser.handle, self.part, int(carry_bytes or 0),
                                                  ctypes.byref(self.handle))
        if rc != _abi.OK:
            raise ParparawError(rc, "parparaw_stream_create")

    def close(self) -> None:
        if self.handle:
            self._lib.parparaw_stream_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def parse_raw(self, host: torch.Tensor, arena: HostArena):
        """One parparaw_stream_parse call: (pp_stream_result, partitions array)."""
        n = host.numel()
        nparts = max(1, (n + self.part - 1) // self.part)
        parts = (_abi.pp_host_partition * nparts)()
        res = _abi.pp_stream_result()
        t0 = time.perf_counter()
        rc = self._lib.parparaw_stream_parse(self.handle, host.data_ptr() if n else None, n,
                                             arena.buf.data_ptr(), arena.buf.numel(), parts, nparts,
                                             ctypes.byref(res))
        self.last_call_ms = (time.perf_counter() - t0) * 1e3  # the library call alone
        if rc != _abi.OK:
            raise ParparawError(rc, "parparaw_stream_parse")
        return res, parts

    def parse(self, host: torch.Tensor, arena: HostArena | None = None) -> list[Partition]:
        """Parses the pinned uint8 host tensor; returns the partitions' columns
        as views of `arena` (a pinned arena sized on demand when None)."""
        own = arena is None
        if own:
            arena = HostArena(2 * host.numel() + (1 << 20))
        while True:
            res, parts = self.parse_raw(host, arena)
            if res.status == _abi.E_CAPACITY and own:
                arena = HostArena(max(2 * arena.buf.numel(), int(res.arena_bytes * 1.25)))
                continue
            break
        if res.status != _abi.OK:
            raise ParparawError(res.status, "streamed parse")
        out = []
        types = self.parser.types
        for k in range(res.num_partitions):
            p = parts[k]
            rows, nb = p.rows, (p.rows + 7) // 8
            cols = []
            for c, t in enumerate(types):
                hc = p.cols[c]
                if t == _abi.SKIP:
                    cols.append({"values": None, "offsets": None, "validity": None})
                    continue
                col = {"validity": arena.view(hc.validity, nb, torch.uint8)}
                if t == _abi.STRING:
                    col["values"] = arena.view(hc.values, hc.values_cap, torch.uint8)
                    col["offsets"] = arena.view(hc.offsets, rows + 1, torch.int64)
                else:
                    col["values"] = arena.view(hc.values, rows, _TORCH_OF[t])
                    col["offsets"] = None
                cols.append(col)
            out.append(Partition(rows, p.row0, p.input_offset, p.input_bytes, cols,
                                 arena.view(p.row_valid, nb, torch.uint8), p.h2d_ms, p.parse_ms, p.d2h_ms))
        return out
