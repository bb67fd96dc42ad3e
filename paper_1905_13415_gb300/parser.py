"""Python binding of the C ABI (include/parparaw.h).

Argument marshalling only: every step of a parse runs in the CUDA library.
PyTorch provides device memory and streams.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import _abi
from .formats import Format

_NP = {_abi.INT32: np.int32, _abi.DATE_D: np.int32, _abi.INT64: np.int64,
       _abi.TIMESTAMP_S: np.int64, _abi.TIMESTAMP_CLF: np.int64, _abi.FLOAT64: np.float64}
_TORCH = {_abi.INT32: torch.int32, _abi.DATE_D: torch.int32, _abi.INT64: torch.int64,
          _abi.TIMESTAMP_S: torch.int64, _abi.TIMESTAMP_CLF: torch.int64, _abi.FLOAT64: torch.float64}


class ParparawError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        super().__init__(f"{what}: {_abi.status_string(code)} ({code})" if what else _abi.status_string(code))


def _ptr(t: torch.Tensor) -> int:
    return t.data_ptr()


def _stream(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


@dataclass
class Result:
    status: int
    final_state: int
    rows: int
    n_rejected: int
    first_invalid_offset: int
    values_bytes_needed: list
    consumed: int = 0

    @property
    def ok(self) -> bool:
        return self.status == _abi.OK


@dataclass
class Inference:
    """Column-count and numeric type inference of one input (Sec. 4.3)."""
    status: int
    records: int
    min_fields: int
    max_fields: int
    first_invalid_offset: int
    types: list  # per field position: a pp_type code, or TYPE_NONE (no non-empty field)


class Output:
    """Caller-owned device buffers for one parse (Arrow-like columns)."""

    def __init__(self, types, rows_cap: int, values_caps, device, result_buf: torch.Tensor | None = None):
        """``result_buf``: RESULT_BYTES of device memory for the parse result
        (a slice of a larger block, say); allocated here when None."""
        self.types = list(types)
        self.rows_cap = int(rows_cap)
        self.device = device
        nbits = (self.rows_cap + 7) // 8
        self.values, self.offsets, self.validity = [], [], []
        for c, t in enumerate(self.types):
            if t == _abi.SKIP:  # a column that is not selected: no buffers
                self.values.append(None)
                self.offsets.append(None)
                self.validity.append(None)
                continue
            if t == _abi.STRING:
                cap = int(values_caps[c])
                self.values.append(torch.empty(max(cap, 1), dtype=torch.uint8, device=device))
                self.offsets.append(torch.empty(self.rows_cap + 1, dtype=torch.int64, device=device))
            else:
                self.values.append(torch.empty(max(self.rows_cap, 1), dtype=_TORCH[t], device=device))
                self.offsets.append(None)
            self.validity.append(torch.empty(max(nbits, 1), dtype=torch.uint8, device=device))
        self.row_valid = torch.empty(max(nbits, 1), dtype=torch.uint8, device=device)
        self.result_buf = (torch.zeros(_abi.RESULT_BYTES, dtype=torch.uint8, device=device) if result_buf is None
                           else result_buf)
        self.values_caps = [int(values_caps[c]) if t == _abi.STRING else 0 for c, t in enumerate(self.types)]
        self.desc = _abi.pp_columns()
        self.desc.num_columns = len(self.types)
        self.desc.rows_cap = self.rows_cap
        for c in range(len(self.types)):
            col = self.desc.cols[c]
            col.values = _ptr(self.values[c]) if self.values[c] is not None else None
            col.offsets = _ptr(self.offsets[c]) if self.offsets[c] is not None else None
            col.validity = _ptr(self.validity[c]) if self.validity[c] is not None else None
            col.values_cap = self.values_caps[c]
        self.desc.row_valid = _ptr(self.row_valid)
        self.desc.result = _ptr(self.result_buf)

    def nbytes(self) -> int:
        n = self.row_valid.numel() + self.result_buf.numel()
        for v, o, m in zip(self.values, self.offsets, self.validity):
            if v is None:
                continue
            n += v.numel() * v.element_size() + m.numel()
            if o is not None:
                n += o.numel() * 8
        return n

    def result(self) -> Result:
        """Reads the result back (synchronises with the device)."""
        raw = self.result_buf.cpu().numpy().tobytes()
        r = _abi.pp_parse_result.from_buffer_copy(raw)
        return Result(r.status, r.final_state, r.rows, r.n_rejected, r.first_invalid_offset,
                      list(r.values_bytes_needed[: len(self.types)]), r.consumed)

    def output_bytes(self, rows: int) -> int:
        """Bytes of the fixed output layout for `rows` rows: values, int64
        offsets, validity bitmaps and row_valid."""
        res = self.result()
        nb = (rows + 7) // 8
        n = nb
        for c, t in enumerate(self.types):
            if t == _abi.SKIP:
                continue
            if t == _abi.STRING:
                n += res.values_bytes_needed[c] + 8 * (rows + 1)
            else:
                n += rows * np.dtype(_NP[t]).itemsize
            n += nb
        return n

    def to_host(self, rows: int | None = None) -> dict:
        """Copies the columns of the first `rows` rows to numpy."""
        if rows is None:
            rows = min(self.result().rows, self.rows_cap)
        nb = (rows + 7) // 8
        cols = []
        for c, t in enumerate(self.types):
            if t == _abi.SKIP:
                cols.append({"type": t, "values": None, "offsets": None, "validity": None})
                continue
            validity = self.validity[c][:nb].cpu().numpy()
            if t == _abi.STRING:
                offs = self.offsets[c][: rows + 1].cpu().numpy()
                end = int(offs[-1]) if rows > 0 else 0
                vals = self.values[c][:end].cpu().numpy()
                cols.append({"type": t, "values": vals, "offsets": offs, "validity": validity})
            else:
                cols.append({"type": t, "values": self.values[c][:rows].cpu().numpy(), "offsets": None,
                             "validity": validity})
        return {"rows": rows, "columns": cols, "row_valid": self.row_valid[:nb].cpu().numpy()}


class Parser:
    """A validated DFA + symbol groups + schema (parparaw_create)."""

    def __init__(self, fmt: Format, schema, tile_config: int = 0, timeout_ms: int | None = None,
                 grid_limit: int | None = None, skip_records: int = 0, utf16le: bool = False):
        """``skip_records``: the first n records (a header, say) are
        recognised but leave no row (Sec. 4.3, skipping records).
        ``utf16le``: the input is UTF-16LE code units (Sec. 4.2); symbols are
        the format's bytes as code points U+0000..U+00FF."""
        self._lib = _abi.load()
        self.format = fmt
        self.types = [_abi.TYPE_NAMES[t] if isinstance(t, str) else int(t) for t in schema]
        tr = np.ascontiguousarray(fmt.transitions, dtype=np.uint8).reshape(-1)
        em = np.ascontiguousarray(fmt.emit, dtype=np.uint8).reshape(-1)
        sym = np.frombuffer(bytes(fmt.symbols), dtype=np.uint8).copy()
        grp = np.asarray(fmt.groups, dtype=np.uint8)
        types = np.asarray(self.types, dtype=np.uint32)
        dfa = _abi.pp_dfa(fmt.num_states, fmt.num_groups, tr.ctypes.data, em.ctypes.data, fmt.start_state,
                          fmt.invalid_state, fmt.accept_mask)
        groups = _abi.pp_symbol_groups(len(sym), sym.ctypes.data if len(sym) else None,
                                       grp.ctypes.data if len(grp) else None, fmt.catch_all)
        sch = _abi.pp_schema(len(types), types.ctypes.data)
        handle = ctypes.c_void_p()
        rc = self._lib.parparaw_create(ctypes.byref(dfa), ctypes.byref(groups), ctypes.byref(sch),
                                       ctypes.byref(handle))
        if rc != _abi.OK:
            raise ParparawError(rc, "parparaw_create")
        self.handle = handle
        self.skip_records = 0
        if tile_config:
            self.set_option(_abi.OPT_TILE_CONFIG, tile_config)
        if timeout_ms:
            self.set_option(_abi.OPT_TIMEOUT_MS, timeout_ms)
        if grid_limit:
            self.set_option(_abi.OPT_GRID_LIMIT, grid_limit)
        if skip_records:
            self.set_option(_abi.OPT_SKIP_RECORDS, skip_records)
        if utf16le:
            self.set_option(_abi.OPT_UTF16LE, 1)

    def set_option(self, option: int, value: int) -> None:
        rc = self._lib.parparaw_set_option(self.handle, option, int(value))
        if rc != _abi.OK:
            raise ParparawError(rc, "parparaw_set_option")
        if option == _abi.OPT_SKIP_RECORDS:
            self.skip_records = int(value)

    def info(self) -> _abi.pp_parser_info:
        info = _abi.pp_parser_info()
        rc = self._lib.parparaw_get_info(self.handle, ctypes.byref(info))
        if rc != _abi.OK:
            raise ParparawError(rc, "parparaw_get_info")
        return info

    def set_kernel_events(self, start, stop) -> None:
        rc = self._lib.parparaw_set_kernel_events(self.handle, start.cuda_event if start else None,
                                                  stop.cuda_event if stop else None)
        if rc != _abi.OK:
            raise ParparawError(rc, "parparaw_set_kernel_events")

    def close(self) -> None:
        if getattr(self, "handle", None):
            self._lib.parparaw_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def allocate(self, rows_cap: int, values_caps, device="cuda", result_buf: torch.Tensor | None = None) -> Output:
        if isinstance(values_caps, int):
            values_caps = [values_caps] * len(self.types)
        return Output(self.types, rows_cap, values_caps, torch.device(device), result_buf)

    def parse_into(self, data: torch.Tensor, out: Output, nbytes: int | None = None, stream=None) -> None:
        """Enqueues the parse of `data` (uint8, CUDA) into `out` on `stream`."""
        n = data.numel() if nbytes is None else int(nbytes)
        rc = self._lib.parparaw_parse(self.handle, _ptr(data) if n else None, n, ctypes.byref(out.desc),
                                      _stream(stream))
        if rc != _abi.OK:
            raise ParparawError(rc, "parparaw_parse")

    def infer(self, data: torch.Tensor, stream=None) -> Inference:
        """Fields per record and the narrowest type of each field position
        (parparaw_infer; this parser's schema is ignored).  Synchronises."""
        buf = torch.zeros(_abi.INFERENCE_BYTES, dtype=torch.uint8, device=data.device)
        st = self._lib.parparaw_infer(self.handle, _ptr(data) if data.numel() else None, data.numel(), _ptr(buf),
                                      _stream(stream))
        if st != _abi.OK:
            raise ParparawError(st, "parparaw_infer")
        r = _abi.pp_inference.from_buffer_copy(buf.cpu().numpy().tobytes())
        return Inference(r.status, r.records, r.min_fields, r.max_fields, r.first_invalid_offset, list(r.type))

    def parse(self, data: torch.Tensor, rows_cap: int | None = None, stream=None) -> tuple[Output, Result]:
        """Parses with outputs sized from the input; retries once with the
        exact sizes the device reports on PP_E_CAPACITY."""
        n = data.numel()
        if rows_cap is None:
            rows_cap = max(1024, n // 16)
        s = torch.cuda.current_stream(data.device) if stream is None else stream
        # outputs allocated (zero fill included) and results read back on the parse's stream
        with torch.cuda.stream(s):
            out = self.allocate(rows_cap, [max(n, 1)] * len(self.types), device=data.device)
            self.parse_into(data, out, stream=s)
            res = out.result()
            if res.status == _abi.E_CAPACITY:
                caps = [max(int(b), 1) for b in res.values_bytes_needed]
                out = self.allocate(max(res.rows, 1), caps, device=data.device)
                self.parse_into(data, out, stream=s)
                res = out.result()
        return out, res


def parse_batch(items, stream=None) -> None:
    """Enqueues one batched parse of [(Parser, data, Output), ...]."""
    lib = _abi.load()
    arr = (_abi.pp_batch_item * len(items))()
    for i, (p, data, out) in enumerate(items):
        arr[i].parser = p.handle.value
        arr[i].input = _ptr(data) if data.numel() else None
        arr[i].len = data.numel()
        arr[i].out = ctypes.pointer(out.desc)
    rc = lib.parparaw_parse_batch(arr, len(items), _stream(stream))
    if rc != _abi.OK:
        raise ParparawError(rc, "parparaw_parse_batch")


class Batch:
    """A prepared batch (parparaw_batch_create): descriptors uploaded once,
    each launch() is kernel launches only."""

    def __init__(self, items):
        self._lib = _abi.load()
        self.items = list(items)  # keeps parsers, inputs and outputs alive
        arr = (_abi.pp_batch_item * len(self.items))()
        for i, (p, data, out) in enumerate(self.items):
            arr[i].parser = p.handle.value
            arr[i].input = _ptr(data) if data.numel() else None
            arr[i].len = data.numel()
            arr[i].out = ctypes.pointer(out.desc)
        handle = ctypes.c_void_p()
        rc = self._lib.parparaw_batch_create(arr, len(self.items), ctypes.byref(handle))
        if rc != _abi.OK:
            raise ParparawError(rc, "parparaw_batch_create")
        self.handle = handle

    def launch(self, stream=None) -> None:
        rc = self._lib.parparaw_batch_launch(self.handle, _stream(stream))
        if rc != _abi.OK:
            raise ParparawError(rc, "parparaw_batch_launch")

    def close(self) -> None:
        if getattr(self, "handle", None):
            torch.cuda.synchronize()
            self._lib.parparaw_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def skip_rows(data: torch.Tensor, rows, terminator: bytes = b"\n", stream=None) -> torch.Tensor:
    """Sec. 4.3, skipping rows (parparaw_skip_rows): ``data`` (a device uint8
    tensor) without the physical lines listed in ``rows`` (row numbers from
    0, strictly increasing).  Returns a new device tensor holding the bytes
    that stay; waits for the pass to learn their count."""
    lib = _abi.load()
    if data.device.type != "cuda" or data.dtype != torch.uint8 or not data.is_contiguous():
        raise ParparawError(_abi.E_ARG, "skip_rows wants a contiguous device uint8 tensor")
    r = torch.as_tensor(list(rows) if not isinstance(rows, torch.Tensor) else rows, dtype=torch.int64)
    if r.numel() > 1 and not bool((r[1:] > r[:-1]).all()):
        raise ParparawError(_abi.E_ARG, "rows must be strictly increasing")
    if r.numel() and int(r[0]) < 0:
        raise ParparawError(_abi.E_ARG, "rows are numbered from 0")
    r = r.to(data.device)
    n = data.numel()
    out = torch.empty(max(n, 1), dtype=torch.uint8, device=data.device)
    out_len = torch.zeros(1, dtype=torch.int64, device=data.device)
    sb = int(lib.parparaw_skip_rows_scratch_bytes(n))
    scratch = torch.empty(sb, dtype=torch.uint8, device=data.device)
    rc = lib.parparaw_skip_rows(data.data_ptr() if n else None, n, r.data_ptr() if r.numel() else None, r.numel(),
                                terminator[0], out.data_ptr(), out_len.data_ptr(), scratch.data_ptr(), sb,
                                _stream(stream))
    if rc != _abi.OK:
        raise ParparawError(rc, "parparaw_skip_rows")
    torch.cuda.synchronize(data.device)
    return out[: int(out_len.item())]
