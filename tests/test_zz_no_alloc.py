"""parparaw_parse_noalloc: the entry point for callers that cannot allocate
device memory on the call path.  Its scratch is one fixed device array shared
by every call, so each call must clear what it needs and leave nothing behind
that changes the next call's result.  Checked here through the C ABI against
parparaw_parse (bit-exact, as every parity test in this suite), over several
calls in a row, plus the up-front rejection of a parse whose scratch would not
fit the array."""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    import paper_1905_13415_gb300 as pkg

    return pkg


def _dev(raw: bytes):
    return torch.frombuffer(bytearray(raw), dtype=torch.uint8).to("cuda")


def _same(a: dict, b: dict):
    assert a["rows"] == b["rows"]
    assert np.array_equal(a["row_valid"], b["row_valid"])
    for ca, cb in zip(a["columns"], b["columns"]):
        assert np.array_equal(ca["validity"], cb["validity"])
        assert np.array_equal(ca["values"].view(np.uint8), cb["values"].view(np.uint8))
        if ca["offsets"] is not None:
            assert np.array_equal(ca["offsets"], cb["offsets"])


def _noalloc(pp, parser, data, out):
    lib = pp._abi.load()
    rc = lib.parparaw_parse_noalloc(parser.handle, data.data_ptr() if data.numel() else None, data.numel(),
                                    ctypes.byref(out.desc), torch.cuda.current_stream().cuda_stream)
    return rc


def test_noalloc_matches_parse_call_after_call(pp):
    cases = []
    for wl, n, seed, cfg in [("mixed", 3000, 1, 2), ("trip", 2500, 2, 0), ("log", 2000, 3, 1)]:
        raw, _ = synth.records(wl, seed, 0, n)
        parser = pp.Parser(pp.formats.by_name(synth.DIALECT[wl]), synth.SCHEMAS[wl], tile_config=cfg)
        data = _dev(raw)
        ref_out, ref_res = parser.parse(data)
        torch.cuda.synchronize()
        assert ref_res.status == 0 and ref_res.rows == n
        cases.append((parser, data, ref_out, ref_res))
    # three different parses in a row, then the first again: stale contents of
    # the shared scratch must not leak into a later result
    for parser, data, ref_out, ref_res in cases + cases[:1]:
        out = parser.allocate(ref_res.rows, [max(int(b), 1) for b in ref_res.values_bytes_needed])
        assert _noalloc(pp, parser, data, out) == 0
        torch.cuda.synchronize()
        res = out.result()
        assert (res.status, res.rows, res.n_rejected, res.first_invalid_offset, res.final_state) == \
            (ref_res.status, ref_res.rows, ref_res.n_rejected, ref_res.first_invalid_offset, ref_res.final_state)
        assert res.values_bytes_needed == ref_res.values_bytes_needed
        _same(out.to_host(res.rows), ref_out.to_host(ref_res.rows))


def test_noalloc_rejects_scratch_beyond_its_array(pp):
    raw, _ = synth.records("mixed", 4, 0, 100)
    parser = pp.Parser(pp.formats.rfc4180_csv(), synth.SCHEMAS["mixed"])
    data = _dev(raw)
    out = parser.allocate(128, [len(raw)] * 8)
    # a row capacity whose reject / null bitmaps alone exceed the fixed array
    out.desc.rows_cap = 8 * pp._abi.NOALLOC_SCRATCH_BYTES
    assert _noalloc(pp, parser, data, out) == pp._abi.E_UNSUPPORTED
    # nothing ran; the next call with a sane capacity works
    out.desc.rows_cap = 128
    assert _noalloc(pp, parser, data, out) == 0
    torch.cuda.synchronize()
    assert out.result().rows == 100
