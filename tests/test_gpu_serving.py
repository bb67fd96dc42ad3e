"""Batched, served and streamed forms of the parse: each result must be
identical to the plain parse of the same input (and so to the oracle)."""
from __future__ import annotations

import random

import numpy as np
import pytest

import oracle as O
import synth
from parity import assert_same, oracle_parse

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
    return torch.frombuffer(bytearray(raw), dtype=torch.uint8).to("cuda") if raw else torch.empty(0, dtype=torch.uint8, device="cuda")


def _inputs(n, seed):
    rng = random.Random(seed)
    out = []
    for i in range(n):
        wl = ["mixed", "log", "review", "trip"][i % 4]
        raw, _ = synth.records(wl, seed * 100 + i, 0, rng.randint(1, 300))
        out.append((wl, raw))
    return out


def test_prepared_batch_launches_repeatably(pp):
    parsers = {wl: pp.Parser(pp.formats.by_name(synth.DIALECT[wl]), synth.SCHEMAS[wl], tile_config=2)
               for wl in synth.SCHEMAS}
    items, refs = [], []
    for wl, raw in _inputs(16, 3):
        ref = oracle_parse(synth.DIALECT[wl], synth.SCHEMAS[wl], raw)
        out = parsers[wl].allocate(max(ref.rows, 1), [max(len(raw), 1)] * len(synth.SCHEMAS[wl]))
        items.append((parsers[wl], _dev(raw), out))
        refs.append(ref)
    b = pp.Batch(items)
    for _ in range(2):
        b.launch()
        torch.cuda.synchronize()
        for (p, data, out), ref in zip(items, refs):
            res = out.result()
            assert_same(out.to_host(res.rows), res, ref, what="prepared batch")
    b.close()


def test_server_result_alone_equals_result_in_the_mix(pp):
    from paper_1905_13415_gb300.serve import Request, Server

    parsers = {wl: pp.Parser(pp.formats.by_name(synth.DIALECT[wl]), synth.SCHEMAS[wl]) for wl in synth.SCHEMAS}
    reqs, alone = [], []
    for i, (wl, raw) in enumerate(_inputs(40, 7)):
        p = parsers[wl]
        data = _dev(raw)
        out, res = p.parse(data)  # alone
        alone.append((out.to_host(res.rows), res))
        reqs.append(Request(i, p, data, max(res.rows, 1), [max(int(x), 1) for x in res.values_bytes_needed]))
    server = Server(arena_bytes=1 << 24, streams=3, max_batch=7, keep_outputs=True)  # small: many rounds
    for r in reqs:
        server.submit(r)
    server.drain()
    torch.cuda.synchronize()
    assert server.rounds >= 6
    for r, (host, res) in zip(reqs, alone):
        got = r.out.result()
        assert (got.status, got.rows, got.n_rejected) == (res.status, res.rows, res.n_rejected)
        mixed = r.out.to_host(got.rows)
        for a, b in zip(mixed["columns"], host["columns"]):
            assert np.array_equal(a["values"].view(np.uint8), b["values"].view(np.uint8))
            assert np.array_equal(a["validity"], b["validity"])
            if a["offsets"] is not None:
                assert np.array_equal(a["offsets"], b["offsets"])
        assert np.array_equal(mixed["row_valid"], host["row_valid"])


def test_server_sizes_requests_and_retries_on_capacity(pp):
    """Requests sized from their length only: inputs with more records than
    one per 16 bytes report PP_E_CAPACITY and are admitted again with the
    exact sizes; every result equals the plain parse."""
    from paper_1905_13415_gb300.serve import Request, Server

    p = pp.Parser(pp.formats.by_name("csv"), ["string", "int32"])
    raws = [b"".join(b"%d,%d\n" % (i % 7, i) for i in range(n)) for n in (10, 300, 2000, 5000)]
    raws += [synth.records("mixed", 90 + i, 0, 50)[0] for i in range(4)]
    ps = [p] * 4 + [pp.Parser(pp.formats.by_name("csv"), synth.SCHEMAS["mixed"])] * 4
    reqs = [Request(i, q, _dev(raw)) for i, (q, raw) in enumerate(zip(ps, raws))]
    server = Server(arena_bytes=1 << 26, streams=2, max_batch=3, keep_outputs=True)
    for r in reqs:
        server.submit(r)
    server.drain()
    torch.cuda.synchronize()
    assert server.retries >= 2  # the short-record inputs outgrow the estimate
    for r, raw, q in zip(reqs, raws, ps):
        out, res = q.parse(_dev(raw))
        got = r.out.result()
        assert got.status == res.status == 0 and got.rows == res.rows == r.rows
        a, b = r.out.to_host(got.rows), out.to_host(res.rows)
        for ca, cb in zip(a["columns"], b["columns"]):
            assert np.array_equal(ca["values"].view(np.uint8), cb["values"].view(np.uint8))
            assert np.array_equal(ca["validity"], cb["validity"])


def test_partial_input_mode(pp):
    raw, _ = synth.records("mixed", 21, 0, 500)
    schema = synth.SCHEMAS["mixed"]
    ref = oracle_parse("csv", schema, raw)
    cut = len(raw) * 2 // 3  # inside some record
    p = pp.Parser(pp.formats.rfc4180_csv(), schema, tile_config=1)
    p.set_option(pp._abi.OPT_PARTIAL_INPUT, 1)
    out, res = p.parse(_dev(raw[:cut]))
    torch.cuda.synchronize()
    assert res.status == 0
    # every record whose delimiter lies before the cut, and nothing else
    tags, _ = O.trace(O.csv6(), raw)
    rd = np.flatnonzero(tags[:cut] == O.RECORD)
    assert res.rows == len(rd) and res.consumed == int(rd[-1]) + 1
    got = out.to_host(res.rows)
    for c, col in enumerate(ref.columns):
        g = got["columns"][c]
        if col.offsets is not None:
            assert np.array_equal(g["offsets"], col.offsets[: res.rows + 1])
        else:
            assert np.array_equal(g["values"].view(np.uint8), col.values[: res.rows].view(np.uint8))


def _bits(bm: np.ndarray, n: int) -> np.ndarray:
    return np.unpackbits(np.asarray(bm, np.uint8), bitorder="little")[:n].astype(bool)


@pytest.mark.parametrize("workload", ["review", "mixed", "log"])
def test_streamed_parse_equals_whole_parse(pp, workload):
    from paper_1905_13415_gb300.stream import StreamParser

    raw, _ = synth.records(workload, 33, 0, {"review": 600, "mixed": 6000, "log": 6000}[workload])
    schema, dialect = synth.SCHEMAS[workload], synth.DIALECT[workload]
    ref = oracle_parse(dialect, schema, raw)
    p = pp.Parser(pp.formats.by_name(dialect), schema, tile_config=2)
    from paper_1905_13415_gb300.stream import HostArena

    host = torch.frombuffer(bytearray(raw), dtype=torch.uint8).pin_memory()
    sp = StreamParser(p, partition_bytes=37_000, carry_bytes=64_000)
    parts = sp.parse(host, HostArena(3 * len(raw) + (1 << 20)) if workload == "mixed" else None)
    assert len(parts) > 3
    assert sum(x.rows for x in parts) == ref.rows
    # every partition reports the device time of its copy in, parse and copy out
    for x in parts:
        assert 0.0 < x.h2d_ms < 1e3 and 0.0 < x.parse_ms < 1e3 and 0.0 < x.d2h_ms < 1e3, x
    for c, col in enumerate(ref.columns):
        if col.offsets is not None:
            fields = []
            for x in parts:
                offs = x.columns[c]["offsets"][: x.rows + 1].numpy()
                vals = x.columns[c]["values"].numpy()
                fields += [bytes(vals[offs[i]:offs[i + 1]]) for i in range(x.rows)]
            assert fields == [ref.field(i, c) for i in range(ref.rows)]
        else:
            vals = np.concatenate([x.columns[c]["values"][: x.rows].numpy() for x in parts])
            assert np.array_equal(vals.view(np.uint8), col.values.view(np.uint8))
        valid = np.concatenate([_bits(x.columns[c]["validity"].numpy(), x.rows) for x in parts])
        assert np.array_equal(valid, _bits(col.validity, ref.rows))


def test_autotune_picks_a_measured_config(pp):
    from paper_1905_13415_gb300.autotune import autotune

    raw, _ = synth.records("mixed", 5, 0, 4000)
    p = pp.Parser(pp.formats.rfc4180_csv(), synth.SCHEMAS["mixed"])
    data = _dev(raw)
    out, res = p.parse(data)
    best, times = autotune([(p, data, out)], reps=2)
    assert best in times and all(t > 0 for t in times.values())
    assert p.info().tile_bytes > 0


def test_stream_entry_outcomes(pp):
    """parparaw_stream_parse through the C ABI: partition offsets and rows,
    an invalid byte in a later partition (offset in the whole input), an
    unterminated end, a record longer than the carry-over region, an arena
    that is too small, and skipped records (first partition only)."""
    from paper_1905_13415_gb300 import _abi
    from paper_1905_13415_gb300.stream import HostArena, StreamParser

    raw, _ = synth.records("mixed", 44, 0, 3000)
    schema = synth.SCHEMAS["mixed"]
    p = pp.Parser(pp.formats.by_name("csv"), schema, tile_config=2)
    host = torch.frombuffer(bytearray(raw), dtype=torch.uint8).pin_memory()
    sp = StreamParser(p, partition_bytes=20_000, carry_bytes=20_000)
    parts = sp.parse(host)
    ref = oracle_parse("csv", schema, raw)
    assert sum(x.rows for x in parts) == ref.rows
    row0 = 0
    for x in parts:  # partitions tile the rows and the input
        assert x.row0 == row0
        row0 += x.rows
    assert parts[0].input_offset == 0 and parts[-1].input_offset + parts[-1].nbytes == len(raw)

    # an invalid byte (a quote inside an unquoted field) in a later partition
    bad = bytearray(raw)
    pos = raw.index(b"\n", 50_000) + 2
    while bad[pos - 1] in b'",\n' or bad[pos] in b'",\n':
        pos += 1
    bad[pos] = ord('"')
    ref_bad = oracle_parse("csv", schema, bytes(bad))
    assert ref_bad.status == O.E_INVALID_INPUT
    res, parts_arr = sp.parse_raw(torch.frombuffer(bad, dtype=torch.uint8).pin_memory(), HostArena(4 * len(raw)))
    assert res.status == _abi.E_INVALID_INPUT and res.first_invalid_offset == ref_bad.first_invalid_offset
    assert res.rows == ref_bad.rows  # every record before the invalid byte

    # an unterminated quote at the end of the input
    unterminated = raw + b'1,"abc'
    res, _ = sp.parse_raw(torch.frombuffer(bytearray(unterminated), dtype=torch.uint8).pin_memory(),
                          HostArena(4 * len(raw)))
    assert res.status == _abi.E_UNTERMINATED

    # a record longer than the carry-over region
    long_rec = raw + b'1,"' + b"x" * 50_000 + b'",2,3.5,2020-01-01T00:00:00,a,2020-01-01T00:00:00,b\n' + raw
    res, _ = sp.parse_raw(torch.frombuffer(bytearray(long_rec), dtype=torch.uint8).pin_memory(),
                          HostArena(8 * len(long_rec)))
    assert res.status == _abi.E_UNSUPPORTED

    # an arena too small: PP_E_CAPACITY with the size the partitions so far need
    res, _ = sp.parse_raw(host, HostArena(4096))
    assert res.status == _abi.E_CAPACITY and res.arena_bytes > 4096 and res.num_partitions == 0
    sp.close()

    # skipped records leave the first partition only
    p2 = pp.Parser(pp.formats.by_name("csv"), schema, tile_config=2, skip_records=5)
    sp2 = StreamParser(p2, partition_bytes=20_000, carry_bytes=20_000)
    parts2 = sp2.parse(host)
    assert sum(x.rows for x in parts2) == ref.rows - 5
    sp2.close()
