"""Skipping records (Sec. 4.3) on the GPU against the oracle: the first n
records leave no row, no string bytes, no conversion and no reject, in every
tile shape, with the skipped records ending inside the first tile, several
tiles in, inside a multi-round tile, at the last record and past it; and
through type inference and the streamed host path."""
from __future__ import annotations

import numpy as np
import pytest

import oracle as O
import synth
from parity import assert_same, oracle_parse

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CONFIGS = list(range(1, 15))


@pytest.fixture(scope="module")
def pp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    import paper_1905_13415_gb300 as pkg

    return pkg


def _dev(raw: bytes):
    return torch.frombuffer(bytearray(raw), dtype=torch.uint8).to("cuda") if raw else torch.empty(
        0, dtype=torch.uint8, device="cuda")


def _parse(pp, dialect, schema, raw, cfg, skip):
    p = pp.Parser(pp.formats.by_name(dialect), schema, tile_config=cfg, skip_records=skip)
    out, res = p.parse(_dev(raw))
    torch.cuda.synchronize()
    return out.to_host(min(res.rows, out.rows_cap)), res


def _skips(nrec: int):
    return sorted({0, 1, 2, 7, nrec // 3, nrec // 2 + 1, nrec - 1, nrec, nrec + 5})


@pytest.mark.parametrize("cfg", CONFIGS)
def test_header_and_bodies(pp, cfg):
    # a header over generated bodies, and a malformed record among the skipped ones
    raw, _ = synth.records("mixed", 77, 0, 3000)
    schema = synth.SCHEMAS["mixed"]
    head = b"id,name,value,when,score,flag,text,day\n"
    for what, data in (("header", head + raw), ("short record skipped", b"1,2\n" + raw)):
        for skip in (1, 2):
            got, res = _parse(pp, "csv", schema, data, cfg, skip)
            assert_same(got, res, oracle_parse("csv", schema, data, skip), what=(what, skip))


@pytest.mark.parametrize("cfg", [0, 1, 2, 10])
@pytest.mark.parametrize("workload,nrec", [("mixed", 4000), ("trip", 3000), ("review", 300), ("log", 3000)])
def test_skip_counts(pp, cfg, workload, nrec):
    raw, _ = synth.records(workload, 78, 0, nrec)
    schema = synth.SCHEMAS[workload]
    dialect = synth.DIALECT[workload]
    for skip in _skips(nrec):
        got, res = _parse(pp, dialect, schema, raw, cfg, skip)
        assert res.rows == max(nrec - skip, 0)
        assert_same(got, res, oracle_parse(dialect, schema, raw, skip), what=(workload, skip))


@pytest.mark.parametrize("cfg", [0, 1, 3, 10])
def test_skip_inside_a_multi_round_tile(pp, cfg):
    # short fields: more fields than one round holds, so the first kept
    # record starts in a later round of the tile
    raw = b"".join(b"%d,%d\n" % (i % 10, i % 7) for i in range(60000))
    schema = ["int32", "string"]
    for skip in (1, 4000, 7001, 20000, 59999):
        got, res = _parse(pp, "csv", schema, raw, cfg, skip)
        assert_same(got, res, oracle_parse("csv", schema, raw, skip), what=skip)


def test_trailing_record_and_rejects(pp):
    schema = ["int32", "string", "float64"]
    raw = b'1,a,2.5\nx,b,1\n3,c\n4,"d\nd",5\n6,e,7'  # a rejected conversion, a short record, no final newline
    for skip in range(0, 7):
        got, res = _parse(pp, "csv", schema, raw, 1, skip)
        assert_same(got, res, oracle_parse("csv", schema, raw, skip), what=skip)


@pytest.mark.parametrize("skip", [1, 3])
def test_inference_skips_the_header(pp, skip):
    raw = b"id,name,score\n" * skip + b"".join(b'%d,"n%d",%d.5\n' % (i, i, i) for i in range(5000))
    ref = O.infer(O.csv6(), raw, skip_records=skip)
    p = pp.Parser(pp.formats.by_name("csv"), ["string"], skip_records=skip)
    got = p.infer(_dev(raw))
    assert (got.status, got.records, got.min_fields, got.max_fields, got.types) == \
        (ref.status, ref.records, ref.min_fields, ref.max_fields, ref.types)
    assert got.types[:3] == [O.INT32, O.STRING, O.FLOAT64]
    kept = p.infer(_dev(raw[:1000]))  # unchanged by the skip: the parser's option applies
    assert kept.records == O.infer(O.csv6(), raw[:1000], skip_records=skip).records


def _bits(v, n):
    return [(int(v[i >> 3]) >> (i & 7)) & 1 for i in range(n)]


def test_streamed_skip_applies_to_the_first_partition_only(pp):
    from paper_1905_13415_gb300.stream import StreamParser

    raw, _ = synth.records("mixed", 79, 0, 6000)
    raw = b"id,name,value,when,score,flag,text,day\n" + raw
    schema = synth.SCHEMAS["mixed"]
    ref = oracle_parse("csv", schema, raw, 1)
    p = pp.Parser(pp.formats.by_name("csv"), schema, tile_config=2, skip_records=1)
    host = torch.frombuffer(bytearray(raw), dtype=torch.uint8).pin_memory()
    parts = StreamParser(p, partition_bytes=37_000, carry_bytes=64_000).parse(host)
    assert len(parts) > 3 and p.skip_records == 1
    assert sum(x.rows for x in parts) == ref.rows
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


def test_batch_items_keep_their_own_skip(pp):
    # one batched launch of parsers with different skips (and a selected
    # column) equals each plain parse against the oracle
    items, refs = [], []
    for k, (workload, n, skip) in enumerate([("mixed", 2000, 0), ("mixed", 1500, 3), ("log", 2500, 1),
                                             ("review", 200, 7), ("trip", 3000, 2999), ("mixed", 10, 20)]):
        raw, _ = synth.records(workload, 80 + k, 0, n)
        schema = list(synth.SCHEMAS[workload])
        if k == 1:
            schema[1] = "skip"
        dialect = synth.DIALECT[workload]
        p = pp.Parser(pp.formats.by_name(dialect), schema, tile_config=2, skip_records=skip)
        data = _dev(raw)
        out = p.allocate(max(n, 1), [len(raw) + 1] * len(schema))
        items.append((p, data, out))
        refs.append(oracle_parse(dialect, schema, raw, skip))
    pp.parse_batch(items)
    torch.cuda.synchronize()
    for k, ((p, data, out), ref) in enumerate(zip(items, refs)):
        res = out.result()
        assert_same(out.to_host(min(res.rows, out.rows_cap)), res, ref, what=("batch item", k))
