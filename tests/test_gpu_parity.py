"""GPU parity: the CUDA path through the C ABI against the oracle, element by
element (bit-exact: the whole output is integer / byte data, and floats are
correctly rounded on both sides).

Tile configurations 1 (512 B) and 2 (3 KiB) put tile and chunk boundaries
inside every construct; 0 is the default shape used by the benchmark."""
from __future__ import annotations

import functools
import json
import os
import random

import numpy as np
import pytest

import oracle as O
import synth
from parity import assert_same, oracle_parse

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden")
CONFIGS = list(range(1, 15))


@pytest.fixture(scope="module")
def pp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    import paper_1905_13415_gb300 as pkg

    return pkg


def to_dev(raw: bytes, offset: int = 0):
    buf = torch.zeros(len(raw) + offset + 16, dtype=torch.uint8)
    buf[offset: offset + len(raw)] = torch.frombuffer(bytearray(raw), dtype=torch.uint8) if raw else buf[:0]
    d = buf.to("cuda")
    return d[offset: offset + len(raw)]


def run(pp, dialect, schema, raw, cfg, offset=0, rows_cap=None, caps=None):
    p = pp.Parser(pp.formats.by_name(dialect), schema, tile_config=cfg)
    data = to_dev(raw, offset)
    if rows_cap is None and caps is None:
        out, res = p.parse(data)
    else:
        out = p.allocate(rows_cap, caps)
        p.parse_into(data, out)
        res = out.result()
    torch.cuda.synchronize()
    rows = min(res.rows, out.rows_cap)
    return out.to_host(rows), res


@pytest.mark.parametrize("cfg", CONFIGS)
def test_worked_examples(pp, cfg):
    cases = json.load(open(os.path.join(GOLD, "worked_examples.json")))["cases"]
    for case in cases:
        raw = case["input"].encode()
        schema = ["string"] * case["columns"]
        got, res = run(pp, case["dialect"], schema, raw, cfg)
        assert_same(got, res, oracle_parse(case["dialect"], schema, raw), what=case["input"])


@pytest.mark.parametrize("cfg", [1, 2])
def test_random_small_inputs(pp, cfg):
    rng = random.Random(cfg)
    for it in range(300):
        n = rng.randint(0, 1200)
        alphabet = b'\n,"\rab' if it % 2 else b'\n,"ab1.'
        raw = bytes(rng.choice(alphabet) for _ in range(n))
        ncol = rng.randint(1, 4)
        schema = [rng.choice(["string", "string", "int32", "float64"]) for _ in range(ncol)]
        got, res = run(pp, "csv", schema, raw, cfg)
        assert_same(got, res, oracle_parse("csv", schema, raw), what=(it, raw[:80]))


@pytest.mark.parametrize("workload,nrows", [("mixed", 2500), ("trip", 3000), ("review", 300), ("log", 3000)])
@pytest.mark.parametrize("cfg", CONFIGS)
def test_generated_workloads(pp, workload, nrows, cfg):
    raw, _ = synth.records(workload, synth.BASE_SEED + 7, 0, nrows)
    schema = synth.SCHEMAS[workload]
    got, res = run(pp, synth.DIALECT[workload], schema, raw, cfg)
    ref = oracle_parse(synth.DIALECT[workload], schema, raw)
    assert ref.rows == nrows and res.status == O.OK
    assert_same(got, res, ref, what=workload)


@functools.lru_cache(maxsize=1)
def _dense_fields(seed: int, nrec: int) -> bytes:
    """Records of 1-3 byte fields (more fields per tile than one field-list
    round holds, in every shape): three string columns among integers,
    quoted fields with doubled quotes, embedded delimiters and newlines,
    empty fields, and now and then a record one field short or long."""
    rng = np.random.default_rng(seed)
    quoted = [b'"' + bytes([a, b]).replace(b'"', b'""') + b'"' for a in b'a,"\n' for b in b'a,"\n']
    plain = [bytes([a]) for a in b"abcxyz"] + [bytes([a, b]) for a in b"abc" for b in b"xyz"]
    nfs = np.where(rng.integers(0, 40, nrec) == 0, rng.choice([5, 7], nrec), 6)
    kind = rng.integers(0, 10, (nrec, 7))
    pick = rng.integers(0, 1 << 30, (nrec, 7))
    out = []
    for i in range(nrec):
        f = []
        for c in range(int(nfs[i])):
            k, x = int(kind[i, c]), int(pick[i, c])
            if c in (1, 3, 4):  # string columns
                f.append(b"" if k == 0 else quoted[x % len(quoted)] if k == 1 else plain[x % len(plain)])
            else:
                f.append(b"%d" % (x % 100))
        out.append(b",".join(f) + b"\n")
    return b"".join(out)


@pytest.mark.parametrize("cfg", CONFIGS)
def test_multi_round_tiles(pp, cfg):
    # tiles with several field-list rounds: the per-column string byte totals
    # taken from the chunk masks must equal what the rounds emit
    raw = _dense_fields(11, 60_000)
    schema = ["int32", "string", "int64", "string", "string", "int32"]
    got, res = run(pp, "csv", schema, raw, cfg)
    ref = oracle_parse("csv", schema, raw)
    assert ref.rows == 60_000
    assert_same(got, res, ref, what=cfg)
    tile = pp.Parser(pp.formats.by_name("csv"), schema, tile_config=cfg).info().tile_bytes
    # more fields per tile than a round holds (at most T/4 and 4960 entries)
    assert raw.count(b",") / (len(raw) / tile) > min(tile / 4, 4960)
    for skip in (3, 20_001):
        p = pp.Parser(pp.formats.by_name("csv"), schema, tile_config=cfg, skip_records=skip)
        out, res = p.parse(to_dev(raw))
        torch.cuda.synchronize()
        assert_same(out.to_host(min(res.rows, out.rows_cap)), res, oracle_parse("csv", schema, raw, skip),
                    what=(cfg, skip))


def _gapped_long_fields(seed: int, nrec: int) -> bytes:
    """Quoted fields of 30-3,000 bytes with doubled quotes (non-data bytes
    inside the field) at random places, in runs, and next to multiples of
    16 and 512 bytes of the field (where long fields are cut into pieces)."""
    rng = np.random.default_rng(seed)
    alphabet = np.frombuffer(b"abcdefgh ,\n", dtype=np.uint8)
    recs = []
    for i in range(nrec):
        n = int(rng.integers(30, 3000))
        body = rng.choice(alphabet, n).tobytes()
        pos = {int(x) for x in rng.integers(0, n, int(rng.integers(0, 6)))}
        if i % 3 == 0:
            pos.add(min(n, max(0, 512 * int(rng.integers(0, n // 512 + 1)) + int(rng.integers(-3, 4)))))
        if i % 5 == 0:
            pos.add(min(n, 16 * int(rng.integers(0, n // 16 + 1))))
        text, last = [], 0
        for q in sorted(pos):
            text += [body[last:q], b'""' * int(rng.integers(1, 4))]
            last = q
        text.append(body[last:])
        recs.append(b'%d,"%s",x%d\n' % (i, b"".join(text), i))
    return b"".join(recs)


@pytest.mark.parametrize("cfg", [1, 2, 3, 10, 13])
def test_long_fields_with_gaps(pp, cfg):
    # the long-field pieces that hold non-data bytes are copied run by run
    raw = _gapped_long_fields(cfg, 2500)
    schema = ["int32", "string", "string"]
    ref = oracle_parse("csv", schema, raw)
    assert ref.status == O.OK and ref.rows == 2500
    got, res = run(pp, "csv", schema, raw, cfg)
    assert_same(got, res, ref, what=cfg)
    # too few value bytes for the long column: the bytes that fit are the oracle's
    cap = ref.columns[1].bytes_total // 2 + 7
    got, res = run(pp, "csv", schema, raw, cfg, rows_cap=ref.rows, caps=[len(raw), cap, len(raw)])
    assert res.status == -6 and res.values_bytes_needed[1] == ref.columns[1].bytes_total
    assert np.array_equal(got["columns"][1]["values"][:cap], ref.columns[1].values[:cap])
    assert np.array_equal(got["columns"][1]["offsets"][: ref.rows + 1], ref.columns[1].offsets[: ref.rows + 1])


@pytest.mark.parametrize("offset", [1, 3, 7, 15])
def test_unaligned_input(pp, offset):
    raw, _ = synth.records("mixed", 5, 0, 500)
    schema = synth.SCHEMAS["mixed"]
    for cfg in (1, 3):
        got, res = run(pp, "csv", schema, raw, cfg, offset=offset)
        assert_same(got, res, oracle_parse("csv", schema, raw), what=(offset, cfg))


def test_empty_and_tiny(pp):
    for raw in [b"", b"\n", b"a", b",", b'"', b"\r\n", b"x" * 17]:
        for cfg in (1, 3):
            got, res = run(pp, "csv", ["string", "string"], raw, cfg)
            assert_same(got, res, oracle_parse("csv", ["string", "string"], raw), what=raw)


def test_invalid_in_the_middle(pp):
    raw, _ = synth.records("mixed", 9, 0, 2000)
    schema = synth.SCHEMAS["mixed"]
    bad = bytearray(raw)
    cut = len(bad) // 2
    while bad[cut] != ord("\n"):
        cut += 1
    bad[cut + 1: cut + 1] = b'ab"c,'
    for cfg in (1, 2, 3):
        got, res = run(pp, "csv", schema, bytes(bad), cfg)
        ref = oracle_parse("csv", schema, bytes(bad))
        assert ref.status == O.E_INVALID_INPUT
        assert_same(got, res, ref, what=cfg)


def test_rejects_and_nulls(pp):
    raw = b"1,a,2.5\n,b,\nx,c,1\n4,d\n5,e,6,7\n99999999999,f,1e3\n-7,\"g\"\"h\",-0.0\n"
    schema = ["int32", "string", "float64"]
    for cfg in CONFIGS:
        got, res = run(pp, "csv", schema, raw, cfg)
        assert_same(got, res, oracle_parse("csv", schema, raw), what=cfg)


def test_integer_edge_cases(pp):
    """Leading zeros, the int32 / int64 limits and one past them, 19- and
    20-digit values, signs and stray bytes, against the oracle."""
    vals = ["0", "-0", "00000000000000000000000042", "2147483647", "2147483648", "-2147483648",
            "-2147483649", "9223372036854775807", "9223372036854775808", "-9223372036854775808",
            "-9223372036854775809", "99999999999999999999", "9999999999999999999",
            "0000000000000000000009223372036854775807", "-00000000000000000000000000000001", "-", "+5",
            "1a", " 1", "", "007"]
    raw = "".join(f"{v},{v}\n" for v in vals).encode()
    schema = ["int32", "int64"]
    for cfg in (1, 2, 10):
        got, res = run(pp, "csv", schema, raw, cfg)
        assert_same(got, res, oracle_parse("csv", schema, raw), what=cfg)


def test_capacity(pp):
    raw, _ = synth.records("mixed", 3, 0, 1000)
    schema = synth.SCHEMAS["mixed"]
    ref = oracle_parse("csv", schema, raw)
    # too few rows: exact row count reported, nothing written past the caps
    got, res = run(pp, "csv", schema, raw, 3, rows_cap=100, caps=[len(raw)] * len(schema))
    assert res.status == O.__dict__.get("E_CAPACITY", -6) and res.rows == ref.rows
    assert_same_prefix = min(100, ref.rows)
    for c, col in enumerate(ref.columns):
        if col.offsets is not None:
            assert np.array_equal(got["columns"][c]["offsets"][: assert_same_prefix + 1],
                                  col.offsets[: assert_same_prefix + 1])
    # too few string bytes: exact byte counts reported
    got, res = run(pp, "csv", schema, raw, 3, rows_cap=ref.rows, caps=[10] * len(schema))
    assert res.status == -6
    for c, col in enumerate(ref.columns):
        if col.offsets is not None:
            assert res.values_bytes_needed[c] == col.bytes_total


def _random_dfa(rng, S, G, with_inv):
    inv = S - 1 if with_inv else 0xFF
    tr = np.zeros((G, S), np.uint8)
    em = np.zeros((G, S), np.uint8)
    for g in range(G):
        for s in range(S):
            if with_inv and s == inv:
                tr[g, s], em[g, s] = inv, 3
            else:
                tr[g, s] = rng.randrange(S)
                em[g, s] = rng.choice([0, 0, 0, 1, 2, 3])
    return tr, em, inv


def test_random_dfas(pp):
    """Arbitrary DFAs (idempotent catch-all or not) give the oracle's result."""
    rng = random.Random(11)
    for it in range(60):
        S = rng.randint(1, 8)
        G = rng.randint(2, 7)
        with_inv = S > 1 and rng.random() < 0.5
        tr, em, inv = _random_dfa(rng, S, G, with_inv)
        if it % 3 == 0:  # make the catch-all (last group) idempotent
            for s in range(S):
                tr[G - 1, s] = tr[G - 1, tr[G - 1, s]]
        syms = bytes(rng.sample(range(256), G - 1))
        accept = [s for s in range(S) if rng.random() < 0.7]
        fmt = pp.formats.Format("rand", tr, em, syms, list(range(G - 1)), G - 1, rng.randrange(S), inv, accept)
        ofmt = O.Format(S, G, tr, em, syms, list(range(G - 1)), G - 1, fmt.start_state, inv, fmt.accept_mask)
        alphabet = list(syms) + [ord("q"), ord("z")]
        raw = bytes(rng.choice(alphabet) for _ in range(rng.randint(0, 3000)))
        schema = ["string"] * rng.randint(1, 3)
        p = pp.Parser(fmt, schema, tile_config=rng.choice([1, 2, 3]))
        out, res = p.parse(to_dev(raw))
        torch.cuda.synchronize()
        ref = O.parse(ofmt, [O.STRING] * len(schema), raw)
        assert_same(out.to_host(min(res.rows, out.rows_cap)), res, ref, what=(it, S, G))


def test_batch_mixed_formats(pp):
    items, refs = [], []
    rng = random.Random(5)
    for i in range(12):
        wl = ["mixed", "log", "review", "trip"][i % 4]
        raw, _ = synth.records(wl, 100 + i, 0, rng.randint(1, 400))
        schema = synth.SCHEMAS[wl]
        p = pp.Parser(pp.formats.by_name(synth.DIALECT[wl]), schema, tile_config=2)
        data = to_dev(raw, offset=i % 5)
        ref = oracle_parse(synth.DIALECT[wl], schema, raw)
        out = p.allocate(max(ref.rows, 1), [max(len(raw), 1)] * len(schema))
        items.append((p, data, out))
        refs.append(ref)
    pp.parse_batch(items)
    torch.cuda.synchronize()
    for (p, data, out), ref in zip(items, refs):
        res = out.result()
        assert_same(out.to_host(res.rows), res, ref, what="batch")


def test_expired_wait_reports_timeout_and_the_context_stays_usable(pp):
    # Failure detection without a GPU fault: with the work queue started past
    # tile 0 (a testing option), tile 0 never publishes, so every later tile's
    # bounded look-back wait runs out; the parse must end with PP_E_TIMEOUT, and
    # the next parse on the same context must be correct.
    raw, _ = synth.records("mixed", 13, 0, 6000)
    schema = synth.SCHEMAS["mixed"]
    p = pp.Parser(pp.formats.rfc4180_csv(), schema, tile_config=2, timeout_ms=20)
    data = to_dev(raw)
    assert (len(raw) + 3071) // 3072 > 20  # many tiles wait on the missing one
    p.set_option(pp._abi.OPT_FIRST_ITEM, 1)
    out, res = p.parse(data, rows_cap=10000)
    torch.cuda.synchronize()
    assert res.status == pp._abi.E_TIMEOUT, res
    p.set_option(pp._abi.OPT_FIRST_ITEM, 0)
    out, res = p.parse(data)
    torch.cuda.synchronize()
    assert_same(out.to_host(res.rows), res, oracle_parse("csv", schema, raw), what="after a timeout")
