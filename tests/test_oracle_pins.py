"""Pins of the oracle to things other than itself.

Each test ties a part of the oracle to what the paper prints (Table 1, the
prefix-sum example of Sec. 2), to hand-worked examples, to algebraic facts of
the method (the composite operator of Sec. 3.1 is associative and composing
chunk vectors reproduces the sequential run for every split), to an
independent format-specific rule (quote parity for RFC-4180 input) or to the
C/Python standard libraries (conversion).
"""
import calendar
import datetime as dt
import itertools
import json
import math
import os
import random

import numpy as np
import pytest

import oracle as O
import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")
NAMES = {"EOR": O.EOR, "ENC": O.ENC, "FLD": O.FLD, "EOF": O.EOF_, "ESC": O.ESC, "INV": O.INV}


def test_csv_dfa_contains_table1():
    """Table 1 (Sec. 4.5): the oracle's CSV DFA restricted to the groups
    \\n, ", ',' and catch-all is the paper's transition table."""
    f = O.csv6()
    sym_to_group = {"\\n": f.group_of(ord("\n")), '"': f.group_of(ord('"')),
                    ",": f.group_of(ord(",")), "*": f.group_of(ord("x"))}
    rows = [l.split() for l in open(os.path.join(GOLD, "table1_csv_dfa.txt")) if not l.startswith("#")]
    assert len(rows) == 4
    for row in rows:
        g = sym_to_group[row[1]]
        assert [int(x) for x in f.next[g]] == [NAMES[s] for s in row[2:8]], row


def test_state_vector_worked_example():
    """The chunk '",' read from each start state EOR, ENC, FLD, EOF, ESC, INV
    (worked by hand from Table 1) ends in ENC, EOF, INV, ENC, ENC, INV."""
    v = O.state_vector(O.csv6(), b'",')
    assert list(v) == [O.ENC, O.EOF_, O.INV, O.ENC, O.ENC, O.INV]


def test_compose_order_and_identity():
    # (a o b)_i = b[a_i]: a maps 0->1, b maps 1->2, so a o b maps 0->2
    a = np.array([1, 1, 2], np.uint8)
    b = np.array([0, 2, 0], np.uint8)
    assert list(O.compose(a, b)) == [2, 2, 0]
    assert list(O.compose(b, a)) == [1, 2, 1]
    ident = np.arange(3, dtype=np.uint8)
    assert list(O.compose(a, ident)) == list(a)
    assert list(O.compose(ident, a)) == list(a)


@pytest.mark.parametrize("S", [1, 2, 3])
def test_compose_associative_exhaustive(S):
    vecs = [np.array(v, np.uint8) for v in itertools.product(range(S), repeat=S)]
    for a in vecs:
        for b in vecs:
            ab = O.compose(a, b)
            for c in vecs:
                assert np.array_equal(O.compose(ab, c), O.compose(a, O.compose(b, c)))


@pytest.mark.parametrize("S", [6, 8])
def test_compose_associative_random(S):
    rng = np.random.default_rng(S)
    for _ in range(2000):
        a, b, c = (rng.integers(0, S, S).astype(np.uint8) for _ in range(3))
        assert np.array_equal(O.compose(O.compose(a, b), c), O.compose(a, O.compose(b, c)))


def _check_all_splits(fmt, s: bytes):
    """Composing the vectors of the chunks of every split of s gives s's
    vector, and its entry for the start state is the sequential end state."""
    L = len(s)
    sub = {(i, j): O.state_vector(fmt, s[i:j]) for i in range(L + 1) for j in range(i, L + 1)}
    whole = sub[(0, L)]
    for mask in range(1 << max(L - 1, 0)):
        cuts = [0] + [k + 1 for k in range(L - 1) if mask >> k & 1] + [L]
        acc = np.arange(fmt.num_states, dtype=np.uint8)
        for i, j in zip(cuts, cuts[1:]):
            acc = sub[(i, j)][acc]  # acc o chunk
        assert np.array_equal(acc, whole), (s, cuts)
    _, states = O.trace(fmt, s)
    end = states[-1] if L else fmt.start_state
    assert whole[fmt.start_state] == end


def test_every_split_csv_exhaustive():
    f = O.csv6()
    for L in range(0, 6):
        for t in itertools.product(b'\n,"\ra', repeat=L):
            _check_all_splits(f, bytes(t))


def test_every_split_log_random():
    f = O.log8()
    rng = random.Random(7)
    for _ in range(300):
        L = rng.randint(1, 8)
        _check_all_splits(f, bytes(rng.choice(b'\n "[]a') for _ in range(L)))


def test_random_splits_long_inputs():
    f = O.csv6()
    raw, _ = synth.records("mixed", 11, 0, 40)
    rng = random.Random(3)
    whole = O.state_vector(f, raw)
    for _ in range(50):
        cuts = sorted({0, len(raw), *rng.sample(range(1, len(raw)), 12)})
        acc = np.arange(6, dtype=np.uint8)
        for i, j in zip(cuts, cuts[1:]):
            acc = O.state_vector(f, raw[i:j])[acc]
        assert np.array_equal(acc, whole)


def _status(name):
    return {"ok": O.OK, "invalid": O.E_INVALID_INPUT, "unterminated": O.E_UNTERMINATED}[name]


def test_worked_examples():
    cases = json.load(open(os.path.join(GOLD, "worked_examples.json")))["cases"]
    for case in cases:
        fmt = O.csv6() if case["dialect"] == "csv" else O.log8()
        data = case["input"].encode()
        r = O.parse(fmt, [O.STRING] * case["columns"], data)
        assert r.status == _status(case["status"]), case
        if "first_invalid" in case:
            assert r.first_invalid_offset == case["first_invalid"], case
        else:
            assert r.first_invalid_offset == -1
        assert r.rows == len(case["rows"]), case
        rejected = set(case.get("rejected", []))
        assert r.n_rejected == len(rejected)
        for i, row in enumerate(case["rows"]):
            assert [r.field(i, c) for c in range(case["columns"])] == [x.encode() for x in row], case
            for c in range(case["columns"]):
                assert r.valid(i, c) == (i not in rejected)


def test_prefix_sum_example_as_string_offsets():
    """Sec. 2's prefix-sum example: fields of lengths 3 5 1 2 9 7 4 2 in one
    string column give Arrow offsets equal to its exclusive sums plus the
    total (the last inclusive sum)."""
    lines = {l.split()[0]: [int(x) for x in l.split()[1:]]
             for l in open(os.path.join(GOLD, "prefix_sum.txt")) if not l.startswith("#")}
    data = b"".join(b"x" * n + b"\n" for n in lines["x"])
    r = O.parse(O.csv6(), [O.STRING], data)
    offs = list(r.columns[0].offsets)
    assert offs[:-1] == lines["exclusive"]
    assert offs[1:] == lines["inclusive"]


def test_quote_parity_cross_check():
    """For RFC-4180 input, a non-quote byte is inside an enclosed field iff an
    odd number of double quotes precede it (the format-specific rule the
    paper avoids, Sec. 2); the DFA context must agree with it."""
    f = O.csv6()
    raw, _ = synth.records("mixed", 5, 0, 400)
    tags, states = O.trace(f, raw)
    before = np.concatenate([[f.start_state], states[:-1]])
    buf = np.frombuffer(raw, np.uint8)
    quotes = np.cumsum(buf == ord('"')) - (buf == ord('"'))
    nonq = buf != ord('"')
    assert np.array_equal((before == O.ENC)[nonq], (quotes % 2 == 1)[nonq])


# ----------------------------------------------------------- conversions

def test_int_conversion_pins():
    rng = random.Random(1)
    for _ in range(3000):
        v = rng.randint(-2**31, 2**31 - 1)
        assert O.convert(O.INT32, str(v).encode()) == (O.CONV_OK, v)
        w = rng.randint(-2**63, 2**63 - 1)
        assert O.convert(O.INT64, str(w).encode()) == (O.CONV_OK, w)
    for txt, ok in [(b"2147483647", True), (b"2147483648", False), (b"-2147483648", True),
                    (b"-2147483649", False), (b"007", True), (b"-0", True), (b"+1", False),
                    (b" 1", False), (b"1 ", False), (b"-", False), (b"1.0", False), (b"0x1", False)]:
        st, v = O.convert(O.INT32, txt)
        assert (st == O.CONV_OK) == ok, txt
        if ok:
            assert v == int(txt)
    assert O.convert(O.INT64, b"9223372036854775807") == (O.CONV_OK, 2**63 - 1)
    assert O.convert(O.INT64, b"9223372036854775808")[0] == O.CONV_FAIL
    assert O.convert(O.INT64, b"-9223372036854775808") == (O.CONV_OK, -2**63)
    assert O.convert(O.INT32, b"") == (O.CONV_EMPTY, 0)
    assert O.convert(O.INT32, b"1" * 65)[0] == O.CONV_FAIL


def test_float_conversion_matches_correct_rounding():
    """Inside the accepted range the result equals Python's correctly rounded
    decimal-to-double conversion."""
    rng = random.Random(2)
    for _ in range(20000):
        frac = rng.randint(0, 22)
        sig = rng.randint(1, 16)
        m = rng.randrange(0, 2**53)
        digits = str(m).rjust(frac + 1, "0")
        txt = (("-" if rng.random() < 0.5 else "") + digits[: len(digits) - frac] +
               ("." + digits[len(digits) - frac:] if frac else ""))
        st, v = O.convert(O.FLOAT64, txt.encode())
        assert st == O.CONV_OK, txt
        ref = float(txt)
        assert v == ref and math.copysign(1, v) == math.copysign(1, ref), txt
        del sig
    for txt, ok in [(b"1.", False), (b".5", False), (b"1e5", False), (b"-", False),
                    (b"9007199254740991", True), (b"9007199254740992", False),
                    (b"0." + b"0" * 21 + b"1", True), (b"0." + b"0" * 22 + b"1", False),
                    (b"-0.00", True), (b"00012.50", True)]:
        st, v = O.convert(O.FLOAT64, txt)
        assert (st == O.CONV_OK) == ok, txt
        if ok:
            assert v == float(txt) and math.copysign(1, v) == math.copysign(1, float(txt))


def test_date_and_timestamp_pins():
    rng = random.Random(3)
    epoch = dt.date(1970, 1, 1)
    for _ in range(3000):
        d = dt.date.fromordinal(rng.randint(dt.date(1, 1, 1).toordinal(), dt.date(9999, 12, 31).toordinal()))
        assert O.convert(O.DATE_D, d.isoformat().encode()) == (O.CONV_OK, (d - epoch).days)
        t = dt.datetime(d.year, d.month, d.day, rng.randint(0, 23), rng.randint(0, 59), rng.randint(0, 59))
        secs = calendar.timegm(t.timetuple())
        iso = f"{t.year:04d}-{t.month:02d}-{t.day:02d}T{t.hour:02d}:{t.minute:02d}:{t.second:02d}"
        assert O.convert(O.TIMESTAMP_S, iso.encode()) == (O.CONV_OK, secs)
        assert O.convert(O.TIMESTAMP_S, iso.replace("T", " ").encode()) == (O.CONV_OK, secs)
        off = rng.randint(-23 * 60, 23 * 60)
        tz = dt.timezone(dt.timedelta(minutes=off))
        ta = t.replace(tzinfo=tz)
        sign = "+" if off >= 0 else "-"
        clf = (f"{t.day:02d}/{t.strftime('%b')}/{t.year:04d}:{t.hour:02d}:{t.minute:02d}:{t.second:02d} "
               f"{sign}{abs(off) // 60:02d}{abs(off) % 60:02d}")
        assert O.convert(O.TIMESTAMP_CLF, clf.encode()) == (O.CONV_OK, int(ta.timestamp()))
    for bad in [b"2021-02-29", b"2020-13-01", b"2020-00-10", b"2020-01-32", b"0000-01-01", b"2020-1-01"]:
        assert O.convert(O.DATE_D, bad)[0] == O.CONV_FAIL, bad
    assert O.convert(O.DATE_D, b"2020-02-29")[0] == O.CONV_OK
    for bad in [b"2020-01-01 24:00:00", b"2020-01-01 00:60:00", b"2020-01-01 00:00:60", b"2020-01-01X00:00:00"]:
        assert O.convert(O.TIMESTAMP_S, bad)[0] == O.CONV_FAIL, bad
    assert O.convert(O.TIMESTAMP_CLF, b"01/Foo/2020:00:00:00 +0000")[0] == O.CONV_FAIL


# ------------------------------------------------------------- round trips

_PYCONV = {
    "int32": lambda t: int(t), "int64": lambda t: int(t), "float64": lambda t: float(t),
    "timestamp": lambda t: calendar.timegm(dt.datetime.strptime(t.decode().replace("T", " "),
                                                                "%Y-%m-%d %H:%M:%S").timetuple()),
    "date": lambda t: (dt.date.fromisoformat(t.decode()) - dt.date(1970, 1, 1)).days,
    "timestamp_clf": lambda t: int(dt.datetime.strptime(t.decode(), "%d/%b/%Y:%H:%M:%S %z").timestamp()),
}
_OTYPE = {"string": O.STRING, "int32": O.INT32, "int64": O.INT64, "float64": O.FLOAT64,
          "timestamp": O.TIMESTAMP_S, "date": O.DATE_D, "timestamp_clf": O.TIMESTAMP_CLF}


@pytest.mark.parametrize("workload,n", [("mixed", 3000), ("trip", 1500), ("review", 150), ("log", 2000)])
def test_generator_round_trip(workload, n):
    """The generator knows every field it wrote; the oracle's parse must give
    back exactly those rows, fields and (through Python's own conversions)
    values."""
    raw, truth = synth.records(workload, synth.BASE_SEED + 99, 0, n)
    schema = synth.SCHEMAS[workload]
    fmt = O.csv6() if synth.DIALECT[workload] == "csv" else O.log8()
    r = O.parse(fmt, [_OTYPE[t] for t in schema], raw)
    assert r.status == O.OK and r.rows == n and r.n_rejected == 0
    for i, rec in enumerate(truth):
        assert len(rec) == len(schema)
        for c, (t, txt) in enumerate(zip(schema, rec)):
            if t == "string":
                assert r.field(i, c) == txt
                assert r.valid(i, c)
            elif txt == b"":
                assert not r.valid(i, c) and r.field(i, c) == 0
            else:
                assert r.valid(i, c)
                assert r.field(i, c) == _PYCONV[t](txt), (i, c, txt)


def test_rejects_and_nulls():
    f = O.csv6()
    types = [O.INT32, O.STRING, O.FLOAT64]
    r = O.parse(f, types, b"1,a,2.5\n,b,\nx,c,1\n4,d\n5,e,6,7\n")
    assert r.rows == 5 and r.n_rejected == 3
    # row 0 valid; row 1 valid with two null numerics
    assert [r.valid(0, c) for c in range(3)] == [True] * 3
    assert [r.valid(1, c) for c in range(3)] == [False, True, False] and (r.row_valid[0] >> 1) & 1
    # row 2: 'x' fails int32 -> rejected; its float still holds its value
    assert not any(r.valid(2, c) for c in range(3)) and r.field(2, 2) == 1.0 and r.field(2, 0) == 0
    # row 3: too few fields; row 4: too many (extra field dropped)
    assert r.field(3, 0) == 4 and r.field(3, 1) == b"d" and r.field(3, 2) == 0.0
    assert r.field(4, 0) == 5 and r.field(4, 2) == 6.0
    assert [(r.row_valid[0] >> k) & 1 for k in range(5)] == [1, 1, 0, 0, 0]


def test_bytes_total_counts_dropped_partial_record():
    r = O.parse(O.csv6(), [O.STRING, O.STRING], b'ab,c\nde,"f')
    assert r.status == O.E_UNTERMINATED and r.rows == 1
    assert r.columns[0].bytes_total == 4 and r.columns[1].bytes_total == 2


# ---------------------------------------------- Sec. 4.3: type inference

@pytest.mark.parametrize("raw,records,mn,mx,types", [
    (b"1,2.5,x\n3,4,y\n", 2, 3, 3, [O.INT32, O.FLOAT64, O.STRING]),    # widest of each position
    (b"1\n2,3\n", 2, 1, 2, [O.INT32, O.INT32]),                         # ragged records
    (b"2147483648,1\n", 1, 2, 2, [O.INT64, O.INT32]),                   # 2^31 needs int64
    (b"-5,,abc\n", 1, 3, 3, [O.INT32, O.NO_TYPE, O.STRING]),            # empty: no type
    (b"1.5e3,007\n", 1, 2, 2, [O.STRING, O.INT32]),                     # no exponent syntax
    (b"99999999999999999999,1\n", 1, 2, 2, [O.STRING, O.INT32]),        # beyond int64 and 2^53
    (b'"12",""\n', 1, 2, 2, [O.INT32, O.NO_TYPE]),                      # quotes are not data
    (b"a,b", 1, 2, 2, [O.STRING, O.STRING]),                            # trailing record
    (b"", 0, 0, 0, []),
])
def test_inference_worked_examples(raw, records, mn, mx, types):
    r = O.infer(O.csv6(), raw)
    assert (r.status, r.records, r.min_fields, r.max_fields) == (O.OK, records, mn, mx)
    assert r.types[: len(types)] == types and all(t == O.NO_TYPE for t in r.types[len(types):])


def test_inference_saturates_the_field_count():
    r = O.infer(O.csv6(), b",".join(b"%d" % i for i in range(300)) + b"\n1\n")
    assert (r.min_fields, r.max_fields) == (1, O.INFER_MAX_FIELDS)
    assert r.types[:64] == [O.INT32] * 64  # only the first 64 positions are typed


@pytest.mark.parametrize("workload", ["mixed", "trip", "review", "log"])
def test_inference_agrees_with_the_schema_and_the_parse(workload):
    # the generator writes every record with the schema's field count, and a
    # parse with the inferred types (no type -> string) rejects nothing
    raw, _ = synth.records(workload, 41, 0, 400)
    fmt = O.csv6() if synth.DIALECT[workload] == "csv" else O.log8()
    r = O.infer(fmt, raw)
    C = len(synth.SCHEMAS[workload])
    assert r.status == O.OK and r.records == 400 and r.min_fields == r.max_fields == C
    types = [O.STRING if t == O.NO_TYPE else t for t in r.types[:C]]
    assert O.parse(fmt, types, raw).n_rejected == 0
    if workload == "trip":  # columns the generator writes as small integers and 2-decimal floats
        assert types[0] == O.INT32 and types[4] == O.FLOAT64 and types[1] == O.STRING


def test_skipped_columns_count_but_keep_nothing():
    # Sec. 4.3, selecting columns: a skipped column's fields still count for
    # the record's field count; every other column is as if it were kept
    raw = b'1,xx,a\n2,"y,y",b\n3\n4,zz,c,9\n5,,d\n'
    full = O.parse(O.csv6(), [O.INT32, O.STRING, O.STRING], raw)
    skip = O.parse(O.csv6(), [O.INT32, O.SKIP, O.STRING], raw)
    assert (skip.rows, skip.n_rejected) == (full.rows, full.n_rejected) == (5, 2)
    assert skip.columns[1].values.size == 0 and skip.columns[1].bytes_total == 0
    for c in (0, 2):
        assert np.array_equal(skip.columns[c].validity, full.columns[c].validity)
        assert [skip.field(r, c) for r in range(5)] == [full.field(r, c) for r in range(5)]
    assert np.array_equal(skip.row_valid, full.row_valid)


@pytest.mark.parametrize("workload,n", [("mixed", 400), ("trip", 300), ("review", 40), ("log", 300)])
def test_skipped_records_equal_the_input_without_them(workload, n):
    # Sec. 4.3, skipping records: skipping the first k records gives what
    # parsing the input with those records' bytes cut off gives (each record
    # ends in the start state, so the cut loses no context)
    raw, _ = synth.records(workload, synth.BASE_SEED + 5, 0, n)
    dialect = synth.DIALECT[workload]
    fmt = O.csv6() if dialect == "csv" else O.log8()
    types = [_OTYPE[t] for t in synth.SCHEMAS[workload]]
    for k in (0, 1, 5, n - 1, n, n + 3):
        cut = _record_start(raw, dialect, k)
        a = O.parse(fmt, types, raw, skip_records=k)
        b = O.parse(fmt, types, raw[cut:])
        assert a.rows == max(n - k, 0)
        assert (a.rows, a.n_rejected, a.status) == (b.rows, b.n_rejected, b.status), k
        for c in range(len(types)):
            assert np.array_equal(a.columns[c].validity, b.columns[c].validity), (k, c)
            assert a.columns[c].bytes_total == b.columns[c].bytes_total, (k, c)
            assert [a.field(r, c) for r in range(a.rows)] == [b.field(r, c) for r in range(b.rows)], (k, c)
        assert np.array_equal(a.row_valid, b.row_valid), k


def _record_start(raw: bytes, dialect: str, n: int) -> int:
    """Byte offset where record n starts, found by a quote-aware scan written
    apart from the oracle (CSV: a newline outside double quotes ends a record;
    the web log: a newline outside quotes and brackets)."""
    quoted = bracket = False
    seen = 0
    if n == 0:
        return 0
    for i, ch in enumerate(raw):
        if ch == 0x22:
            quoted = not quoted
        elif dialect != "csv" and not quoted and ch in (0x5B, 0x5D):
            bracket = ch == 0x5B
        elif ch == 0x0A and not quoted and not bracket:
            seen += 1
            if seen == n:
                return i + 1
    return len(raw)


def test_skipped_records_leave_no_rejects_and_keep_validation():
    # a malformed record that is skipped is not rejected, while an invalid
    # byte inside a skipped record still fails the input
    raw = b'1\n2,b\n3,c\n'
    assert O.parse(O.csv6(), [O.INT32, O.STRING], raw).n_rejected == 1
    s = O.parse(O.csv6(), [O.INT32, O.STRING], raw, skip_records=1)
    assert (s.rows, s.n_rejected) == (2, 0) and s.field(0, 1) == b'b'
    bad = b'1,"x"y\n2,b\n'
    a = O.parse(O.csv6(), [O.INT32, O.STRING], bad)
    b = O.parse(O.csv6(), [O.INT32, O.STRING], bad, skip_records=1)
    assert a.status == b.status != 0 and a.first_invalid_offset == b.first_invalid_offset


def test_inference_skips_a_header_record():
    # a header row makes every column a string; skipped (Sec. 4.3), the
    # types are those of the body, as if the header were cut off
    body = b'1,a,2.5\n70000000000,"b,c",3\n,d,-1000.5\n'
    raw = b'id,name,score\n' + body
    s = O.infer(O.csv6(), raw)
    assert s.types[:3] == [O.STRING] * 3 and s.records == 4
    k = O.infer(O.csv6(), raw, skip_records=1)
    b = O.infer(O.csv6(), body)
    assert k.types[:3] == [O.INT64, O.STRING, O.FLOAT64] and k.records == 3
    assert (k.types, k.records, k.min_fields, k.max_fields, k.status) == \
        (b.types, b.records, b.min_fields, b.max_fields, b.status)
    assert O.infer(O.csv6(), raw, skip_records=9).records == 0


def _lines_without(raw: bytes, rows, term: bytes = b"\n") -> bytes:
    """The definition of skipping rows written with bytes.split: a row is a
    physical line with its terminator; the last one may lack it."""
    parts = raw.split(term)
    lines = [p + term for p in parts[:-1]] + ([parts[-1]] if parts[-1] else [])
    drop = set(rows)
    return b"".join(line for i, line in enumerate(lines) if i not in drop)


def test_skip_rows_matches_the_line_split_definition():
    # Sec. 4.3, skipping rows: the pruning pass against bytes.split
    rng = random.Random(11)
    for it in range(400):
        term = b"\n" if it % 3 else b";"
        raw = bytes(rng.choice(b'ab"\n,;') for _ in range(rng.randint(0, 300)))
        nl = raw.count(term) + 1
        rows = sorted(rng.sample(range(nl + 3), rng.randint(0, min(nl + 3, 12))))
        assert O.skip_rows(raw, rows, term[0]) == _lines_without(raw, rows, term), (it, raw, rows)


def test_skip_rows_is_not_skip_records():
    # rows are physical lines: dropping a header row equals skipping the
    # header record, but dropping a row inside a quoted field breaks the record
    body = b'1,"x\ny"\n2,z\n'
    raw = b"id,name\n" + body
    a = O.parse(O.csv6(), [O.INT32, O.STRING], O.skip_rows(raw, [0]))
    b = O.parse(O.csv6(), [O.INT32, O.STRING], raw, skip_records=1)
    assert (a.rows, a.field(0, 1), a.field(1, 1)) == (b.rows, b.field(0, 1), b.field(1, 1)) == (2, b"x\ny", b"z")
    c = O.parse(O.csv6(), [O.INT32, O.STRING], O.skip_rows(raw, [1]))  # leaves 'y",..' : a stray quote
    assert c.status == O.E_INVALID_INPUT


# ------------------------------------------------ Sec. 4.2: UTF-16 symbols

_TEXT_ALPHABET = ["a", "b", "z", "1", " ", "é", "ß", "€", "漢", "字", "😀", "🚀", "𝄞"]


def _random_utf8_csv(rng, records):
    """Records of [int32, string, string, float64] whose strings hold
    multi-byte and astral characters, some quoted with delimiters inside."""
    lines = []
    for _ in range(records):
        def text():
            s = "".join(rng.choice(_TEXT_ALPHABET) for _ in range(rng.randint(0, 8)))
            if rng.random() < 0.4:
                return '"' + s.replace('"', '""') + rng.choice(["", ",", "\n", '""']) + '"'
            return s
        lines.append(f"{rng.randint(-99, 999)},{text()},{text()},{rng.randint(0, 999)}.{rng.randint(0, 99):02d}\n")
    return "".join(lines)


def test_utf16_parse_equals_the_utf8_parse_transcoded():
    """Sec. 4.2 pinned against Python's own codecs: a CSV input parsed as
    UTF-16LE code units gives the rows, statuses, numbers and validity of the
    same input parsed as UTF-8 bytes, and each string field's UTF-16LE bytes
    decode to the same text as its UTF-8 bytes."""
    rng = random.Random(42)
    f8, f16 = O.csv6(), O.csv6().as_utf16le()
    types = [O.INT32, O.STRING, O.STRING, O.FLOAT64]
    for it in range(40):
        text = _random_utf8_csv(rng, rng.randint(1, 30))
        if it % 5 == 4:  # an invalid input: a quote inside an unquoted field
            cut = rng.randrange(len(text))
            text = text[:cut] + 'x"' + text[cut:]
        r8 = O.parse(f8, types, text.encode("utf-8"))
        r16 = O.parse(f16, types, text.encode("utf-16-le"))
        assert (r16.status, r16.rows, r16.n_rejected, r16.final_state) == (r8.status, r8.rows, r8.n_rejected,
                                                                           r8.final_state)
        if r8.first_invalid_offset >= 0:  # the same code point, counted in each encoding's bytes
            cp = len(text.encode("utf-8")[: r8.first_invalid_offset].decode("utf-8"))
            assert r16.first_invalid_offset == len(text[:cp].encode("utf-16-le"))
        for c, t in enumerate(types):
            assert np.array_equal(r16.columns[c].validity, r8.columns[c].validity)
            for r in range(r8.rows):
                if t == O.STRING:
                    assert r16.field(r, c).decode("utf-16-le") == r8.field(r, c).decode("utf-8")
                else:
                    assert r16.field(r, c) == r8.field(r, c)
        assert np.array_equal(r16.row_valid, r8.row_valid)


def test_utf16_numeric_text_must_be_ascii():
    f16 = O.csv6().as_utf16le()
    raw = "12,x\n１２,y\n".encode("utf-16-le")  # the second number uses fullwidth digits
    r = O.parse(f16, [O.INT32, O.STRING], raw)
    assert r.rows == 2 and r.n_rejected == 1
    assert r.field(0, 0) == 12 and not r.valid(1, 0)


def test_utf16_chunk_vectors_compose_at_every_split():
    """Sec. 4.2 with Sec. 3.1: chunk vectors (a chunk skips the low half of a
    surrogate pair begun in the previous chunk) compose to the whole input's
    vector at every code-unit boundary, also inside surrogate pairs."""
    rng = random.Random(7)
    f16 = O.csv6().as_utf16le()
    alphabet = [",", "\n", '"', "\r", "a", "é", "😀", "𝄞"]
    for _ in range(60):
        text = "".join(rng.choice(alphabet) for _ in range(rng.randint(1, 12)))
        raw = text.encode("utf-16-le")
        n = len(raw)
        whole = O.state_vector_at(f16, raw, 0, n)
        seq = O.state_vector(O.csv6(), b"")  # identity
        assert len(whole) == len(seq)
        for k in range(0, n + 1, 2):
            a, b = O.state_vector_at(f16, raw, 0, k), O.state_vector_at(f16, raw, k, n)
            assert np.array_equal(O.compose(a, b), whole), (text, k)
        for k1 in range(2, n, 2):  # three chunks
            k2 = min(n, k1 + 2 * rng.randint(1, 3))
            v = O.compose(O.compose(O.state_vector_at(f16, raw, 0, k1), O.state_vector_at(f16, raw, k1, k2)),
                          O.state_vector_at(f16, raw, k2, n))
            assert np.array_equal(v, whole), (text, k1, k2)


def test_utf16_whole_vector_is_the_sequential_run():
    """The whole input's vector is, per start state, the state where the
    sequential parse of the UTF-8 form ends (the symbol sequences agree)."""
    rng = random.Random(8)
    for _ in range(30):
        text = "".join(rng.choice([",", "\n", '"', "a", "é", "😀"]) for _ in range(rng.randint(1, 15)))
        v16 = O.state_vector_at(O.csv6().as_utf16le(), text.encode("utf-16-le"), 0, len(text.encode("utf-16-le")))
        v8 = O.state_vector(O.csv6(), text.encode("utf-8"))
        assert np.array_equal(v16, v8), text


def test_utf16_reads_a_surrogate_pair_as_one_symbol():
    """With a DFA whose catch-all flips between two states, the final state
    is the parity of the number of code points (Python's count), not of the
    code units: a surrogate pair is one symbol (Sec. 4.2)."""
    nxt = np.array([[1, 0]], np.uint8)  # one group, the catch-all: toggle
    emt = np.zeros((1, 2), np.uint8)
    f16 = O.Format(2, 1, nxt, emt, b"", [], 0, 0, 0xFF, 3, True)
    rng = random.Random(9)
    for _ in range(50):
        text = "".join(rng.choice(["a", "é", "😀", "𝄞", "漢"]) for _ in range(rng.randint(0, 9)))
        raw = text.encode("utf-16-le")
        assert O.state_vector_at(f16, raw, 0, len(raw))[0] == len(text) % 2, text
        r = O.parse(f16, [O.STRING], raw)
        assert r.final_state == len(text) % 2
