"""Parity at the benchmark's full sizes, in the launch configuration the
benchmark times, element by element against the oracle.

- the exact 1e6-byte mixed CSV input of the latency line, compared whole;
- the 1e9-byte trip-like CSV and the 4.8e9-byte review-like CSV, tile shape
  picked by the autotuner on the resident input (as the benchmark picks it),
  one plain parse each: every record is compared.  The output is too
  large for one oracle run, so the oracle parses the input in pieces of whole
  records (record i of a workload depends only on the seed and i, and a piece
  starts in the start state after a record delimiter, so its parse is rows
  [r0, r1) of the whole parse); the pieces run on all host cores;
- the 10,000-input batch (~6e9 bytes, half CSV, half web logs), tile shape
  picked by the autotuner, one prepared persistent launch: every input is
  compared whole.

Properties that hold at any size (row count equal to the generator's, monotone
offsets ending at the reported byte totals) are checked as well.
"""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import synth
from parity import assert_rows_equal, assert_same, oracle_parse

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

WORKERS = max(1, min(32, os.cpu_count() or 1))


def ordered_map(fn, args):
    """fn over args on WORKERS threads (the oracle and the generator release
    the GIL), results in order, at most 2 * WORKERS of them held at once."""
    args = list(args)
    with ThreadPoolExecutor(WORKERS) as ex:
        futs = [ex.submit(fn, a) for a in args[: 2 * WORKERS]]
        for k in range(len(args)):
            r = futs[k].result()
            futs[k] = None
            if k + 2 * WORKERS < len(args):
                futs.append(ex.submit(fn, args[k + 2 * WORKERS]))
            yield r


@pytest.fixture(scope="module")
def pp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    import paper_1905_13415_gb300 as pkg

    return pkg


def test_mixed_1mb_bench_input(pp):
    """The 1e6-byte input whose parse latency the benchmark reports, whole."""
    seed = synth.BASE_SEED + 1
    raw = synth.generate("mixed", seed, 1_000_000).tobytes()
    schema = synth.SCHEMAS["mixed"]
    p = pp.Parser(pp.formats.by_name("csv"), schema)
    data = torch.frombuffer(bytearray(raw), dtype=torch.uint8).cuda()
    out, res = p.parse(data)
    ref = oracle_parse("csv", schema, raw)
    assert ref.status == 0 and ref.rows > 10_000
    assert_same(out.to_host(res.rows), res, ref, what="mixed 1e6")


@pytest.mark.parametrize("workload,seed_off,size,piece",
                         [("trip", 2, 1_000_000_000, 200_000), ("review", 3, 4_800_000_000, 100_000)])
def test_full_size_every_record(pp, workload, seed_off, size, piece):
    seed = synth.BASE_SEED + seed_off
    schema, dialect = synth.SCHEMAS[workload], synth.DIALECT[workload]
    host = torch.empty(size, dtype=torch.uint8, pin_memory=True)
    n, rows = synth.generate_into(workload, seed, size, host.data_ptr(), size)
    data = host[:n].to("cuda")
    del host
    p = pp.Parser(pp.formats.by_name(dialect), schema)
    out = p.allocate(rows + 16, [n] * len(schema))
    from paper_1905_13415_gb300.autotune import autotune_plain

    autotune_plain(p, data, out, reps=3)  # the tile shape the benchmark picks the same way
    p.parse_into(data, out)
    torch.cuda.synchronize()
    res = out.result()
    assert res.status == 0 and res.rows == rows and res.n_rejected == 0, res
    for c, t in enumerate(out.types):
        if out.offsets[c] is not None:
            offs = out.offsets[c][: rows + 1]
            assert int(offs[0]) == 0
            assert bool((offs[1:] >= offs[:-1]).all()), c
            assert int(offs[rows]) == int(res.values_bytes_needed[c]), c

    def oracle_piece(r0):
        r1 = min(r0 + piece, rows)
        raw = synth.record_bytes(workload, seed, r0, r1 - r0)
        return r1, len(raw), oracle_parse(dialect, schema, raw)

    covered = 0
    for r0, (r1, nbytes, ref) in zip(range(0, rows, piece), ordered_map(oracle_piece, range(0, rows, piece))):
        assert ref.status == 0, (workload, r0)
        assert_rows_equal(out, r0, r1, ref, what=(workload, r0, r1))
        covered += nbytes
    assert covered == n  # the pieces are exactly the input
    del out, data
    torch.cuda.empty_cache()


def test_full_size_batch(pp):
    from paper_1905_13415_gb300 import Batch, Parser, formats
    from paper_1905_13415_gb300.autotune import autotune

    n_inputs, total = 10_000, 6_000_000_000
    sizes, kinds, seeds = synth.batch_plan(n_inputs, total, synth.BASE_SEED + 4)
    host = torch.empty(int(sizes.sum()), dtype=torch.uint8, pin_memory=True)
    offs, lens, rows = synth.generate_batch_into(kinds, seeds, sizes, host.data_ptr())
    data = host.to("cuda")
    parsers = {k: Parser(formats.by_name(synth.DIALECT[k]), synth.SCHEMAS[k]) for k in ("mixed", "log")}
    items = []
    for i in range(n_inputs):
        p = parsers[kinds[i]]
        d = data[int(offs[i]): int(offs[i]) + int(lens[i])]
        out = p.allocate(max(int(rows[i]), 1), [max(int(lens[i]), 1)] * len(p.types))
        items.append((p, d, out))
    rng = np.random.default_rng(7)
    autotune([items[i] for i in sorted(rng.choice(n_inputs, size=400, replace=False))], reps=2)
    b = Batch(items)
    b.launch()
    torch.cuda.synchronize()
    b.close()
    hv = host.numpy()

    def oracle_input(i):
        raw = hv[int(offs[i]): int(offs[i]) + int(lens[i])]
        return oracle_parse(synth.DIALECT[kinds[i]], synth.SCHEMAS[kinds[i]], raw)

    for i, ref in enumerate(ordered_map(oracle_input, range(n_inputs))):  # every input, compared whole
        p, d, out = items[i]
        res = out.result()
        assert res.status == 0 and res.rows == int(rows[i]) and res.n_rejected == 0, (i, res)
        assert_same(out.to_host(res.rows), res, ref, what=f"batch input {i}")
    del items, data
    torch.cuda.empty_cache()
