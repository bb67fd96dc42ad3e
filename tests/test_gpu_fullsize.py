"""Parity at the benchmark's full sizes, in the launch configuration the
benchmark times.

- the 1e9-byte trip-like CSV and the 4.8e9-byte review-like CSV, default tile
  shape, one plain parse each;
- the 10,000-input batch (~6e9 bytes, half CSV, half web logs), tile shape
  picked by the autotuner, one prepared persistent launch.

These outputs are too large for the oracle as a whole, so every sampled
record is regenerated alone (record i of a workload depends only on the seed
and i) and parsed by the oracle, and compared field by field with row i of the
GPU output; the properties that hold at any size (row count equal to the
generator's, monotone offsets that end at the reported byte totals, no
rejects, every value valid) are checked on the whole output.  Sampled batch
inputs are compared whole with the oracle.
"""
from __future__ import annotations

import numpy as np
import pytest

import synth
from parity import assert_same, oracle_parse

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SAMPLES = 1500


@pytest.fixture(scope="module")
def pp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    import paper_1905_13415_gb300 as pkg

    return pkg


def _bit(bm: torch.Tensor, rows: torch.Tensor) -> np.ndarray:
    r = rows.to(bm.device)
    return ((bm[r >> 3] >> (r & 7)) & 1).cpu().numpy().astype(bool)


@pytest.mark.parametrize("workload,seed_off,size", [("trip", 2, 1_000_000_000), ("review", 3, 4_800_000_000)])
def test_full_size_sampled_records(pp, workload, seed_off, size):
    seed = synth.BASE_SEED + seed_off
    schema, dialect = synth.SCHEMAS[workload], synth.DIALECT[workload]
    host = torch.empty(size, dtype=torch.uint8, pin_memory=True)
    n, rows = synth.generate_into(workload, seed, size, host.data_ptr(), size)
    data = host[:n].to("cuda")
    del host
    p = pp.Parser(pp.formats.by_name(dialect), schema)  # the default shape, as benchmarked
    out = p.allocate(rows + 16, [n] * len(schema))
    p.parse_into(data, out)
    torch.cuda.synchronize()
    res = out.result()
    assert res.status == 0 and res.rows == rows and res.n_rejected == 0, res
    assert res.first_invalid_offset == -1 or res.first_invalid_offset >= n

    # properties of the whole output
    nb = (rows + 7) // 8
    full = torch.full((nb,), 0xFF, dtype=torch.uint8, device="cuda")
    if rows % 8:
        full[-1] = (1 << (rows % 8)) - 1
    assert torch.equal(out.row_valid[:nb], full)
    for c, t in enumerate(out.types):
        assert torch.equal(out.validity[c][:nb], full), c
        if out.offsets[c] is not None:
            offs = out.offsets[c][: rows + 1]
            assert int(offs[0]) == 0
            assert bool((offs[1:] >= offs[:-1]).all()), c
            assert int(offs[rows]) == int(res.values_bytes_needed[c]), c

    # sampled records against the oracle, each parsed alone
    rng = np.random.default_rng(seed)
    sample = np.unique(np.concatenate([[0, rows - 1], rng.choice(rows, size=min(SAMPLES, rows), replace=False)]))
    idx = torch.from_numpy(sample.astype(np.int64))
    got_cols = []
    for c, t in enumerate(out.types):
        if out.offsets[c] is not None:
            lo = out.offsets[c][idx.cuda()].cpu().numpy()
            hi = out.offsets[c][(idx + 1).cuda()].cpu().numpy()
            vals = out.values[c]
            got_cols.append([bytes(vals[int(a):int(b)].cpu().numpy()) for a, b in zip(lo, hi)])
        else:
            got_cols.append(out.values[c][idx.cuda()].cpu().numpy())
    valid = [_bit(out.validity[c], idx) for c in range(len(out.types))]
    for k, i in enumerate(sample):
        raw, _ = synth.records(workload, seed, int(i), 1)
        ref = oracle_parse(dialect, schema, raw)
        assert ref.rows == 1 and ref.status == 0
        for c, col in enumerate(ref.columns):
            if col.offsets is not None:
                assert got_cols[c][k] == ref.field(0, c), (workload, int(i), c)
            else:
                assert got_cols[c][k].tobytes() == col.values[:1].tobytes(), (workload, int(i), c)
            assert valid[c][k] == bool(col.validity[0] & 1), (workload, int(i), c)
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
    for i, (p, d, out) in enumerate(items):
        res = out.result()
        assert res.status == 0 and res.rows == int(rows[i]) and res.n_rejected == 0, (i, res)
    # the smallest, the largest and a sample in between, each compared whole
    order = np.argsort(lens)
    pick = sorted({int(order[0]), int(order[-1]), *map(int, rng.choice(n_inputs, size=10, replace=False))})
    for i in pick:
        if int(lens[i]) > 300_000_000:
            continue
        p, d, out = items[i]
        raw = host[int(offs[i]): int(offs[i]) + int(lens[i])].numpy().tobytes()
        res = out.result()
        ref = oracle_parse(synth.DIALECT[kinds[i]], synth.SCHEMAS[kinds[i]], raw)
        assert_same(out.to_host(res.rows), res, ref, what=f"batch input {i}")
    del items, data
    torch.cuda.empty_cache()
