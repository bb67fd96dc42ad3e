#!/usr/bin/env python3
"""Benchmark: raw-input parse GB/s on device and its HBM roofline fraction.

Default workload: the 4.8e9-byte review-like CSV (9 columns, always-quoted
text of mean 700 B with commas, line breaks and doubled quotes), a seeded
synthetic stand-in for the yelp reviews dataset.  One step = one whole
parse (init, tile and finalize kernels) of the resident input.

Prints one JSON line (rank 0).  --impl reference times the oracle (the plain
sequential CPU parser) on the host cores instead.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (synth workload, seed offset, default bytes, description)
    "review": ("review", 3, 4_800_000_000,
               "review-like CSV (yelp-like), 9 columns, quoted text mean 700 B, LF"),
    "trip": ("trip", 2, 1_000_000_000, "trip-record CSV (NYC-taxi-like), 18 columns, CRLF, no quotes"),
    "mixed": ("mixed", 1, 1_000_000, "RFC-4180 CSV, 8 mixed columns, 30% quoted strings"),
}


def csv_hash_of_sources() -> str:
    """Hash of the sources the parse is built from (the row-pruning pre-pass,
    a separate unit that the parse never runs, is left out)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1905_13415_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        if f == "pp_rows.cu":
            continue
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def measured_peak_gbs():
    try:
        d = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def recorded_traffic(workload: str, tile_config: int):
    """DRAM bytes per launch of the tile kernel from the committed ncu
    summary, if it was taken on the current kernel sources with the same
    tile shape."""
    path = os.path.join(ROOT, "profiles", "pp_tile_kernel_traffic.txt")
    if not os.path.exists(path):
        return None
    src = csv_hash_of_sources()
    for line in open(path):
        parts = line.split()
        if (len(parts) >= 5 and not line.startswith("#") and parts[0] == workload and parts[1] == src
                and parts[2] == str(tile_config)):
            return {"bytes_per_launch": float(parts[3]), "scaled_from": " ".join(parts[4:])}
    return None


class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [l.strip().split(",") for l in self.file if l.strip()]
        os.unlink(self.file.name)
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = max(mx, float(r[2]))
            except (ValueError, IndexError):
                continue
            for name, v in zip(names, r[4:8]):
                if v.strip().lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(backend: str = "nccl"):
    """One process per GPU (torchrun): each rank parses its own replica of the
    workload; the ranks only agree on the timing."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group(backend)
    return world, rank, local


def max_over_ranks(values, world: int, device):
    """Each timing's maximum over the ranks: the slowest replica sets the step."""
    if world <= 1:
        return [float(v) for v in values]
    import torch

    t = torch.tensor([float(v) for v in values], device=device, dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return [float(x) for x in t]


def whole_job_rate(world: int, bytes_per_rank: int, step_ms: float) -> float:
    """GB/s of all replicas together (every rank parses bytes_per_rank per step)."""
    return world * bytes_per_rank / (step_ms * 1e-3) / 1e9


def oracle_rate(workload_name: str, raw_sample, schema, dialect):
    """Times the oracle (single thread) on a sample; returns (GB/s, seconds)."""
    import oracle
    from tests.parity import OTYPE

    fmt = oracle.csv6() if dialect == "csv" else oracle.log8()
    t0 = time.perf_counter()
    r = oracle.parse(fmt, [OTYPE[t] for t in schema], raw_sample)
    dt = time.perf_counter() - t0
    assert r.status == 0
    return len(raw_sample) / dt / 1e9, dt


def run_reference(args):
    """--impl reference: the oracle as it stands, on the host cores."""
    import numpy as np

    import synth

    world, rank, _ = int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")), 0
    if rank != 0:
        return 0
    wl, seed_off, default_n, desc = WORKLOADS[args.workload]
    sample = min(args.size or default_n, args.ref_sample)
    raw = synth.generate(wl, synth.BASE_SEED + seed_off, sample)
    schema, dialect = synth.SCHEMAS[wl], synth.DIALECT[wl]
    for _ in range(args.warmup):
        oracle_rate(wl, raw, schema, dialect)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_rate(wl, raw, schema, dialect)
    dt = time.perf_counter() - t0
    value = args.steps * len(raw) / dt / 1e9
    line = {
        "impl": "reference", "metric": "raw-input parse GB/s", "value": round(value, 4), "unit": "GB/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(dt / args.steps * 1e3, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": desc, "input_bytes": args.size or default_n,
                   "sample_bytes_per_step": len(raw)},
        "cpu_baseline": {"value": round(value, 4), "unit": "GB/s", "cores": 1, "kind": "oracle",
                         "sample": f"first {len(raw)} bytes (whole records) of the workload per step"},
        "e2e": {"value": round(value, 4), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def _bits_of(bm, n: int):
    import numpy as np

    return np.unpackbits(np.asarray(bm, np.uint8), bitorder="little")[:n]


def output_digest_parts(pieces, types) -> list:
    """Per column, SHA-256 of its logical content over a sequence of row
    ranges [(rows, columns dict list, row_valid)]: string bytes and field
    lengths, fixed-width values, validity bits; then row_valid bits."""
    import numpy as np

    # one hash per stream (values, field lengths, validity) of each column
    hs = [[hashlib.sha256() for _ in range(3)] for _ in range(len(types))] + [[hashlib.sha256()]]
    for rows, cols, row_valid in pieces:
        for c, t in enumerate(types):
            col = cols[c]
            if col["values"] is None:
                continue
            if col["offsets"] is not None:
                offs = np.asarray(col["offsets"][: rows + 1], np.int64)
                hs[c][0].update(np.asarray(col["values"][int(offs[0]): int(offs[-1])], np.uint8).tobytes())
                hs[c][1].update(np.diff(offs).tobytes())
            else:
                hs[c][0].update(np.asarray(col["values"][:rows]).tobytes())
            hs[c][2].update(_bits_of(col["validity"], rows).tobytes())
        hs[-1][0].update(_bits_of(row_valid, rows).tobytes())
    return ["/".join(h.hexdigest()[:16] for h in col) for col in hs]


def output_digest_device(out, rows: int) -> list:
    """output_digest_parts of a device Output (copied to the host)."""
    h = out.to_host(rows)
    return output_digest_parts([(rows, h["columns"], h["row_valid"])], out.types)


def output_digest_partitions(parts, types) -> list:
    """output_digest_parts of a streamed parse's host partitions."""
    pieces = []
    for x in parts:
        cols = [{k: (v.numpy() if v is not None else None) for k, v in col.items()} for col in x.columns]
        pieces.append((x.rows, cols, x.row_valid.numpy()))
    return output_digest_parts(pieces, types)


def roofline_line(algo_bytes: int, kern_ms: float, peak: float, peak_kind: str, traffic=None) -> dict:
    """HBM roofline of the tile kernel: algorithmic bytes (input read once +
    the exact output layout) over the kernel's CUDA-event time."""
    achieved = algo_bytes / (kern_ms * 1e-3) / 1e9
    return {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "peak_kind": peak_kind, "kernel": "pp_tile_kernel",
            "kernel_ms": round(kern_ms, 4), "algorithmic_bytes": int(algo_bytes), "traffic": traffic}


def pick_tile_shape(args, parser, data, out) -> dict:
    """The tile shape of a plain-parse line: --tile-config when given, else
    the autotuner's pick (every candidate shape times a parse of the resident
    input before the timed region)."""
    from paper_1905_13415_gb300.autotune import autotune_plain

    if args.tile_config:
        return {"tile_config": args.tile_config, "tile_shape": "fixed by --tile-config"}
    best, ms = autotune_plain(parser, data, out, reps=3)
    return {"tile_config": best, "tile_shape": "autotuned on the resident input",
            "autotune_ms": {str(k): round(v, 3) for k, v in ms.items()}}


def run_other_configs(args, dev, log):
    """The two other plain-parse configurations: the 1 MB mixed CSV (latency of
    one parse: median of many, inputs resident) and the 1e9-byte trip-record
    CSV (GB/s, timed like the main workload)."""
    import numpy as np
    import torch

    import synth
    from paper_1905_13415_gb300 import Parser, formats

    out = {}
    stream = torch.cuda.current_stream()
    for name, size, reps in (("mixed", 1_000_000, 200), ("trip", 1_000_000_000, 10)):
        wl, seed_off, _, desc = WORKLOADS[name]
        host = torch.empty(size, dtype=torch.uint8, pin_memory=True)
        n, rows = synth.generate_into(wl, synth.BASE_SEED + seed_off, size, host.data_ptr(), size)
        data = host[:n].to(dev)
        p = Parser(formats.by_name(synth.DIALECT[wl]), synth.SCHEMAS[wl], tile_config=args.tile_config)
        o, res = p.parse(data, rows_cap=rows + 16)
        assert res.status == 0 and res.rows == rows, (name, res)
        o = p.allocate(rows + 16, [max(int(b), 1) for b in res.values_bytes_needed], device=dev)
        tuned = pick_tile_shape(args, p, data, o)
        for _ in range(3):
            p.parse_into(data, o, stream=stream)
        ms, kms = [], []
        ks, kt = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for ev in (ks, kt):
            ev.record(stream)
        p.set_kernel_events(ks, kt)
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            p.parse_into(data, o, stream=stream)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            kms.append(ks.elapsed_time(kt))
        p.set_kernel_events(None, None)
        med, kmed = float(np.median(ms)), float(np.median(kms))
        algo = n + o.output_bytes(rows)
        peak, peak_kind = measured_peak_gbs()
        out[name] = {"workload": desc, "input_bytes": n, "rows": rows, **tuned, "ms_median": round(med, 4),
                     "GB/s": round(n / (med * 1e-3) / 1e9, 3), "runs": reps,
                     "note": "one parse (init, tile, finalize kernels) per run, input resident",
                     "roofline": roofline_line(algo, kmed, peak, peak_kind,
                                               (recorded_traffic(name, tuned["tile_config"]) or {}).get("bytes_per_launch")
                                               if size == WORKLOADS[name][2] else None)}
        log(f"{name}: {n} B in {med:.3f} ms (median of {reps})")
        if name == "trip":  # column-count and type inference over the same input (Sec. 4.3)
            inf = p.infer(data)
            assert inf.status == 0 and inf.records == rows
            t = []
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                p.infer(data, stream=stream)  # includes reading the 96-byte result back
                e1.record(stream)
                e1.synchronize()
                t.append(e0.elapsed_time(e1))
            imed = float(np.median(t))
            out["trip_infer"] = {"input_bytes": n, "ms_median": round(imed, 4),
                                 "GB/s": round(n / (imed * 1e-3) / 1e9, 3), "runs": reps,
                                 "min_fields": inf.min_fields, "max_fields": inf.max_fields}
            out["trip_skip_rows"] = time_skip_rows(data, rows, reps, stream)
        del o, data, host
        torch.cuda.empty_cache()
    return out


def time_skip_rows(data, rows, reps, stream):
    """Skipping rows (Sec. 4.3) over a resident input: every 100th line
    dropped by the pruning pre-pass (parparaw_skip_rows), buffers allocated
    once, device time of the pass alone."""
    import numpy as np
    import torch

    from paper_1905_13415_gb300 import _abi

    lib = _abi.load()
    n = data.numel()
    drop = torch.arange(0, rows, 100, dtype=torch.int64, device=data.device)
    outb = torch.empty(n, dtype=torch.uint8, device=data.device)
    out_len = torch.zeros(1, dtype=torch.int64, device=data.device)
    sb = int(lib.parparaw_skip_rows_scratch_bytes(n))
    scratch = torch.empty(sb, dtype=torch.uint8, device=data.device)

    def once():
        rc = lib.parparaw_skip_rows(data.data_ptr(), n, drop.data_ptr(), drop.numel(), 0x0A, outb.data_ptr(),
                                    out_len.data_ptr(), scratch.data_ptr(), sb, stream.cuda_stream)
        assert rc == _abi.OK, rc

    for _ in range(3):
        once()
    t = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        once()
        e1.record(stream)
        e1.synchronize()
        t.append(e0.elapsed_time(e1))
    kept = int(out_len.item())
    assert 0 < kept < n
    med = float(np.median(t))
    return {"input_bytes": n, "rows_dropped": int(drop.numel()), "bytes_kept": kept, "ms_median": round(med, 4),
            "GB/s": round(n / (med * 1e-3) / 1e9, 3), "runs": reps,
            "note": "every 100th line pruned before the parse; 3 reads of the input, 1 write of what stays"}


def run_batched(args, dev, log):
    """Config 4: 10,000 inputs (log-normal sizes 1 KB..64 MB, ~6e9 B, half CSV,
    half web logs) in one persistent launch per step, tile shape autotuned."""
    import numpy as np
    import torch

    import synth
    from paper_1905_13415_gb300 import Batch, Parser, formats
    from paper_1905_13415_gb300.autotune import autotune, time_batch

    n = args.batch_inputs
    sizes, kinds, seeds = synth.batch_plan(n, args.batch_bytes, synth.BASE_SEED + 4)
    host = torch.empty(int(sizes.sum()), dtype=torch.uint8, pin_memory=True)
    t0 = time.perf_counter()
    offs, lens, rows = synth.generate_batch_into(kinds, seeds, sizes, host.data_ptr())
    gen_s = time.perf_counter() - t0
    data = host.to(dev)
    parsers = {k: Parser(formats.by_name(synth.DIALECT[k]), synth.SCHEMAS[k]) for k in ("mixed", "log")}
    items = []
    for i in range(n):
        p = parsers[kinds[i]]
        d = data[int(offs[i]): int(offs[i]) + int(lens[i])]
        out = p.allocate(max(int(rows[i]), 1), [max(int(lens[i]), 1)] * len(p.types), device=dev)
        items.append((p, d, out))
    total = int(lens.sum())
    # autotune on a sample of the inputs
    rng = np.random.default_rng(7)
    sample = [items[i] for i in sorted(rng.choice(n, size=min(400, n), replace=False))]
    best, tuned = autotune(sample, reps=3)
    # one prepared batch, timed
    stream = torch.cuda.current_stream()
    b = Batch(items)
    for _ in range(args.warmup):
        b.launch(stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    steps = max(3, min(args.steps, 10))
    kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for a, z in kev:
        a.record(stream)
        z.record(stream)
    timer = items[0][0]  # the batch's first parser carries the tile-kernel events
    e0.record(stream)
    for k in range(steps):
        timer.set_kernel_events(*kev[k])
        b.launch(stream)
    e1.record(stream)
    torch.cuda.synchronize()
    timer.set_kernel_events(None, None)
    batch_ms = e0.elapsed_time(e1) / steps
    kern_ms = statistics.mean(a.elapsed_time(z) for a, z in kev)
    b.close()
    bad = 0
    algo = 0
    for i, (p, d, out) in enumerate(items):
        res = out.result()
        if res.status != 0 or res.rows != int(rows[i]):
            bad += 1
        algo += int(lens[i]) + out.output_bytes(res.rows)
    peak, peak_kind = measured_peak_gbs()
    # the plain per-input loop on the same inputs
    for p, d, out in items[:50]:
        p.parse_into(d, out, stream=stream)
    torch.cuda.synchronize()
    e0.record(stream)
    for p, d, out in items:
        p.parse_into(d, out, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    loop_ms = e0.elapsed_time(e1)
    # What the batch costs beyond its bytes: each format's inputs parsed as
    # one large input of the same bytes (the plain rate without per-input
    # tails), and the tiles lost to partial last tiles of small inputs.
    tile = parsers["mixed"].info().tile_bytes
    tiles = int(sum((int(x) + tile - 1) // tile for x in lens))
    whole_ms = 0.0
    for kind in ("mixed", "log"):
        nbytes = int(sum(int(lens[i]) for i in range(n) if kinds[i] == kind))
        big = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
        m, r = synth.generate_into(kind, synth.BASE_SEED + 40, nbytes, big.data_ptr(), nbytes)
        dbig = big[:m].to(dev)
        p = parsers[kind]
        o = p.allocate(r + 16, [max(m, 1)] * len(p.types), device=dev)
        p.parse_into(dbig, o, stream=stream)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(3):
            p.parse_into(dbig, o, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        whole_ms += e0.elapsed_time(e1) / 3 * nbytes / max(m, 1)
        del o, dbig, big
    del items, data
    torch.cuda.empty_cache()
    log(f"batched: {total} B in {batch_ms:.2f} ms, loop {loop_ms:.2f} ms, generator {gen_s:.1f} s")
    return {"value": round(total / (batch_ms * 1e-3) / 1e9, 3), "unit": "GB/s", "inputs": n, "bytes": total,
            "ms_per_step": round(batch_ms, 3), "steps": steps, "launches_per_step": 3,
            "tile_config": best, "autotune_ms": {str(k): round(v, 3) for k, v in tuned.items()},
            "roofline": roofline_line(algo, kern_ms, peak, peak_kind),
            "plain_loop": {"value": round(total / (loop_ms * 1e-3) / 1e9, 3), "unit": "GB/s",
                           "ms": round(loop_ms, 2), "launches": 3 * n},
            "bad_results": bad,
            "same_bytes_as_two_large_inputs_ms": round(whole_ms, 3),
            "batch_over_large_inputs": round(batch_ms / whole_ms, 3) if whole_ms > 0 else None,
            "tiles": tiles, "tiles_if_concatenated": (total + tile - 1) // tile,
            "workload": "10,000 inputs, log-normal sizes 1 KB..64 MB (~6e9 B), half RFC-4180 CSV, half web logs"}


def run_served(args, dev, log):
    """Config 5: Poisson arrivals at 2,000 req/s for 60 s; request sizes
    log-normal (median 64 KB, sigma 2) clipped to 4 KB..256 MB, payloads drawn
    from a device-resident pool of mixed-CSV / review-CSV / web-log inputs;
    requests sized from their length only (capacity retries); admission capped
    by a 40 GB output arena; p50 / p99 latency (arrival to the host seeing the
    result, and to the device completing it) against the plain per-request
    parse, then a sweep of higher rates until the plain loop saturates."""
    import numpy as np
    import torch

    import synth
    from paper_1905_13415_gb300 import Parser, formats
    from paper_1905_13415_gb300.serve import Request, Server, run_trace, run_trace_plain

    rng = np.random.default_rng(synth.BASE_SEED + 5)
    npool = args.serve_pool
    sizes = np.clip(np.exp(np.log(64 << 10) + 2.0 * rng.standard_normal(npool)), 4 << 10, 256 << 20).astype(np.uint64)
    kinds = [("mixed", "review", "log")[i % 3] for i in range(npool)]
    seeds = (synth.BASE_SEED + 5) * 1000 + np.arange(npool, dtype=np.uint64)
    host = torch.empty(int(sizes.sum()), dtype=torch.uint8, pin_memory=True)
    offs, lens, _ = synth.generate_batch_into(kinds, seeds, sizes, host.data_ptr())
    data = host.to(dev)
    parsers = {k: Parser(formats.by_name(synth.DIALECT[k]), synth.SCHEMAS[k]) for k in ("mixed", "review", "log")}

    def trace(rate, seconds, seed):
        r = np.random.default_rng(seed)
        nreq = int(rate * seconds)
        return np.cumsum(r.exponential(1.0 / rate, nreq)), r.integers(0, npool, nreq)

    def make(picks, keep=()):
        keep = set(keep)
        return [Request(j, parsers[kinds[i]], data[int(offs[i]): int(offs[i]) + int(lens[i])], keep=j in keep)
                for j, i in enumerate(picks)]

    def payload_digest(i):
        out, res = parsers[kinds[i]].parse(data[int(offs[i]): int(offs[i]) + int(lens[i])])
        return res.status, output_digest_device(out, res.rows)

    rate, secs = args.serve_rate, args.serve_seconds
    arrivals, picks = trace(rate, secs, synth.BASE_SEED + 5)
    check = sorted(rng.choice(len(picks), size=min(200, len(picks)), replace=False).tolist())
    reqs = make(picks, keep=check)
    served = run_trace(Server(arena_bytes=40 << 30, streams=4, device=dev), reqs, arrivals)
    # outputs of a sample of served requests against the plain parse of the same payload
    want = {}
    bad = 0
    for j in check:
        i = int(picks[j])
        if i not in want:
            want[i] = payload_digest(i)
        r = reqs[j]
        got = (r.status, output_digest_device(r.out, r.rows))
        bad += got != want[i]
        r.out = None
    served["checked"] = len(check)
    served["mismatched"] = bad
    assert bad == 0, "served outputs differ from the plain parse"
    del reqs
    plain = run_trace_plain(make(picks), arrivals, device=dev)
    log(f"served: {served}; plain: {plain}")
    sweep = []
    for k, sweep_rate in enumerate(args.serve_sweep):
        arr, pk = trace(sweep_rate, args.sweep_seconds, synth.BASE_SEED + 50 + k)
        s_res = run_trace(Server(arena_bytes=40 << 30, streams=4, device=dev), make(pk), arr)
        p_res = run_trace_plain(make(pk), arr, device=dev)
        offered = float(lens[pk].sum()) / args.sweep_seconds / 1e9
        sweep.append({"rate_per_s": sweep_rate, "seconds": args.sweep_seconds, "offered_GB/s": round(offered, 4),
                      "served": s_res, "plain": p_res})
        log(f"sweep {sweep_rate}/s: served {s_res['gbs']} GB/s p99 {s_res['p99_ms']} ms; "
            f"plain {p_res['gbs']} GB/s p99 {p_res['p99_ms']} ms")
        if p_res["wall_s"] > 1.5 * args.sweep_seconds:  # the plain loop no longer keeps up: saturated
            break
    del data, host
    torch.cuda.empty_cache()
    return {"value": served["gbs"], "unit": "GB/s", "p50_ms": served["p50_ms"], "p99_ms": served["p99_ms"],
            "p50_device_ms": served["p50_device_ms"], "p99_device_ms": served["p99_device_ms"],
            "requests": len(picks), "seconds": secs, "rate_per_s": rate, "rounds": served["rounds"],
            "capacity_retries": served["capacity_retries"], "wall_s": served["wall_s"],
            "checked": served["checked"], "mismatched": served["mismatched"], "plain": plain, "sweep": sweep,
            "workload": f"Poisson {rate}/s for {secs} s; log-normal sizes 4 KB..256 MB (median 64 KB); "
                        f"pool of {npool} mixed-CSV / review-CSV / web-log payloads; 40 GB arena; "
                        f"requests sized from their length (one row per 16 B, string columns as long as the input), "
                        f"PP_E_CAPACITY retried with the exact sizes",
            "latency": "arrival to the host seeing the result (p50_ms, p99_ms) and to the device completing it "
                       "(p50_device_ms, p99_device_ms); the difference is host dispatch and polling"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="review", choices=sorted(WORKLOADS))
    ap.add_argument("--size", type=int, default=0, help="input bytes (default: the workload's size)")
    ap.add_argument("--tile-config", type=int, default=0, help="tile shape (default: autotuned per workload)")
    ap.add_argument("--cpu-sample", type=int, default=1_500_000_000,
                    help="bytes of the workload the CPU baseline parses")
    ap.add_argument("--ref-sample", type=int, default=256_000_000)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--partition-bytes", type=int, default=512 << 20)
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-others", action="store_true", help="skip the 1 MB and 1 GB plain-parse lines")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--batch-inputs", type=int, default=10_000)
    ap.add_argument("--batch-bytes", type=int, default=6_000_000_000)
    ap.add_argument("--serve-seconds", type=float, default=60.0)
    ap.add_argument("--serve-sweep", type=float, nargs="*", default=[4000.0, 8000.0, 16000.0, 32000.0, 64000.0])
    ap.add_argument("--sweep-seconds", type=float, default=5.0)
    ap.add_argument("--serve-rate", type=float, default=2000.0)
    ap.add_argument("--serve-pool", type=int, default=1500)
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch

    import __graft_entry__
    import synth

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    __graft_entry__.build()
    from paper_1905_13415_gb300 import Parser, formats

    wl, seed_off, default_n, desc = WORKLOADS[args.workload]
    target = args.size or default_n
    schema, dialect = synth.SCHEMAS[wl], synth.DIALECT[wl]

    # ------------------------------------------------------------ input
    host_in = torch.empty(target, dtype=torch.uint8, pin_memory=True)
    t0 = time.perf_counter()
    n, gen_rows = synth.generate_into(wl, synth.BASE_SEED + seed_off, target, host_in.data_ptr(), target)
    gen_s = time.perf_counter() - t0
    host_in = host_in[:n]
    data = host_in.to(dev)
    torch.cuda.synchronize()

    parser = Parser(formats.by_name(dialect), schema, tile_config=args.tile_config)
    out, res = parser.parse(data, rows_cap=gen_rows + 16)
    torch.cuda.synchronize()
    assert res.status == 0 and res.rows == gen_rows and res.n_rejected == 0, (res, gen_rows)
    # exactly sized outputs for the timed loop (and the device-to-host copies)
    out = parser.allocate(res.rows, [max(int(b), 1) for b in res.values_bytes_needed], device=dev)
    parser.parse_into(data, out)
    res = out.result()
    assert res.status == 0 and res.rows == gen_rows
    rows = res.rows
    tuned = pick_tile_shape(args, parser, data, out)
    algo_bytes = n + out.output_bytes(rows)  # input read once + exact output layout
    out_bytes_estimate = out.output_bytes(rows)

    stream = torch.cuda.current_stream()
    nev = args.steps
    k_start = [torch.cuda.Event(enable_timing=True) for _ in range(nev)]
    k_stop = [torch.cuda.Event(enable_timing=True) for _ in range(nev)]
    for ev in (*k_start, *k_stop):  # torch creates the CUDA event on first record
        ev.record(stream)

    for _ in range(args.warmup):
        parser.parse_into(data, out, stream=stream)
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(args.steps):
        parser.set_kernel_events(k_start[i], k_stop[i])
        parser.parse_into(data, out, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    parser.set_kernel_events(None, None)
    clocks = sampler.stop()
    step_ms = e0.elapsed_time(e1) / args.steps
    kern_ms = statistics.mean(a.elapsed_time(b) for a, b in zip(k_start, k_stop))
    step_ms, kern_ms = max_over_ranks([step_ms, kern_ms], world, dev)
    res = out.result()
    assert res.status == 0 and res.rows == rows

    value = whole_job_rate(world, n, step_ms)
    peak, peak_kind = measured_peak_gbs()
    achieved = algo_bytes / (kern_ms * 1e-3) / 1e9
    # the recorded traffic is per launch of the workload's full size
    traffic = recorded_traffic(args.workload, tuned["tile_config"]) if target == default_n else None

    # ------------------------------------------------- end to end (host)
    # Through the library's streaming entry (parparaw_stream_parse): pinned
    # host input -> device, parse, columns -> a pinned host arena, partitions
    # overlapped on three streams with on-device carry-over (Sec. 4.4).
    e2e = None
    if not args.no_e2e:
        from paper_1905_13415_gb300.stream import HostArena, StreamParser

        ref_digest = output_digest_device(out, rows)  # the plain device parse, for the check below
        del out
        torch.cuda.empty_cache()
        sp = StreamParser(parser, partition_bytes=args.partition_bytes, device=dev)
        arena = HostArena(int(out_bytes_estimate * 1.1) + (64 << 20))  # reused by every step

        def e2e_step():
            parts = sp.parse(host_in, arena)
            return sum(x.rows for x in parts), parts

        for _ in range(max(1, min(args.warmup, 2))):
            got_rows, parts = e2e_step()
        assert got_rows == rows, (got_rows, rows)
        d2h = sum(sum(v.numel() * v.element_size() for v in col.values() if v is not None) + x.row_valid.numel()
                  for x in parts for col in x.columns)
        del parts
        if world > 1:
            torch.distributed.barrier()
        ksteps = max(10, min(args.steps, 20))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_step_ms, call_ms, dev_ms = [], [], []
        for _ in range(ksteps):
            ts = time.perf_counter()
            got_rows, parts = e2e_step()  # returns with the library's streams drained
            e2e_step_ms.append((time.perf_counter() - ts) * 1e3)
            call_ms.append(sp.last_call_ms)
            # the library's device times of the step's partitions, summed: copy in, parse, copy out
            dev_ms.append([round(sum(getattr(x, k) for x in parts), 2) for k in ("h2d_ms", "parse_ms", "d2h_ms")])
        torch.cuda.synchronize()
        e2e_ms = (time.perf_counter() - t0) * 1e3 / ksteps
        verified = output_digest_partitions(parts, parser.types) == ref_digest  # the last timed step's output
        assert verified, "streamed output differs from the plain parse"
        del parts
        (e2e_ms,) = max_over_ranks([e2e_ms], world, dev)
        e2e = {"value": round(whole_job_rate(world, n, e2e_ms), 3), "unit": "GB/s",
               "h2d_bytes_per_step": n, "d2h_bytes_per_step": int(d2h), "ms_per_step": round(e2e_ms, 3),
               "median_ms": round(statistics.median(e2e_step_ms), 3),
               "median_GB/s": round(n / (statistics.median(e2e_step_ms) * 1e-3) / 1e9, 3),
               "steps": ksteps, "step_ms": [round(x, 2) for x in e2e_step_ms],
               "library_call_ms": [round(x, 2) for x in call_ms],
               "device_ms_h2d_parse_d2h": dev_ms,
               "api": "parparaw_stream_parse (C ABI; partitions overlapped, carry-over on the device)",
               "partition_bytes": args.partition_bytes,
               "verified": "per-column SHA-256 of the last timed step's output equals the plain device parse's"}
        sp.close()

    # ------------------------------------------------------ CPU baseline
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        sample_n = min(args.cpu_sample, n)
        # the generator is deterministic, so this is a whole-record prefix of the input
        raw = synth.generate(wl, synth.BASE_SEED + seed_off, sample_n)
        last = len(raw)
        rate, secs = oracle_rate(wl, raw[:last], schema, dialect)
        cpu = {"value": round(rate, 4), "unit": "GB/s", "cores": 1, "kind": "oracle",
               "sample": f"first {last} bytes (whole records) of the same input, {secs:.1f} s single-threaded"}

    def log(msg):
        print(msg, file=sys.stderr, flush=True)

    batched = served = others = None
    if rank == 0 and world == 1 and not args.no_others:
        others = run_other_configs(args, dev, log)
    if rank == 0 and world == 1 and not args.no_batch:
        batched = run_batched(args, dev, log)
    if rank == 0 and world == 1 and not args.no_serve:
        served = run_served(args, dev, log)

    if rank == 0:
        line = {
            "metric": "raw-input parse GB/s", "value": round(value, 3), "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(step_ms, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic",
            "config": {"workload": desc, "input_bytes": n, "rows": rows, "columns": len(schema),
                       "tile_bytes": parser.info().tile_bytes, "parallelism": f"replicas x{world}",
                       **tuned,
                       "l2": "input larger than L2 (no flush needed)", "generator_s": round(gen_s, 2)},
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4), "peak_kind": peak_kind,
                         "kernel": "pp_tile_kernel", "kernel_ms": round(kern_ms, 4),
                         "algorithmic_bytes": algo_bytes,
                         "traffic": traffic["bytes_per_launch"] if traffic else None,
                         "traffic_source": (f"ncu DRAM bytes, {traffic['scaled_from']} "
                                            "(profiles/pp_tile_kernel_traffic.txt)") if traffic else
                                           ("no capture of the current kernel sources at this tile shape"
                                            if target == default_n else "recorded for the full size only")},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": 3 * args.steps,
            "batched": batched,
            "served": served,
            "other_configs": others,
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
