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
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1905_13415_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def measured_peak_gbs():
    try:
        d = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def recorded_traffic(workload: str):
    """DRAM bytes per launch of the tile kernel from the committed ncu
    summary, if it was taken on the current kernel sources."""
    path = os.path.join(ROOT, "profiles", "pp_tile_kernel_traffic.txt")
    if not os.path.exists(path):
        return None
    src = csv_hash_of_sources()
    for line in open(path):
        parts = line.split()
        if len(parts) >= 4 and not line.startswith("#") and parts[0] == workload and parts[1] == src:
            return {"bytes_per_launch": float(parts[2]), "scaled_from": parts[3]}
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


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    return world, rank, local


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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="review", choices=sorted(WORKLOADS))
    ap.add_argument("--size", type=int, default=0, help="input bytes (default: the workload's size)")
    ap.add_argument("--tile-config", type=int, default=0)
    ap.add_argument("--cpu-sample", type=int, default=1_500_000_000,
                    help="bytes of the workload the CPU baseline parses")
    ap.add_argument("--ref-sample", type=int, default=256_000_000)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
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
    algo_bytes = n + out.output_bytes(rows)  # input read once + exact output layout

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
    if world > 1:
        t = torch.tensor([step_ms, kern_ms], device=dev, dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        step_ms, kern_ms = float(t[0]), float(t[1])
    res = out.result()
    assert res.status == 0 and res.rows == rows

    value = world * n / (step_ms * 1e-3) / 1e9
    peak, peak_kind = measured_peak_gbs()
    achieved = algo_bytes / (kern_ms * 1e-3) / 1e9
    traffic = recorded_traffic(args.workload)

    # ------------------------------------------------- end to end (host)
    e2e = None
    if not args.no_e2e:
        host_out = []
        d2h = 0
        for t_ in [*out.values, *[o for o in out.offsets if o is not None], *out.validity, out.row_valid,
                   out.result_buf]:
            host_out.append((t_, torch.empty(t_.shape, dtype=t_.dtype, pin_memory=True)))
            d2h += t_.numel() * t_.element_size()
        dev_in = torch.empty_like(data)

        def e2e_step():
            dev_in.copy_(host_in, non_blocking=True)
            parser.parse_into(dev_in, out, stream=stream)
            for d, h in host_out:
                h.copy_(d, non_blocking=True)

        for _ in range(max(1, args.warmup)):
            e2e_step()
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        ksteps = max(3, min(args.steps, 10))
        s0.record(stream)
        for _ in range(ksteps):
            e2e_step()
        s1.record(stream)
        torch.cuda.synchronize()
        e2e_ms = s0.elapsed_time(s1) / ksteps
        if world > 1:
            t = torch.tensor([e2e_ms], device=dev, dtype=torch.float64)
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            e2e_ms = float(t[0])
        e2e = {"value": round(world * n / (e2e_ms * 1e-3) / 1e9, 3), "unit": "GB/s",
               "h2d_bytes_per_step": n, "d2h_bytes_per_step": d2h, "ms_per_step": round(e2e_ms, 3),
               "steps": ksteps}
        del dev_in

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

    if rank == 0:
        line = {
            "metric": "raw-input parse GB/s", "value": round(value, 3), "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(step_ms, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic",
            "config": {"workload": desc, "input_bytes": n, "rows": rows, "columns": len(schema),
                       "tile_bytes": parser.info().tile_bytes, "parallelism": f"replicas x{world}",
                       "l2": "input larger than L2 (no flush needed)", "generator_s": round(gen_s, 2)},
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4), "peak_kind": peak_kind,
                         "kernel": "pp_tile_kernel", "kernel_ms": round(kern_ms, 4),
                         "algorithmic_bytes": algo_bytes,
                         "traffic": traffic["bytes_per_launch"] if traffic else None},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": 3 * args.steps,
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
