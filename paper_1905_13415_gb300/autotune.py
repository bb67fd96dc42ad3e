"""Tile-shape autotuner.

The tile shape fixes threads per block, bytes per thread (the paper's chunk
size, Sec. 5 sweeps it) and therefore bytes per tile.  The best shape depends
on the input mix (record length, share of special symbols, input sizes of a
batch), so it is measured: every candidate parses a sample of the real inputs
(one batched launch per repetition, or one plain parse of a single input,
CUDA events on the launching stream) and the fastest is set on the parsers.
"""
from __future__ import annotations

import statistics

import torch

from . import _abi
from .parser import Batch

# (config, threads x bytes per thread [blocks per SM]): every shape but the
# 32-thread test shape
CANDIDATES = {2: "64x48", 3: "256x112", 4: "128x208", 5: "128x112/4", 6: "128x112/6", 7: "128x48/8",
              8: "256x80/3", 9: "256x96/3", 10: "448x64", 11: "512x48", 12: "256x112/3", 13: "384x128",
              14: "448x128"}


def time_batch(items, reps: int = 3, warmup: int = 1, stream=None) -> float:
    """Median milliseconds of one batched parse of `items` [(parser, data, out)]."""
    stream = stream or torch.cuda.current_stream()
    b = Batch(items)
    try:
        for _ in range(warmup):
            b.launch(stream)
        times = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            b.launch(stream)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
    finally:
        b.close()
    return statistics.median(times)


def autotune(items, configs=None, reps: int = 3) -> tuple[int, dict]:
    """Times each tile configuration on the sample `items` and sets the
    fastest on every parser that appears in them.  Returns (config, {config:
    ms})."""
    parsers = []
    for p, _, _ in items:
        if all(p is not q for q in parsers):
            parsers.append(p)
    results = {}
    for cfg in configs or CANDIDATES:
        for p in parsers:
            p.set_option(_abi.OPT_TILE_CONFIG, cfg)
        results[cfg] = time_batch(items, reps=reps)
    best = min(results, key=results.get)
    for p in parsers:
        p.set_option(_abi.OPT_TILE_CONFIG, best)
    return best, results


def time_plain(parser, data, out, reps: int = 3, warmup: int = 1, stream=None) -> float:
    """Median milliseconds of one plain parse of `data` into `out`."""
    stream = stream or torch.cuda.current_stream()
    for _ in range(warmup):
        parser.parse_into(data, out, stream=stream)
    times = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        parser.parse_into(data, out, stream=stream)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    return statistics.median(times)


def autotune_plain(parser, data, out, configs=None, reps: int = 3, stream=None) -> tuple[int, dict]:
    """Times each tile configuration on one plain parse of `data` (a device
    input) into `out` and sets the fastest on `parser`.  Returns (config,
    {config: ms})."""
    results = {}
    for cfg in configs or CANDIDATES:
        parser.set_option(_abi.OPT_TILE_CONFIG, cfg)
        results[cfg] = time_plain(parser, data, out, reps=reps, stream=stream)
    best = min(results, key=results.get)
    parser.set_option(_abi.OPT_TILE_CONFIG, best)
    return best, results
