"""Autotuner for the batched form: picks the launch shape of
ck_multi_insert (threads per block, resident blocks per SM, keys per tile)
by timing fills of the actual tables with CUDA events, fastest wins.  One
thread drives one insertion in this design, so threads per insertion is
fixed at 1; the chain cap stays at the workload's value (a lower cap would
change results)."""
from __future__ import annotations

import itertools

import torch

from . import multi as M


def _fill_ms(mt, kt, vt, st, stream, reps=1):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    best = None
    for _ in range(reps):
        mt.clear(stream)
        e0.record(stream)
        mt.insert(kt, vt, st, stream=stream)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    return best


def tune(mt, kt, vt, st, stream=None, blocks=(128, 256), per_sm=(0, 4), tiles=(1024, 4096, 16384), reps=3):
    """Time every (block, blocks_per_sm, tile) combination, each the best of
    `reps` fills (the first fill of a shape also warms it); leave the
    fastest set on `mt` and return (best, [(config, ms), ...])."""
    stream = stream or torch.cuda.current_stream()
    results = []
    for b, p, t in itertools.product(blocks, per_sm, tiles):
        mt.set_param(M.MULTI_BLOCK, b)
        mt.set_param(M.MULTI_BLOCKS_PER_SM, p)
        mt.set_param(M.MULTI_TILE, t)
        _fill_ms(mt, kt, vt, st, stream)  # warm-up
        results.append(({"block": b, "blocks_per_sm": p, "tile": t}, _fill_ms(mt, kt, vt, st, stream, reps)))
    best = min(results, key=lambda r: r[1])[0]
    mt.set_param(M.MULTI_BLOCK, best["block"])
    mt.set_param(M.MULTI_BLOCKS_PER_SM, best["blocks_per_sm"])
    mt.set_param(M.MULTI_TILE, best["tile"])
    return best, results
