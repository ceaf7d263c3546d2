"""Autotuner of the batched persistent launch.

Times candidate tunings (threads per CTA of the batched MC leg, histories per work-queue chunk,
resident CTAs per SM, streams for the per-problem branches) on the batch's own time steps and
keeps the fastest. Every candidate runs one untimed step first (graphs are recorded there), then
`steps` timed steps with CUDA events on the batch stream. The problems advance while tuning, as in
the first steps of a run; results do not depend on the tuning (the batch is exact per problem).
"""
from __future__ import annotations

import itertools

DEFAULT_SPACE = {"block": (128, 256), "chunk": (1024, 4096, 16384), "ctas_per_sm": (0,), "streams": (8, 32)}


def candidates(space: dict | None = None) -> list[dict]:
    sp = dict(DEFAULT_SPACE)
    if space:
        sp.update(space)
    keys = list(sp)
    return [dict(zip(keys, v)) for v in itertools.product(*(sp[k] for k in keys))]


def tune_batch(batch, steps: int = 2, space: dict | None = None, use_graph: int = 1) -> dict:
    import torch
    best, best_ms, table = None, float("inf"), []
    for cand in candidates(space):
        batch.set_tuning(use_graph=use_graph, **cand)
        batch.step(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(batch.stream)
        batch.step(steps)
        e1.record(batch.stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        table.append({**cand, "ms_per_step": ms})
        if ms < best_ms:
            best, best_ms = cand, ms
    batch.set_tuning(use_graph=use_graph, **best)
    return {"best": best, "ms_per_step": best_ms, "table": table}
