"""Autotuners: of the batched persistent launch, and of one problem's leg and census.

tune_batch times candidate tunings (threads per CTA of the batched MC leg, histories per
work-queue chunk, resident CTAs per SM, streams for the per-problem branches) on the batch's own
time steps and keeps the fastest. Every candidate runs one untimed step first (graphs are recorded
there), then `steps` timed steps with CUDA events on the batch stream. The problems advance while
tuning, as in the first steps of a run; results do not depend on the tuning (the batch is exact
per problem).

tune_problem times one problem's creation-time knobs: the copies of the fixed-point tally arrays
(more copies spread the leg's atomic adds to hot cells, fewer keep the copies in L2), the
privatisation tile (priv_tile: the side of the window of cells whose tallies each CTA keeps in
shared memory, placed on the densest source region; 0: none), the leg's sort interval (leg_sort_every = K: 0 runs the fused leg, K >= 1 the
phased leg, whose live histories are sorted by cell every K segments) and the census sort interval
(with census_order >= 1, the census is sorted and combed in cell order on every sort_every-th step
only). The copies, the tile and the leg's sort interval never change a result; the census sort interval
does (an unsorted comb samples each cell's weight less evenly), so it is searched only when the
space names it, and the caller accepts the variance that comes with a longer interval.
"""
from __future__ import annotations

import itertools

DEFAULT_SPACE = {"block": (128, 256), "chunk": (1024, 4096, 16384), "ctas_per_sm": (0,), "streams": (8, 32)}
PROBLEM_SPACE = {"tally_copies": (1, 4), "priv_tile": (0, 8, 16), "leg_sort_every": (0, 8)}
L2_FLUSH_BYTES = 256 << 20


def candidates(space: dict | None = None, default: dict | None = None) -> list[dict]:
    sp = dict(DEFAULT_SPACE if default is None else default)
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


def tune_problem(spec, steps: int = 4, warmup: int = 3, space: dict | None = None, stream=None) -> dict:
    """Time each candidate (a fresh problem of spec with those knobs, `warmup` untimed steps, then
    `steps` steps of device time each after an L2 flush) and return the fastest spec with the table.
    Per-step device time is the problem's own (CUDA events around each step on its stream)."""
    import torch
    from . import hyb
    stream = stream if stream is not None else torch.cuda.Stream()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    best, best_ms, table = None, float("inf"), []
    with torch.cuda.stream(stream):
        # the knobs the space names (by default PROBLEM_SPACE); the others keep the spec's values
        for cand in candidates(space, {}) if space else candidates(None, PROBLEM_SPACE):
            P = hyb.Problem(spec.with_(**cand), stream=stream)
            try:
                P.step(warmup, stats=False)
                ms = 0.0
                for _ in range(steps):
                    flush.zero_()
                    ms += P.step(1)[0]["ms"]
            finally:
                P.close()
            ms /= steps
            table.append({**cand, "ms_per_step": ms})
            if ms < best_ms:
                best, best_ms = cand, ms
    torch.cuda.synchronize()
    return {"best": best, "spec": spec.with_(**best), "ms_per_step": best_ms, "table": table}
