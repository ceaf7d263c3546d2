"""History-sharded MC leg across ranks, emulated by two gloo processes on the CPU.

Histories of one leg are independent, so a leg shards by contiguous slices of the global
history index (census bank slots, then source births): every rank draws exactly the points it
would draw in a one-rank run, and one sum all-reduce of the tallies and counters is the only
exchange. Two CPU ranks run the oracle on their slices and all-reduce with gloo; the result must
equal the one-rank leg (integer counts and per-history records exactly, tallies to rounding).
"""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest

INT_KEYS = ("histories", "segments", "collisions", "leaked", "census", "killed", "reached_limit", "errors")
WORLD = 2


def _spec_and_bank():
    from paper_2511_16821_gb300 import workloads as W
    spec = W.checkerboard(n_s=2, n_hist=3000, cells_per_block=2)
    bank = W.random_bank(spec, 2000, seed=4)
    return spec, bank


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, out_dir: str) -> None:
    import torch
    import torch.distributed as dist
    import oracle as O
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    spec, bank = _spec_and_bank()
    n = bank["n"] + spec.n_hist
    h0, h1 = rank * n // world, (rank + 1) * n // world
    r = O.mc_leg_range(spec, 1, bank, h0, h1)
    assert r["rc"] == 0
    tal = torch.from_numpy(np.concatenate([r["pre"], r["post"], r["mom"].ravel()]))
    dist.all_reduce(tal)
    ints = torch.tensor([r["stats"][k] for k in INT_KEYS], dtype=torch.int64)
    dist.all_reduce(ints)
    # per-history records: gather the slices (padded to a common length) in rank order
    m = (n + world - 1) // world
    rec = torch.full((m, 4), -1, dtype=torch.int32)
    rec[: h1 - h0] = torch.from_numpy(r["hist"])
    parts = [torch.empty_like(rec) for _ in range(world)]
    dist.all_gather(parts, rec)
    if rank == 0:
        hist = np.concatenate([p.numpy()[: (q + 1) * n // world - q * n // world] for q, p in enumerate(parts)])
        np.savez(os.path.join(out_dir, "sharded.npz"), tal=tal.numpy(), ints=ints.numpy(), hist=hist)
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_leg_equals_one_rank(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    import oracle as O
    O.lib()                                   # build the oracle once, before the ranks start
    spec, bank = _spec_and_bank()
    mp.spawn(_rank_main, args=(WORLD, _free_port(), str(tmp_path)), nprocs=WORLD, join=True)
    got = np.load(tmp_path / "sharded.npz")
    full = O.mc_leg(spec, 1, bank, want_hist=True)
    want_tal = np.concatenate([full["pre"], full["post"], full["mom"].ravel()])
    assert [int(v) for v in got["ints"]] == [full["stats"][k] for k in INT_KEYS]
    assert np.array_equal(got["hist"], full["hist"])
    assert np.allclose(got["tal"], want_tal, rtol=1e-12, atol=1e-15 * np.max(np.abs(want_tal)))
