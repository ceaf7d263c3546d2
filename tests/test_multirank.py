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


# ------------------------------------------------------------------------------------------------
# The library's exchange block (hyb_mc_leg_range / hyb_mc_leg_reduce_finish) under an all-reduce:
# int64 words summed element-wise, 128-bit values carried as four 32-bit limbs (value = sum_i
# limb_i 2^(32 i) mod 2^128, the top limb signed). Ranks hold random 128-bit values (positive and
# negative, up to 2^125 in size, as the FP64 path's fixed-point tallies and weight sums can be); the
# limb-wise gloo sum, reassembled, must be their exact sum modulo 2^128, and plain int64 words (the
# FP32 path's tallies) must sum as two's-complement integers.
# ------------------------------------------------------------------------------------------------
M128 = (1 << 128) - 1


def _values(rank: int, n: int) -> list[int]:
    rng = np.random.default_rng(100 + rank)
    out = []
    for _ in range(n):
        mag = int(rng.integers(0, 1 << 62)) << int(rng.integers(0, 64))
        out.append(-mag if rng.integers(0, 2) else mag)
    return out


def _to_limbs(v: int) -> list[int]:
    u = v & M128
    limbs = [(u >> (32 * i)) & 0xFFFFFFFF for i in range(4)]
    if limbs[3] >= 1 << 31:               # the top limb is signed
        limbs[3] -= 1 << 32
    return limbs


def _from_limbs(w: list[int]) -> int:
    return sum(int(x) << (32 * i) for i, x in enumerate(w)) & M128


def _exchange_rank(rank: int, world: int, port: int, out_dir: str) -> None:
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    vals = _values(rank, 64)
    blk = torch.tensor([x for v in vals for x in _to_limbs(v)], dtype=torch.int64)
    rng = np.random.default_rng(7 + rank)
    words = torch.from_numpy(rng.integers(-(1 << 62), 1 << 62, 64, dtype=np.int64))
    dist.all_reduce(blk)
    dist.all_reduce(words)
    if rank == 0:
        np.savez(os.path.join(out_dir, "xblk.npz"), blk=blk.numpy(), words=words.numpy())
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_exchange_block_sums_exactly_under_allreduce(tmp_path, world):
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    mp.spawn(_exchange_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    got = np.load(tmp_path / "xblk.npz")
    limbs = got["blk"].reshape(-1, 4)
    want = [sum(_values(r, 64)[i] for r in range(world)) & M128 for i in range(64)]
    assert [_from_limbs(list(map(int, row))) for row in limbs] == want
    w = sum(np.random.default_rng(7 + r).integers(-(1 << 62), 1 << 62, 64, dtype=np.int64).astype(object)
            for r in range(world))
    wrap = [((int(x) + (1 << 63)) % (1 << 64)) - (1 << 63) for x in w]
    assert [int(x) for x in got["words"]] == wrap
