"""The oracle's MC leg over history-index slices in worker processes -- TEST INFRASTRUCTURE.

Histories of a leg are independent (Sec. 2.3: each history draws its own point), so the leg over
[0, N) equals the sum of the legs over contiguous slices [h_r, h_{r+1}): records and margins are
the slices' rows in order, integer counters add exactly, and the FP64 tallies add to rounding (the
one-process sums differ by reassociation only, ~1e-16 relative). The workers are started with the
``spawn`` method (never forked from a process that holds a CUDA context) and each loads its own
copy of the oracle library.
"""
from __future__ import annotations

import multiprocessing as mp
import os
import pickle
import tempfile

import numpy as np

_INT_STATS = ("histories", "segments", "collisions", "leaked", "census", "killed", "reached_limit", "errors")
_W_STATS = ("w_source", "w_absorbed", "w_leaked", "w_census", "w_handoff", "w_killed")


_cache: dict = {}


def _slice_leg(args):
    path, step, h0, h1, kw = args
    import oracle
    if path not in _cache:             # the problem and bank travel once per worker, as a file
        _cache.clear()
        with open(path, "rb") as f:
            _cache[path] = pickle.load(f)
    spec, bank = _cache[path]
    return oracle.mc_leg(spec, step, bank, h0=h0, h1=h1, **kw)


def _steps(args):
    spec, nsteps, elem, bank = args
    import oracle
    out = []
    for k in range(nsteps):
        r = oracle.step(spec, k, bank, elem=elem)
        bank = r["bank"]
        out.append(r)
    return out


def merge(parts: list[dict]) -> dict:
    """Sum of slice results (tallies, segment counts, statistics) with rows concatenated."""
    out = {k: sum(p[k] for p in parts) for k in ("pre", "post", "mom", "pre_n", "post_n")}
    st = {k: sum(int(p["stats"][k]) for p in parts) for k in _INT_STATS}
    st.update({k: float(sum(p["stats"][k] for p in parts)) for k in _W_STATS})
    st["sn_iterations"] = 0
    out["stats"] = st
    out["rc"] = max(p["rc"] for p in parts)
    for k in ("hist", "margin"):
        if k in parts[0]:
            out[k] = np.concatenate([p[k] for p in parts])
    return out


class Pool:
    """A spawn-started pool of `nproc` oracle workers (default: the host's cores)."""

    def __init__(self, nproc: int | None = None):
        self.nproc = nproc or os.cpu_count() or 1
        self._pool = mp.get_context("spawn").Pool(self.nproc)

    def mc_leg(self, spec, step: int, bank: dict | None, nslices: int | None = None, **kw) -> dict:
        """The oracle's mc_leg(spec, step, bank, **kw) over all histories, run as `nslices`
        contiguous index slices (default: 4 per worker) and merged."""
        import oracle
        n = oracle.n_histories(spec, bank)
        ns = max(1, min(nslices or 4 * self.nproc, n))
        cuts = [n * r // ns for r in range(ns + 1)]
        if n == 0:
            return oracle.mc_leg(spec, step, bank, **kw)
        fd, path = tempfile.mkstemp(suffix=".pkl", prefix="oracle_leg_")
        try:
            with os.fdopen(fd, "wb") as f:
                pickle.dump((spec, bank), f, protocol=pickle.HIGHEST_PROTOCOL)
            kw = dict(kw, elem=kw.get("elem", oracle._elem_default))
            jobs = [(path, step, cuts[r], cuts[r + 1], kw) for r in range(ns) if cuts[r + 1] > cuts[r]]
            return merge(self._pool.map(_slice_leg, jobs))
        finally:
            os.unlink(path)

    def steps(self, specs: list, nsteps: int, elem: int | None = None, banks: list | None = None) -> list[list[dict]]:
        """Whole hybrid steps 0 .. nsteps-1 of each problem (oracle.step, one problem per worker,
        starting from its bank or from the problem's zero initial data): per problem the list of
        the steps' results."""
        import oracle
        el = oracle._elem_default if elem is None else elem
        jobs = [(sp, nsteps, el, None if banks is None else banks[i]) for i, sp in enumerate(specs)]
        return self._pool.map(_steps, jobs, chunksize=1)

    def close(self):
        self._pool.close()
        self._pool.join()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
