"""Thin ctypes binding of the C ABI in ``include/hyb.h`` (argument marshalling only).

Every step of the hybrid path runs in the sm_103a kernels of ``libhyb.so``; PyTorch provides the
device workspace (one caching-allocator block per problem) and the CUDA stream. There is no CPU
fallback: without the library or a CUDA device every entry point raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build
from .workloads import ProblemSpec

HYB_OK, HYB_EINVAL, HYB_ENOMEM, HYB_ECUDA, HYB_ETIMEOUT, HYB_ESTATE, HYB_EBOUNDS, HYB_ECAPACITY = range(8)
FP32, FP64 = 0, 1
SOBOL, PRNG, HALTON = 0, 1, 2
NS_INF = 2147483647
STREAM_INIT, STREAM_LEG_CENSUS, STREAM_LEG_SOURCE, STREAM_REMAP_SOURCE, STREAM_REMAP_COMB = range(5)
TALLY = {"pre": 0, "post": 1, "handoff": 2, "sn_phi": 3, "flux": 4, "pre_raw": 5, "post_raw": 6}
SOBOL_DIMS = 65


class HybError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"hyb status {status}: {msg}")
        self.status = status


class Desc(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("lx", C.c_double), ("ly", C.c_double),
                ("sigma_a", C.POINTER(C.c_double)), ("sigma_s", C.POINTER(C.c_double)),
                ("Q", C.POINTER(C.c_double)), ("ic_cell_w", C.POINTER(C.c_double)),
                ("c", C.c_double), ("dt", C.c_double), ("n_s", C.c_int32), ("sampler", C.c_int32),
                ("n_hist", C.c_int64), ("seed", C.c_uint64), ("precision", C.c_int32),
                ("sn_order", C.c_int32), ("handoff_full", C.c_int32), ("sn_max_iter", C.c_int32),
                ("sn_tol", C.c_double), ("w_min", C.c_double), ("census_cap", C.c_int64),
                ("sn_warm_start", C.c_int32), ("census_order", C.c_int32), ("sn_accel", C.c_int32),
                ("remap_variant", C.c_int32), ("n_s_cell", C.POINTER(C.c_int32)), ("sn_layout", C.c_int32),
                ("seg_limit", C.c_int32), ("wait_limit", C.c_int32), ("tally_copies", C.c_int32),
                ("sort_every", C.c_int32), ("leg_sort_every", C.c_int32), ("priv_tile", C.c_int32),
                ("pad4", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [(k, C.c_int64) for k in ("histories", "segments", "collisions", "leaked", "census",
                                         "killed", "reached_limit", "errors")] + \
               [(k, C.c_double) for k in ("w_source", "w_absorbed", "w_leaked", "w_census",
                                          "w_handoff", "w_killed")] + \
               [("sn_iterations", C.c_int32), ("combed", C.c_int32), ("bank_size", C.c_int64),
                ("ms", C.c_float), ("pad", C.c_int32), ("tally_adds", C.c_int64),
                ("ms_leg", C.c_float), ("ms_sn", C.c_float), ("ms_remap", C.c_float), ("ms_leg_kernel", C.c_float)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if k not in ("pad", "pad1")}


class Tuning(C.Structure):
    _fields_ = [("block", C.c_int32), ("chunk", C.c_int32), ("ctas_per_sm", C.c_int32), ("streams", C.c_int32),
                ("use_graph", C.c_int32), ("pad", C.c_int32)]


_lib = None


def lib():
    """Load libhyb.so (building it in-tree first when the sources are newer)."""
    global _lib
    if _lib is None:
        path = _build.OUT
        if _build.stale():
            path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError("libhyb.so is missing; run __graft_entry__.build()")
        L = C.CDLL(path)
        P = C.c_void_p
        L.hyb_status_string.restype = C.c_char_p
        L.hyb_last_error.restype = C.c_char_p
        L.hyb_last_error.argtypes = [P]
        L.hyb_workspace_size.argtypes = [C.POINTER(Desc), C.POINTER(C.c_size_t)]
        L.hyb_priv_window.argtypes = [C.POINTER(Desc)] + [C.POINTER(C.c_int32)] * 3
        L.hyb_create_problem.argtypes = [C.POINTER(Desc), P, C.c_size_t, P, C.POINTER(P)]
        L.hyb_destroy_problem.argtypes = [P]
        L.hyb_mc_leg.argtypes = [P, C.POINTER(Stats)]
        L.hyb_mc_leg_trace.argtypes = [P, P, C.POINTER(Stats)]
        L.hyb_leg_exchange_bytes.argtypes = [P, C.POINTER(C.c_size_t)]
        L.hyb_mc_leg_range.argtypes = [P, C.c_int64, C.c_int64, P, C.c_size_t, P]
        L.hyb_mc_leg_reduce_finish.argtypes = [P, P, C.c_size_t, C.POINTER(Stats)]
        L.hyb_collided_solve.argtypes = [P, C.POINTER(Stats)]
        L.hyb_remap.argtypes = [P, C.POINTER(Stats)]
        L.hyb_step.argtypes = [P, C.c_int32, C.POINTER(Stats)]
        L.hyb_step_async.argtypes = [P, C.c_int32]
        L.hyb_remap_stats.argtypes = [P, C.POINTER(Stats)]
        L.hyb_get_tally.argtypes = [P, C.c_int32, P, C.c_size_t, C.c_int32]
        L.hyb_set_sn_phi.argtypes = [P, P, C.c_size_t]
        L.hyb_get_bank.argtypes = [P] + [P] * 6 + [C.POINTER(C.c_int64)]
        L.hyb_set_bank.argtypes = [P] + [P] * 6 + [C.c_int64]
        L.hyb_set_bank_native.argtypes = [P] + [P] * 6 + [C.c_int64]
        L.hyb_bank_capacity.argtypes = [P, C.POINTER(C.c_int64)]
        L.hyb_set_step.argtypes = [P, C.c_int64]
        L.hyb_get_step.argtypes = [P, C.POINTER(C.c_int64)]
        L.hyb_points.argtypes = [C.c_uint64, C.c_int64, C.c_int32, C.c_int32, C.c_int64, C.c_int64,
                                 C.c_int32, P, P]
        L.hyb_sobol_table.argtypes = [C.c_int32, P]
        L.hyb_cdf_scratch_bytes.argtypes = [C.c_int32, C.c_int32, C.POINTER(C.c_size_t)]
        L.hyb_batch_create.argtypes = [C.POINTER(P), C.c_int32, P, C.POINTER(P)]
        L.hyb_batch_set_tuning.argtypes = [P, C.POINTER(Tuning)]
        L.hyb_batch_set_problems.argtypes = [P, C.POINTER(P), C.c_int32]
        L.hyb_batch_step.argtypes = [P, C.c_int32, C.POINTER(Stats)]
        L.hyb_batch_destroy.argtypes = [P]
        L.hyb_batch_last_error.restype = C.c_char_p
        L.hyb_batch_last_error.argtypes = [P]
        L.hyb_build_cdf.argtypes = [P, C.c_int32, C.c_int32, P, P, P, P, P, C.c_size_t, P]
        L.hyb_quadrature.argtypes = [C.c_int32, P, P, P, C.POINTER(C.c_int32)]
        L.hyb_atomic_rate.argtypes = [C.c_int64, C.c_int64, P, C.POINTER(C.c_double)]
        _lib = L
    return _lib


def _check(status: int, handle=None) -> None:
    if status != HYB_OK:
        msg = lib().hyb_last_error(handle).decode()
        raise HybError(status, msg or lib().hyb_status_string(status).decode())


def _torch_cuda():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("a CUDA device is required: the hybrid path has no CPU fallback")
    return torch


def _dptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(C.POINTER(C.c_double))


def make_desc(spec: ProblemSpec) -> tuple[Desc, list]:
    keep = []

    def arr(x):
        if x is None:
            return None
        a = np.ascontiguousarray(np.asarray(x, dtype=np.float64).ravel())
        keep.append(a)
        return _dptr(a)

    d = Desc(nx=spec.nx, ny=spec.ny, lx=spec.lx, ly=spec.ly, sigma_a=arr(spec.sigma_a),
             sigma_s=arr(spec.sigma_s), Q=arr(spec.Q), ic_cell_w=arr(spec.ic), c=spec.c, dt=spec.dt,
             n_s=spec.n_s, sampler=spec.sampler, n_hist=spec.n_hist, seed=spec.seed,
             precision=spec.precision, sn_order=spec.sn_order, handoff_full=spec.handoff_full,
             sn_max_iter=spec.sn_max_iter, sn_tol=spec.sn_tol, w_min=spec.w_min,
             census_cap=spec.census_cap, sn_warm_start=spec.sn_warm_start, census_order=spec.census_order,
             sn_accel=spec.sn_accel, remap_variant=spec.remap_variant, sn_layout=spec.sn_layout,
             seg_limit=spec.seg_limit, wait_limit=spec.wait_limit, tally_copies=spec.tally_copies,
             sort_every=spec.sort_every, leg_sort_every=spec.leg_sort_every, priv_tile=spec.priv_tile)
    if spec.n_s_cell is not None:
        lim = np.ascontiguousarray(np.asarray(spec.n_s_cell, dtype=np.int32).ravel())
        keep.append(lim)
        d.n_s_cell = lim.ctypes.data_as(C.POINTER(C.c_int32))
    return d, keep


def workspace_size(spec: ProblemSpec) -> int:
    d, keep = make_desc(spec)
    n = C.c_size_t(0)
    _check(lib().hyb_workspace_size(C.byref(d), C.byref(n)))
    return int(n.value)


def priv_window(spec: ProblemSpec) -> tuple[int, int, int]:
    """(x0, y0, side) of the leg's shared-memory window for this problem (side 0: none)."""
    d, keep = make_desc(spec)
    x0, y0, s = C.c_int32(0), C.c_int32(0), C.c_int32(0)
    _check(lib().hyb_priv_window(C.byref(d), C.byref(x0), C.byref(y0), C.byref(s)))
    return x0.value, y0.value, s.value


class Problem:
    """One hybrid problem resident on the device (bank, tallies, CDFs, S_N state)."""

    def __init__(self, spec: ProblemSpec, stream=None, workspace=None):
        torch = _torch_cuda()
        self.spec = spec
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        d, keep = make_desc(spec)
        nbytes = C.c_size_t(0)
        _check(lib().hyb_workspace_size(C.byref(d), C.byref(nbytes)))
        self.ws_bytes = int(nbytes.value)
        if workspace is None:
            workspace = torch.empty(self.ws_bytes, dtype=torch.uint8, device="cuda")
        elif workspace.numel() * workspace.element_size() < self.ws_bytes:
            raise ValueError("workspace tensor too small")
        self.workspace = workspace
        h = C.c_void_p()
        _check(lib().hyb_create_problem(C.byref(d), C.c_void_p(workspace.data_ptr()), self.ws_bytes,
                                        C.c_void_p(self.stream.cuda_stream), C.byref(h)))
        self.h = h
        self.ncells = spec.nx * spec.ny

    def close(self) -> None:
        if getattr(self, "h", None):
            lib().hyb_destroy_problem(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # --- the hybrid step -------------------------------------------------------------------
    def mc_leg(self, stats: bool = True, trace=None) -> dict | None:
        s = Stats()
        ps = C.byref(s) if stats else None
        if trace is not None:
            _check(lib().hyb_mc_leg_trace(self.h, C.c_void_p(trace.data_ptr()), ps), self.h)
        else:
            _check(lib().hyb_mc_leg(self.h, ps), self.h)
        return s.as_dict() if stats else None

    # --- history-sharded leg --------------------------------------------------------------
    def exchange_block(self):
        """A zeroed device int64 tensor of the leg's exchange-block size."""
        torch = _torch_cuda()
        n = C.c_size_t(0)
        _check(lib().hyb_leg_exchange_bytes(self.h, C.byref(n)), self.h)
        return torch.zeros(int(n.value) // 8, dtype=torch.int64, device="cuda")

    def mc_leg_range(self, h0: int, h1: int, block, trace=None) -> None:
        """The leg over global history indices [h0, h1) into `block` (see exchange_block)."""
        _check(lib().hyb_mc_leg_range(self.h, h0, h1, C.c_void_p(block.data_ptr()), block.numel() * 8,
                                      C.c_void_p(trace.data_ptr()) if trace is not None else None), self.h)

    def mc_leg_reduce_finish(self, block, stats: bool = True) -> dict | None:
        """Make the (summed) exchange block the problem's leg."""
        s = Stats()
        _check(lib().hyb_mc_leg_reduce_finish(self.h, C.c_void_p(block.data_ptr()), block.numel() * 8,
                                              C.byref(s) if stats else None), self.h)
        return s.as_dict() if stats else None

    def collided_solve(self, stats: bool = True) -> dict | None:
        s = Stats()
        _check(lib().hyb_collided_solve(self.h, C.byref(s) if stats else None), self.h)
        return s.as_dict() if stats else None

    def remap(self, stats: bool = True) -> dict | None:
        s = Stats()
        _check(lib().hyb_remap(self.h, C.byref(s) if stats else None), self.h)
        return s.as_dict() if stats else None

    def step_async(self, n: int = 1) -> None:
        """n steps without statistics and without the final synchronisation (hyb_step_async): the
        last remap may still run on the problem's stream when this returns."""
        _check(lib().hyb_step_async(self.h, n), self.h)

    def remap_stats(self) -> dict:
        """Statistics of the last remap (of step or remap)."""
        s = Stats()
        _check(lib().hyb_remap_stats(self.h, C.byref(s)), self.h)
        return s.as_dict()

    def step(self, n: int = 1, stats: bool = True) -> list[dict] | None:
        arr = (Stats * max(n, 1))()
        _check(lib().hyb_step(self.h, n, arr if stats else None), self.h)
        return [arr[i].as_dict() for i in range(n)] if stats else None

    # --- data ------------------------------------------------------------------------------
    def tally(self, which: str) -> np.ndarray:
        n = self.ncells * (4 if which in ("handoff", "sn_phi") else 1)
        out = np.zeros(n)
        _check(lib().hyb_get_tally(self.h, TALLY[which], out.ctypes.data_as(C.c_void_p), n, 0), self.h)
        return out.reshape(self.ncells, 4) if n != self.ncells else out

    def tally_to(self, which: str, dst) -> None:
        """Copy a tally into a device tensor (float64, right size), asynchronously on the problem's
        stream."""
        _check(lib().hyb_get_tally(self.h, TALLY[which], C.c_void_p(dst.data_ptr()), dst.numel(), 1), self.h)

    def set_sn_phi(self, phi: np.ndarray) -> None:
        a = np.ascontiguousarray(phi, dtype=np.float64).ravel()
        _check(lib().hyb_set_sn_phi(self.h, a.ctypes.data_as(C.c_void_p), a.size), self.h)

    def capacity(self) -> int:
        c = C.c_int64(0)
        _check(lib().hyb_bank_capacity(self.h, C.byref(c)), self.h)
        return int(c.value)

    def bank(self) -> dict:
        cap = self.capacity()
        cell = np.zeros(cap, np.int32)
        f = [np.zeros(cap) for _ in range(5)]
        n = C.c_int64(cap)
        _check(lib().hyb_get_bank(self.h, cell.ctypes.data_as(C.c_void_p),
                                  *[a.ctypes.data_as(C.c_void_p) for a in f], C.byref(n)), self.h)
        k = int(n.value)
        return {"cell": cell[:k], "fx": f[0][:k], "fy": f[1][:k], "ox": f[2][:k], "oy": f[3][:k],
                "w": f[4][:k], "n": k}

    def set_bank(self, b: dict) -> None:
        n = int(b.get("n", len(b["w"])))
        cell = np.ascontiguousarray(b["cell"][:n], dtype=np.int32)
        f = [np.ascontiguousarray(b[k][:n], dtype=np.float64) for k in ("fx", "fy", "ox", "oy", "w")]
        _check(lib().hyb_set_bank(self.h, cell.ctypes.data_as(C.c_void_p),
                                  *[a.ctypes.data_as(C.c_void_p) for a in f], n), self.h)

    def set_bank_native(self, cell, fx, fy, ox, oy, w, n: int | None = None) -> None:
        """Replace the bank from arrays already in the problem's layout (torch tensors, page-locked
        host or device, int32 cells and float32/float64 values by the problem precision). The copy
        is asynchronous on the problem's stream; invalid particles are reported by the next step."""
        arrs = (cell, fx, fy, ox, oy, w)
        n = int(cell.numel()) if n is None else n
        want = "torch.float64" if self.spec.precision == FP64 else "torch.float32"
        if str(cell.dtype) != "torch.int32" or any(str(a.dtype) != want for a in arrs[1:]):
            raise TypeError(f"set_bank_native needs int32 cells and {want} values")
        if any(not a.is_contiguous() or a.numel() < n for a in arrs):
            raise ValueError("set_bank_native needs contiguous arrays of at least n values")
        _check(lib().hyb_set_bank_native(self.h, *[C.c_void_p(a.data_ptr()) for a in arrs], n), self.h)

    def set_step(self, k: int) -> None:
        _check(lib().hyb_set_step(self.h, k), self.h)

    @property
    def step_index(self) -> int:
        s = C.c_int64(0)
        _check(lib().hyb_get_step(self.h, C.byref(s)), self.h)
        return int(s.value)


def sobol_table(ndims: int) -> np.ndarray:
    out = np.zeros((ndims, 32), np.uint32)
    _check(lib().hyb_sobol_table(ndims, out.ctypes.data_as(C.c_void_p)))
    return out


def quadrature(order: int):
    ox, oy, w = np.zeros(40), np.zeros(40), np.zeros(40)
    m = C.c_int32(40)
    _check(lib().hyb_quadrature(order, ox.ctypes.data_as(C.c_void_p), oy.ctypes.data_as(C.c_void_p),
                                w.ctypes.data_as(C.c_void_p), C.byref(m)))
    return ox[:m.value], oy[:m.value], w[:m.value]


def points(seed: int, step: int, stream_id: int, sampler: int, i0: int, n: int, ndims: int, stream=None):
    """Point-set integers on the device, shape (n, ndims), as a torch int32 tensor (bit pattern)."""
    torch = _torch_cuda()
    out = torch.empty((n, ndims), dtype=torch.int32, device="cuda")
    s = stream if stream is not None else torch.cuda.current_stream()
    _check(lib().hyb_points(C.c_uint64(seed), step, stream_id, sampler, i0, n, ndims,
                            C.c_void_p(out.data_ptr()), C.c_void_p(s.cuda_stream)))
    return out


def atomic_rate(n_addr: int, n_ops: int = 1 << 28, stream=None) -> float:
    """Measured 64-bit global atomic additions per second to n_addr random addresses."""
    torch = _torch_cuda()
    s = stream if stream is not None else torch.cuda.current_stream()
    r = C.c_double(0.0)
    _check(lib().hyb_atomic_rate(n_addr, n_ops, C.c_void_p(s.cuda_stream), C.byref(r)))
    return float(r.value)


def build_cdf(w, nx: int, ny: int, stream=None):
    """Integer 2-D CDF of the device cell weights w (torch float64, nx*ny) with a torch-owned
    scratch block; returns (q, row_pre, col_pre, W_qmax) device tensors."""
    torch = _torch_cuda()
    nbytes = C.c_size_t(0)
    _check(lib().hyb_cdf_scratch_bytes(nx, ny, C.byref(nbytes)))
    scratch = torch.empty(int(nbytes.value), dtype=torch.uint8, device="cuda")
    q = torch.empty(nx * ny, dtype=torch.int64, device="cuda")
    rp = torch.empty(ny + 1, dtype=torch.int64, device="cuda")
    cp = torch.empty(ny * (nx + 1), dtype=torch.int64, device="cuda")
    wq = torch.empty(2, dtype=torch.float64, device="cuda")
    s = stream if stream is not None else torch.cuda.current_stream()
    _check(lib().hyb_build_cdf(C.c_void_p(w.data_ptr()), nx, ny, C.c_void_p(q.data_ptr()),
                               C.c_void_p(rp.data_ptr()), C.c_void_p(cp.data_ptr()), C.c_void_p(wq.data_ptr()),
                               C.c_void_p(scratch.data_ptr()), scratch.numel(), C.c_void_p(s.cuda_stream)))
    return q, rp, cp, wq


class Batch:
    """Many problems advanced together: one CUDA graph per step, the MC legs of all problems in
    one persistent work-queue launch. The problems must outlive the batch and are stepped only
    through it while it exists."""

    def __init__(self, problems: list, stream=None, tuning: dict | None = None):
        torch = _torch_cuda()
        self.problems = list(problems)
        self.stream = stream if stream is not None else torch.cuda.Stream()
        torch.cuda.synchronize()
        arr = (C.c_void_p * len(self.problems))(*[p.h.value for p in self.problems])
        h = C.c_void_p()
        st = lib().hyb_batch_create(arr, len(self.problems), C.c_void_p(self.stream.cuda_stream), C.byref(h))
        if st != HYB_OK:
            raise HybError(st, lib().hyb_batch_last_error(None).decode())
        self.h = h
        if tuning:
            self.set_tuning(**tuning)

    def _check(self, st):
        if st != HYB_OK:
            raise HybError(st, lib().hyb_batch_last_error(self.h).decode())

    def set_tuning(self, block=256, chunk=4096, ctas_per_sm=0, streams=8, use_graph=1):
        t = Tuning(block=block, chunk=chunk, ctas_per_sm=ctas_per_sm, streams=streams, use_graph=int(use_graph), pad=0)
        self._check(lib().hyb_batch_set_tuning(self.h, C.byref(t)))
        self.tuning = dict(block=block, chunk=chunk, ctas_per_sm=ctas_per_sm, streams=streams, use_graph=int(use_graph))

    def set_problems(self, problems: list) -> None:
        """Replace the resident problems, keeping streams, events and device buffers."""
        self.problems = list(problems)
        arr = (C.c_void_p * len(self.problems))(*[p.h.value for p in self.problems])
        self._check(lib().hyb_batch_set_problems(self.h, arr, len(self.problems)))

    def step(self, n: int = 1, stats: bool = True):
        arr = (Stats * len(self.problems))()
        self._check(lib().hyb_batch_step(self.h, n, arr if stats else None))
        return [arr[i].as_dict() for i in range(len(self.problems))] if stats else None

    def close(self):
        if getattr(self, "h", None):
            lib().hyb_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
