"""Parity oracle for the scatter-limited hybrid (Q)MC / S_N method -- TEST INFRASTRUCTURE.

A ctypes wrapper over ``oracle.cpp``: plain, single-threaded FP64 C++ that restates the paper
(Krotz & McClarren, PHYSOR 2026) step by step and shares no code with the CUDA library. Only
``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference legs may
import it; the product path never does.

Paper map: Sec. 2.2 (hybrid time step, Eq. (R) remap), Sec. 2.3 (scatter-limited MC leg),
Sec. 2.4 (QMC points), App. B (Erlang transfer law, used as a pin).
"""
from __future__ import annotations

import contextlib
import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")

NS_INF = 2147483647
# Evaluation of the direction and optical-depth maps sin/cos(2 pi u), -log u (Sec. 2.3-2.4):
# LIBM = the host libm (the default, the plain reading of the paper's maps); SERIES = explicit
# series in a fixed operation order, pinned to a 40-digit reference (the recipe the GPU FP64 path
# also follows, so comparing with it checks the rest of that path bit for bit).
LIBM, SERIES = 0, 1
_elem_default = LIBM


@contextlib.contextmanager
def elementary(mode: int):
    """Evaluate the maps with `mode` (LIBM or SERIES) inside the block."""
    global _elem_default
    old = _elem_default
    _elem_default = mode
    try:
        yield
    finally:
        _elem_default = old
STREAM_INIT, STREAM_LEG_CENSUS, STREAM_LEG_SOURCE, STREAM_REMAP_SOURCE, STREAM_REMAP_COMB = range(5)
FATE_LEAKED, FATE_CENSUS, FATE_KILLED, FATE_ERROR = range(4)


def build(force: bool = False) -> str:
    """Compile liboracle.so with g++ (no FMA contraction, plain -O2)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared",
                               _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


class _Problem(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("lx", C.c_double), ("ly", C.c_double),
                ("sigma_a", C.POINTER(C.c_double)), ("sigma_s", C.POINTER(C.c_double)),
                ("Q", C.POINTER(C.c_double)), ("c", C.c_double), ("dt", C.c_double),
                ("n_s", C.c_int32), ("sampler", C.c_int32), ("n_hist", C.c_int64),
                ("seed", C.c_uint64), ("sn_order", C.c_int32), ("handoff_full", C.c_int32),
                ("w_min", C.c_double), ("census_cap", C.c_int64), ("sn_tol", C.c_double),
                ("sn_max_iter", C.c_int32), ("census_order", C.c_int32), ("remap_variant", C.c_int32),
                ("n_s_cell", C.POINTER(C.c_int32)), ("elem", C.c_int32), ("sort_every", C.c_int32)]


class _Bank(C.Structure):
    _fields_ = [("n", C.c_int64), ("cap", C.c_int64), ("cell", C.POINTER(C.c_int32)),
                ("fx", C.POINTER(C.c_double)), ("fy", C.POINTER(C.c_double)),
                ("ox", C.POINTER(C.c_double)), ("oy", C.POINTER(C.c_double)),
                ("w", C.POINTER(C.c_double))]


class _Stats(C.Structure):
    _fields_ = [(k, C.c_int64) for k in ("histories", "segments", "collisions", "leaked", "census",
                                         "killed", "reached_limit", "errors")] + \
               [(k, C.c_double) for k in ("w_source", "w_absorbed", "w_leaked", "w_census",
                                          "w_handoff", "w_killed")] + \
               [("sn_iterations", C.c_int32), ("pad", C.c_int32)]


def _stats_dict(s: _Stats) -> dict:
    return {k: getattr(s, k) for k, _ in _Stats._fields_ if k != "pad"}


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _lib.or_mix64.restype = C.c_uint64
        _lib.or_mix64.argtypes = [C.c_uint64]
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double)) if a is not None else None


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32)) if a is not None else None


@dataclass
class _Keep:
    """Holds the numpy arrays a ctypes struct points into."""
    sa: np.ndarray
    ss: np.ndarray
    q: np.ndarray | None
    nsc: np.ndarray | None = None


def _problem(spec, elem: int | None = None) -> tuple[_Problem, _Keep]:
    sa = np.ascontiguousarray(spec.sigma_a, dtype=np.float64).ravel()
    ss = np.ascontiguousarray(spec.sigma_s, dtype=np.float64).ravel()
    q = None if spec.Q is None else np.ascontiguousarray(spec.Q, dtype=np.float64).ravel()
    nsc = getattr(spec, "n_s_cell", None)
    nsc = None if nsc is None else np.ascontiguousarray(nsc, dtype=np.int32).ravel()
    p = _Problem(nx=spec.nx, ny=spec.ny, lx=spec.lx, ly=spec.ly, sigma_a=_dp(sa), sigma_s=_dp(ss),
                 Q=_dp(q), c=spec.c, dt=spec.dt, n_s=spec.n_s, sampler=spec.sampler,
                 n_hist=spec.n_hist, seed=spec.seed, sn_order=spec.sn_order,
                 handoff_full=spec.handoff_full, w_min=spec.w_min, census_cap=spec.census_cap,
                 sn_tol=spec.sn_tol, sn_max_iter=spec.sn_max_iter,
                 census_order=getattr(spec, "census_order", 0),
                 remap_variant=getattr(spec, "remap_variant", 0),
                 n_s_cell=None if nsc is None else nsc.ctypes.data_as(C.POINTER(C.c_int32)),
                 elem=_elem_default if elem is None else elem,
                 sort_every=getattr(spec, "sort_every", 0))
    return p, _Keep(sa, ss, q, nsc)


def empty_bank(cap: int) -> dict:
    return {"cell": np.zeros(cap, np.int32), "fx": np.zeros(cap), "fy": np.zeros(cap),
            "ox": np.zeros(cap), "oy": np.zeros(cap), "w": np.zeros(cap), "n": 0}


def _bank(b: dict | None) -> _Bank | None:
    if b is None:
        return None
    for k in ("fx", "fy", "ox", "oy", "w"):
        b[k] = np.ascontiguousarray(b[k], dtype=np.float64)
    b["cell"] = np.ascontiguousarray(b["cell"], dtype=np.int32)
    cap = len(b["w"])
    return _Bank(n=int(b.get("n", cap)), cap=cap, cell=_ip(b["cell"]), fx=_dp(b["fx"]),
                 fy=_dp(b["fy"]), ox=_dp(b["ox"]), oy=_dp(b["oy"]), w=_dp(b["w"]))


def _trim(b: dict, n: int) -> dict:
    out = {k: v[:n].copy() for k, v in b.items() if k != "n"}
    out["n"] = n
    return out


def mix64(z: int) -> int:
    return lib().or_mix64(z)


def sobol_table(ndims: int) -> np.ndarray:
    V = np.zeros((ndims, 32), np.uint32)
    rc = lib().or_sobol_table(ndims, V.ctypes.data_as(C.POINTER(C.c_uint32)))
    assert rc == 0
    return V


def points(seed: int, step: int, stream: int, sampler: int, i0: int, n: int, ndims: int) -> np.ndarray:
    out = np.zeros((n, ndims), np.uint32)
    rc = lib().or_points(C.c_uint64(seed), C.c_int64(step), C.c_int32(stream), C.c_int32(sampler),
                         C.c_int64(i0), C.c_int64(n), C.c_int32(ndims),
                         out.ctypes.data_as(C.POINTER(C.c_uint32)))
    assert rc == 0
    return out


def quadrature(order: int):
    ox, oy, oz, w = (np.zeros(64) for _ in range(4))
    m = lib().or_quadrature(order, _dp(ox), _dp(oy), _dp(oz), _dp(w))
    assert m > 0
    return ox[:m], oy[:m], oz[:m], w[:m]


def init_bank(spec, ic_cell_w: np.ndarray, elem: int | None = None) -> dict:
    p, keep = _problem(spec, elem)
    b = empty_bank(spec.n_hist)
    cb = _bank(b)
    icw = np.ascontiguousarray(ic_cell_w, dtype=np.float64).ravel()
    rc = lib().or_init_bank(C.byref(p), _dp(icw), C.byref(cb))
    assert rc == 0
    return _trim(b, cb.n)


def sample_births(spec, step: int, n: int, elem: int | None = None):
    p, keep = _problem(spec, elem)
    cell = np.zeros(n, np.int32)
    fx, fy, ox, oy, tf = (np.zeros(n) for _ in range(5))
    w0 = C.c_double(0)
    rc = lib().or_sample_births(C.byref(p), C.c_int64(step), C.c_int64(n), _ip(cell), _dp(fx), _dp(fy),
                                _dp(ox), _dp(oy), _dp(tf), C.byref(w0))
    assert rc == 0
    return dict(cell=cell, fx=fx, fy=fy, ox=ox, oy=oy, t_frac=tf, w0=w0.value)


def n_histories(spec, bank: dict | None) -> int:
    """Histories of a leg: the bank's particles, then n_hist births when Q is not zero."""
    nb = 0 if bank is None else int(bank.get("n", len(bank["w"])))
    has_src = spec.Q is not None and float(np.sum(spec.Q)) > 0
    return nb + (spec.n_hist if has_src else 0)


def mc_leg(spec, step: int, bank: dict | None, want_hist: bool = False, want_census: bool = False,
           want_margin: bool = False, h0: int = 0, h1: int | None = None, skip: np.ndarray | None = None,
           elem: int | None = None):
    """Returns dict(pre, post, mom, stats, pre_n, post_n, hist?, margin?, census?); tallies are raw
    track-length sums. Only histories with global index in [h0, h1) and skip[h] == 0 are tracked
    (skip: uint8 per history, or None); hist / margin rows cover those, in index order."""
    p, keep = _problem(spec, elem)
    nc = spec.nx * spec.ny
    pre, post, mom = np.zeros(nc), np.zeros(nc), np.zeros(4 * nc)
    st = _Stats()
    cb = _bank(bank)
    nh = n_histories(spec, bank)
    h1 = nh if h1 is None else min(h1, nh)
    nr = max(h1 - h0, 0)
    hist = np.zeros((max(nr, 1), 4), np.int32) if want_hist else None
    marg = np.zeros(max(nr, 1)) if want_margin else None
    cens = empty_bank(max(nh, 1)) if want_census else None
    cc = _bank(cens)
    pre_n, post_n = np.zeros(nc, np.int64), np.zeros(nc, np.int64)
    if skip is not None:
        skip = np.ascontiguousarray(skip, dtype=np.uint8)
        assert skip.size >= nh
    P64 = C.POINTER(C.c_int64)
    rc = lib().or_mc_leg_ex(C.byref(p), C.c_int64(step), C.byref(cb) if cb else None, C.c_int64(h0), C.c_int64(h1),
                            skip.ctypes.data_as(C.c_void_p) if skip is not None else None, _dp(pre), _dp(post),
                            _dp(mom), C.byref(st), _ip(hist) if hist is not None else None, _dp(marg),
                            C.byref(cc) if cc else None, pre_n.ctypes.data_as(P64), post_n.ctypes.data_as(P64))
    s = _stats_dict(st)
    out = dict(pre=pre, post=post, mom=mom.reshape(nc, 4), stats=s, rc=rc, pre_n=pre_n, post_n=post_n)
    if want_hist:
        out["hist"] = hist[: s["histories"]]
    if want_margin:
        out["margin"] = marg[: s["histories"]]
    if want_census:
        out["census"] = _trim(cens, cc.n)
    return out


def mc_leg_range(spec, step: int, bank: dict | None, h0: int, h1: int, elem: int | None = None):
    """The leg over global history indices [h0, h1) (bank slots first, then births), as one rank
    of a history-sharded leg: dict(pre, post, mom, stats, hist) for that range only."""
    p, keep = _problem(spec, elem)
    nc = spec.nx * spec.ny
    pre, post, mom = np.zeros(nc), np.zeros(nc), np.zeros(4 * nc)
    st = _Stats()
    cb = _bank(bank)
    hist = np.zeros((max(h1 - h0, 1), 4), np.int32)
    rc = lib().or_mc_leg_range(C.byref(p), C.c_int64(step), C.byref(cb) if cb else None, C.c_int64(h0),
                               C.c_int64(h1), _dp(pre), _dp(post), _dp(mom), C.byref(st), _ip(hist))
    s = _stats_dict(st)
    return dict(pre=pre, post=post, mom=mom.reshape(nc, 4), stats=s, rc=rc, hist=hist[: s["histories"]])


def sn_solve(spec, mom: np.ndarray, elem: int | None = None):
    p, keep = _problem(spec, elem)
    nc = spec.nx * spec.ny
    m = np.ascontiguousarray(mom, dtype=np.float64).ravel()
    phi = np.zeros(4 * nc)
    it = C.c_int32(0)
    rc = lib().or_sn_solve(C.byref(p), _dp(m), _dp(phi), C.byref(it))
    assert rc == 0
    return phi.reshape(nc, 4), it.value


def dg_sweep(nx, ny, lx, ly, sig, ox, oy, S, in_x=None, in_y=None):
    sig = np.ascontiguousarray(sig, dtype=np.float64).ravel()
    S = np.ascontiguousarray(S, dtype=np.float64).ravel()
    in_x = None if in_x is None else np.ascontiguousarray(in_x, dtype=np.float64).ravel()
    in_y = None if in_y is None else np.ascontiguousarray(in_y, dtype=np.float64).ravel()
    psi = np.zeros(4 * nx * ny)
    lib().or_dg_sweep(C.c_int32(nx), C.c_int32(ny), C.c_double(lx), C.c_double(ly), _dp(sig),
                      C.c_double(ox), C.c_double(oy), _dp(S), _dp(in_x), _dp(in_y), _dp(psi))
    return psi.reshape(nx * ny, 4)


def remap_density(spec, pre, post, phi, elem: int | None = None):
    p, keep = _problem(spec, elem)
    nc = spec.nx * spec.ny
    f = np.zeros(4 * nc)
    args = [None if a is None else np.ascontiguousarray(a, dtype=np.float64).ravel() for a in (pre, post, phi)]
    lib().or_remap_density(C.byref(p), *[_dp(a) for a in args], _dp(f))
    return f.reshape(nc, 4)


def remap(spec, step: int, bank: dict | None, pre, post, phi, elem: int | None = None):
    p, keep = _problem(spec, elem)
    nb = 0 if bank is None else int(bank.get("n", len(bank["w"])))
    cap = nb + spec.n_hist
    out = empty_bank(max(cap, 1))
    cb, co = _bank(bank), _bank(out)
    st = _Stats()
    combed = C.c_int32(0)
    args = [np.ascontiguousarray(a, dtype=np.float64).ravel() for a in (pre, post, phi)]
    rc = lib().or_remap(C.byref(p), C.c_int64(step), C.byref(cb) if cb else None,
                        *[_dp(a) for a in args], C.byref(co), C.byref(st), C.byref(combed))
    assert rc == 0, rc
    res = _trim(out, co.n)
    return res, _stats_dict(st), bool(combed.value)


def phase_keys(spec, bank: dict, elem: int | None = None):
    """The census_order-2 keys of the particles of a bank and the bits per coordinate."""
    p, keep = _problem(spec, elem)
    cb = _bank(bank)
    n = int(bank.get("n", len(bank["w"])))
    out = np.zeros(max(n, 1), np.uint32)
    bits = lib().or_phase_keys(C.byref(p), C.byref(cb), out.ctypes.data_as(C.c_void_p))
    return out[:n], bits


def remap_additive(spec, step: int, bank: dict | None, leg_census: dict | None, post, phi, elem: int | None = None):
    """Steps 3' and 4' (the previous hybrids' remap): the leg census followed by the survivors of
    births from sigma_s (phi_post + phi_c), combed. bank: the step-start bank."""
    p, keep = _problem(spec, elem)
    nb = 0 if bank is None else int(bank.get("n", len(bank["w"])))
    nl = 0 if leg_census is None else int(leg_census.get("n", len(leg_census["w"])))
    out = empty_bank(max(nl + spec.n_hist, 1))
    cb, cl, co = _bank(bank), _bank(leg_census), _bank(out)
    st = _Stats()
    combed = C.c_int32(0)
    args = [np.ascontiguousarray(a, dtype=np.float64).ravel() for a in (post, phi)]
    rc = lib().or_remap_additive(C.byref(p), C.c_int64(step), C.byref(cb) if cb else None,
                                 C.byref(cl) if cl else None, *[_dp(a) for a in args], C.byref(co),
                                 C.byref(st), C.byref(combed))
    assert rc == 0, rc
    return _trim(out, co.n), _stats_dict(st), bool(combed.value)


def step(spec, step_index: int, bank: dict | None, elem: int | None = None):
    p, keep = _problem(spec, elem)
    nc = spec.nx * spec.ny
    nb = 0 if bank is None else int(bank.get("n", len(bank["w"])))
    cap = nb + 2 * spec.n_hist
    out = empty_bank(max(cap, 1))
    cb, co = _bank(bank), _bank(out)
    flux, pre, post, mom, phi = np.zeros(nc), np.zeros(nc), np.zeros(nc), np.zeros(4 * nc), np.zeros(4 * nc)
    ls, rs = _Stats(), _Stats()
    rc = lib().or_step(C.byref(p), C.c_int64(step_index), C.byref(cb) if cb else None, C.byref(co),
                       _dp(flux), _dp(pre), _dp(post), _dp(mom), _dp(phi), C.byref(ls), C.byref(rs))
    assert rc == 0, rc
    return dict(bank=_trim(out, co.n), flux=flux, pre=pre, post=post, mom=mom.reshape(nc, 4),
                phi=phi.reshape(nc, 4), leg=_stats_dict(ls), remap=_stats_dict(rs))


def build_cdf(nx: int, ny: int, w: np.ndarray):
    """The integer 2-D CDF (q, row_pre, col_pre) of the cell weights w (sign ignored)."""
    w = np.ascontiguousarray(w, dtype=np.float64).ravel()
    q = np.zeros(nx * ny, np.int64)
    rp = np.zeros(ny + 1, np.int64)
    cp = np.zeros(ny * (nx + 1), np.int64)
    P = C.POINTER(C.c_int64)
    lib().or_build_cdf(C.c_int32(nx), C.c_int32(ny), _dp(w), q.ctypes.data_as(P), rp.ctypes.data_as(P),
                       cp.ctypes.data_as(P))
    return q, rp, cp


def sincos_2pi(u: np.ndarray, elem: int | None = None):
    u = np.ascontiguousarray(u, dtype=np.float64)
    s, c = np.zeros_like(u), np.zeros_like(u)
    lib().or_sincos_2pi(_dp(u), C.c_int64(u.size), _dp(s), _dp(c), C.c_int32(_elem_default if elem is None else elem))
    return s, c


def neg_log(u: np.ndarray, elem: int | None = None):
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.zeros_like(u)
    lib().or_neg_log(_dp(u), C.c_int64(u.size), _dp(out), C.c_int32(_elem_default if elem is None else elem))
    return out
