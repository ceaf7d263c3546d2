"""Shared checks of the GPU parity tests: the CUDA path's leg results against the oracle's.

Bars: integers bit-exact; FP64 tallies within 1e-12 relative per cell; FP32 within 1e-4 relative
on the cells a tally resolves (above 1e-3 of its peak, at least 32 scored segments), every cell
above 1e-3 of the peak within 1e-2, and the tally-weighted error within 1e-5; records that differ
from the oracle's only at decisions within rounding of a tie, each reported with its margin.
"""
import math

import numpy as np

FP64_RTOL = 1e-12
FP32_RTOL = 1e-4


def check_counts(g, o):
    for k in ("histories", "segments", "collisions", "leaked", "census", "killed", "reached_limit", "errors"):
        assert g[k] == o[k], (k, g[k], o[k])
    for k in ("w_source", "w_absorbed", "w_leaked", "w_census", "w_handoff", "w_killed"):
        assert math.isclose(g[k], o[k], rel_tol=1e-12, abs_tol=1e-14 * max(1.0, abs(o["w_source"]))), (k, g[k], o[k])


def rel_err(g, o, floor):
    return np.abs(g - o) / np.maximum(np.abs(o), floor)


def check_fp64_tallies(g, o):
    for key in ("pre", "post"):
        a, b = g[key], o[key]
        assert np.all(np.abs(a - b) <= FP64_RTOL * np.abs(b) + 1e-300), (key, np.max(rel_err(a, b, 1e-300)))
        assert np.all((a == 0) == (b == 0)), key
    m_g, m_o = g["mom"], o["mom"]
    bound = np.abs(m_o[:, :1])            # |m_j| <= m_0 since |P_j| <= 1 on the cell
    assert np.all(np.abs(m_g[:, 0] - m_o[:, 0]) <= FP64_RTOL * np.abs(m_o[:, 0]) + 1e-300)
    assert np.all(np.abs(m_g[:, 1:] - m_o[:, 1:]) <= FP64_RTOL * (np.abs(m_o[:, 1:]) + bound) + 1e-300)


def start_weights(spec, bank):
    """w_start of every history of a leg, in index order (bank slots, then births of w0 each)."""
    nb = 0 if bank is None else int(bank["n"])
    ws = [np.abs(np.asarray(bank["w"][:nb], np.float64))] if nb else []
    if spec.Q is not None and np.sum(spec.Q) > 0:
        area = (spec.lx / spec.nx) * (spec.ly / spec.ny)
        ws.append(np.full(spec.n_hist, float(np.sum(spec.Q)) * area * spec.dt / spec.n_hist))
    return np.concatenate(ws) if ws else np.zeros(0)


# A record of the FP64 path that differs from the libm oracle's must come from a decision whose two
# smallest event distances lie within rounding of each other: relative gap below this in the oracle
# (the two evaluations of the direction and depth maps differ in the last bit).
FLIP_MARGIN_FP64 = 1e-10


def flips(g, o):
    """Indices of the histories whose records differ, with the oracle's decision margins."""
    if not g["hist"].size:
        return np.zeros(0, np.int64), np.zeros(0)
    mism = np.nonzero(np.any(g["hist"] != o["hist"], axis=1))[0]
    return mism, o["margin"][mism] if "margin" in o else np.full(mism.size, np.nan)


# FP64 against the libm oracle, a cell of any support: the last-bit differences of the maps place a
# sliver segment (a collision or census point a few 1e-15 cm from a face) with a relative length
# error far above 1e-16; measured up to 2.5e-12 in single-segment cells of the 112^2 benchmark leg
# (cells with >= 4 segments stay within 1.1e-14).
FP64_RTOL_UNRESOLVED = 1e-9


def check_fp64_libm(g, o, spec, bank, name):
    """The FP64 path against the libm oracle: its direction and optical-depth maps differ from
    libm's in the last bit, so a record may differ only where a decision ties to rounding; every
    flip is reported with its margin. Tallies: 1e-12 relative on every cell with >= 32 scored
    segments, 1e-9 on every cell, apart from the flipped histories, each of which moves at most
    2 w_start c dt of track length (x sigma_s,max for the hand-off moments)."""
    mism, marg = flips(g, o)
    print(f"\nFP64 vs libm oracle {name}: {mism.size} of {len(o['hist'])} records differ; margins "
          f"{np.array2string(marg, precision=2)}; smallest margin overall {np.min(o['margin']) if o['margin'].size else 1:.2e}")
    assert np.all(marg < FLIP_MARGIN_FP64), (mism[:5], marg[:5])
    ws = start_weights(spec, bank)
    A = 2.0 * spec.c * spec.dt * float(np.sum(ws[mism])) if mism.size else 0.0
    gs, os_ = g["stats"], o["stats"]
    assert gs["histories"] == os_["histories"]
    slack = int(np.sum(g["hist"][mism, 3]) + np.sum(o["hist"][mism, 3])) if mism.size else 0
    for k in ("segments", "collisions", "leaked", "census", "killed", "reached_limit", "errors"):
        assert abs(gs[k] - os_[k]) <= slack, (k, gs[k], os_[k])
    rep = {}
    for key, cnt in (("pre", o["pre_n"]), ("post", o["post_n"])):
        a, b = g[key], o[key]
        err = np.abs(a - b) - A
        res = cnt >= MIN_SEGMENTS
        assert np.all(err[res] <= FP64_RTOL * np.abs(b[res]) + 1e-300), (key, np.max(rel_err(a[res], b[res], 1e-300)))
        assert np.all(err <= FP64_RTOL_UNRESOLVED * np.abs(b) + 1e-300), (key, np.max(rel_err(a, b, 1e-300)))
        rep[key] = float(np.max(rel_err(a, b, 1e-300))) if a.size else 0.0
    m_g, m_o = g["mom"], o["mom"]
    Am = A * float(np.max(spec.sigma_s)) if mism.size else 0.0
    bound = np.abs(m_o[:, :1])
    res = o["post_n"] >= MIN_SEGMENTS
    e0 = np.abs(m_g[:, 0] - m_o[:, 0]) - Am
    e1 = np.abs(m_g[:, 1:] - m_o[:, 1:]) - Am
    assert np.all(e0[res] <= FP64_RTOL * np.abs(m_o[res, 0]) + 1e-300)
    assert np.all(e1[res] <= FP64_RTOL * (np.abs(m_o[res, 1:]) + bound[res]) + 1e-300)
    assert np.all(e0 <= FP64_RTOL_UNRESOLVED * np.abs(m_o[:, 0]) + 1e-300)
    assert np.all(e1 <= FP64_RTOL_UNRESOLVED * (np.abs(m_o[:, 1:]) + bound) + 1e-300)
    print(f"  FP64 vs libm {name}: max rel tally difference, every cell {rep}")
    if not mism.size:
        check_counts(gs, os_)


MIN_SEGMENTS = 32
# Unrestricted FP32 bound (every cell above 1e-3 of its tally's peak, whatever its support): a cell
# scored by a few segments can hold a sliver segment a few 1e-7 cm long whose FP32 length carries a
# percent-level relative error (measured maximum 2.7e-3 on the 112^2 benchmark leg).
FP32_RTOL_UNRESOLVED = 1e-2


# FP32 in optically thick cells (sigma_t dx of order 1 or more): a history that crosses a face just
# short of its next collision keeps the small difference of two nearly equal optical depths, so the
# next flight's length carries a relative error far above FP32's 6e-8 and a resolved cell's tally
# can be off by a few 1e-4 (measured 2.0e-4 on a batch problem with sigma_t dx up to 2.4, 2.8e-4 on
# the 1024^2 diffusive mesh with sigma_t dx up to 10).
FP32_RTOL_THICK = 5e-4


def fp32_check(g, o, name, without=None, rtol=FP32_RTOL):
    """FP32 tracking against the FP64 oracle: record flips are reported with their margins, not
    failed (FP32 rounding, amplified where the remaining optical depth cancels, moves a decision
    whose gap is small), and the tallies are graded with the flipped histories taken out of both
    sides (`without(indices) -> (g, o)` reruns both legs without them): 1e-4 relative on the cells
    they resolve (>= 32 scored segments, above 1e-3 of the peak), every cell above 1e-3 of the peak
    within 1e-2 (the worst cell's segment count reported), the tally-weighted mean within 1e-5."""
    mism, marg = flips(g, o)
    print(f"\nFP32 {name}: history flips {mism.size}/{len(o['hist'])} with margins "
          f"{np.array2string(marg, precision=2)}")
    assert mism.size <= max(4, len(o["hist"]) // 20000)
    if mism.size:
        assert without is not None, "flipped histories need a regrade without them"
        g, o = without(mism)
    rep = fp32_report(g, o)
    raw = fp32_report(g, o, min_seg=0)
    wtd = fp32_weighted(g, o)
    worst = fp32_worst(g, o)
    print(f"  FP32 {name}{' (flipped histories taken out)' if mism.size else ''}: max rel err (cells >= 1e-3 "
          f"peak, >= {MIN_SEGMENTS} segments) {rep}; unrestricted {raw} (worst cell: {worst}); weighted {wtd}")
    for k, v in rep.items():
        assert v < rtol, (k, v)
    for k, v in raw.items():
        assert v < FP32_RTOL_UNRESOLVED, (k, v)
    for k, v in wtd.items():
        assert v < 1e-5, (k, v)
    return rep, raw, wtd


def fp32_worst(g, o, frac=1e-3):
    """Segments scored in the cell of the largest unrestricted relative error, per tally."""
    out = {}
    for key, cnt in (("pre", o["pre_n"]), ("post", o["post_n"])):
        a, b = g[key], o[key]
        peak = np.max(np.abs(b)) if b.size else 0
        sel = np.nonzero(np.abs(b) >= frac * peak)[0] if peak > 0 else np.zeros(0, np.int64)
        if sel.size:
            k = sel[np.argmax(rel_err(a[sel], b[sel], 1e-300))]
            out[key] = f"cell {k}: {int(cnt[k])} segments, rel err {float(rel_err(a[k:k+1], b[k:k+1], 1e-300)[0]):.1e}"
    return out


def fp32_report(g, o, frac=1e-3, min_seg=MIN_SEGMENTS):
    """Max relative FP32 error of every tally on cells above `frac` of its peak that hold at least
    `min_seg` scored segments (pre/post: their own counts; moments: the post counts).

    FP32 tracking carries directions and positions to ~6e-8 relative, so its trajectory sits
    ~1e-8 cm from the FP64 one after a step; a cell whose tally is one short segment ending on a
    nearby face then differs by up to ~1e-3 relative. Such a cell holds a single history (its
    Monte Carlo error is ~100 %); the bar applies to cells the tally resolves (>= 32 segments,
    statistical error <= 18 %), and the tally-weighted error bounds the sparse rest."""
    rep = {}
    cnt = {"pre": o["pre_n"], "post": o["post_n"]}
    for key in ("pre", "post"):
        a, b = g[key], o[key]
        peak = np.max(np.abs(b)) if b.size else 0
        sel = (np.abs(b) >= frac * peak) & (cnt[key] >= min_seg) if peak > 0 else np.zeros_like(b, bool)
        rep[key] = float(np.max(rel_err(a[sel], b[sel], 1e-300))) if sel.any() else 0.0
    for j in range(4):
        a, b = g["mom"][:, j], o["mom"][:, j]
        peak = np.max(np.abs(o["mom"][:, 0])) if o["mom"].size else 0
        sel = (np.abs(o["mom"][:, 0]) >= frac * peak) & (o["post_n"] >= min_seg) if peak > 0 \
            else np.zeros_like(b, bool)
        rep[f"mom{j}"] = float(np.max(np.abs(a[sel] - b[sel]) / np.abs(o["mom"][sel, 0]))) if sel.any() else 0.0
    return rep


def fp32_weighted(g, o):
    """Tally-weighted mean relative FP32 error (sum |g - o| / sum |o|) per tally."""
    return {k: float(np.sum(np.abs(g[k] - o[k])) / max(np.sum(np.abs(o[k])), 1e-300)) for k in ("pre", "post")}
