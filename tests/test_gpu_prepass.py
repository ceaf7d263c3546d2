"""The bank pre-pass of the Eq. (R) remap and the births drawn ahead.

hyb_step re-streams the step-start bank's slots on a side stream while the collided solve runs
(the straight sigma_t-attenuated flight to t_{n+1} needs neither the collided flux nor the remap
density), and the remap's pass A then streams only the births; on the same stream it draws the
next step's source births (they depend on the step index alone), which the next leg takes. The
same steps taken through the separate calls (mc_leg, collided_solve, remap: births drawn by the
leg, every slot streamed by pass A) give the same leg statistics, the same census bit for bit --
cells, positions, directions, weights -- the same fluxes and the same remap counters; the remap's
weight statistics, summed at the bank's own fixed-point scale for the bank slots, agree to
rounding. Covered: FP32 and FP64, a comb and a census that fits, a census sorted by cell, and a
pre-pass left pending by a failed step, ordered before the next leg.
"""
import numpy as np
import pytest

from paper_2511_16821_gb300 import workloads as W

pytestmark = pytest.mark.gpu

BANK_KEYS = ("cell", "fx", "fy", "ox", "oy", "w")


def _same_bank(a, b, what):
    assert a["n"] == b["n"], what
    for k in BANK_KEYS:
        assert np.array_equal(a[k][:a["n"]], b[k][:b["n"]]), (what, k)


@pytest.mark.parametrize("prec", [W.FP32, W.FP64])
@pytest.mark.parametrize("cap,order", [(0, 0), (10 ** 9, 0), (0, 1)])
def test_step_with_prepass_equals_separate_calls(prec, cap, order):
    from paper_2511_16821_gb300 import hyb
    spec = W.checkerboard(n_s=2, n_hist=40_000, cells_per_block=5).with_(
        precision=prec, census_cap=cap, census_order=order, sn_warm_start=1)
    A = hyb.Problem(spec)
    B = hyb.Problem(spec)
    for k in range(4):
        sa = A.step(1)[0]
        lb = B.mc_leg()
        # from the second step on, A's leg takes births drawn beside the previous solve
        for key in ("histories", "segments", "collisions", "leaked", "census", "killed", "tally_adds",
                    "w_source", "w_absorbed", "w_census", "w_handoff"):
            assert sa[key] == lb[key], (k, key, sa[key], lb[key])
        B.collided_solve()
        rb = B.remap()
        _same_bank(A.bank(), B.bank(), (prec, cap, order, k))
        assert np.array_equal(A.tally("flux"), B.tally("flux")), k
        assert sa["bank_size"] == rb["bank_size"] and sa["combed"] == rb["combed"], k
        ra = A.remap_stats()
        for key in ("histories", "segments", "leaked", "killed", "errors", "census", "combed"):
            assert ra[key] == rb[key], (k, key, ra[key], rb[key])
    A.close()
    B.close()


@pytest.mark.parametrize("prec", [W.FP32, W.FP64])
def test_remap_statistics_with_prepass(prec):
    """The remap statistics after a step with the pre-pass (bank slots summed at their own scale)
    against the same remap without it."""
    from paper_2511_16821_gb300 import hyb
    spec = W.checkerboard(n_s=2, n_hist=40_000, cells_per_block=5).with_(precision=prec, sn_warm_start=1)
    A = hyb.Problem(spec)
    A.step(2)
    bank = A.bank()
    A.set_bank(bank)
    A.set_step(2)
    A.step(1)
    ra = A.remap_stats()
    B = hyb.Problem(spec)
    B.step(2)
    B.set_bank(bank)
    B.set_step(2)
    B.mc_leg()
    B.collided_solve()
    rb = B.remap()
    for k in ("histories", "segments", "leaked", "killed", "errors", "census", "combed", "bank_size"):
        assert ra[k] == rb[k], (k, ra[k], rb[k])
    tol = 1e-6 if prec == W.FP32 else 1e-13
    for k in ("w_source", "w_absorbed", "w_leaked", "w_killed", "w_census"):
        assert abs(ra[k] - rb[k]) <= tol * max(abs(rb[k]), abs(rb["w_source"])), (k, ra[k], rb[k])
    _same_bank(A.bank(), B.bank(), prec)
    A.close()
    B.close()


def test_pending_prepass_ordered_before_the_next_leg():
    """A step that fails in the collided solve (its pipeline wait bound exhausted) leaves its bank
    pre-pass pending; the next call that reuses the staging buffer (here the next leg, after
    set_bank and set_step) is ordered after it and the pre-pass is forgotten: that leg equals the
    leg of a fresh problem on the same bank and step."""
    from paper_2511_16821_gb300 import hyb
    base = W.homogeneous(n=256, L=4.0, sigma_a=0.1, sigma_s=1.0, Q=1.0, n_hist=20_000, dt=0.1, n_s=0,
                         precision=W.FP32).with_(sn_order=8)
    bank = W.random_bank(base, 15_000, seed=3)
    P = hyb.Problem(base.with_(wait_limit=1))
    P.set_bank(bank)
    P.set_step(1)
    with pytest.raises(hyb.HybError) as e:
        P.step(1)
    assert e.value.status == hyb.HYB_ETIMEOUT
    P.set_bank(bank)
    P.set_step(1)
    sa = P.mc_leg()
    Q = hyb.Problem(base)
    Q.set_bank(bank)
    Q.set_step(1)
    sb = Q.mc_leg()
    for k in ("histories", "segments", "collisions", "leaked", "census", "w_source", "w_census", "w_handoff"):
        assert sa[k] == sb[k], (k, sa[k], sb[k])
    for t in ("pre_raw", "post_raw", "handoff"):
        assert np.array_equal(P.tally(t), Q.tally(t)), t
    P.close()
    Q.close()


@pytest.mark.parametrize("next_step", [1, 5])
def test_births_drawn_ahead_only_for_their_step(next_step):
    """After a step, the births of step 1 lie ready; a leg of step 1 takes them, a leg of any other
    step (set_step) draws its own: either leg equals a fresh problem's leg of that step."""
    from paper_2511_16821_gb300 import hyb
    spec = W.checkerboard(n_s=2, n_hist=40_000, cells_per_block=5).with_(precision=W.FP64, sn_warm_start=1)
    bank = W.random_bank(spec, 30_000, seed=7)
    A = hyb.Problem(spec)
    A.set_bank(bank)
    A.step(1)
    A.set_bank(bank)
    A.set_step(next_step)
    sa = A.mc_leg()
    B = hyb.Problem(spec)
    B.set_bank(bank)
    B.set_step(next_step)
    sb = B.mc_leg()
    for k in ("histories", "segments", "collisions", "leaked", "census", "killed", "tally_adds",
              "w_source", "w_census", "w_handoff"):
        assert sa[k] == sb[k], (k, sa[k], sb[k])
    for t in ("pre_raw", "post_raw", "handoff"):
        assert np.array_equal(A.tally(t), B.tally(t)), t
    A.close()
    B.close()
