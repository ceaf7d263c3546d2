"""The tuning knobs of a problem: tally copies (the privatisation of the leg's fixed-point
tallies) and the census sort interval.

Tally copies only spread the leg's atomic additions over more addresses; the normalisation sums
the copies exactly, so every tally and counter is the same bit for bit for any number of copies.
The sort interval changes the census (the comb runs along a sorted census only on every
sort_every-th step), so it is checked against the oracle taking the same steps.
"""
import numpy as np
import pytest

from paper_2511_16821_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    import torch
    from paper_2511_16821_gb300 import hyb
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    hyb.lib()
    return hyb


@pytest.mark.parametrize("prec", [W.FP32, W.FP64])
def test_tally_copies_do_not_change_the_leg(H, prec):
    """Copies of the tally arrays and the shared-memory window (priv_tile: the source block's cells
    and beyond; 32 is wider than the 25-cell source block, 7 straddles its edge) change where the
    integer additions land, never their sums."""
    hyb = H
    spec = W.checkerboard(n_s=2, n_hist=60_000, cells_per_block=5).with_(precision=prec)
    bank = W.random_bank(spec, 40_000, seed=5)
    ref = None
    for copies, priv in ((0, 0), (1, 0), (3, 0), (8, 0), (0, 7), (1, 16), (4, 32)):
        P = hyb.Problem(spec.with_(tally_copies=copies, priv_tile=priv))
        P.set_bank(bank)
        P.set_step(2)
        st = P.mc_leg()
        got = (st, {t: P.tally(t) for t in ("pre_raw", "post_raw", "handoff")})
        P.close()
        if ref is None:
            ref = got
            continue
        for k in ("histories", "segments", "collisions", "tally_adds", "w_source", "w_absorbed", "w_handoff"):
            assert got[0][k] == ref[0][k], (copies, priv, k)
        for t in ("pre_raw", "post_raw", "handoff"):
            assert np.array_equal(got[1][t], ref[1][t]), (copies, priv, t)


@pytest.mark.parametrize("order", [1, 2])
def test_sort_interval_matches_oracle(H, orc, order):
    """FP64, census sorted on every second step only, three steps of the pure-MC census path (a
    pulse) and of the hybrid remap with the comb (a small checkerboard): banks cell for cell and
    fluxes to rounding against the oracle taking the same steps."""
    cb = W.checkerboard(n_s=2, n_hist=6000, cells_per_block=2)
    for spec in (W.pulse(n_hist=4096).with_(n_s=W.NS_INF), cb.with_(census_cap=3000)):
        spec = spec.with_(precision=W.FP64, sn_tol=1e-13, census_order=order, sort_every=2)
        P = H.Problem(spec)
        ob = orc.init_bank(spec, spec.ic, elem=orc.SERIES) if spec.ic is not None else None
        for k in range(3):
            st = P.step(1)[0]
            r = orc.step(spec, k, ob, elem=orc.SERIES)
            ob = r["bank"]
            gb = P.bank()
            assert gb["n"] == ob["n"] and st["bank_size"] == ob["n"], (spec.name, k)
            assert np.array_equal(gb["cell"], ob["cell"]), (spec.name, k)
            assert np.allclose(gb["w"], ob["w"], rtol=1e-10, atol=0), (spec.name, k)
            f = P.tally("flux")
            assert np.allclose(f, r["flux"], rtol=1e-9, atol=1e-12 * np.max(np.abs(r["flux"]))), (spec.name, k)
        P.close()


def test_tune_problem_picks_a_timed_candidate(H):
    """The single-problem tuner times every candidate of the space and returns the fastest, as a
    spec with those knobs; the tuned problem's step equals the default problem's (copies never
    change a result)."""
    from paper_2511_16821_gb300 import autotune
    spec = W.checkerboard(n_s=2, n_hist=40_000, cells_per_block=5).with_(precision=W.FP32, census_order=1)
    r = autotune.tune_problem(spec, steps=2, warmup=3, space={"tally_copies": (1, 4), "sort_every": (1, 2)})
    assert len(r["table"]) == 4
    assert all(t["ms_per_step"] > 0 for t in r["table"])
    assert r["ms_per_step"] == min(t["ms_per_step"] for t in r["table"])
    assert r["spec"].tally_copies == r["best"]["tally_copies"] and r["spec"].sort_every == r["best"]["sort_every"]
    a = H.Problem(spec.with_(sort_every=r["best"]["sort_every"]))
    b = H.Problem(r["spec"])
    sa, sb = a.step(2), b.step(2)
    for x, y in zip(sa, sb):
        for k in ("histories", "segments", "census", "combed", "bank_size", "w_census"):
            assert x[k] == y[k], k
    assert np.array_equal(a.tally("flux"), b.tally("flux"))
    a.close()
    b.close()
