"""The phased MC leg (leg_sort_every = K): histories advance at most K segments per phase and the
live ones are compacted and sorted by cell between phases. Every history does the fused leg's
arithmetic on the same points and every sum is an order-free integer sum, so the leg equals the
fused leg bit for bit: per-history records (final cell, fate, scatters, segments), counters,
weight statistics and raw tallies; and whole steps equal theirs (banks, fluxes). Covered: FP32 and
FP64, K = 1 (a phase per segment), 3 and 16, N_s = 0, 2 and infinity (the census kept as
particles), a leg without births."""
import numpy as np
import pytest

from paper_2511_16821_gb300 import workloads as W

pytestmark = pytest.mark.gpu

KEYS = ("histories", "segments", "collisions", "leaked", "census", "killed", "reached_limit", "errors",
        "tally_adds", "w_source", "w_absorbed", "w_leaked", "w_census", "w_handoff", "w_killed")


def _leg(spec, bank, step):
    import torch
    from paper_2511_16821_gb300 import hyb
    P = hyb.Problem(spec.with_(ic=None))
    P.set_bank(bank)
    P.set_step(step)
    n = int(bank["n"]) + (spec.n_hist if spec.Q is not None else 0)
    tr = torch.full((max(n, 1), 4), -7, dtype=torch.int32, device="cuda")
    st = P.mc_leg(trace=tr)
    out = (st, {t: P.tally(t) for t in ("pre_raw", "post_raw", "handoff")}, tr.cpu().numpy())
    P.close()
    return out


@pytest.mark.parametrize("prec", [W.FP32, W.FP64])
@pytest.mark.parametrize("n_s", [0, 2])
def test_phased_leg_equals_fused(prec, n_s):
    spec = W.checkerboard(n_s=n_s, n_hist=50_000, cells_per_block=5).with_(precision=prec)
    bank = W.random_bank(spec, 40_000, seed=11)
    ref = _leg(spec, bank, 2)
    for k in (1, 3, 16):
        got = _leg(spec.with_(leg_sort_every=k), bank, 2)
        for key in KEYS:
            assert got[0][key] == ref[0][key], (k, key, got[0][key], ref[0][key])
        for t in ref[1]:
            assert np.array_equal(got[1][t], ref[1][t]), (k, t)
        assert np.array_equal(got[2], ref[2]), k


def test_phased_leg_bank_only():
    spec = W.pulse(n_hist=20_000).with_(precision=W.FP32)
    bank = W.random_bank(spec, 15_000, seed=12)
    ref = _leg(spec, bank, 1)
    got = _leg(spec.with_(leg_sort_every=2), bank, 1)
    for key in KEYS:
        assert got[0][key] == ref[0][key], key
    for t in ref[1]:
        assert np.array_equal(got[1][t], ref[1][t]), t
    assert np.array_equal(got[2], ref[2])


@pytest.mark.parametrize("prec,n_s", [(W.FP32, 2), (W.FP64, 2), (W.FP32, W.NS_INF)])
def test_phased_steps_equal_fused(prec, n_s):
    """Three whole steps: the phased leg gives the fused steps' banks and fluxes bit for bit."""
    from paper_2511_16821_gb300 import hyb
    spec = W.checkerboard(n_s=n_s, n_hist=40_000, cells_per_block=5).with_(precision=prec, sn_warm_start=1)
    out = []
    for k in (0, 2):
        P = hyb.Problem(spec.with_(leg_sort_every=k))
        st = P.step(3)
        out.append((P.tally("flux"), P.bank(), st))
        P.close()
    (fa, ba, sa), (fb, bb, sb) = out
    assert np.array_equal(fa, fb)
    assert ba["n"] == bb["n"]
    for key in ("cell", "fx", "fy", "ox", "oy", "w"):
        assert np.array_equal(ba[key][:ba["n"]], bb[key][:bb["n"]]), key
    for x, y in zip(sa, sb):
        for key in ("histories", "segments", "census", "bank_size", "w_census", "sn_iterations"):
            assert x[key] == y[key], key


@pytest.mark.parametrize("prec", [W.FP32, W.FP64])
def test_phased_leg_segment_bound(prec):
    """Histories that reach the segment bound end as errors in the phase that reaches it (the
    phases stay bounded) and the leg returns HYB_ETIMEOUT, as the fused leg does; without the
    bound the phased leg equals the fused one on these long histories."""
    from paper_2511_16821_gb300 import hyb
    spec = W.homogeneous(n=64, L=1.0, sigma_a=0.0, sigma_s=0.5, Q=1.0, n_hist=2000, dt=10.0, n_s=1,
                         precision=prec)
    for k in (0, 3):
        P = hyb.Problem(spec.with_(seg_limit=8, leg_sort_every=k))
        with pytest.raises(hyb.HybError) as e:
            P.mc_leg()
        assert e.value.status == hyb.HYB_ETIMEOUT, k
        P.close()
    res = []
    for k in (0, 5):
        P = hyb.Problem(spec.with_(leg_sort_every=k))
        st = P.mc_leg()
        res.append((st, P.tally("pre_raw"), P.tally("post_raw")))
        P.close()
    assert res[0][0]["segments"] > 8 * res[0][0]["histories"] // 2
    for key in KEYS:
        assert res[0][0][key] == res[1][0][key], key
    assert np.array_equal(res[0][1], res[1][1]) and np.array_equal(res[0][2], res[1][2])
