"""Batched persistent execution: problems of the batched distribution (mesh side, sigma_t,
scattering ratio, N_s and history count drawn per problem) stepped together through one graph per
step give exactly the results of stepping each problem alone -- fluxes, census banks and counters
bit for bit, since every kernel works on one problem's data and all tallies are order-free."""
import numpy as np
import pytest

from paper_2511_16821_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _problems(n, seed, **kw):
    return [W.random_batch_problem(seed, p, max_side=64, **kw).with_(n_hist=min(20000, W.random_batch_problem(seed, p).n_hist),
                                                                     sn_warm_start=1)
            for p in range(n)]


@pytest.mark.parametrize("prec,order", [(W.FP32, 0), (W.FP64, 0), (W.FP32, 1)])
def test_batch_equals_alone(prec, order):
    import torch
    from paper_2511_16821_gb300 import hyb
    specs = [sp.with_(census_order=order) for sp in _problems(6, 3, precision=prec)]
    alone = []
    for sp in specs:
        P = hyb.Problem(sp)
        st = P.step(3)
        alone.append((P.tally("flux"), P.bank(), st[-1]))
        P.close()
    probs = [hyb.Problem(sp) for sp in specs]
    B = hyb.Batch(probs, tuning=dict(block=256, chunk=1024, streams=4))
    bst = B.step(3)
    torch.cuda.synchronize()
    for i, P in enumerate(probs):
        flux, bank, st = alone[i]
        assert np.array_equal(P.tally("flux"), flux), i
        b = P.bank()
        assert b["n"] == bank["n"]
        for k in ("cell", "fx", "fy", "ox", "oy", "w"):
            assert np.array_equal(b[k], bank[k]), (i, k)
        for k in ("histories", "segments", "collisions", "leaked", "census", "killed", "reached_limit"):
            assert bst[i][k] == st[k], (i, k)
        assert bst[i]["bank_size"] == st["bank_size"]
        assert bst[i]["w_source"] == st["w_source"] and bst[i]["w_census"] == st["w_census"]
    B.close()
    # tuning (including eager, graph-free issue) does not change results
    for tun in (dict(block=128, chunk=8192, streams=1), dict(block=256, chunk=2048, streams=3, use_graph=0)):
        probs2 = [hyb.Problem(sp) for sp in specs]
        B2 = hyb.Batch(probs2, tuning=tun)
        B2.step(3)
        for i, P in enumerate(probs2):
            assert np.array_equal(P.tally("flux"), alone[i][0]), (i, tun)
            assert np.array_equal(P.bank()["w"], alone[i][1]["w"]), (i, tun)
        B2.close()


def test_batch_rejects_halton_and_infinite_ns():
    """... a census sorted on some steps only (a step graph replays one sort decision), and the
    phased leg (its phases wait on the host)."""
    from paper_2511_16821_gb300 import hyb
    base = _problems(2, 5, precision=W.FP32)
    for bad in (base[1].with_(sampler=W.HALTON), base[1].with_(n_s=W.NS_INF),
                base[1].with_(census_order=1, sort_every=2), base[1].with_(leg_sort_every=2)):
        probs = [hyb.Problem(base[0]), hyb.Problem(bad)]
        with pytest.raises(hyb.HybError) as e:
            hyb.Batch(probs)
        assert e.value.status == hyb.HYB_EINVAL
        for P in probs:
            P.close()
