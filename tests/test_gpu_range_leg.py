"""The history-sharded MC leg and the bounded device loops.

Sharded leg (Sec. 2.3: histories are independent, each drawing its own point): the leg over
disjoint index ranges that cover [bank slots | births], with the exchange blocks summed as int64
words (what an all-reduce does) and finished, equals the whole leg bit for bit -- tallies, hand-off
moments, counters, weight sums and per-history records -- on the FP32 and FP64 paths, and the step
continues from it (collided solve, remap) exactly as from the whole leg.

Bounded loops: a history that reaches the per-problem segment bound, and a collided-solve pipeline
wait that reaches its poll bound, end their kernels with a status word the host maps to
HYB_ETIMEOUT; the context stays usable (a following problem steps normally).
"""
import numpy as np
import pytest

from paper_2511_16821_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _problem(spec, bank, step):
    from paper_2511_16821_gb300 import hyb
    P = hyb.Problem(spec)
    P.set_bank(bank)
    P.set_step(step)
    return P


@pytest.mark.parametrize("prec", [W.FP32, W.FP64])
def test_sharded_leg_equals_whole_leg(prec):
    import torch
    spec = W.checkerboard(n_s=2, n_hist=50_000, cells_per_block=5).with_(precision=prec)
    bank = W.random_bank(spec, 30_000, seed=1)
    N = 80_000
    A = _problem(spec, bank, 2)
    ta = torch.full((N, 4), -7, dtype=torch.int32, device="cuda")
    sa = A.mc_leg(trace=ta)
    B = _problem(spec, bank, 2)
    tb = torch.full((N, 4), -7, dtype=torch.int32, device="cuda")
    cuts = [(0, 12_345), (12_345, 30_000), (30_000, 30_000), (30_000, 61_111), (61_111, 10 ** 9)]
    total = B.exchange_block()
    for h0, h1 in cuts:
        blk = B.exchange_block()
        B.mc_leg_range(h0, h1, blk, trace=tb)
        total += blk
    sb = B.mc_leg_reduce_finish(total)
    for k in ("histories", "segments", "collisions", "leaked", "census", "killed", "reached_limit", "errors",
              "tally_adds", "w_source", "w_absorbed", "w_leaked", "w_census", "w_handoff", "w_killed"):
        assert sa[k] == sb[k], (k, sa[k], sb[k])
    for t in ("pre_raw", "post_raw", "pre", "post", "handoff"):
        assert np.array_equal(A.tally(t), B.tally(t)), t
    assert torch.equal(ta, tb)
    A.collided_solve()
    B.collided_solve()
    A.remap()
    B.remap()
    assert np.array_equal(A.tally("flux"), B.tally("flux"))
    ba, bb = A.bank(), B.bank()
    assert all(np.array_equal(ba[k], bb[k]) for k in ("cell", "fx", "fy", "ox", "oy", "w"))
    A.close()
    B.close()


def test_sharded_leg_rejects_bad_ranges_and_blocks():
    import torch
    from paper_2511_16821_gb300 import hyb
    spec = W.checkerboard(n_s=1, n_hist=1000, cells_per_block=1)
    P = hyb.Problem(spec)
    blk = P.exchange_block()
    for h0, h1 in ((-1, 5), (10, 3)):
        with pytest.raises(hyb.HybError) as e:
            P.mc_leg_range(h0, h1, blk)
        assert e.value.status == hyb.HYB_EINVAL
    with pytest.raises(hyb.HybError) as e:
        P.mc_leg_range(0, 10, blk[: blk.numel() // 2])
    assert e.value.status == hyb.HYB_ENOMEM
    # a remap needs a finished leg: the shard alone is not one
    P.mc_leg_range(0, 100, blk)
    with pytest.raises(hyb.HybError) as e:
        P.remap()
    assert e.value.status == hyb.HYB_ESTATE
    P.close()
    del torch


@pytest.mark.parametrize("prec", [W.FP32, W.FP64])
def test_segment_bound_returns_timeout(prec):
    # a 64 x 64 non-absorbing mesh crossed for c dt = 10 cm: histories run tens of segments, the
    # bound of 8 ends them as errors
    from paper_2511_16821_gb300 import hyb
    spec = W.homogeneous(n=64, L=1.0, sigma_a=0.0, sigma_s=0.5, Q=1.0, n_hist=2000, dt=10.0, n_s=1,
                         precision=prec).with_(seg_limit=8)
    P = hyb.Problem(spec)
    with pytest.raises(hyb.HybError) as e:
        P.mc_leg()
    assert e.value.status == hyb.HYB_ETIMEOUT
    P.close()
    ok = hyb.Problem(spec.with_(seg_limit=0))
    st = ok.mc_leg()
    assert st["errors"] == 0 and st["segments"] > 8 * st["histories"] // 2
    ok.close()


@pytest.mark.parametrize("prec", [W.FP32, W.FP64])
def test_sweep_wait_bound_returns_timeout(prec):
    # 256 x 256 cells: 8 row strips per ordinate, each waiting on the one below; one poll per wait
    # cannot see the traces of a strip that has not yet run its first steps
    from paper_2511_16821_gb300 import hyb
    base = W.homogeneous(n=256, L=4.0, sigma_a=0.1, sigma_s=1.0, Q=1.0, n_hist=20_000, dt=0.1, n_s=0,
                         precision=prec).with_(sn_order=8)
    P = hyb.Problem(base.with_(wait_limit=1))
    P.mc_leg()
    with pytest.raises(hyb.HybError) as e:
        P.collided_solve()
    assert e.value.status == hyb.HYB_ETIMEOUT
    P.close()
    Q = hyb.Problem(base)
    st = Q.step(1)[0]
    assert st["sn_iterations"] >= 1
    Q.close()
