"""The device times a step reports: the whole step, its three phases, and the MC leg kernel alone
(events around its launch), which lies inside the leg phase."""
import pytest

from paper_2511_16821_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_leg_kernel_time_inside_the_leg_phase():
    from paper_2511_16821_gb300 import hyb
    P = hyb.Problem(W.checkerboard(n_s=2, n_hist=100_000, cells_per_block=5).with_(sn_warm_start=1))
    for st in P.step(3):
        assert 0 < st["ms_leg_kernel"] <= st["ms_leg"] + 1e-3
        assert abs(st["ms"] - (st["ms_leg"] + st["ms_sn"] + st["ms_remap"])) < 1e-3
    lg = P.mc_leg()
    assert 0 < lg["ms_leg_kernel"] <= lg["ms"] + 1e-3
    P.close()
