"""Asynchronous stepping (hyb_step_async) and the asynchronous device tally copy.

Steps launched without the final synchronisation, each followed by the next bank upload and a
device copy of the flux queued on the problem's stream, give the same census, fluxes and step
index as synchronous steps; an error inside the collided solve is still returned by the call
(its stop test reads the status word), and an unchecked step's status is read by the next
synchronising call.
"""
import numpy as np
import pytest

from paper_2511_16821_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [W.FP32, W.FP64])
def test_async_steps_equal_synchronous_steps(prec):
    import torch
    from paper_2511_16821_gb300 import hyb
    spec = W.checkerboard(n_s=2, n_hist=40_000, cells_per_block=5).with_(precision=prec, sn_warm_start=1)
    A = hyb.Problem(spec)
    B = hyb.Problem(spec)
    fa = torch.empty(spec.nx * spec.ny, dtype=torch.float64, device="cuda")
    for k in range(3):
        A.step(1)
        B.step_async(1)
        B.tally_to("flux", fa)          # queued behind the remap, no host wait
        torch.cuda.synchronize()
        assert np.array_equal(A.tally("flux"), fa.cpu().numpy()), k
    assert A.step_index == B.step_index == 3
    ba, bb = A.bank(), B.bank()
    assert ba["n"] == bb["n"]
    for key in ("cell", "fx", "fy", "ox", "oy", "w"):
        assert np.array_equal(ba[key][:ba["n"]], bb[key][:bb["n"]]), key
    # the synchronising call after the async steps reads a clean status
    st = B.remap_stats()
    assert st["errors"] == 0
    A.close()
    B.close()


def test_async_step_reports_a_solve_error():
    from paper_2511_16821_gb300 import hyb
    base = W.homogeneous(n=256, L=4.0, sigma_a=0.1, sigma_s=1.0, Q=1.0, n_hist=20_000, dt=0.1, n_s=0,
                         precision=W.FP32).with_(sn_order=8)
    P = hyb.Problem(base.with_(wait_limit=1))
    with pytest.raises(hyb.HybError) as e:
        P.step_async(1)
    assert e.value.status == hyb.HYB_ETIMEOUT
    P.close()
