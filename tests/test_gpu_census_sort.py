"""The census sort at the benchmark size: 2 x 10^6 remap slots (about a thousand tiles of the
one-sweep radix sort, a ragged last tile). Without a comb the remap keeps every survivor, so the
census sorted by cell must be exactly the slot-order census of the same remap under a stable sort
by cell (every field bit for bit); with the comb, the sorted census is in cell order and has the
size the comb gives."""
import numpy as np
import pytest

from paper_2511_16821_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FIELDS = ("cell", "fx", "fy", "ox", "oy", "w")


def _remap_bank(spec, bank):
    from paper_2511_16821_gb300 import hyb
    P = hyb.Problem(spec)
    P.set_bank(bank)
    P.set_step(2)
    P.mc_leg()
    P.collided_solve()
    st = P.remap()
    b = P.bank()
    P.close()
    return b, st


@pytest.mark.parametrize("prec", [W.FP32, W.FP64])
def test_cell_order_is_the_stable_sort_of_slot_order(prec):
    from paper_2511_16821_gb300 import hyb
    spec = W.checkerboard(n_s=2, n_hist=1_000_000).with_(precision=prec, sn_warm_start=1)
    P = hyb.Problem(spec)
    P.step(2)
    bank = P.bank()
    P.close()
    big = spec.with_(census_cap=4_000_000)   # above the 2 x 10^6 slots: no comb
    b0, s0 = _remap_bank(big.with_(census_order=0), bank)
    b1, s1 = _remap_bank(big.with_(census_order=1), bank)
    assert not s0["combed"] and not s1["combed"]
    assert b0["n"] == b1["n"] and b0["n"] > 1_000_000
    n = b0["n"]
    perm = np.argsort(b0["cell"][:n], kind="stable")
    for k in FIELDS:
        assert np.array_equal(b1[k][:n], b0[k][:n][perm]), k
    # with the comb (the default capacity): cell order, the comb's size
    b2, s2 = _remap_bank(spec.with_(census_order=1), bank)
    assert s2["combed"]
    c = b2["cell"][:b2["n"]]
    assert b2["n"] == s2["bank_size"] and np.all(np.diff(c) >= 0)
