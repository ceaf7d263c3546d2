"""Serving with continuous batching: requests arriving while others run are admitted as memory and
slots allow, all resident problems advance together each tick, and every request's result equals
solving it alone (bit for bit)."""
import numpy as np
import pytest

from paper_2511_16821_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _specs(n, seed):
    out = []
    for i in range(n):
        sp = W.random_batch_problem(seed, i, max_side=32)
        out.append(sp.with_(n_hist=min(sp.n_hist, 5000), sn_warm_start=1))
    return out


def test_served_results_equal_alone():
    from paper_2511_16821_gb300 import hyb
    from paper_2511_16821_gb300.serve import Server
    specs = _specs(8, 11)
    ticks = [0, 0, 1, 2, 2, 3, 5, 6]
    steps = [3, 1, 4, 2, 5, 3, 2, 4]
    srv = Server(budget_bytes=64e9)
    done = srv.run_schedule(list(zip(ticks, specs, steps)))
    srv.close()
    assert len(done) == 8
    assert srv.rebuilds >= 3            # membership changed while requests were in flight
    for r in done:
        P = hyb.Problem(r.spec)
        P.step(r.steps)
        assert np.array_equal(r.flux, P.tally("flux")), r.rid
        assert len(r.step_latency) == r.steps
        P.close()


def test_admission_respects_memory_budget():
    from paper_2511_16821_gb300 import hyb
    from paper_2511_16821_gb300.serve import Server
    specs = _specs(6, 12)
    sizes = [hyb.workspace_size(s) for s in specs]
    budget = sum(sorted(sizes)[-2:]) + 1          # at most two of the largest at once
    srv = Server(budget_bytes=budget)
    done = srv.run_schedule([(0, s, 2) for s in specs])
    srv.close()
    assert len(done) == 6
    assert srv.peak_used <= budget
    assert any(r.t_admit > r.t_arrival for r in done)   # some waited for memory
