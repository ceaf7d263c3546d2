"""Host logic of the serving loop (no device): the Poisson request stream and the latency summary."""
import math

import numpy as np

from paper_2511_16821_gb300 import serve
from paper_2511_16821_gb300 import workloads as W


def test_poisson_arrivals_rate_and_requests():
    lam, dur = 200.0, 20.0
    arr = serve.poisson_arrivals(lam, dur, seed=3, max_side=64)
    t = np.array([a[0] for a in arr])
    assert np.all(np.diff(t) > 0) and t[-1] <= dur
    # count ~ Poisson(lam dur): within 4 standard deviations
    assert abs(len(arr) - lam * dur) < 4 * math.sqrt(lam * dur)
    # exponential gaps: mean 1/lam, coefficient of variation ~1
    g = np.diff(np.concatenate([[0.0], t]))
    assert abs(g.mean() * lam - 1) < 0.05 and abs(g.std() / g.mean() - 1) < 0.05
    steps = np.array([a[2] for a in arr])
    assert steps.min() >= 1 and steps.max() <= 64
    for _, spec, _ in arr[:50]:
        assert spec.nx in (32, 64) and spec.nx == spec.ny
        assert 0.05 <= spec.dt <= 0.2 and 0 <= spec.n_s <= 4 and spec.sn_warm_start == 1
    # the same seed, the same stream
    arr2 = serve.poisson_arrivals(lam, dur, seed=3, max_side=64)
    assert [a[0] for a in arr2] == [a[0] for a in arr] and [a[2] for a in arr2] == [a[2] for a in arr]


def test_poisson_arrivals_history_cap():
    arr = serve.poisson_arrivals(50.0, 5.0, seed=1, max_side=32, hist_cap=1234)
    assert arr and all(spec.n_hist <= 1234 for _, spec, _ in arr)


class _Req:
    def __init__(self, lat, hist):
        self.step_latency = lat
        self.histories = hist


def test_latency_summary_percentiles():
    done = [_Req([0.001 * i for i in range(1, 51)], 100), _Req([0.001 * i for i in range(51, 101)], 300)]
    out = serve.latency_summary(10.0, 5.0, [None] * 3, done, [_Req([1.0], 600)], 2.0, path="x")
    lat = np.array([0.001 * i for i in range(1, 101)] + [1.0])
    assert out["steps"] == 101 and out["requests_done"] == 2 and out["requests_unfinished"] == 1
    assert math.isclose(out["p50_ms"], np.percentile(lat, 50) * 1e3)
    assert math.isclose(out["p99_ms"], np.percentile(lat, 99) * 1e3)
    assert math.isclose(out["histories_per_s"], 1000 / 2.0) and out["path"] == "x" and out["arrived"] == 3
    empty = serve.latency_summary(1.0, 1.0, [], [], [], 0.0)
    assert math.isnan(empty["p50_ms"]) and empty["histories_per_s"] == 0.0
