"""Host logic of the benchmark (no device): the FP32 tally-error report and the launch count."""
import numpy as np

import bench
from paper_2511_16821_gb300 import workloads as W


def _tallies(n=100, seed=0):
    rng = np.random.default_rng(seed)
    o = {"pre": rng.uniform(1, 2, n), "post": rng.uniform(1, 2, n), "mom": rng.uniform(1, 2, (n, 4)),
         "pre_n": np.full(n, 100), "post_n": np.full(n, 100)}
    g = {"pre": o["pre"].copy(), "post": o["post"].copy(), "mom": o["mom"].copy()}
    return g, o


def test_tally_error_definitions():
    g, o = _tallies()
    g["pre"][5] *= 1 + 3e-5                  # a resolved cell
    g["post"][7] *= 1 + 2e-3                 # a cell scored by few segments: out of the resolved set
    o["post_n"][7] = 3
    o["pre"][9] = 1e-6                       # below 1e-3 of the peak: in neither set
    g["pre"][9] = 2e-6
    e = bench.tally_error(g, o)
    assert np.isclose(e["pre"]["resolved_max"], 3e-5, rtol=1e-6) and np.isclose(e["pre"]["max"], 3e-5, rtol=1e-6)
    assert e["post"]["resolved_max"] == 0.0 and np.isclose(e["post"]["max"], 2e-3, rtol=1e-6)
    w = abs(g["pre"] - o["pre"]).sum() / abs(o["pre"]).sum()
    assert np.isclose(e["pre"]["weighted"], w)
    # moments: relative to the zeroth moment's magnitude, resolved by the post-limit segments
    g["mom"][11, 2] += 1e-4 * abs(o["mom"][11, 0])
    e = bench.tally_error(g, o)
    assert np.isclose(e["mom2"]["resolved_max"], 1e-4, rtol=1e-6) and e["mom1"]["max"] == 0.0


def test_launches_per_step():
    spec = W.checkerboard(n_s=2, n_hist=1000)
    # leg + normalisation, three side-stream kernels, source + (sweep + reduction) per iteration +
    # finish, five remap kernels
    assert bench.launches_per_step(spec, 6) == 2 + 3 + (1 + 12 + 1) + 5
    assert bench.launches_per_step(spec, 1) - bench.launches_per_step(spec, 0) == 2
