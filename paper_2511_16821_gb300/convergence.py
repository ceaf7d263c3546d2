"""QMC versus pseudorandom error convergence of the hybrid on the GPU.

The paper compares the error of the hybrid's scalar flux against the particle count for Halton
points and pseudorandom numbers and fits err ~ c N^alpha (Sec. 3, Table 1: alpha near -0.5 for
MC and -0.6 to -0.7 for QMC). Here the same study runs on a synthetic heterogeneous problem with
Sobol points under a digital shift, Halton points under a shift modulo 1 and the counter PRNG:
for every history count N and seed
the hybrid advances `steps` time steps, and the error is the relative L2 norm, over cells, of the
end-of-step scalar flux (MC pre + post tallies and the collided S_N flux) against a reference
computed with many more histories (the mean over a few Sobol shifts). The error at each N is the
root mean square over seeds, and alpha is the least-squares slope of log(error) against log(N).

    python -m paper_2511_16821_gb300.convergence            # the full study, printed as JSON
"""
from __future__ import annotations

import json
import math

import numpy as np

from . import hyb
from . import workloads as W


def problem(n_hist: int, seed: int, sampler: int, n_s: int = 2, precision: int = W.FP32,
            census_order: int = 0, sigma_scale: float = 1.0, remap_variant: int = 0,
            cap_factor: int = 1) -> W.ProblemSpec:
    """Checkerboard of 7x7 one-centimetre blocks at 4 cells per block (28x28), S4, absorber /
    scatterer blocks (cross sections times sigma_scale), Q = 1 in the centre block, dt = 0.1.
    remap_variant 1: steps 3'/4' of the previous hybrids; cap_factor: census cap in units of
    n_hist (large: no comb)."""
    order = ("slot", "cell", "phase-space")[census_order]
    sp = W.checkerboard(n_s=n_s, n_hist=n_hist, seed=seed, precision=precision, sampler=sampler, cells_per_block=4)
    name = f"checkerboard28 x{sigma_scale:g} N_s={'inf' if n_s == W.NS_INF else n_s}, census in {order} order"
    if remap_variant:
        name += ", remap 3'/4'"
    if cap_factor != 1:
        name += f", census cap {cap_factor} n_hist"
    return sp.with_(sigma_a=sp.sigma_a * sigma_scale, sigma_s=sp.sigma_s * sigma_scale, sn_order=4, sn_tol=1e-6,
                    census_order=census_order, remap_variant=remap_variant, census_cap=cap_factor * n_hist,
                    name=name)


def end_flux(spec: W.ProblemSpec, steps: int) -> np.ndarray:
    with hyb.Problem(spec) as p:
        p.step(steps, stats=False)
        return p.tally("flux")


def fit_alpha(ns, errs) -> float:
    x = np.log(np.asarray(ns, dtype=float))
    y = np.log(np.asarray(errs, dtype=float))
    return float(np.polyfit(x, y, 1)[0])


def study(log2_n=range(10, 21), seeds=range(16), steps: int = 4, ref_log2: int = 24, ref_seeds=range(100, 104),
          n_s: int = 2, census_order: int = 0, sigma_scale: float = 1.0, remap_variant: int = 0,
          cap_factor: int = 1, spec_fn=problem) -> dict:
    import torch
    mk = lambda n, s, smp: spec_fn(n, s, smp, n_s, census_order=census_order, sigma_scale=sigma_scale,   # noqa: E731
                                   remap_variant=remap_variant, cap_factor=cap_factor)
    ref = np.mean([end_flux(mk(1 << ref_log2, s, W.SOBOL), steps) for s in ref_seeds], axis=0)
    nref = float(np.linalg.norm(ref))
    out = {"workload": mk(1, 0, W.SOBOL).name, "steps": steps, "reference_histories": 1 << ref_log2,
           "reference_shifts": len(list(ref_seeds)), "seeds": len(list(seeds)), "metric": "relative L2 error of the "
           "end-of-step scalar flux, RMS over seeds"}
    for name, sampler in (("sobol", W.SOBOL), ("halton", W.HALTON), ("prng", W.PRNG)):
        ns, errs = [], []
        for k in log2_n:
            n = 1 << k
            e2 = [float(np.linalg.norm(end_flux(mk(n, s, sampler), steps) - ref)) ** 2 for s in seeds]
            ns.append(n)
            errs.append(math.sqrt(sum(e2) / len(e2)) / nref)
        out[name] = {"n": ns, "err": errs, "alpha": fit_alpha(ns, errs)}
    torch.cuda.synchronize()
    return out


def ns_sweep(n_s_values=(0, 1, 2, 5, 10, 20, W.NS_INF), log2_n=range(10, 19, 2), seeds=range(8),
             ref_log2: int = 22, ref_seeds=range(100, 104), sigma_scale: float = 1.0) -> list:
    """The analogue of the paper's Table 1 on the synthetic problem: for each scatter limit N_s,
    the source iterations of the collided solve (from zero, stop at 1e-6 relative change) and the
    convergence rates alpha of one step's flux error with Sobol points, Halton points and the
    counter PRNG.
    N_s = infinity is the pure (Q)MC method (no collided stage)."""
    import torch
    rows = []
    for n_s in n_s_values:
        with hyb.Problem(problem(1 << 16, 0, W.SOBOL, n_s, sigma_scale=sigma_scale).with_(sn_warm_start=0)) as p:
            st = p.step(1)[0]
        r = study(log2_n=log2_n, seeds=seeds, steps=1, ref_log2=ref_log2, ref_seeds=ref_seeds, n_s=n_s,
                  sigma_scale=sigma_scale)
        rows.append({"n_s": "inf" if n_s == W.NS_INF else n_s, "sn_iterations": st["sn_iterations"],
                     "alpha_sobol": r["sobol"]["alpha"], "alpha_halton": r["halton"]["alpha"],
                     "alpha_prng": r["prng"]["alpha"], "err_sobol": r["sobol"]["err"][-1],
                     "err_halton": r["halton"]["err"][-1], "err_prng": r["prng"]["err"][-1],
                     "n_max": r["sobol"]["n"][-1], "workload": r["workload"]})
    torch.cuda.synchronize()
    return rows


if __name__ == "__main__":
    # one step (the MC leg from the source, then the collided solve) and four steps (census
    # particles re-streamed through the remap), at N_s = 0 (5 point dimensions) and N_s = 2 (11),
    # and four steps with the census in cell order
    for n_s in (0, 2):
        for steps in (1, 4):
            print(json.dumps(study(steps=steps, n_s=n_s)), flush=True)
    print(json.dumps(study(steps=4, n_s=2, census_order=1)), flush=True)
    print(json.dumps(study(steps=4, n_s=2, census_order=2)), flush=True)
    # the previous hybrids' remap (steps 3'/4'), and both remaps without a comb (census cap 8 n_hist)
    print(json.dumps(study(steps=4, n_s=2, remap_variant=1)), flush=True)
    print(json.dumps(study(steps=4, n_s=2, cap_factor=8, ref_log2=22)), flush=True)
    print(json.dumps(study(steps=4, n_s=2, remap_variant=1, cap_factor=8, ref_log2=22)), flush=True)
    print(json.dumps({"ns_sweep": ns_sweep()}), flush=True)
    print(json.dumps({"ns_sweep": ns_sweep(sigma_scale=10.0)}), flush=True)
