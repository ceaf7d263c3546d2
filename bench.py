"""Benchmark of the GB300 hybrid (Q)MC / S_N step.

Workload (the one-GPU benchmark configuration): the 7x7-block checkerboard on a 112x112 mesh
(absorber sigma_a = 10 / scatterer sigma_s = 1, Q = 1 in the centre block, vacuum boundaries),
10^6 source histories per step plus the census bank (10^6 after the comb), dt = 0.1, S8, Sobol
points with a digital shift. One step = the whole hybrid step: MC leg, collided S_N-DG solve,
remap and census (Sec. 2.2 steps 1-4). Headline: FP32 tracking with int64 fixed-point tallies;
the FP64 path is measured beside it.

value     = MC-leg histories per second of whole-step time (device events, L2 flushed between
            steps; inputs resident in HBM)
e2e       = the same through the public C ABI with the census bank copied in from page-locked host
            memory (the problem's own layout, hyb_set_bank_native) and the step flux copied back
            every step
cpu_baseline / --impl reference = the single-threaded FP64 oracle on the host cores, on a
            bounded sample of the same workload.
Under torchrun (N > 1) each rank runs an independent problem replica (weak scaling, no
data-path collective); the barrier and the max over ranks of the timed region are kept.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2511_16821_gb300 import workloads as W  # noqa: E402

N_S = 2
N_HIST = 1_000_000
L2_FLUSH_BYTES = 512 << 20
METRIC = "histories/s"


def peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {"hbm_gbs": d.get("hbm_gbs", 6800.0), "src": "measured", "sm_max_mhz": d.get("sm_max_mhz", 2070.0)}
    return {"hbm_gbs": 6800.0, "src": "fallback", "sm_max_mhz": 2070.0}


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.rows = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for n, v in zip(names, r[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
            except (ValueError, IndexError):
                continue
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


CENSUS_ORDER = 0
PRIV_TILE = -1          # the library's automatic window (none at the benchmark's N_s = 2)
SN_ACCEL = 0
WARM = 1


# DRAM bytes (read + write) of one launch of the FP32 leg kernel on this workload, from one ncu
# capture without a cache flush (profiles/mc_leg_kernel_fp32_checkerboard112_ns2.md), with the
# SHA-256 of the sources the kernel is built from at that capture: the value is reported only while
# they are unchanged.
LEG_TRAFFIC_BYTES = 52_232_192 + 27_894_272
LEG_TRAFFIC_SOURCES_SHA256 = "3c69b6e98eac016ad25f1ab0ce29b90f17ed692f76428436a6cd901bcfa402a7"
LEG_SOURCES = ("mc_leg.cu", "hyb_device.cuh", "hyb_internal.h")


def leg_sources_sha256() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in LEG_SOURCES:
        with open(os.path.join(ROOT, "paper_2511_16821_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def leg_traffic():
    if LEG_TRAFFIC_BYTES is None or leg_sources_sha256() != LEG_TRAFFIC_SOURCES_SHA256:
        return None
    return LEG_TRAFFIC_BYTES


def spec_for(precision: int, n_hist: int = N_HIST, n_s: int | None = None, seed: int = 0,
             warm: int | None = None) -> W.ProblemSpec:
    """The benchmark workload; source iteration starts from the previous step's collided flux
    (the same fixed point, fewer sweeps)."""
    warm = WARM if warm is None else warm
    n_s = N_S if n_s is None else n_s
    return W.checkerboard(n_s=n_s, n_hist=n_hist, seed=seed, precision=precision).with_(sn_warm_start=warm,
                                                                                       census_order=CENSUS_ORDER,
                                                                                       sn_accel=SN_ACCEL,
                                                                                       priv_tile=PRIV_TILE)


def launches_per_step(spec: W.ProblemSpec, sn_iters: int) -> int:
    """Kernels of this library launched by one single-problem step (memsets not counted)."""
    leg = 2                                   # leg kernel, normalisation (births: drawn in the step before)
    side = 3                                  # beside the collided solve: bank pre-pass scalars, bank re-stream,
                                              # the next step's births
    sn = 1 + 2 * sn_iters + 1                 # source (with the starting iterate); sweep + reduce per iteration;
                                              # finish (copy, flux)
    remap = 2 + 3                             # density with the CDF reduction, CDF rows (marginal, guides,
                                              # scalars); births' pass, scan, write (with the finish)
    return leg + side + sn + remap

def run_gpu(args, rank: int, world: int) -> dict:
    import torch
    from paper_2511_16821_gb300 import hyb

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    res = {}
    for prec in ([W.FP32, W.FP64] if not args.fp32_only else [W.FP32]):
        spec = spec_for(prec, seed=rank)
        with torch.cuda.stream(stream):
            P = hyb.Problem(spec, stream=stream)
            for _ in range(args.warmup):
                P.step(1)
            torch.cuda.synchronize()
            if world > 1:
                import torch.distributed as dist
                dist.barrier()
            hist = segs = 0
            phase = {"mc_leg": [], "collided_sn": [], "remap": []}
            sn_it, step_ms, leg_k = [], [], []
            clk = Clocks(dev.index)
            with clk:
                t0 = time.perf_counter()
                for k in range(args.steps):
                    flush.zero_()
                    st = P.step(1)[0]      # CUDA events on the problem stream around each phase
                    step_ms.append(st["ms"])
                    hist += st["histories"]
                    segs += st["segments"]
                    phase["mc_leg"].append(st["ms_leg"])
                    phase["collided_sn"].append(st["ms_sn"])
                    phase["remap"].append(st["ms_remap"])
                    sn_it.append(st["sn_iterations"])
                    # the leg kernel alone (events at its launch), with its tally additions
                    leg_k.append((st["ms_leg_kernel"], st["tally_adds"], st["histories"], st["segments"]))
                torch.cuda.synchronize()
                if world > 1:
                    dist.barrier()
                wall = time.perf_counter() - t0
            res[prec] = dict(spec=spec, P=P, hist=hist, segs=segs, step_ms=step_ms, wall=wall, leg_kernel=leg_k,
                             clocks=clk.summary(), sn_iters=sn_it, bank=st["bank_size"],
                             phase_ms={k: statistics.median(v) for k, v in phase.items()})
    return res


def leg_profile(prec: int, reps: int = 5) -> dict:
    """The benchmark leg on its steady-state census bank (step 2; the leg's source births drawn
    beside the previous step's collided solve, as in a step): the inputs of the oracle's all-cores
    leg (bank, step, workload) and the raw tallies for the FP32 error against it, with the leg's
    device time (events around the leg kernel and its normalisation; the roofline itself takes
    the leg kernel's time inside the timed steps)."""
    import torch
    from paper_2511_16821_gb300 import hyb
    spec = spec_for(prec)
    P = hyb.Problem(spec)
    P.step(2)                      # a steady-state census bank
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    ms, hist, segs, adds, nb = [], 0, 0, 0, 0
    for _ in range(reps):
        flush.zero_()
        torch.cuda.synchronize()
        P.set_step(2)
        st = P.mc_leg()
        ms.append(st["ms"])
        hist, segs, adds = st["histories"], st["segments"], st["tally_adds"]
    bank = P.bank()
    nb = bank["n"]
    tallies = {"pre": P.tally("pre_raw"), "post": P.tally("post_raw"), "mom": P.tally("handoff")}
    P.close()
    return dict(ms=statistics.median(ms), histories=hist, segments=segs, tally_adds=adds, bank=nb,
                ncells=spec.ncells, bank_host=bank, tallies=tallies, step=2, spec=spec)


def tally_error(g: dict, o: dict, frac: float = 1e-3, min_seg: int = 32) -> dict:
    """FP32 tallies against the FP64 oracle's: per tally the largest relative error on the cells it
    resolves (above `frac` of its peak with >= min_seg scored segments), on every cell above `frac`
    of the peak, and the tally-weighted mean relative error."""
    out = {}
    cnt = {"pre": o["pre_n"], "post": o["post_n"]}
    for key in ("pre", "post", "mom0", "mom1", "mom2", "mom3"):
        if key.startswith("mom"):
            j = int(key[3])
            a, b, ref, n = g["mom"][:, j], o["mom"][:, j], np.abs(o["mom"][:, 0]), o["post_n"]
        else:
            a, b, ref, n = g[key], o[key], np.abs(o[key]), cnt[key]
        peak = float(np.max(ref)) if ref.size else 0.0
        err = np.abs(a - b) / np.maximum(ref, 1e-300)
        sel = ref >= frac * peak if peak > 0 else np.zeros_like(ref, bool)
        res = sel & (n >= min_seg)
        out[key] = {"resolved_max": float(np.max(err[res])) if res.any() else 0.0,
                    "max": float(np.max(err[sel])) if sel.any() else 0.0,
                    "weighted": float(np.sum(np.abs(a - b)) / max(float(np.sum(np.abs(b))), 1e-300))}
    return out


def e2e_measure(spec: W.ProblemSpec, steps: int) -> dict:
    """Public-API end to end: every step's census bank crosses from page-locked host memory (the
    problem's layout) and every step's flux is read back into page-locked host memory, all inside
    the timed region. The steps run through hyb_step_async, which returns once the remap is
    queued, so the host queues the next step's upload and this step's flux read-back while the
    remap runs. The uploads are double-buffered: step k+1's bank is copied to a device staging
    buffer on a second stream during step k, and hyb_set_bank_native takes it from there (a device
    copy on the problem's stream, with the device-side particle checks)."""
    import torch
    from paper_2511_16821_gb300 import hyb
    P = hyb.Problem(spec)
    P.step(1)
    host_bank = P.bank()
    n = int(host_bank["n"])
    esz = 4 if spec.precision == W.FP32 else 8
    fdt = np.float32 if spec.precision == W.FP32 else np.float64
    pinned = [torch.from_numpy(np.ascontiguousarray(host_bank["cell"][:n], dtype=np.int32)).pin_memory()]
    pinned += [torch.from_numpy(np.ascontiguousarray(host_bank[k][:n], dtype=fdt)).pin_memory()
               for k in ("fx", "fy", "ox", "oy", "w")]
    # histories per step of this input (every timed step starts from the same bank)
    P.set_bank_native(*pinned, n=n)
    hist_per_step = P.step(1)[0]["histories"]
    staging = [[torch.empty_like(t, device="cuda") for t in pinned] for _ in range(2)]
    copy_stream = torch.cuda.Stream()
    uploaded = [torch.cuda.Event() for _ in range(2)]   # staging buffer b holds its step's bank
    consumed = [torch.cuda.Event() for _ in range(2)]   # the problem has copied staging buffer b
    flux_dev = torch.empty(spec.nx * spec.ny, dtype=torch.float64, device="cuda")
    flux_host = [torch.empty(spec.nx * spec.ny, dtype=torch.float64).pin_memory() for _ in range(2)]

    def upload(b):
        with torch.cuda.stream(copy_stream):
            copy_stream.wait_event(consumed[b])
            for d, h in zip(staging[b], pinned):
                d.copy_(h, non_blocking=True)
            uploaded[b].record(copy_stream)

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    upload(0)
    for k in range(steps):
        b = k % 2
        P.stream.wait_event(uploaded[b])
        P.set_bank_native(*staging[b], n=n)
        consumed[b].record(P.stream)
        if k + 1 < steps:
            upload(1 - b)
        P.step_async(1)
        P.tally_to("flux", flux_dev)
        with torch.cuda.stream(P.stream):
            flux_host[b].copy_(flux_dev, non_blocking=True)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    P.remap_stats()                       # reads the status word of the last, unchecked step
    assert np.isfinite(flux_host[(steps - 1) % 2].numpy()).all()
    return {"value": hist_per_step * steps / dt, "unit": METRIC, "steps": steps,
            "h2d_bytes_per_step": int(host_bank["n"]) * (4 + 5 * esz),
            "d2h_bytes_per_step": int(spec.nx * spec.ny * 8),
            "pipeline": "hyb_step_async; the next step's bank uploaded from page-locked memory on a second "
                        "stream during the current step; the flux read back into page-locked memory"}


def cpu_baseline(n_hist: int, steps: int, leg: dict | None = None) -> dict:
    """The FP64 oracle on the host cores: (1) one thread, whole hybrid steps on a bounded sample of
    the workload (same mesh, N_s, dt and quadrature; n_hist histories per step); (2) every core
    (one spawn-started process per core over contiguous history-index slices, integer counters
    summed) on the benchmark's own MC leg (its census bank and step), whose result also gives the
    FP32 path's tally error against the oracle."""
    import oracle
    oracle.build()
    spec = spec_for(W.FP64, n_hist=n_hist, warm=0)
    bank = None
    hist = 0
    t0 = time.perf_counter()
    for k in range(steps):
        r = oracle.step(spec, k, bank)
        bank = r["bank"]
        hist += r["leg"]["histories"]
    dt = time.perf_counter() - t0
    one = {"value": hist / dt, "unit": METRIC, "cores": 1,
           "sample": f"{steps} full hybrid steps of the checkerboard-112 workload at {n_hist} "
                     f"histories/step (FP64 oracle, one thread)", "seconds": round(dt, 2)}
    out = dict(one, kind="oracle")
    if leg is None:
        return out
    from oracle.parallel import Pool
    ncores = os.cpu_count() or 1
    ospec = leg["spec"].with_(precision=W.FP64)
    with Pool(ncores) as pool:
        pool.mc_leg(ospec, leg["step"], None, nslices=ncores)     # start-up of the workers, untimed
        t0 = time.perf_counter()
        o = pool.mc_leg(ospec, leg["step"], leg["bank_host"])
        dt = time.perf_counter() - t0
    n = o["stats"]["histories"]
    out.update({"value": n / dt, "cores": ncores, "seconds": round(dt, 2),
                "sample": f"the benchmark's MC leg ({leg['bank']} census particles + births, step "
                          f"{leg['step']}) on {ncores} processes over index slices (FP64 oracle)",
                "one_core": one})
    out["fp32_tally_error"] = tally_error(leg["tallies"], o)
    return out


def batched_measure(n_problems: int = 256, steps: int = 3, seed: int = 0, sn_accel: int = 0,
                    single: bool = True) -> dict:
    """The batched workload: n problems of the batched distribution (FP32 tracking, int64
    tallies), one graph per step after autotuning, against the plain single-problem path over the
    same problems (each stepped alone, one after the other). sn_accel: Anderson depth of the
    problems' collided solves (0: plain source iteration)."""
    import torch
    from paper_2511_16821_gb300 import hyb
    from paper_2511_16821_gb300.autotune import tune_batch
    specs = [W.random_batch_problem(seed, p).with_(sn_warm_start=1, sn_accel=sn_accel) for p in range(n_problems)]
    stream = torch.cuda.Stream()
    probs = [hyb.Problem(sp, stream=stream) for sp in specs]
    B = hyb.Batch(probs, stream=stream)
    tune = tune_batch(B, steps=1, space={"block": (256,), "chunk": (2048, 8192, 32768), "streams": (16, 48)})
    # steady state: a problem whose source iteration outgrows its cap in the step graphs is finished
    # eagerly and the graphs are re-captured with a larger cap, a one-off cost of ~20 ms for 256
    # problems; three steps let the caps settle before the timed ones
    B.step(3)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    st = B.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    hist = sum(x["histories"] for x in st)
    # the batched leg launch against the atomic roofline (its tally additions over its device time,
    # events around the launch inside the step), with the HBM view of the banks' pick-ups
    adds = sum(x["tally_adds"] for x in st)
    ms_leg = st[-1]["ms_leg"]
    nbank = sum(x["histories"] for x in st) - sum(sp.n_hist for sp in specs)
    peak = hyb.atomic_rate(6 * sum(sp.nx * sp.ny for sp in specs))
    B.close()
    for P in probs:
        P.close()
    out = {"problems": n_problems, "sn_accel": sn_accel, "histories_per_step": hist, "ms_per_step": ms,
           "histories_per_s": hist / (ms / 1e3), "tuning": tune["best"],
           "roofline": {"bound": "atomic", "kernel": "mc_leg_batch_kernel<float>",
                        "achieved": adds / (ms_leg / 1e3) / 1e9, "peak": peak / 1e9, "unit": "Gatomic/s",
                        "frac": adds / (ms_leg / 1e3) / peak, "leg_ms": ms_leg, "tally_adds": adds,
                        "hbm": {"bytes": 24 * nbank, "achieved": 24 * nbank / (ms_leg / 1e3) / 1e9,
                                "unit": "GB/s"}}}
    if not single:
        return out
    # plain path: each problem alone, the same number of steps, one after the other
    alone = [hyb.Problem(sp, stream=stream) for sp in specs]
    for P in alone:
        P.step(1, stats=False)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h2 = 0
    for P in alone:
        for x in P.step(steps):
            h2 += x["histories"]
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    for P in alone:
        P.close()
    out["single_problem_path"] = {"histories_per_s": h2 / dt, "ms_per_step_all": 1e3 * dt / steps}
    return out


# (tally_copies, priv_tile); the first is the library's default (automatic copies and window)
LEG_PLACEMENTS = ((0, -1), (0, 0), (1, 0), (4, 0), (1, 16), (4, 16), (4, 8))


def leg_ns_sweep(atomic_peak: float, reps: int = 5) -> list:
    """The benchmark leg at the checkerboard family's scatter limits N_s = 0, 1, 2, 4: the leg
    kernel's device time (CUDA events at its launch, median of `reps` launches on the step-2 bank,
    the L2 flushed before each) with the default tally placement and with the best of
    LEG_PLACEMENTS (global copies of the tally arrays x the shared-memory window over the source
    block); its tally additions over that time against the measured atomic rate."""
    import torch
    from paper_2511_16821_gb300 import hyb
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    out = []
    for ns in (0, 1, 2, 4):
        spec = spec_for(W.FP32, n_s=ns)
        P0 = hyb.Problem(spec)
        P0.step(2)
        bank = P0.bank()
        P0.close()
        rows = []
        for copies, priv in LEG_PLACEMENTS:
            P = hyb.Problem(spec.with_(tally_copies=copies, priv_tile=priv))
            P.set_bank(bank)
            ms = []
            for _ in range(reps):
                flush.zero_()
                torch.cuda.synchronize()
                P.set_step(2)
                st = P.mc_leg()
                ms.append(st["ms_leg_kernel"])
            P.close()
            m = statistics.median(ms)
            rate = st["tally_adds"] / (m / 1e3)
            rows.append({"tally_copies": copies, "priv_tile": priv, "leg_kernel_ms": m,
                         "achieved": rate / 1e9, "frac": rate / atomic_peak})
        best = min(rows, key=lambda r: r["leg_kernel_ms"])
        out.append({"n_s": ns, "histories": st["histories"], "segments": st["segments"],
                    "tally_adds": st["tally_adds"], "unit": "Gatomic/s", "default": rows[0], "best": best})
    return out


def census_order_measure(steps: int = 5, order: int = 1) -> dict:
    """The benchmark workload with the census sorted before the comb (FP32), by cell (order 1) or by
    cell and phase space (order 2): device time per step. At equal histories their multi-step
    flux errors are lower (convergence.py)."""
    import torch
    from paper_2511_16821_gb300 import hyb
    spec = spec_for(W.FP32).with_(census_order=order)
    stream = torch.cuda.Stream()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    with torch.cuda.stream(stream):
        P = hyb.Problem(spec, stream=stream)
        P.step(3)
        ms, hist = 0.0, 0
        for _ in range(steps):
            flush.zero_()
            st = P.step(1)[0]
            ms += st["ms"]
            hist += st["histories"]
        P.close()
    torch.cuda.synchronize()
    return {"census_order": ("slot", "cell", "phase space")[order], "histories_per_s": hist / (ms / 1e3),
            "ms_per_step": ms / steps}


def large_measure(steps: int = 2, n_hist: int = 100_000_000, sn_accel: int = 0) -> dict:
    """The large diffusive workload: 1024^2 cells over 10 x 10 cm, random 8 x 8-cell blocks with
    sigma_t in {1, 10, 1000} (scattering ratio 0.999 in the thickest, 0.5 elsewhere), N_s = 8,
    10^8 births per step, dt = 0.01, S8, FP32 tracking. One untimed step fills the census; the
    timed steps carry 10^8 census particles plus 10^8 births each. sn_accel: Anderson depth of
    the collided solve (0: plain source iteration)."""
    import torch
    from paper_2511_16821_gb300 import hyb
    spec = W.large(n=1024, n_hist=n_hist, precision=W.FP32).with_(sn_warm_start=1, sn_accel=sn_accel)
    stream = torch.cuda.Stream()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    with torch.cuda.stream(stream):
        P = hyb.Problem(spec, stream=stream)
        P.step(1)
        ms, hist, segs, it, phase = 0.0, 0, 0, [], {"mc_leg": 0.0, "collided_sn": 0.0, "remap": 0.0}
        for _ in range(steps):
            flush.zero_()
            st = P.step(1)[0]
            ms += st["ms"]
            hist += st["histories"]
            segs += st["segments"]
            it.append(st["sn_iterations"])
            phase["mc_leg"] += st["ms_leg"] / steps
            phase["collided_sn"] += st["ms_sn"] / steps
            phase["remap"] += st["ms_remap"] / steps
        P.close()
    torch.cuda.synchronize()
    return {"workload": "large diffusive 1024x1024, N_s=8, 1e8 births/step + census, dt=0.01, S8, FP32",
            "sn_accel": sn_accel,
            "histories_per_s": hist / (ms / 1e3), "segments_per_s": segs / (ms / 1e3), "ms_per_step": ms / steps,
            "phase_ms": phase, "sn_iterations": it}


def serving_measure(lam: float, duration: float, seed: int = 0, hist_cap: int | None = None,
                    plain: bool = False, drain: float = 30.0) -> dict:
    """Poisson arrivals of rate lam for `duration` seconds through the continuous-batching server
    (120 GB admission budget), then at most `drain` seconds more; with plain=True also the plain
    single-problem path on the same request stream."""
    from paper_2511_16821_gb300.serve import Server, run_poisson_plain
    srv = Server(budget_bytes=120e9)
    res = srv.run_poisson(lam, duration, seed=seed, hist_cap=hist_cap, drain=drain)
    srv.close()
    if plain:
        res["plain_single_problem"] = run_poisson_plain(lam, duration, seed=seed, hist_cap=hist_cap, drain=drain)
    return res


def reference_arm(args, rank: int, world: int) -> None:
    """The oracle (one thread, FP64) on the benchmark workload: whole hybrid steps at the
    benchmark's 10^6 histories/step when warm-up plus timed steps fit in about two minutes (about
    4 s per step on one core), else at a proportionally smaller history count, stated in the line."""
    if rank != 0:
        return
    n_hist = N_HIST if (args.steps + args.warmup) * 5.0 <= 150.0 else \
        max(10_000, int(N_HIST * 150.0 / (5.0 * (args.steps + args.warmup))))
    import oracle
    oracle.build()
    spec = spec_for(W.FP64, n_hist=n_hist, warm=0)
    bank = None
    for k in range(args.warmup):
        bank = oracle.step(spec, k, bank)["bank"]
    hist = 0
    t0 = time.perf_counter()
    for k in range(args.steps):
        r = oracle.step(spec, args.warmup + k, bank)
        bank = r["bank"]
        hist += r["leg"]["histories"]
    dt = time.perf_counter() - t0
    v = hist / dt
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": METRIC, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_block(),
            "cpu_baseline": {"value": v, "unit": METRIC, "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} whole hybrid steps at {n_hist} histories/step "
                                       f"(after {args.warmup} untimed ones), one thread"},
            "e2e": {"value": v, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def config_block() -> dict:
    return {"workload": "checkerboard 7x7 blocks, 112x112 mesh, N_s=2, 1e6 histories/step, dt=0.1, S8",
            "mesh": "112x112", "n_s": N_S, "n_hist": N_HIST, "sampler": "sobol+digital shift",
            "sn_order": 8, "dt": 0.1, "l2": "flushed (512 MiB write) before every timed step",
            "histories_counted": "MC-leg histories per step: the census bank's pick-ups (1e6 after the "
                                 "comb) plus the 1e6 source births"}


def main():
    global CENSUS_ORDER, SN_ACCEL, WARM, N_S, PRIV_TILE
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--fp32-only", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched and serving measurements")
    ap.add_argument("--no-large", action="store_true", help="skip the large-mesh measurement")
    ap.add_argument("--serve-sweep", default="", help="comma-separated arrival rates: run only the serving sweep")
    ap.add_argument("--serve-seconds", type=float, default=10.0)
    ap.add_argument("--serve-drain", type=float, default=30.0, help="seconds served after the arrival window")
    ap.add_argument("--serve-plain", action="store_true",
                    help="also serve the same request stream through the plain single-problem path")
    ap.add_argument("--lean", action="store_true",
                    help="timed steps only (FP32, no profile/e2e/CPU legs): the case used for ncu captures")
    ap.add_argument("--sn-accel", type=int, default=0, help="Anderson depth of the collided solve (0: plain SI)")
    ap.add_argument("--sn-warm", type=int, default=1, choices=[0, 1, 2],
                    help="source-iteration start: 0 zero, 1 previous step's flux, 2 linear extrapolation")
    ap.add_argument("--census-order", type=int, default=0, choices=[0, 1, 2],
                    help="census in slot order (0), sorted by cell (1) or by cell and phase space (2) "
                         "before the comb")
    ap.add_argument("--lean-n-s", type=int, default=N_S,
                    help="with --lean: the scatter limit of the checkerboard (profiling other members of the family)")
    ap.add_argument("--lean-priv-tile", type=int, default=-1,
                    help="with --lean: the leg's shared-memory window of cells (priv_tile; -1 automatic)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if (args.lean_n_s != N_S or args.lean_priv_tile != -1) and not args.lean:
        ap.error("--lean-n-s and --lean-priv-tile change the workload: --lean runs only")
    N_S = args.lean_n_s
    PRIV_TILE = args.lean_priv_tile
    CENSUS_ORDER = args.census_order
    SN_ACCEL = args.sn_accel
    WARM = args.sn_warm

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="gloo" if args.impl == "reference" else "nccl")
    if args.impl == "reference":
        reference_arm(args, rank, world)
        return

    import torch
    if args.serve_sweep:
        if rank == 0:
            for lam in [float(x) for x in args.serve_sweep.split(",")]:
                print(json.dumps({"serving": serving_measure(lam, args.serve_seconds, plain=args.serve_plain,
                                                             drain=args.serve_drain)}), flush=True)
        return
    if args.lean:
        args.fp32_only = args.no_cpu = args.no_e2e = args.no_batch = args.no_large = True
    res = run_gpu(args, rank, world)
    if args.lean:
        if rank == 0:
            r = res[W.FP32]
            print(json.dumps({"lean": True, "ms_per_step": sum(r["step_ms"]) / args.steps,
                              "phase_ms": r["phase_ms"], "sn_iterations": r["sn_iters"],
                              "leg_kernel_ms": statistics.median([x[0] for x in r["leg_kernel"]])}), flush=True)
        return
    r32 = res[W.FP32]
    tot_ms = sum(r32["step_ms"])
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([tot_ms], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        tot_ms = float(t.item())
        h = torch.tensor([float(r32["hist"]), float(r32["segs"])], dtype=torch.float64, device="cuda")
        dist.all_reduce(h)
        hist_all, segs_all = h[0].item(), h[1].item()
    else:
        hist_all, segs_all = r32["hist"], r32["segs"]
    if rank != 0:
        return
    value = hist_all / (tot_ms / 1000.0)
    pk = peaks()
    prof = leg_profile(W.FP32)
    # The MC leg's roofline (the hot path's target): its algorithmic work is one fixed-point tally
    # addition per pre-limit segment and five per post-limit segment (all counted by the kernel:
    # hyb_leg_stats.tally_adds) plus its read stream: 24 B per bank particle (births are generated
    # in the kernel: 0 B). Its bound is the rate of 64-bit global atomic additions to the tally
    # footprint (measured live with hyb_atomic_rate on 6 x ncells addresses); the HBM view is
    # reported beside it.
    from paper_2511_16821_gb300 import hyb
    atomic_peak = hyb.atomic_rate(6 * prof["ncells"])
    # the leg kernel alone, in every timed step (CUDA events at its launch, on the problem's stream):
    # per step its tally additions over its duration; the median over the timed steps
    lk = [x for x in r32["leg_kernel"] if x[0] > 0]
    leg_ms = statistics.median([x[0] for x in lk])
    adds_rate = statistics.median([x[1] / (x[0] / 1e3) for x in lk])
    n_src = r32["spec"].n_hist
    leg_bytes = statistics.median([(x[2] - n_src) * 24 for x in lk])      # bank particles picked up
    hbm_achieved = statistics.median([(x[2] - n_src) * 24 / (x[0] / 1e3) for x in lk]) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": config_block(),
        "segments_per_s": segs_all / (tot_ms / 1000.0),
        "sn_iterations": r32["sn_iters"],
        "phase_ms": r32["phase_ms"],
        "roofline": {"bound": "atomic", "kernel": "mc_leg_kernel<float>", "achieved": adds_rate / 1e9,
                     "peak": atomic_peak / 1e9, "unit": "Gatomic/s", "frac": adds_rate / atomic_peak,
                     "target_frac": 0.5,
                     "traffic": leg_traffic(),
                     "peak_src": "measured live: hyb_atomic_rate, 64-bit adds to 6 x ncells random addresses",
                     "leg_ms": leg_ms, "leg_histories": int(statistics.median([x[2] for x in lk])),
                     "leg_segments": int(statistics.median([x[3] for x in lk])),
                     "tally_adds": int(statistics.median([x[1] for x in lk])),
                     "timed_in": "the timed steps (events around the leg kernel launch)",
                     "leg_phase_ms": r32["phase_ms"]["mc_leg"],
                     "hbm": {"achieved": hbm_achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                             "frac": hbm_achieved / pk["hbm_gbs"], "bytes": leg_bytes, "peak_src": pk["src"]}},
        "gpu_launches": launches_per_step(r32["spec"], int(np.mean(r32["sn_iters"]) + 0.5)) * args.steps,
        "clocks": r32["clocks"],
    }
    # the remap phase against HBM: 24 B read per copied census particle and 24 B written per
    # census survivor (the bank of the next step); births are generated (0 B)
    rb = r32["bank"] * 24 * 2
    rms = r32["phase_ms"]["remap"]
    line["roofline_remap"] = {"bound": "hbm", "kernel": "remap phase (density, CDF, count, scan, write)",
                              "achieved": rb / (rms / 1e3) / 1e9, "peak": pk["hbm_gbs"], "unit": "GB/s",
                              "frac": rb / (rms / 1e3) / 1e9 / pk["hbm_gbs"], "bytes": rb, "ms": rms,
                              "peak_src": pk["src"]}
    if W.FP64 in res:
        r64 = res[W.FP64]
        ms64 = sum(r64["step_ms"])
        lk64 = [x for x in r64["leg_kernel"] if x[0] > 0]
        ms64k = statistics.median([x[0] for x in lk64])
        rate64 = statistics.median([x[1] / (x[0] / 1e3) for x in lk64])
        bank64 = statistics.median([x[2] - r64["spec"].n_hist for x in lk64])
        line["fp64"] = {"value": r64["hist"] / (ms64 / 1000.0), "unit": METRIC,
                        "segments_per_s": r64["segs"] / (ms64 / 1000.0), "ms_per_step": ms64 / args.steps,
                        "phase_ms": r64["phase_ms"],
                        "roofline": {"bound": "atomic", "kernel": "mc_leg_kernel<double>",
                                     "achieved": rate64 / 1e9, "peak": atomic_peak / 1e9,
                                     "unit": "Gatomic/s", "frac": rate64 / atomic_peak,
                                     "leg_ms": ms64k, "tally_adds": int(statistics.median([x[1] for x in lk64])),
                                     "timed_in": "the timed steps (events around the leg kernel launch)",
                                     "hbm": {"achieved": bank64 * 44 / (ms64k / 1e3) / 1e9, "peak": pk["hbm_gbs"],
                                             "unit": "GB/s", "frac": bank64 * 44 / (ms64k / 1e3) / 1e9 / pk["hbm_gbs"],
                                             "bytes": bank64 * 44}}}
    if not args.no_e2e:
        line["e2e"] = e2e_measure(spec_for(W.FP32), max(2, min(args.steps, 20)))
    line["leg_ns_sweep"] = leg_ns_sweep(atomic_peak)
    if CENSUS_ORDER == 0:
        line["census_cell_order"] = census_order_measure(order=1)
        line["census_phase_order"] = census_order_measure(order=2)
    if not args.no_large:
        line["large"] = large_measure(sn_accel=4)
        line["large_plain_si"] = large_measure(sn_accel=0)
    if not args.no_batch:
        line["batched"] = batched_measure()
        line["batched_anderson"] = batched_measure(sn_accel=4, single=False)
        line["serving"] = serving_measure(100.0, 3.0, plain=True, drain=10.0)
    if not args.no_cpu:
        cb = cpu_baseline(n_hist=200_000, steps=2, leg=prof)
        line["fp32_tally_error"] = cb.pop("fp32_tally_error")
        line["cpu_baseline"] = cb
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
