"""Seeded synthetic problem descriptions and particle banks.

This module holds no arithmetic of the transport method: it only builds the inputs (mesh,
cross sections, sources, initial weights, random banks) that both the CUDA path and the CPU
oracle consume. Problems are shaped like the paper's (Sec. 3: heterogeneous materials, a
localised source, vacuum boundaries) and like the benchmark configurations of this library:

* ``pulse``         16x16 homogeneous square, unit pulse in the 2x2 centre cells, N_s = 1
* ``checkerboard``  7x7 blocks of 1 cm on a 112x112 mesh, absorber / scatterer, Q = 1 centre
* ``random_batch``  the batched-problem distribution (mesh side, sigma_t, ratio, N_s, N_src)
* ``large``         1024x1024 diffusive mesh with random 8x8-cell material blocks
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace

import numpy as np

FP32, FP64 = 0, 1
SOBOL, PRNG, HALTON = 0, 1, 2
NS_INF = 2147483647


@dataclass
class ProblemSpec:
    """A hybrid transport problem on the uniform Cartesian mesh [0,lx] x [0,ly].

    Arrays are row-major per cell, index iy*nx + ix. Q is the angle-integrated emission rate
    density (particles per unit area per unit time); ic the total initial weight per cell
    (isotropic, uniform in the cell, at t = 0).
    """
    nx: int
    ny: int
    lx: float
    ly: float
    sigma_a: np.ndarray
    sigma_s: np.ndarray
    Q: np.ndarray | None = None
    ic: np.ndarray | None = None
    c: float = 1.0
    dt: float = 0.1
    n_s: int = 1
    n_hist: int = 10_000
    seed: int = 0
    sampler: int = SOBOL
    precision: int = FP64
    sn_order: int = 4
    handoff_full: int = 1
    w_min: float = 0.0
    census_cap: int = 0
    sn_tol: float = 1e-10
    sn_max_iter: int = 500
    sn_warm_start: int = 0
    census_order: int = 0
    sn_accel: int = 0
    remap_variant: int = 0          # 0: Eq. (R) relabelling remap; 1: steps 3'/4' of the previous hybrids
    n_s_cell: np.ndarray | None = None   # per-cell scatter limits in [0, n_s] (space-dependent N_s)
    sn_layout: int = 0              # sweep memory layout: 0 automatic, 1 padded mesh, 2 wavefront order
    seg_limit: int = 0              # segments per history before HYB_ETIMEOUT (0: the default 2^20)
    wait_limit: int = 0             # polls of a device wait (solve pipeline, sort look-back) before HYB_ETIMEOUT (0: 2^22)
    tally_copies: int = 0           # copies of the fixed-point tally arrays (0: automatic)
    sort_every: int = 0             # census_order >= 1: sort on the steps n with n mod sort_every == 0 (0, 1: all)
    leg_sort_every: int = 0         # 0: fused leg; K >= 1: phases of K segments, live histories sorted by cell between
    priv_tile: int = -1             # fused leg: a window of priv_tile^2 cells' tallies in each CTA's shared memory
                                    # (-1: 16 x 16 where N_s = 0 and the source is concentrated there, else none)
    name: str = field(default="problem")

    @property
    def ncells(self) -> int:
        return self.nx * self.ny

    def with_(self, **kw) -> "ProblemSpec":
        return replace(self, **kw)


def pulse(n_hist: int = 10_000, seed: int = 0, precision: int = FP64, sampler: int = SOBOL,
          n_s: int = 1) -> ProblemSpec:
    """1x1 cm, 16x16 cells, sigma_s = 1, sigma_a = 0.1, unit pulse in cells ix,iy in {7,8}."""
    n = 16
    ic = np.zeros((n, n))
    ic[7:9, 7:9] = 0.25
    return ProblemSpec(nx=n, ny=n, lx=1.0, ly=1.0, sigma_a=np.full(n * n, 0.1),
                       sigma_s=np.full(n * n, 1.0), Q=None, ic=ic.ravel(), c=1.0, dt=0.05,
                       n_s=n_s, n_hist=n_hist, seed=seed, sampler=sampler, precision=precision,
                       sn_order=4, name="pulse16")


def checkerboard(n_s: int = 2, n_hist: int = 1_000_000, seed: int = 0, precision: int = FP64,
                 sampler: int = SOBOL, cells_per_block: int = 16) -> ProblemSpec:
    """7x7 blocks of 1 cm; block (I,J) scatters iff I+J is even; Q = 1 in the centre block."""
    nb, cpb = 7, cells_per_block
    n = nb * cpb
    I = np.arange(n) // cpb
    blk_i, blk_j = np.meshgrid(I, I, indexing="xy")     # blk_i: column block, blk_j: row block
    scat = ((blk_i + blk_j) % 2) == 0
    sa = np.where(scat, 0.0, 10.0)
    ss = np.where(scat, 1.0, 0.0)
    Q = np.where((blk_i == 3) & (blk_j == 3), 1.0, 0.0)
    return ProblemSpec(nx=n, ny=n, lx=7.0, ly=7.0, sigma_a=sa.ravel(), sigma_s=ss.ravel(),
                       Q=Q.ravel(), ic=None, c=1.0, dt=0.1, n_s=n_s, n_hist=n_hist, seed=seed,
                       sampler=sampler, precision=precision, sn_order=8, name=f"checkerboard{n}")


def _splitmix(state: int):
    """A splitmix64 stream (Steele, Lea & Flood 2014) used only to draw problem parameters."""
    M = (1 << 64) - 1
    while True:
        state = (state + 0x9E3779B97F4A7C15) & M
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
        yield (z ^ (z >> 31)) / 2.0 ** 64


def random_batch_problem(base_seed: int, p: int, precision: int = FP32, dt: float = 0.1,
                         max_side: int = 256) -> ProblemSpec:
    """Problem p of the batched distribution: side in {32,64,128,256} (capped at max_side),
    L ~ U[1,10] cm, per-cell sigma_t log-uniform in [0.1, 100], ratio ~ U[0, 0.99],
    N_s ~ U{0..4}, N_src log-uniform in [1e4, 1e6], Q = 1 uniform, S4."""
    g = _splitmix((base_seed << 32) ^ (p * 0x632BE59BD9B4E019 & ((1 << 64) - 1)))
    sides = [s for s in (32, 64, 128, 256) if s <= max_side]
    side = sides[min(int(next(g) * len(sides)), len(sides) - 1)]
    L = 1.0 + 9.0 * next(g)
    n_s = min(int(next(g) * 5), 4)
    n_hist = int(round(10.0 ** (4.0 + 2.0 * next(g))))
    cell_seed = int(next(g) * 2 ** 63)
    rng = np.random.default_rng(cell_seed)
    st = 10.0 ** rng.uniform(-1.0, 2.0, side * side)
    ratio = rng.uniform(0.0, 0.99, side * side)
    ss = ratio * st
    sa = st - ss
    return ProblemSpec(nx=side, ny=side, lx=L, ly=L, sigma_a=sa, sigma_s=ss,
                       Q=np.ones(side * side), ic=None, c=1.0, dt=dt, n_s=n_s, n_hist=n_hist,
                       seed=base_seed * 100003 + p, sampler=SOBOL, precision=precision,
                       sn_order=4, name=f"batch{base_seed}_{p}")


def large(seed: int = 0, n_hist: int = 100_000_000, precision: int = FP32, n: int = 1024,
          block: int = 8) -> ProblemSpec:
    """10x10 cm, n x n cells, (n/block)^2 material blocks with sigma_t in {1,10,1000};
    scattering ratio 0.999 where sigma_t = 1000, else 0.5; Q = 1 uniform; N_s = 8; S8."""
    rng = np.random.default_rng(seed)
    nb = n // block
    choice = rng.integers(0, 3, size=(nb, nb))
    st_blk = np.array([1.0, 10.0, 1000.0])[choice]
    rt_blk = np.where(st_blk == 1000.0, 0.999, 0.5)
    st = np.kron(st_blk, np.ones((block, block)))
    rt = np.kron(rt_blk, np.ones((block, block)))
    ss = st * rt
    sa = st - ss
    return ProblemSpec(nx=n, ny=n, lx=10.0, ly=10.0, sigma_a=sa.ravel(), sigma_s=ss.ravel(),
                       Q=np.ones(n * n), ic=None, c=1.0, dt=0.01, n_s=8, n_hist=n_hist, seed=seed,
                       sampler=SOBOL, precision=precision, sn_order=8, name=f"large{n}")


def homogeneous(n: int = 8, L: float = 1.0, sigma_a: float = 0.1, sigma_s: float = 1.0,
                Q: float | None = 1.0, **kw) -> ProblemSpec:
    """A homogeneous n x n square, optionally with a uniform source."""
    return ProblemSpec(nx=n, ny=n, lx=L, ly=L, sigma_a=np.full(n * n, sigma_a),
                       sigma_s=np.full(n * n, sigma_s),
                       Q=None if Q is None else np.full(n * n, Q), **kw)


def random_bank(spec: ProblemSpec, n: int, seed: int, w_scale: float = 1.0) -> dict:
    """A census bank of n particles with seeded random cells, in-cell offsets, isotropic
    in-plane directions (|Omega_xy| <= 1) and positive weights."""
    rng = np.random.default_rng(seed)
    dx, dy = spec.lx / spec.nx, spec.ly / spec.ny
    cell = rng.integers(0, spec.nx * spec.ny, n).astype(np.int32)
    mu = rng.uniform(-1, 1, n)
    ph = rng.uniform(0, 2 * np.pi, n)
    s = np.sqrt(1 - mu * mu)
    return {"cell": cell, "fx": rng.uniform(0, dx, n), "fy": rng.uniform(0, dy, n),
            "ox": s * np.cos(ph), "oy": s * np.sin(ph),
            "w": w_scale * rng.uniform(0.5, 1.5, n), "n": n}
