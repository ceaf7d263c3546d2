"""Pins of the oracle's MC leg (Sec. 2.3) and source sampling.

Checks rest on exact rational geometry, closed forms (implicit capture w e^{-sigma l}, the
track-length integral, the Poisson/Erlang law of App. B), numerical quadrature, the N_s = 0
reduction to the uncollided split (Sec. 2.2/2.3), and the particle balance.
"""
import math
from fractions import Fraction as F

import numpy as np
import pytest
from scipy import integrate

from paper_2511_16821_gb300 import workloads as W


def one_particle_bank(cell, fx, fy, ox, oy, w=1.0):
    return {"cell": np.array([cell], np.int32), "fx": np.array([fx]), "fy": np.array([fy]),
            "ox": np.array([ox]), "oy": np.array([oy]), "w": np.array([w]), "n": 1}


def rational_track(nx, ny, dx, dy, cell, fx, fy, ox, oy, L):
    """Exact straight-line walk (Fractions): returns [(cell, l)] and fate ('census'|'leaked').
    Ties: a simultaneous x and y face hit moves diagonally; a face at exactly the census
    distance counts as a crossing."""
    ix, iy = cell % nx, cell // nx
    fx, fy, ox, oy, dx, dy, rem = map(F, (fx, fy, ox, oy, dx, dy, L))
    segs = []
    while True:
        tx = (dx - fx) / ox if ox > 0 else (fx / (-ox) if ox < 0 else None)
        ty = (dy - fy) / oy if oy > 0 else (fy / (-oy) if oy < 0 else None)
        cands = [t for t in (tx, ty) if t is not None]
        tf = min(cands) if cands else None
        if tf is None or tf > rem:
            segs.append((iy * nx + ix, rem))
            return segs, "census", iy * nx + ix
        segs.append((iy * nx + ix, tf))
        rem -= tf
        fx += ox * tf
        fy += oy * tf
        if tx is not None and tx == tf:
            ix += 1 if ox > 0 else -1
            fx = F(0) if ox > 0 else dx
        if ty is not None and ty == tf:
            iy += 1 if oy > 0 else -1
            fy = F(0) if oy > 0 else dy
        if not (0 <= ix < nx and 0 <= iy < ny):
            return segs, "leaked", min(max(iy, 0), ny - 1) * nx + min(max(ix, 0), nx - 1)


CASES = [
    # (cell, fx/dx, fy/dy, ox, oy, c*dt)
    (9, 0.375, 0.25, 0.3, 0.4, 2.0),
    (14, 0.5, 0.5, -0.6, 0.25, 1.7),
    (9, 0.5, 0.5, 0.5, 0.5, 3.0),       # diagonal through exact corners
    (20, 0.125, 0.75, 1.0, 0.0, 1.3),    # axis aligned
    (33, 0.625, 0.875, 0.0, -0.8, 0.9),
    (21, 0.25, 0.5, -0.7, -0.7, 5.0),    # leaks through a corner region
]


@pytest.mark.parametrize("case", CASES)
def test_uncollided_geometry_and_tally_exact(orc, case):
    cell, ax, ay, ox, oy, L = case
    nx, ny, lx, ly = 6, 7, 1.5, 2.1
    rng = np.random.default_rng(cell)
    sa = rng.uniform(0.2, 3.0, nx * ny)
    spec = W.ProblemSpec(nx=nx, ny=ny, lx=lx, ly=ly, sigma_a=sa, sigma_s=np.zeros(nx * ny),
                         Q=None, c=2.0, dt=L / 2.0, n_s=2, n_hist=1)
    dx, dy = lx / nx, ly / ny
    fx, fy = ax * dx, ay * dy
    bank = one_particle_bank(cell, fx, fy, ox, oy, 1.0)
    r = orc.mc_leg(spec, 0, bank, want_hist=True, want_census=True)
    segs, fate, last = rational_track(nx, ny, dx, dy, cell, fx, fy, ox, oy, spec.c * spec.dt)
    # exact per-cell tally w_in (1 - e^{-sigma l}) / sigma with w_in = exp(-sum sigma l)
    expect = np.zeros(nx * ny)
    tau = 0.0
    for k, l in segs:
        l = float(l)
        expect[k] += math.exp(-tau) * (-math.expm1(-sa[k] * l)) / sa[k]
        tau += sa[k] * l
    assert np.allclose(r["pre"], expect, rtol=1e-13, atol=1e-16)
    assert np.all(r["post"] == 0)
    h = r["hist"][0]
    assert h[0] == last
    assert h[1] == (1 if fate == "census" else 0)
    n_zero = sum(1 for _, l in segs if l == 0)
    assert h[3] == len(segs) - n_zero or h[3] == len(segs)
    if fate == "census":
        assert r["census"]["n"] == 1
        assert math.isclose(r["census"]["w"][0], math.exp(-tau), rel_tol=1e-13)
    else:
        assert math.isclose(r["stats"]["w_leaked"], math.exp(-tau), rel_tol=1e-13)


def test_ns0_reduces_to_uncollided_leg(orc):
    # N_s = 0: no collisions, no pre tally; the post leg is the uncollided leg with sigma_t, so it
    # equals the pre tally of a purely absorbing run with sigma_a' = sigma_t (Sec. 2.3, N_s = 0).
    base = W.checkerboard(n_s=0, n_hist=4000, cells_per_block=4)
    rng = np.random.default_rng(4)
    sa = base.sigma_a + rng.uniform(0, 0.5, base.ncells)
    ss = base.sigma_s + rng.uniform(0, 0.5, base.ncells)
    A = base.with_(sigma_a=sa, sigma_s=ss, n_s=0)
    B = base.with_(sigma_a=sa + ss, sigma_s=np.zeros(base.ncells), n_s=3)
    bank = W.random_bank(base, 3000, seed=9)
    ra = orc.mc_leg(A, 2, bank, want_hist=True)
    rb = orc.mc_leg(B, 2, bank, want_hist=True)
    assert ra["stats"]["collisions"] == 0 and np.all(ra["pre"] == 0)
    assert ra["stats"]["reached_limit"] == ra["stats"]["histories"]
    assert np.array_equal(ra["hist"][:, [0, 1, 3]], rb["hist"][:, [0, 1, 3]])
    assert np.allclose(ra["post"], rb["pre"], rtol=1e-13, atol=0)
    # hand-off weight = (sigma_s/sigma_t) x absorbed weight of the uncollided run, per cell
    st = sa + ss
    assert np.allclose(ra["mom"][:, 0], ss * rb["pre"], rtol=1e-12, atol=0)
    assert math.isclose(ra["stats"]["w_handoff"], float(np.sum(ss * rb["pre"])), rel_tol=1e-12)
    assert math.isclose(ra["stats"]["w_absorbed"], float(np.sum(sa * rb["pre"])), rel_tol=1e-12)
    assert math.isclose(rb["stats"]["w_absorbed"], float(np.sum(st * rb["pre"])), rel_tol=1e-12)


@pytest.mark.parametrize("which", ["pulse", "checker", "killing"])
def test_particle_balance(orc, which):
    if which == "pulse":
        spec = W.pulse(n_hist=5000)
        bank = orc.init_bank(spec, spec.ic)
    elif which == "checker":
        spec = W.checkerboard(n_s=2, n_hist=5000, cells_per_block=4)
        bank = W.random_bank(spec, 2000, seed=1)
    else:
        spec = W.checkerboard(n_s=4, n_hist=5000, cells_per_block=4).with_(w_min=0.5)
        bank = W.random_bank(spec, 2000, seed=2)
    r = orc.mc_leg(spec, 1, bank)
    s = r["stats"]
    out = s["w_absorbed"] + s["w_leaked"] + s["w_census"] + s["w_handoff"] + s["w_killed"]
    assert math.isclose(s["w_source"], out, rel_tol=1e-13)
    assert s["leaked"] + s["census"] + s["killed"] == s["histories"]
    if which == "killing":
        assert s["killed"] > 0
    # absorbed weight in the pre-limit legs equals sigma_a x pre tally (implicit capture)
    sa = spec.sigma_a
    st = spec.sigma_a + spec.sigma_s
    absorbed = float(np.sum(sa * r["pre"])) + float(np.sum(np.where(st > 0, sa / np.where(st > 0, st, 1), 0) * st * r["post"]))
    assert math.isclose(s["w_absorbed"], absorbed, rel_tol=1e-12)
    assert math.isclose(s["w_handoff"], float(np.sum(r["mom"][:, 0])), rel_tol=1e-12)


def test_infinite_medium_zero_variance(orc):
    # Far from the boundary and with N_s never reached, implicit capture makes every history's
    # weight w0 exp(-sigma_a c dt) however often it scatters (Sec. 2.3, unlimited case).
    n = 41
    spec = W.homogeneous(n=n, L=41.0, sigma_a=0.7, sigma_s=2.0, Q=None, c=1.0, dt=0.25, n_s=14,
                         n_hist=1)
    centre = (n // 2) * n + n // 2
    N = 4000
    bank = {"cell": np.full(N, centre, np.int32), "fx": np.full(N, 0.5), "fy": np.full(N, 0.5),
            "ox": np.cos(np.linspace(0, 6, N)) * 0.9, "oy": np.sin(np.linspace(0, 6, N)) * 0.9,
            "w": np.ones(N), "n": N}
    r = orc.mc_leg(spec, 0, bank, want_census=True)
    s = r["stats"]
    assert s["leaked"] == 0 and s["reached_limit"] == 0 and s["collisions"] > N / 4
    assert np.allclose(r["census"]["w"], math.exp(-0.7 * 0.25), rtol=1e-14)


@pytest.mark.parametrize("n_s", [1, 2, 40])
def test_scatter_count_is_poisson_erlang(orc, n_s):
    # Census-born histories in an infinite homogeneous medium: inter-scatter times are
    # Exp(sigma_s c), so the scatter count at t_{n+1} is Poisson(lambda), lambda = sigma_s c dt,
    # truncated at N_s; P(reach N_s) = 1 - e^{-lambda} sum_{j<N_s} lambda^j/j!  (App. B tail).
    n = 41
    lam = 1.3
    spec = W.homogeneous(n=n, L=410.0, sigma_a=0.0, sigma_s=lam, Q=None, c=1.0, dt=1.0,
                         n_s=n_s, n_hist=1)
    centre = (n // 2) * n + n // 2
    N = 2 ** 14
    bank = {"cell": np.full(N, centre, np.int32), "fx": np.full(N, 5.0), "fy": np.full(N, 5.0),
            "ox": np.full(N, 0.6), "oy": np.full(N, -0.3), "w": np.ones(N), "n": N}
    r = orc.mc_leg(spec, 0, bank, want_hist=True)
    nfin = r["hist"][:, 2]
    assert r["stats"]["leaked"] == 0
    pois = [math.exp(-lam) * lam ** j / math.factorial(j) for j in range(60)]
    for j in range(min(n_s, 6)):
        p = pois[j]
        assert abs(np.mean(nfin == j) - p) < 4 * math.sqrt(p * (1 - p) / N) + 1e-3
    p_reach = 1.0 - sum(pois[:n_s])
    got = np.mean(nfin == n_s)
    assert abs(got - p_reach) < 4 * math.sqrt(max(p_reach * (1 - p_reach), 1e-12) / N) + 1e-3
    assert r["stats"]["reached_limit"] == int(np.sum(nfin == n_s))


@pytest.mark.parametrize("sig", [0.05, 0.9, 7.0])
def test_handoff_moments_match_quadrature(orc, sig):
    # Post-limit (N_s = 0) single segment inside one cell: m_j = sigma_s int w0 e^{-sigma_t s}
    # P_j(xi(s), eta(s)) ds, P = (1, xi, eta, xi eta), compared with adaptive quadrature.
    ss = 0.4 * sig
    spec = W.homogeneous(n=1, L=10.0, sigma_a=sig - ss, sigma_s=ss, Q=None, c=1.0, dt=0.9,
                         n_s=0, n_hist=1)
    fx, fy, ox, oy = 3.0, 6.5, 0.55, -0.35
    r = orc.mc_leg(spec, 0, one_particle_bank(0, fx, fy, ox, oy, 2.0))
    l = 0.9

    def P(j, s):
        xi = 2 * (fx + ox * s) / 10.0 - 1
        eta = 2 * (fy + oy * s) / 10.0 - 1
        return (1.0, xi, eta, xi * eta)[j]

    for j in range(4):
        val, _ = integrate.quad(lambda s: ss * 2.0 * math.exp(-sig * s) * P(j, s), 0, l,
                                epsabs=0, epsrel=1e-13, limit=200)
        assert math.isclose(r["mom"][0, j], val, rel_tol=1e-12, abs_tol=1e-15)
    assert math.isclose(r["post"][0], 2.0 * (-math.expm1(-sig * l)) / sig, rel_tol=1e-14)


def test_uniform_source_is_stratified(orc):
    # Q uniform on a 16x16 mesh: cell choice reduces to (floor(u0 nx), floor(u1 ny)); dims 0-1
    # of the shifted Sobol set form a (0,2)-net, so 256 births fill each cell exactly once.
    spec = W.homogeneous(n=16, L=2.0, Q=3.0, dt=0.5, n_hist=256, seed=11)
    b = orc.sample_births(spec, 4, 256)
    assert np.array_equal(np.sort(b["cell"]), np.arange(256))
    assert math.isclose(b["w0"] * 256, 3.0 * 4.0 * 0.5, rel_tol=1e-15)
    # single row: the in-row position is exactly u0 * L
    row = W.ProblemSpec(nx=8, ny=1, lx=2.0, ly=0.5, sigma_a=np.ones(8), sigma_s=np.zeros(8),
                        Q=np.ones(8), n_hist=100, seed=2)
    b = orc.sample_births(row, 0, 100)
    P = orc.points(2, 0, 2, 0, 0, 100, 2)
    u0 = (P[:, 0].astype(np.float64) + 0.5) / 2 ** 32
    x = (b["cell"] % 8) * 0.25 + b["fx"]
    assert np.allclose(x, u0 * 2.0, rtol=0, atol=1e-15)
    u2 = (P[:, 1].astype(np.float64) + 0.5) / 2 ** 32
    assert np.allclose(b["fy"], u2 * 0.5, rtol=0, atol=1e-15)


@pytest.mark.parametrize("nx,ny", [(4096, 2048), (4096, 4096)])
def test_cdf_total_fits_on_the_largest_meshes(orc, nx, ny):
    # uniform weights on the largest accepted meshes: the quantisation 2^B with B = min(40, 62 -
    # ceil(log2 ncells)) keeps the total at 2^62 (2^40 per cell would overflow int64 from 2^23 cells
    # on); every prefix is non-negative and strictly increasing, and a point's cell is the
    # uniform map floor(u n)
    q, rp, cp = orc.build_cdf(nx, ny, np.ones(nx * ny))
    B = min(40, 62 - int(math.ceil(math.log2(nx * ny))))
    assert np.all(q == 2 ** B)
    assert int(rp[-1]) == nx * ny * 2 ** B <= 2 ** 62
    assert np.all(np.diff(rp) == nx * 2 ** B)
    row = cp.reshape(ny, nx + 1)
    assert np.all(np.diff(row, axis=1) == 2 ** B)


def test_cdf_quantisation_unchanged_below_2_22_cells(orc):
    # meshes up to 2^22 cells keep the 2^40 scale
    w = np.random.default_rng(1).uniform(0.1, 1, 2048 * 2048)
    q, rp, _ = orc.build_cdf(2048, 2048, w)
    assert np.array_equal(q, np.rint(w / w.max() * 2.0 ** 40).astype(np.int64))


def test_decision_margins_and_history_subsets(orc):
    # margins lie in [0, 1] and are small only where two event distances nearly tie; a leg over a
    # subset (index range, skip mask) tracks exactly those histories: the records of the subsets
    # are the whole leg's rows, and the counters and tallies of complementary subsets add up
    spec = W.checkerboard(n_s=2, n_hist=3000, cells_per_block=3)
    bank = W.random_bank(spec, 1000, seed=2)
    full = orc.mc_leg(spec, 1, bank, want_hist=True, want_margin=True)
    m = full["margin"]
    n = full["stats"]["histories"]
    assert n == 4000 and m.shape == (n,) and np.all((m >= 0) & (m <= 1))
    skip = np.zeros(n, np.uint8)
    skip[::7] = 1
    a = orc.mc_leg(spec, 1, bank, want_hist=True, want_margin=True, skip=skip)
    b = orc.mc_leg(spec, 1, bank, want_hist=True, want_margin=True, skip=1 - skip)
    assert np.array_equal(a["hist"], full["hist"][skip == 0]) and np.array_equal(b["hist"], full["hist"][skip == 1])
    assert np.array_equal(a["margin"], m[skip == 0])
    for k in ("histories", "segments", "collisions", "leaked", "census", "killed", "reached_limit"):
        assert a["stats"][k] + b["stats"][k] == full["stats"][k], k
    for k in ("pre", "post", "mom"):
        assert np.allclose(a[k] + b[k], full[k], rtol=1e-13, atol=1e-300), k
    r = orc.mc_leg(spec, 1, bank, want_hist=True, h0=1500, h1=2500)
    assert np.array_equal(r["hist"], full["hist"][1500:2500])
    # a history whose two smallest event distances are equal (an exact corner: start at the cell's
    # centre moving along the diagonal) has margin 0
    one = W.homogeneous(n=2, L=2.0, sigma_a=0.1, sigma_s=0.0, Q=None, n_hist=1, dt=10.0, n_s=0)
    c = math.sqrt(0.5)
    bk = {"cell": np.array([0], np.int32), "fx": np.array([0.5]), "fy": np.array([0.5]),
          "ox": np.array([c]), "oy": np.array([c]), "w": np.array([1.0]), "n": 1}
    r1 = orc.mc_leg(one, 0, bk, want_margin=True)
    assert r1["margin"][0] == 0.0


def test_nonuniform_source_cell_frequencies(orc):
    # Births land in cells in proportion to Q * area (integer CDF), to within the 1-D Sobol
    # stratification error of the row/column picks.
    rng = np.random.default_rng(5)
    Q = rng.uniform(0, 1, 64) ** 3
    spec = W.ProblemSpec(nx=8, ny=8, lx=1.0, ly=3.0, sigma_a=np.ones(64), sigma_s=np.zeros(64),
                         Q=Q, n_hist=2 ** 16, seed=3)
    b = orc.sample_births(spec, 0, 2 ** 16)
    freq = np.bincount(b["cell"], minlength=64) / 2 ** 16
    assert np.allclose(freq, Q / Q.sum(), atol=2e-4)
    iy = b["cell"] // 8
    assert np.all(b["fx"] >= 0) and np.all(b["fx"] <= 1.0 / 8)
    assert np.all(b["fy"] >= 0) and np.all(b["fy"] <= 3.0 / 8)
    del iy


def test_direction_is_isotropic(orc):
    spec = W.homogeneous(n=4, Q=1.0, n_hist=2 ** 14)
    b = orc.sample_births(spec, 0, 2 ** 14)
    r2 = b["ox"] ** 2 + b["oy"] ** 2
    # in-plane projection of an isotropic 3-D direction: <Ox^2> = <Oy^2> = 1/3, |Oxy| <= 1
    assert np.all(r2 <= 1 + 1e-15)
    assert abs(np.mean(b["ox"] ** 2) - 1 / 3) < 1e-3 and abs(np.mean(b["oy"] ** 2) - 1 / 3) < 1e-3
    assert abs(np.mean(b["ox"])) < 1e-3 and abs(np.mean(b["oy"] * b["ox"])) < 1e-3
    assert abs(np.mean(b["t_frac"]) - 0.5) < 1e-4


# ------------------------------------------------------------------------------------------------
# space-dependent N_s (per-cell scatter limits)
# ------------------------------------------------------------------------------------------------
def _cb_limits(spec, scatter_limit, absorber_limit=0):
    """Per-cell limits on the checkerboard: absorber cells (sigma_s = 0) and scatterer cells."""
    return np.where(spec.sigma_s > 0, scatter_limit, absorber_limit).astype(np.int32)


def test_uniform_cell_limits_equal_scalar_ns(orc):
    spec = W.checkerboard(n_s=2, n_hist=3000, cells_per_block=4)
    bank = W.random_bank(spec, 1500, seed=5)
    a = orc.mc_leg(spec, 1, bank, want_hist=True)
    b = orc.mc_leg(spec.with_(n_s_cell=np.full(spec.ncells, 2, np.int32)), 1, bank, want_hist=True)
    for k in ("pre", "post", "mom", "hist"):
        assert np.array_equal(a[k], b[k]), k
    assert a["stats"] == b["stats"]


def test_zero_cell_limits_equal_ns0(orc):
    """All limits 0 under a larger n_s: no scatter anywhere, every segment post-limit: the N_s = 0
    leg bit for bit (the optical depths drawn for the larger n_s are never used)."""
    spec = W.checkerboard(n_s=3, n_hist=3000, cells_per_block=4)
    bank = W.random_bank(spec, 1500, seed=6)
    a = orc.mc_leg(spec.with_(n_s=0), 1, bank, want_hist=True)
    b = orc.mc_leg(spec.with_(n_s_cell=np.zeros(spec.ncells, np.int32)), 1, bank, want_hist=True)
    for k in ("pre", "post", "mom", "hist"):
        assert np.array_equal(a[k], b[k]), k
    assert a["stats"] == b["stats"]


def test_cell_limits_split_the_tallies_by_region(orc):
    """A segment is pre-limit exactly when the scatter count is below the limit of its cell: no
    pre-limit track length in zero-limit cells, and no post-limit track length (nor hand-off) in
    cells whose limit no history reaches; the leg balance still closes."""
    spec = W.checkerboard(n_s=12, n_hist=4000, cells_per_block=4)
    rng = np.random.default_rng(3)
    lim = np.where(rng.uniform(size=spec.ncells) < 0.5, 0, 12).astype(np.int32)
    spec = spec.with_(n_s_cell=lim)
    bank = W.random_bank(spec, 2000, seed=7)
    r = orc.mc_leg(spec, 1, bank, want_hist=True)
    assert r["stats"]["collisions"] > 0
    assert np.max(r["hist"][:, 2]) < 12
    assert np.all(r["pre"][lim == 0] == 0.0)
    assert np.all(r["post"][lim == 12] == 0.0) and np.all(r["mom"][lim == 12] == 0.0)
    assert np.any(r["pre"][lim == 12] > 0) and np.any(r["post"][lim == 0] > 0)
    s = r["stats"]
    out = s["w_absorbed"] + s["w_leaked"] + s["w_census"] + s["w_handoff"] + s["w_killed"]
    assert math.isclose(s["w_source"], out, rel_tol=1e-13)
    assert math.isclose(s["w_handoff"], float(np.sum(r["mom"][:, 0])), rel_tol=1e-12)


def test_zero_limits_in_non_scattering_cells_give_the_pure_mc_leg(orc):
    """Limit 0 where sigma_s = 0 (nothing to hand off there: post-limit attenuation with sigma_t =
    sigma_a is the pre-limit implicit capture) and a limit no history reaches elsewhere: the leg is
    the N_s = infinity leg, its pre tally split into pre + post by region, weights and census alike."""
    spec = W.checkerboard(n_s=20, n_hist=3000, cells_per_block=4)
    bank = W.random_bank(spec, 1500, seed=8)
    lim = _cb_limits(spec, 20, 0)
    a = orc.mc_leg(spec.with_(n_s=W.NS_INF), 1, bank, want_hist=True, want_census=True)
    b = orc.mc_leg(spec.with_(n_s_cell=lim), 1, bank, want_hist=True, want_census=True)
    assert np.max(b["hist"][:, 2]) < 20
    assert np.array_equal(a["pre"], b["pre"] + b["post"])
    assert np.all(b["mom"] == 0.0) and b["stats"]["w_handoff"] == 0.0
    assert np.array_equal(a["hist"][:, :2], b["hist"][:, :2]) and np.array_equal(a["hist"][:, 3], b["hist"][:, 3])
    for k in ("cell", "fx", "fy", "ox", "oy", "w"):
        assert np.array_equal(a["census"][k], b["census"][k]), k
    for k in ("w_absorbed", "w_leaked", "w_census"):
        assert a["stats"][k] == b["stats"][k], k
