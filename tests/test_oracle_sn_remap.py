"""Pins of the oracle's collided S_N-DG stage (Sec. 2.2 step 2) and the remap (step 3, Eq. (R)).

S_N-DG: sphere-moment identities of the quadrature, exact reproduction of a bilinear
manufactured solution (the DG space contains it), the thick infinite-medium limit
phi = q / (sigma_a + 1/(c dt)), and source iteration against a dense direct solve.
Remap: a pure absorber remaps to exactly the MC-leg census, birth weights integrate the remap
source, uniform sources give stratified births, bilinear in-cell sampling has the right
moments, the comb conserves weight and count.
"""
import math

import numpy as np
import pytest

from paper_2511_16821_gb300 import workloads as W

FOURPI = 4 * math.pi


@pytest.mark.parametrize("order,count", [(4, 12), (8, 40)])
def test_quadrature_sphere_moments(orc, order, count):
    ox, oy, oz, w = orc.quadrature(order)
    assert len(w) == count and np.all(w > 0) and np.all(oz > 0)
    assert np.allclose(ox ** 2 + oy ** 2 + oz ** 2, 1.0, atol=1e-15)
    assert math.isclose(w.sum(), FOURPI, rel_tol=1e-14)
    for comp in (ox, oy, oz):
        assert math.isclose(np.sum(w * comp ** 2), FOURPI / 3, rel_tol=1e-13)
    for comp in (ox, oy, ox * oy):          # odd in-plane moments vanish (the z-half is mirrored)
        assert abs(np.sum(w * comp)) < 1e-13
    for p in range(2, order // 2 + 1):   # even moments up to mu^N are exact
        assert math.isclose(np.sum(w * oz ** (2 * p)), FOURPI / (2 * p + 1), rel_tol=1e-12)


@pytest.mark.parametrize("ox,oy", [(0.35, 0.8), (-0.6, 0.3), (-0.2, -0.9), (0.7, -0.5)])
def test_dg_reproduces_bilinear_solution(orc, ox, oy):
    nx, ny, lx, ly = 5, 4, 2.0, 1.2
    hx, hy = lx / nx / 2, ly / ny / 2
    rng = np.random.default_rng(3)
    sig = rng.uniform(0.5, 4.0, nx * ny)
    al, be, ga, de = 1.3, -0.4, 0.7, 0.25
    a = np.zeros((nx * ny, 4))
    S = np.zeros((nx * ny, 4))
    norm = np.array([1, 1 / 3, 1 / 3, 1 / 9])
    A = 4 * hx * hy
    for iy in range(ny):
        for ix in range(nx):
            k = iy * nx + ix
            xc, yc = (2 * ix + 1) * hx, (2 * iy + 1) * hy
            a[k] = [al + be * xc + ga * yc + de * xc * yc, (be + de * yc) * hx, (ga + de * xc) * hy,
                    de * hx * hy]
            s = sig[k] * a[k] + np.array([ox * be + oy * ga + ox * de * yc + oy * de * xc,
                                          oy * de * hx, ox * de * hy, 0.0])
            S[k] = A * norm * s
    xb = 0.0 if ox > 0 else lx
    yb = 0.0 if oy > 0 else ly
    in_x = np.array([[al + be * xb + ga * (2 * iy + 1) * hy + de * xb * (2 * iy + 1) * hy,
                      (ga + de * xb) * hy] for iy in range(ny)])
    in_y = np.array([[al + be * (2 * ix + 1) * hx + ga * yb + de * (2 * ix + 1) * hx * yb,
                      (be + de * yb) * hx] for ix in range(nx)])
    psi = orc.dg_sweep(nx, ny, lx, ly, sig, ox, oy, S, in_x, in_y)
    assert np.allclose(psi, a, rtol=1e-12, atol=1e-13)


def test_sn_thick_infinite_medium_limit(orc):
    n, L = 24, 24.0
    spec = W.homogeneous(n=n, L=L, sigma_a=5.0, sigma_s=5.0, Q=None, c=1.0, dt=0.1, n_s=1,
                         sn_order=4, sn_tol=1e-13)
    A = (L / n) ** 2
    m0 = 0.37
    mom = np.zeros((n * n, 4))
    mom[:, 0] = m0
    phi, it = orc.sn_solve(spec, mom)
    q = m0 / (A * spec.dt)                       # emission per unit area per unit time
    expect = q / (5.0 + 1.0 / (spec.c * spec.dt))
    centre = (n // 2) * n + n // 2
    assert math.isclose(phi[centre, 0], expect, rel_tol=1e-10)
    assert np.all(np.abs(phi[centre, 1:]) < 1e-10 * expect)
    assert it > 2


def test_source_iteration_matches_direct_solve(orc):
    nx, ny = 3, 2
    rng = np.random.default_rng(8)
    spec = W.ProblemSpec(nx=nx, ny=ny, lx=1.5, ly=0.8, sigma_a=rng.uniform(0.1, 1, 6),
                         sigma_s=rng.uniform(0.5, 3, 6), Q=None, dt=0.2, n_s=1, sn_order=8,
                         sn_tol=1e-15, sn_max_iter=2000)
    mom = rng.uniform(0, 1, (6, 4)) * np.array([1, 0.2, 0.2, 0.05])
    phi, it = orc.sn_solve(spec, mom)
    ox, oy, oz, w = orc.quadrature(8)
    A = (1.5 / nx) * (0.8 / ny)
    norm = np.array([1, 1 / 3, 1 / 3, 1 / 9])
    sig = spec.sigma_a + spec.sigma_s + 1 / (spec.c * spec.dt)

    def F(ph):
        S = (spec.sigma_s[:, None] / FOURPI) * ph.reshape(6, 4) * A * norm + mom / (FOURPI * spec.dt)
        out = np.zeros((6, 4))
        for m in range(len(w)):
            out += w[m] * orc.dg_sweep(nx, ny, 1.5, 0.8, sig, ox[m], oy[m], S)
        return out.ravel()

    f0 = F(np.zeros(24))
    J = np.stack([F(np.eye(24)[k]) - f0 for k in range(24)], axis=1)
    direct = np.linalg.solve(np.eye(24) - J, f0)
    assert np.allclose(phi.ravel(), direct, rtol=1e-11, atol=1e-14)


def _absorber(n=12, **kw):
    rng = np.random.default_rng(1)
    return W.ProblemSpec(nx=n, ny=n, lx=2.0, ly=2.0, sigma_a=rng.uniform(0.5, 3, n * n),
                         sigma_s=np.zeros(n * n), Q=None, dt=0.3, n_s=2, **kw)


def test_pure_absorber_remap_equals_mc_census(orc):
    spec = _absorber(n_hist=100, census_cap=10 ** 6)
    bank = W.random_bank(spec, 3000, seed=4)
    r = orc.mc_leg(spec, 0, bank, want_census=True)
    nc = spec.ncells
    out, st, combed = orc.remap(spec, 0, bank, r["pre"], r["post"], np.zeros((nc, 4)))
    c = r["census"]
    assert not combed and out["n"] == c["n"]
    assert np.array_equal(out["cell"], c["cell"])
    for k in ("fx", "fy", "ox", "oy", "w"):
        assert np.allclose(out[k], c[k], rtol=1e-14, atol=1e-15)


def test_remap_birth_weight_integrates_source(orc):
    spec = W.checkerboard(n_s=1, n_hist=5000, cells_per_block=4)
    bank = W.random_bank(spec, 1000, seed=3)
    r = orc.mc_leg(spec, 0, bank)
    phi, _ = orc.sn_solve(spec, r["mom"])
    # with cell-constant densities every birth carries w = W / N exactly
    phi0 = phi.copy()
    phi0[:, 1:] = 0.0
    f = orc.remap_density(spec, r["pre"], r["post"], phi0)
    A = (spec.lx / spec.nx) * (spec.ly / spec.ny)
    Wsrc = float(np.sum(np.abs(f[:, 0]) * A * spec.dt))
    out, st, _ = orc.remap(spec, 0, bank, r["pre"], r["post"], phi0)
    assert math.isclose(st["w_source"], float(bank["w"].sum()) + Wsrc, rel_tol=1e-12)
    f = orc.remap_density(spec, r["pre"], r["post"], phi)
    # remap source = Q + sigma_s (phi_pre + phi_post + phi_c): check the density by hand
    T = (r["pre"] + r["post"]) / (A * spec.dt)
    assert np.allclose(f[:, 0], spec.Q + spec.sigma_s * (T + phi[:, 0]), rtol=1e-14)
    assert np.allclose(f[:, 1:], spec.sigma_s[:, None] * phi[:, 1:], rtol=1e-14)


def test_uniform_remap_source_is_stratified(orc):
    n = 16
    spec = W.ProblemSpec(nx=n, ny=n, lx=1.0, ly=1.0, sigma_a=np.ones(n * n), sigma_s=np.zeros(n * n),
                         Q=np.full(n * n, 2.0), c=1e-12, dt=1.0, n_hist=n * n, seed=5)
    out, st, combed = orc.remap(spec, 3, None, np.zeros(n * n), np.zeros(n * n), np.zeros((n * n, 4)))
    assert out["n"] == n * n and not combed
    assert np.array_equal(np.sort(out["cell"]), np.arange(n * n))


def test_bilinear_in_cell_sampling_moments(orc):
    spec = W.ProblemSpec(nx=1, ny=1, lx=2.0, ly=3.0, sigma_a=np.ones(1), sigma_s=np.ones(1),
                         Q=None, c=1e-12, dt=1.0, n_hist=2 ** 14, seed=9, census_cap=2 ** 20)
    f = np.array([[1.0, 0.4, -0.3, 0.2]])   # all nodal values positive: inverse CDF
    out, st, _ = orc.remap(spec, 0, None, np.zeros(1), np.zeros(1), f)
    xi = 2 * out["fx"] / 2.0 - 1
    eta = 2 * out["fy"] / 3.0 - 1
    assert np.allclose(out["w"], out["w"][0], rtol=0)
    assert abs(np.mean(xi) - 0.4 / 3) < 2e-4
    assert abs(np.mean(eta) + 0.3 / 3) < 2e-4
    assert abs(np.mean(xi * eta) - 0.2 / 9) < 2e-4
    # negative nodal value: uniform positions, weight factor f(xi, eta)/|f0|
    g = np.array([[1.0, 0.9, 0.5, 0.1]])
    out, st, _ = orc.remap(spec, 0, None, np.zeros(1), np.zeros(1), g)
    xi = 2 * out["fx"] / 2.0 - 1
    eta = 2 * out["fy"] / 3.0 - 1
    wbar = 1.0 * 6.0 * 1.0 / 2 ** 14
    expect = wbar * (1.0 + 0.9 * xi + 0.5 * eta + 0.1 * xi * eta)
    assert np.allclose(out["w"], expect, rtol=1e-9)
    assert abs(np.mean(xi)) < 2e-4 and np.any(out["w"] < 0)


def test_comb_conserves_count_and_weight(orc):
    spec = _absorber(n_hist=1)
    bank = W.random_bank(spec, 1000, seed=12)
    nc = spec.ncells
    z = np.zeros(nc)
    full, _, c0 = orc.remap(spec.with_(census_cap=10 ** 6), 0, bank, z, z, np.zeros((nc, 4)))
    cap = 300
    out, st, combed = orc.remap(spec.with_(census_cap=cap), 0, bank, z, z, np.zeros((nc, 4)))
    assert combed and not c0 and out["n"] == cap
    assert math.isclose(out["w"].sum(), full["w"].sum(), rel_tol=1e-12)
    assert np.allclose(out["w"], full["w"].sum() / cap, rtol=1e-12)
    # copies of survivor j ~ cap * w_j / sum w, within one
    key = {(int(c), float(x), float(y)): j for j, (c, x, y) in enumerate(zip(full["cell"], full["fx"], full["fy"]))}
    cnt = np.zeros(full["n"])
    for c, x, y in zip(out["cell"], out["fx"], out["fy"]):
        cnt[key[(int(c), float(x), float(y))]] += 1
    ideal = cap * full["w"] / full["w"].sum()
    assert np.all(np.abs(cnt - ideal) < 1.0 + 1e-9)


def test_pure_mc_step_total_is_exact(orc):
    # N_s = infinity (pure MC, Sec. 3 non-hybrid runs): no remap; with implicit capture and no
    # leakage the census total is W exp(-sigma_a c t) exactly at every step.
    n = 20
    spec = W.homogeneous(n=n, L=20.0, sigma_a=0.4, sigma_s=1.5, Q=None, dt=0.1, n_s=W.NS_INF,
                         n_hist=3000, census_cap=3000)
    ic = np.zeros(n * n)
    ic[(n // 2) * n + n // 2] = 1.0
    bank = orc.init_bank(spec, ic)
    for k in range(3):
        r = orc.step(spec, k, bank)
        bank = r["bank"]
        assert math.isclose(bank["w"].sum(), math.exp(-0.4 * 0.1 * (k + 1)), rel_tol=1e-12)


def test_hybrid_infinite_medium_decay(orc):
    # The hybrid step keeps the infinite-medium total decaying as exp(-sigma_a c t) up to the
    # step-averaging error of the scattering source, O(sigma_s sigma_t (c dt)^2) per step; the
    # error must shrink when dt is halved.
    def run(dt, steps):
        n = 16
        spec = W.homogeneous(n=n, L=16.0, sigma_a=0.5, sigma_s=1.0, Q=None, dt=dt, n_s=1,
                             n_hist=4000, sn_order=4)
        ic = np.zeros(n * n)
        ic[(n // 2) * n + n // 2] = 1.0
        bank = orc.init_bank(spec, ic)
        for k in range(steps):
            bank = orc.step(spec, k, bank)["bank"]
        return abs(bank["w"].sum() / math.exp(-0.5 * dt * steps) - 1.0)

    e1 = run(0.1, 4)
    e2 = run(0.05, 8)
    assert e1 < 4 * 1.0 * 1.5 * 0.1 ** 2
    assert e2 < e1


def _remap_inputs(orc, seed=3):
    spec = W.checkerboard(n_s=1, n_hist=3000, cells_per_block=2)
    bank = W.random_bank(spec, 2000, seed=seed)
    r = orc.mc_leg(spec, 0, bank)
    phi, _ = orc.sn_solve(spec, r["mom"])
    return spec, bank, r, phi


def test_census_cell_order_is_a_stable_sort(orc):
    """Without a comb the cell-ordered census holds the same particles as the slot-ordered one,
    ordered by cell and, within a cell, in slot order (a stable sort)."""
    spec, bank, r, phi = _remap_inputs(orc)
    spec = spec.with_(census_cap=10 ** 7)
    a, _, ca = orc.remap(spec, 0, bank, r["pre"], r["post"], phi)
    b, _, cb = orc.remap(spec.with_(census_order=1), 0, bank, r["pre"], r["post"], phi)
    assert not ca and not cb and a["n"] == b["n"]
    order = np.argsort(a["cell"], kind="stable")
    for k in ("cell", "fx", "fy", "ox", "oy", "w"):
        assert np.array_equal(b[k], a[k][order]), k


@pytest.mark.parametrize("order", [1, 2])
def test_census_sort_interval(orc, order):
    """With sort_every = 3 the sorted order applies on the steps n with n mod 3 == 0 only: the
    census of step 3 (and 0) equals the sorted one, that of steps 1 and 2 the slot-ordered one."""
    spec, bank, r, phi = _remap_inputs(orc)
    spec = spec.with_(census_cap=r["stats"]["census"] // 2 + 1)   # a comb along the census order
    for step in (0, 1, 2, 3):
        a, _, _ = orc.remap(spec.with_(census_order=order, sort_every=3), step, bank, r["pre"], r["post"], phi)
        want = order if step % 3 == 0 else 0
        b, _, _ = orc.remap(spec.with_(census_order=want), step, bank, r["pre"], r["post"], phi)
        assert a["n"] == b["n"], step
        for k in ("cell", "fx", "fy", "ox", "oy", "w"):
            assert np.array_equal(a[k], b[k]), (step, k)
    # and sorting on every step differs from never sorting, so the check above can fail
    c, _, _ = orc.remap(spec.with_(census_order=order), 1, bank, r["pre"], r["post"], phi)
    d, _, _ = orc.remap(spec.with_(census_order=0), 1, bank, r["pre"], r["post"], phi)
    assert not np.array_equal(c["cell"], d["cell"])


def test_cell_ordered_comb_keeps_each_cell_within_one_copy(orc):
    """A systematic comb along the cell-ordered census gives every cell the number of copies its
    quantised weight asks for, rounded up or down: its census weight is within one copy weight
    of its pre-comb weight. Along slot order the same comb misses cells by several copies."""
    spec, bank, r, phi = _remap_inputs(orc)
    full, _, _ = orc.remap(spec.with_(census_cap=10 ** 7), 0, bank, r["pre"], r["post"], phi)
    cap = full["n"] // 3
    nc = spec.nx * spec.ny
    want = np.bincount(full["cell"], weights=np.abs(full["w"]), minlength=nc)
    devs = {}
    for order in (0, 1):
        b, _, combed = orc.remap(spec.with_(census_cap=cap, census_order=order), 0, bank, r["pre"], r["post"], phi)
        assert combed and b["n"] == cap
        wcopy = float(np.abs(b["w"][0]))
        assert np.allclose(np.abs(b["w"]), wcopy, rtol=1e-15)
        got = np.bincount(b["cell"], weights=np.abs(b["w"]), minlength=nc)
        devs[order] = float(np.max(np.abs(got - want)) / wcopy)
    assert devs[1] <= 1.0 + 1e-6, devs
    assert devs[0] > 1.5, devs


# ------------------------------------------------------------------------------------------------
# steps 3'/4' of the previous hybrids (additive remap, remap_variant = 1)
# ------------------------------------------------------------------------------------------------
def test_additive_remap_pure_absorber_keeps_the_leg_census(orc):
    """Without scattering the Eq. (R') source sigma_s (phi_post + phi_c) is zero whatever Q is:
    the new census is the MC leg's census itself (the relabelling remap instead re-streams the
    bank and adds births from Q)."""
    spec = _absorber(n_hist=400, census_cap=10 ** 6).with_(Q=np.full(144, 0.7), remap_variant=1)
    bank = W.random_bank(spec, 2000, seed=6)
    r = orc.mc_leg(spec, 0, bank, want_census=True)
    nc = spec.ncells
    out, st, combed = orc.remap_additive(spec, 0, bank, r["census"], r["post"], np.zeros((nc, 4)))
    c = r["census"]
    assert not combed and st["histories"] == 0 and out["n"] == c["n"]
    for k in ("cell", "fx", "fy", "ox", "oy", "w"):
        assert np.array_equal(out[k], c[k]), k
    rel, _, _ = orc.remap(spec, 0, bank, r["pre"], r["post"], np.zeros((nc, 4)))
    assert rel["n"] > c["n"]


def test_additive_step_is_pure_mc_when_no_history_reaches_the_limit(orc):
    """When no history reaches N_s there is no hand-off, the collided flux is zero and so is the
    Eq. (R') source: a 3'/4' step is then the N_s = infinity step, bank for bank (same comb
    quantisation base: the step-start bank's max |w| and the birth weight)."""
    n = 10
    spec = W.homogeneous(n=n, L=2.0, sigma_a=0.3, sigma_s=0.05, Q=1.0, dt=0.2, n_s=12, n_hist=1500,
                         census_cap=900)
    bank = W.random_bank(spec, 1200, seed=8)
    for order in (0, 1):
        a = orc.step(spec.with_(remap_variant=1, census_order=order), 2, bank)
        b = orc.step(spec.with_(n_s=W.NS_INF, census_order=order), 2, bank)
        assert a["leg"]["reached_limit"] == 0 and np.all(a["phi"] == 0.0)
        assert a["bank"]["n"] == b["bank"]["n"] == 900
        for k in ("cell", "fx", "fy", "ox", "oy", "w"):
            assert np.array_equal(a["bank"][k], b["bank"][k]), (order, k)
        assert np.array_equal(a["flux"], b["flux"])


def test_additive_births_integrate_the_collided_emission(orc):
    """The Eq. (R') births carry sigma_s (phi_post + phi_c) A dt in total (each w = W / N for
    cell-constant densities) and their weight is conserved: start = absorbed + leaked + census."""
    spec = W.checkerboard(n_s=1, n_hist=4000, cells_per_block=4).with_(remap_variant=1, census_cap=10 ** 7)
    bank = W.random_bank(spec, 1500, seed=2)
    r = orc.mc_leg(spec, 0, bank, want_census=True)
    phi, _ = orc.sn_solve(spec, r["mom"])
    phi[:, 1:] = 0.0
    phi[:, 0] = np.maximum(phi[:, 0], 0.0)   # non-negative densities: every birth carries +W / N
    A = (spec.lx / spec.nx) * (spec.ly / spec.ny)
    W_exp = float(np.sum(spec.sigma_s * (r["post"] / (A * spec.dt) + phi[:, 0]) * A * spec.dt))
    assert W_exp > 0
    out, st, combed = orc.remap_additive(spec, 0, bank, r["census"], r["post"], phi)
    assert not combed and st["histories"] == spec.n_hist
    assert math.isclose(st["w_source"], W_exp, rel_tol=1e-12)
    w_births = out["w"][r["census"]["n"]:].sum()
    assert math.isclose(st["w_source"], st["w_absorbed"] + st["w_leaked"] + st["w_killed"] + w_births,
                        rel_tol=1e-12)
    # the leg census leads the new census unchanged
    assert np.array_equal(out["w"][:r["census"]["n"]], r["census"]["w"])


def test_additive_hybrid_infinite_medium_decay(orc):
    """Like the relabelling step, the 3'/4' step keeps the infinite-medium total decaying as
    exp(-sigma_a c t) up to the step-averaging error of the collided emission, shrinking with dt."""
    def run(dt, steps):
        n = 16
        spec = W.homogeneous(n=n, L=16.0, sigma_a=0.5, sigma_s=1.0, Q=None, dt=dt, n_s=1,
                             n_hist=4000, sn_order=4, remap_variant=1, census_cap=6000)
        ic = np.zeros(n * n)
        ic[(n // 2) * n + n // 2] = 1.0
        bank = orc.init_bank(spec, ic)
        for k in range(steps):
            bank = orc.step(spec, k, bank)["bank"]
        return abs(bank["w"].sum() / math.exp(-0.5 * dt * steps) - 1.0)

    e1 = run(0.1, 4)
    e2 = run(0.05, 8)
    assert e1 < 4 * 1.0 * 1.5 * 0.1 ** 2
    assert e2 < e1


# ------------------------------------------------------------------------------------------------
# census in phase-space order (census_order = 2)
# ------------------------------------------------------------------------------------------------
def _deinterleave(sub, b):
    q = [np.zeros_like(sub) for _ in range(3)]
    for i in range(b):
        for d in range(3):
            q[d] |= ((sub >> (3 * i + d)) & 1) << i
    return q


def test_phase_key_groups_by_cell_and_orders_within_it(orc):
    """The key is the cell index above a Morton interleave of three b-bit coordinates, and those
    coordinates follow the in-cell x, the in-cell y and the polar angle of the direction
    (checked against an arctangent), each cut into 2^b equal bins."""
    spec = W.checkerboard(n_s=1, n_hist=10, cells_per_block=2)
    bank = W.random_bank(spec, 20000, seed=11)
    keys, b = orc.phase_keys(spec, bank)
    assert b == 5                                     # 196 cells: 8 cell bits, 3 x 5 = 15 sub-key bits
    keys = keys.astype(np.int64)
    assert np.array_equal(keys >> (3 * b), bank["cell"])
    qx, qy, qa = _deinterleave(keys & ((1 << 3 * b) - 1), b)
    dx, dy = spec.lx / spec.nx, spec.ly / spec.ny
    ang = np.mod(np.arctan2(bank["oy"], bank["ox"]), 2 * np.pi)
    for q, v in ((qx, bank["fx"] / dx), (qy, bank["fy"] / dy), (qa, ang)):
        o = np.argsort(v, kind="stable")
        assert np.all(np.diff(q[o]) >= 0)             # monotone in the coordinate
        counts = np.bincount(q, minlength=1 << b)
        assert counts.min() > 0.5 * len(q) / (1 << b) if q is not qa else counts.min() > 0
    # x and y bins are equal widths: the bin of a value is its fraction of the cell, scaled
    assert np.all(np.abs(qx - bank["fx"] / dx * (1 << b)) <= 1.0)


def test_phase_census_order_is_a_stable_sort_by_key(orc):
    """Without a comb the phase-ordered census holds the slot-ordered census's particles, sorted
    stably by their keys (so also by cell)."""
    spec, bank, r, phi = _remap_inputs(orc)
    spec = spec.with_(census_cap=10 ** 7)
    a, _, ca = orc.remap(spec, 0, bank, r["pre"], r["post"], phi)
    b, _, cb = orc.remap(spec.with_(census_order=2), 0, bank, r["pre"], r["post"], phi)
    assert not ca and not cb and a["n"] == b["n"]
    keys, _ = orc.phase_keys(spec, a)
    order = np.argsort(keys, kind="stable")
    for k in ("cell", "fx", "fy", "ox", "oy", "w"):
        assert np.array_equal(b[k], a[k][order]), k
    assert np.all(np.diff(b["cell"]) >= 0)


def test_phase_ordered_comb_keeps_each_cell_within_one_copy(orc):
    spec, bank, r, phi = _remap_inputs(orc)
    full, _, _ = orc.remap(spec.with_(census_cap=10 ** 7), 0, bank, r["pre"], r["post"], phi)
    cap = full["n"] // 3
    out, _, combed = orc.remap(spec.with_(census_cap=cap, census_order=2), 0, bank, r["pre"], r["post"], phi)
    assert combed and out["n"] == cap
    wc = out["w"][0]
    nc = spec.ncells
    before = np.bincount(full["cell"], weights=full["w"], minlength=nc)
    after = np.bincount(out["cell"], weights=out["w"], minlength=nc)
    assert np.all(np.abs(after - before) <= wc * (1 + 1e-9))
